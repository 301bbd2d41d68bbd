"""What the trained network gains over the inversion without it (BASELINE config 5).

Seeded and deterministic (every kernel reduces in a fixed order): forward solves on the data
mesh generate noisy injured-minus-healthy S differences and tear targets, the network trains on
the GPU, and the regularised inversion on a different, coarser mesh starts once from the
healthy permittivity and once from healthy plus the network's proposal.
"""
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_learned_start_beats_plain_start():
    from paper_2311_05322_gb300 import inversion
    r = inversion.run("test", seed=3, plain=False)
    net = r["network"]
    assert net["epoch_loss_first_last"][1] < 0.5 * net["epoch_loss_first_last"][0]
    assert net["test_mse"] < net["zero_predictor_mse"]            # generalises beyond predicting zero
    base, learned = r["inversion"]["mixed"]["J"], r["inversion"]["mixed_learned"]["J"]
    assert base[-1] < base[0]                                     # the inversion reduces the misfit
    assert learned[0] < base[0]                                   # the network's start fits the data better
    assert min(learned) <= min(base)                              # and stays ahead over the same iterations
