"""What the trained network gains over the inversion without it.

Seeded and deterministic (every kernel reduces in a fixed order): forward solves on the data
mesh generate noisy injured-minus-healthy S differences and tear targets, the network trains on
the GPU, and the inversion on a different, coarser mesh starts once from the healthy
permittivity and once from healthy plus the network's proposal, for four held-out tears whose
sizes span the 2-10 mm range.  The network can only help where the tear's signal rises above
the 40 dB noise: for every tear with a positive noise-weighted SNR its start must fit the data
better than the healthy start.
"""
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_learned_start_over_several_tears():
    from paper_2311_05322_gb300 import inversion
    r = inversion.run("test", seed=3, plain=False, tears=4, reciprocal=False)
    net = r["network"]
    assert net["epoch_loss_first_last"][1] < 0.5 * net["epoch_loss_first_last"][0]
    assert net["test_mse"] < net["zero_predictor_mse"]            # generalises beyond predicting zero
    above = [c for c in r["cases"] if c["snr_db"] > 0.0]
    assert above, [c["snr_db"] for c in r["cases"]]               # the largest tears rise above the noise
    for c in r["cases"]:
        base = c["inversion"]["mixed"]["J"]
        assert base[-1] < base[0]                                 # every inversion reduces the misfit
    for c in above:
        base, learned = c["inversion"]["mixed"]["J"], c["inversion"]["mixed_learned"]["J"]
        assert learned[0] < base[0], (c["snr_db"], learned[0], base[0])
