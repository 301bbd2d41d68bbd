"""The allocation-free preconditioner apply against the regular one and the oracle.

mw_apply_preconditioner_noalloc serves callers that cannot allocate device memory when they
apply the preconditioner; it must give the same result as mw_apply_preconditioner, call after
call, while its gathered operand lives in the library's fixed scratch array.  This file is
collected last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

from oracle import assemble as asm
from oracle import oras
from phantom import EPS_MATCHING, box_partition, kuhn_mesh

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_noalloc_apply_matches_regular_apply_twice():
    from paper_2311_05322_gb300 import mw
    m = kuhn_mesh(6, 5, 4, lo=(-0.03, -0.025, -0.02), hi=(0.03, 0.025, 0.02))
    rng = np.random.default_rng(77)
    eps = EPS_MATCHING + rng.uniform(-6, 6, m.n_tet) + 1j * rng.uniform(-4, 4, m.n_tet)
    c = mw.Context(0)
    c.set_mesh(m.xyz, m.tets)
    c.assemble([1e9], np.stack([eps.real, eps.imag], 1), EPS_MATCHING)
    c.setup_preconditioner(4, box_partition(m, (2, 2, 1), seed=7), 1, mw.MW_PREC_BF16)
    E = c.info.n_edge
    sysm = asm.build_system(m.xyz, m.tets)
    P = oras.ORAS(sysm, box_partition(m, (2, 2, 1), seed=7), 4, 1, eps, 1e9, EPS_MATCHING)
    P.apply_many = lambda R: np.stack([P.apply(R[:, k]) for k in range(R.shape[1])], 1)
    for call, ncols in enumerate((24, 7)):
        X = rng.normal(size=(E, ncols)) + 1j * rng.normal(size=(E, ncols))
        x64 = torch.from_numpy(X).to(torch.complex64).cuda()          # the value both paths see
        ref = torch.empty((E, ncols), dtype=torch.complex128, device="cuda")
        c.apply_preconditioner(0, x64.to(torch.complex128), ref, ncols)
        z = torch.full((E, ncols), float("nan"), dtype=torch.complex64, device="cuda")
        c.apply_preconditioner_noalloc(0, x64, z, ncols)
        torch.cuda.synchronize()
        a = z.cpu().numpy().astype(np.complex128)
        b = ref.cpu().numpy()
        # same kernels on the same inputs: equal up to FP32 rounding (the BF16 apply bar in the
        # parity tests is 1e-2 against the FP64 operator)
        assert np.all(np.isfinite(a)), f"call {call}: rows left unwritten"
        assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(b), f"call {call}"
        # and against the oracle's ORAS operator (exact sparse-LU subdomain solves, FP64), at the
        # bar of the BF16 tensor-core apply in the parity tests
        zo = P.apply_many(x64.cpu().numpy().astype(np.complex128))
        assert np.linalg.norm(a - zo) <= 1e-2 * np.linalg.norm(zo), f"call {call}"
    c.close()


def test_noalloc_rejects_operand_above_the_fixed_scratch():
    from paper_2311_05322_gb300 import mw
    m = kuhn_mesh(24, 24, 16, lo=(-0.06, -0.06, -0.04), hi=(0.06, 0.06, 0.04))
    c = mw.Context(0)
    c.set_mesh(m.xyz, m.tets)
    c.assemble([1e9], np.tile([44.0, -20.0], (m.n_tet, 1)), EPS_MATCHING)
    c.setup_preconditioner(144, box_partition(m, (6, 6, 4), seed=7), 1, mw.MW_PREC_BF16)
    E = c.info.n_edge
    x = torch.zeros((E, 128), dtype=torch.complex64, device="cuda")
    z = torch.zeros_like(x)
    with pytest.raises(mw.MWError) as ei:
        c.apply_preconditioner_noalloc(0, x, z, 128)
    assert ei.value.status == mw.MW_EINVAL and "fixed scratch" in str(ei.value)
    c.close()
