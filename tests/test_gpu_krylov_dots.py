"""Error of the mixed-precision Arnoldi dot products against FP64 dots at the bench's size.

The solver keeps the Krylov basis in complex64 and forms h_i = V_i^H w by FP32 products summed
in FP32 over one row tile (TR = 8 * 256 / R rows), then in FP64 across tiles and blocks.  On the
same FP32 inputs, the exact (FP64) dots differ from that by at most about (TR + 4) * 2^-24 times
sum_rows |v_i| |w| per column (first-order bound of recursive FP32 summation plus the complex
product's rounding).  This test measures the difference on seeded vectors of the headline
workload's shape (1,558,914 rows, 32 columns) and checks it against that bound.
"""
import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("n_rows,n_cols,nvec", [(1558914, 32, 6), (200003, 16, 5), (99991, 64, 3)])
def test_streaming_dots_error_against_fp64(n_rows, n_cols, nvec):
    from paper_2311_05322_gb300 import mw
    rng = np.random.default_rng(n_rows % 1000 + n_cols)
    vstride = (n_rows * n_cols + 31) // 32 * 32          # the solver's 256-byte vector spacing
    V = np.zeros(nvec * vstride, np.complex64)
    for i in range(nvec):
        V[i * vstride:i * vstride + n_rows * n_cols] = (rng.standard_normal(n_rows * n_cols, np.float32)
                                                        + 1j * rng.standard_normal(n_rows * n_cols, np.float32))
    w = (rng.standard_normal(n_rows * n_cols, np.float32)
         + 1j * rng.standard_normal(n_rows * n_cols, np.float32)).astype(np.complex64)
    c = mw.Context(0)
    h = c.krylov_dots(torch.from_numpy(V).cuda(), torch.from_numpy(w).cuda(), nvec, vstride, n_rows, n_cols)
    c.close()
    w64 = w.reshape(n_rows, n_cols).astype(np.complex128)
    tr = 8 * 256 // n_cols
    worst = 0.0
    for i in range(nvec):
        Vi = V[i * vstride:i * vstride + n_rows * n_cols].reshape(n_rows, n_cols).astype(np.complex128)
        exact = np.sum(np.conj(Vi) * w64, axis=0)
        scale = np.sum(np.abs(Vi) * np.abs(w64), axis=0)
        err = np.abs(h[i] - exact)
        assert np.all(err <= (tr + 4) * 2.0 ** -24 * scale), (i, (err / scale).max())
        worst = max(worst, float((err / scale).max()))
    print(f"\nstreaming dots {n_rows}x{n_cols}: max |h - h_fp64| / sum|v||w| = {worst:.3e} "
          f"(bound {(tr + 4) * 2.0 ** -24:.3e})")
