"""One inversion evaluation split over processes by transmitter columns (one process per GPU).

The forward solves of different transmitters are independent, and so are their adjoint solves
once the adjoint weights are known (Sec. IV-D: J of Eq. sahar:2 couples the columns only through
the S-matrix).  The split therefore has exactly two exchanges per evaluation:
  1. each process solves its window of transmitter columns and all-gathers the S columns, so
     every process holds the whole S (cost and adjoint weights need every entry);
  2. each process solves the adjoints of its own columns and forms their share of the per-tet
     gradient G_T = sum_j lambda_j^T M^T x_j; one all-reduce sums the shares.
The Tikhonov term depends on eps only and is added once, after the sum, on every process.

The solver calls are passed in (`forward_cols`, `gradient_cols`): on a GPU they are the
library's mw_forward_cols / mw_gradient_cols; the module itself holds no arithmetic of the
method beyond the sums of the two collectives.
"""
from __future__ import annotations

import numpy as np


def column_window(rank: int, world: int, n: int) -> tuple[int, int]:
    """Contiguous, balanced windows: (first column, column count) of `rank` among `world`."""
    base, rem = divmod(n, world)
    return rank * base + min(rank, rem), base + (1 if rank < rem else 0)


class ColumnShardedEvaluation:
    """Driver of the split.  `dist` is torch.distributed (initialised); collective buffers live
    on `device` (a CUDA device for NCCL, the CPU for gloo)."""

    def __init__(self, dist, n_src: int, n_freq: int, device="cpu"):
        self.dist = dist
        self.rank = dist.get_rank()
        self.world = dist.get_world_size()
        if n_src < self.world:
            raise ValueError(f"{n_src} transmitters cannot be split over {self.world} processes")
        self.n_src, self.n_freq, self.device = n_src, n_freq, device
        self.j0, self.nl = column_window(self.rank, self.world, n_src)
        self.nl_max = column_window(0, self.world, n_src)[1]

    def gather_columns(self, S_cols: np.ndarray) -> np.ndarray:
        """All-gather of the windows' S columns ([n_freq][n_src][nl] each) into the whole S
        ([n_freq][n_src][n_src]); windows are padded to the widest for the collective."""
        import torch
        nf, ns = self.n_freq, self.n_src
        buf = torch.zeros((nf, ns, self.nl_max, 2), dtype=torch.float64)
        buf[:, :, :self.nl, 0] = torch.from_numpy(np.ascontiguousarray(S_cols.real))
        buf[:, :, :self.nl, 1] = torch.from_numpy(np.ascontiguousarray(S_cols.imag))
        buf = buf.to(self.device)
        parts = [torch.empty_like(buf) for _ in range(self.world)]
        self.dist.all_gather(parts, buf)
        S = np.empty((nf, ns, ns), dtype=np.complex128)
        for r, p in enumerate(parts):
            j0, nl = column_window(r, self.world, ns)
            q = p[:, :, :nl].cpu().numpy()
            S[:, :, j0:j0 + nl] = q[..., 0] + 1j * q[..., 1]
        return S

    def sum_gradient(self, g_part: np.ndarray) -> np.ndarray:
        import torch
        t = torch.from_numpy(np.ascontiguousarray(g_part, dtype=np.float64)).to(self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return t.cpu().numpy()

    def evaluate(self, forward_cols, gradient_cols, S_obs, S_empty, alpha: float = 0.0, tikhonov=None):
        """J, dJ/d(Re eps, Im eps) [n_tet][2] and the whole S of one evaluation.
        forward_cols(j0, nl) -> S columns of the window; gradient_cols(S, S_obs, S_empty) ->
        (J of the whole S, the window's share of the data gradient); tikhonov() -> (R, dR)."""
        S = self.gather_columns(forward_cols(self.j0, self.nl))
        J, g_part = gradient_cols(S, S_obs, S_empty)
        g = self.sum_gradient(g_part)
        if alpha != 0.0:
            R, gR = tikhonov()
            J += alpha * R
            g = g + alpha * gR
        return J, g, S
