"""CPU FP64 oracle for the edge-element Maxwell hot path of arXiv 2311.05322.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package: only `tests/`,
`__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may call it.  It shares no code
with the CUDA library (no kernels, headers, tables or helpers); both sides read their inputs from
the seeded generators in `phantom/`, which hold none of the method's arithmetic.

Everything is plain numpy/scipy in float64 / complex128, written to be checked against the
paper by eye:
  topology.py  canonical edges, signs, faces, CSR pattern            (Sec. IV-D, Nedelec r=1)
  elements.py  Whitney element and boundary-face matrices            (Eq. m2)
  assemble.py  A_f = K - k0^2 M_eps + i k0 sqrt(eps_bg) B            (Eq. m2, k^2 = k0^2 eps_r)
  sources.py   dipole -> edge current, right-hand sides               (Eq. m1 with a volume source)
  solve.py     sparse direct solve, S-matrix                          (Eq. s1, dipole form)
  inverse.py   cost, adjoint, per-tet gradient, Tikhonov, L-BFGS      (Eq. sahar:2, Sec. IV-D)
  oras.py      one-level ORAS and right-preconditioned GMRES          (Sec. IV-C)
  ports.py     TE10 waveguide ports, metal walls, port S-matrix       (Eq. m1-m2 boundary terms, Eq. s1)
  nn.py        FP64 forward/backward of the learned initialiser network
Functions whose parity has no independent pin say "parity unpinned" in their docstring.
"""
