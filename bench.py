"""Benchmark of the microwave-tomography hot path on GB300: Maxwell RHS-solves/s at rel.res 1e-8.

One step = one evaluation of the regularised inversion (Sec. IV-D) on the shoulder-scale
phantom: eps -> matrix reassembly, 32 forward dipole solves, S-matrix, cost and adjoint
sources, 32 adjoint solves (GMRES(50) + ORAS, FP64 true relative residual <= 1e-8 per column),
per-tet adjoint gradient and Tikhonov term.  RHS-solves per step = 2 x transmitters x frequencies.

  value  device-resident: eps, S_obs, S_empty and the gradient stay in HBM (CUDA events on the
         library's stream around K steps).
  e2e    the public host-buffer API (mw_assemble + mw_gradient): eps and S in from pinned host
         memory, gradient and cost back to the host, inside the timed region.
Under torchrun (N > 1) the ranks split one evaluation by transmitter columns (strong scaling; an
all-gather of S and an all-reduce of the gradient per evaluation, paper_2311_05322_gb300.sharded);
`--replicas` runs independent evaluations per rank instead (weak scaling).  Rank 0 prints one
JSON line.  `--impl reference` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Maxwell RHS-solves/s at rel.res 1e-8"
UNIT = "RHS-solves/s"


def _args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--cells", default="80x80x34")
    ap.add_argument("--n-src", type=int, default=32)
    ap.add_argument("--antennas", default="dipoles", choices=["dipoles", "waveguides"],
                    help="z-dipole ring, or ceramic-filled TE10 waveguides on three side walls (Eq. m1 ports)")
    ap.add_argument("--freqs", default="1.0e9", help="comma-separated frequencies (Hz)")
    ap.add_argument("--parts", default="22x22x10")
    ap.add_argument("--overlap", type=int, default=1)
    ap.add_argument("--prec", default="bf16", choices=["bf16", "fp32", "sparse", "sparse_bf16"],
                    help="subdomain solves: dense inverses applied in BF16 (tensor cores) or FP32, or sparse "
                         "multifrontal factors (large subdomains)")
    ap.add_argument("--alpha", type=float, default=1e-3)
    ap.add_argument("--z-storage", default="bf16", choices=["bf16", "fp32"],
                    help="storage of the preconditioned Krylov vectors on the tensor-core path")
    ap.add_argument("--inner-tol", type=float, default=1e-2,
                    help="residual reduction of each inner FGMRES cycle (GMRES-IR); 1e-2 measured fastest")
    ap.add_argument("--plain-cols", type=int, default=1, help="columns timed on the plain FP64 path (0 = skip)")
    ap.add_argument("--plain-factor", default="fp64", choices=["fp64", "fp32"],
                    help="subdomain inverses of the plain FP64 path factorised in FP64 (setup, outside the timing) "
                         "or in FP32 and applied in FP64")
    ap.add_argument("--fp64-batch-cols", type=int, default=4,
                    help="columns timed as one FP64 block (isolates the batching gain; 0 = skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--graphs", action="store_true", help="replay restart cycles from captured CUDA graphs")
    ap.add_argument("--cpu-sample-subdomains", type=int, default=24)
    ap.add_argument("--cpu-cores", type=int, default=0, help="host processes of the oracle baseline (0 = all cores)")
    ap.add_argument("--no-legs", action="store_true", help="skip the three-frequency, sparse, training and time-to-misfit legs")
    ap.add_argument("--replicas", action="store_true",
                    help="N > 1: independent evaluations per rank instead of the column split of one evaluation")
    ap.add_argument("--inversion-leg", default="bench", choices=["none", "tiny", "bench", "test", "reduced"],
                    help="scale of the time-to-misfit leg of the default run")
    ap.add_argument("--study", default=None, choices=["tiny", "reduced"],
                    help="antenna-count design study (Sec. V): err / ctr for N = 96/64/32/16 at 23/15/10 dB")
    ap.add_argument("--inversion", default=None, choices=["tiny", "bench", "test", "reduced", "full"],
                    help="time-to-misfit of the regularised inversion instead of RHS-solves/s")
    ap.add_argument("--tears", type=int, default=1, help="held-out tears of the --inversion run")
    ap.add_argument("--alphas", default="", help="Tikhonov sweep of the --inversion run (comma-separated)")
    ap.add_argument("--plain", action="store_true", help="--inversion: run the plain FP64 arm at every scale")
    return ap.parse_args(argv)


def _dims(s):
    return tuple(int(x) for x in s.split("x"))


# ---------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if p[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------------------
def waveguide_counts(n_src: int):
    """Guides per side wall (x = lo, x = hi, y = lo, y = hi): the x = lo wall, where the torso
    enters the box, stays open; the others share n_src as evenly as they can."""
    base, rem = divmod(n_src, 3)
    return (0,) + tuple(base + (1 if k < rem else 0) for k in range(3))


def make_workload(a):
    from phantom import EPS_CERAMIC, box_partition, port_chamber, random_tear, shoulder
    cells = _dims(a.cells)
    freqs = tuple(float(f) for f in a.freqs.split(","))
    healthy = shoulder(cells, n_src=a.n_src, freqs=freqs)
    injured = shoulder(cells, n_src=a.n_src, freqs=freqs, tear=random_tear(2001))
    if a.antennas == "waveguides":
        fv, lab, ps, guide = port_chamber(healthy.mesh, waveguide_counts(a.n_src), a_cells=5, b_cells=2, depth=4)
        for w in (healthy, injured):
            w.eps[guide] = EPS_CERAMIC
            w.extra["ports"] = (fv, lab, ps, guide)
    parts = _dims(a.parts)
    part = box_partition(healthy.mesh, parts, seed=7)
    return healthy, injured, parts, part


def oras_traffic_ratio(parts: str):
    """DRAM traffic per algorithmic byte of the ORAS apply from the committed ncu summary, or
    None when the summary was taken on another partition or the two kernels' source no longer
    matches the one the counters were taken on."""
    import hashlib
    prof = os.path.join(ROOT, "profiles", "oras_apply_traffic_shoulder80x80x34.md")
    src = os.path.join(ROOT, "paper_2311_05322_gb300", "csrc", "k_oras_tc.cu")
    if not (os.path.exists(prof) and os.path.exists(src)):
        return None
    kv = dict(l.split(": ", 1) for l in open(prof).read().splitlines() if ": " in l and not l.startswith("|"))
    if kv.get("partition", "").strip() != parts:
        return None
    text = open(src).read()

    def body(sig):
        i = text.find(sig)
        if i < 0:
            return ""
        return text[i:text.index("\n}\n", i) + 3]
    gather, mma = body("gather_b_kernel("), body("__global__ void __launch_bounds__(kThreadsTc, 2) oras_tc_kernel")
    if not gather or not mma:
        return None
    h = hashlib.sha256((gather + mma).encode()).hexdigest()
    if kv.get("kernel_source_sha256", "").strip() != h:
        return None
    return float(kv["traffic_per_algorithmic_byte"])


def aggregate(units_per_rank: float, seconds: float, world: int, dist=None):
    """Whole-job throughput under weak scaling: every rank solves its own units; the job time is
    the slowest rank's (one all_reduce MAX of a scalar, no exchange on the data path)."""
    if dist is not None and world > 1:
        import torch
        dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([seconds], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        seconds = float(t.item())
    return units_per_rank * world / seconds, seconds


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs"), d.get("bf16_tflops"), d.get("bf16_tflops_sustained"), "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


def measured_alu_peaks(dev):
    """FP32 (TF32 off) and FP64 dense GEMM rates of this GPU, measured here with torch.matmul
    (cuBLAS) and CUDA events, best of 5 after 2 warm-ups: the peaks the FP32- and FP64-bound
    kernels are rated against."""
    import torch
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for name, dt, n in (("fp32_tflops", torch.float32, 8192), ("fp64_tflops", torch.float64, 4096)):
            g = torch.Generator(device=dev).manual_seed(1)
            a = torch.randn(n, n, dtype=dt, device=dev, generator=g)
            b = torch.randn(n, n, dtype=dt, device=dev, generator=g)
            for _ in range(2):
                torch.matmul(a, b)
            best = float("inf")
            for _ in range(5):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            out[name] = 2.0 * n ** 3 / (best * 1e-3) / 1e12
            del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    out["how"] = "torch.matmul fp32 8192^3 (TF32 off) and fp64 4096^3, best of 5, CUDA events"
    return out


# What bounds each kernel class of the library's profiler, and the work it is rated by.
CLASS_BOUND = {"spmm": "hbm", "oras_apply": "hbm", "cgs_dots": "hbm", "cgs_update": "hbm", "residual_fp64": "hbm",
               "reassemble": "hbm", "gradient": "fp64", "factor": "fp32", "nn_gemm": "fp32", "nn_conv": "fp32",
               "nn_other": "hbm"}


def rate_classes(prof, hbm, alu):
    """Per class: device ms, launches, achieved GB/s and TFLOP/s of algorithmic work, and the
    fraction of the peak of its bound (HBM copy rate, or the measured FP32 / FP64 GEMM rate)."""
    out = {}
    for k, v in prof.items():
        if v["launches"] == 0 or v["ms"] <= 0:
            continue
        sec = v["ms"] * 1e-3
        gbs = v["bytes"] / sec / 1e9
        tfs = v.get("flops", 0.0) / sec / 1e12
        bound = CLASS_BOUND.get(k, "hbm")
        if bound == "hbm":
            peak, ach, unit = hbm, gbs, "GB/s"
        else:
            peak, ach, unit = alu.get(f"{bound}_tflops"), tfs, "TFLOP/s"
        out[k] = {"ms": v["ms"], "launches": v["launches"], "GBs": gbs, "TFLOPs": tfs, "bound": bound,
                  "achieved": ach, "peak": peak, "unit": unit, "frac": (ach / peak) if peak else None}
    return out


# ---------------------------------------------------------------------------------------
# CPU oracle sample (baseline, not a target)
# ---------------------------------------------------------------------------------------
class OracleColumnSample:
    """Oracle cost of one column solve, from timed pieces of one Arnoldi step on the full
    workload: the oracle's FP64 matvec, its ORAS subdomain solves on a random sample of
    subdomains (scaled to all), one modified Gram-Schmidt pass at the mean Krylov depth; times
    the Arnoldi steps per column.  The untimed setup (system, sampled subdomain factorisations)
    runs once; run() times one sample."""

    def __init__(self, w, part, n_sub, overlap, iters_per_col, n_sample_subs, seed=0, ports=None):
        import scipy.sparse.linalg as spla

        from oracle import assemble as asm
        from oracle import oras as ooras
        t0 = time.perf_counter()
        self.w, self.n_sub, self.iters = w, n_sub, iters_per_col
        self.sysm = asm.build_system(w.mesh.xyz, w.mesh.tets, with_pattern=False)
        self.rng = np.random.default_rng(seed)
        pick = self.rng.choice(n_sub, size=min(n_sample_subs, n_sub), replace=False)
        subs, _ = ooras.build_subdomains(self.sysm, part, n_sub, overlap, which=pick)
        self.zface, free = None, None
        if ports is not None:
            from oracle import ports as oports
            fv, lab, ps, _ = ports
            P = oports.make_ports(ps.origin, ps.u, ps.v, ps.a, ps.eps_fill)
            bnd = oports.classify(self.sysm, P, fv, lab)
            self.zface = oports.face_coefficients(w.freqs[0], w.eps_bg, bnd)
            free = ~bnd.metal
        self.lus = []
        for sub in subs:
            B = ooras.local_matrix(self.sysm, sub, w.eps, w.freqs[0], w.eps_bg, self.zface)
            if free is not None:                       # metal edges are not unknowns
                fl = np.nonzero(free[sub.dofs])[0]
                B = B[fl][:, fl].tocsc()
                sub = ooras.Subdomain(sub.tets, sub.dofs[fl], np.nonzero(np.isin(fl, sub.owned))[0], sub.iface,
                                      sub.iface_tet)
            self.lus.append((sub, spla.splu(B)))
        self.setup_s = time.perf_counter() - t0

    def run(self):
        from oracle import assemble as asm
        w, rng = self.w, self.rng
        E = self.sysm.topo.n_edge
        x = rng.normal(size=(E, 1)) + 1j * rng.normal(size=(E, 1))
        t = time.perf_counter()
        for _ in range(2):
            y = asm.apply_system(self.sysm, w.eps, w.freqs[0], w.eps_bg, x, self.zface)[:, 0]
        t_mv = (time.perf_counter() - t) / 2
        x = x[:, 0]
        z = np.zeros(E, dtype=complex)
        t = time.perf_counter()
        for sub, lu in self.lus:
            yy = lu.solve(np.ascontiguousarray(x[sub.dofs]))
            z[sub.dofs[sub.owned]] = yy[sub.owned]
        t_p = (time.perf_counter() - t) * self.n_sub / len(self.lus)
        depth = max(1, int(round(min(self.iters, 50) / 2)))
        V = rng.normal(size=(depth, E)) + 0j
        t = time.perf_counter()
        wv = y.copy()
        for i in range(depth):
            h = np.vdot(V[i], wv)
            wv = wv - h * V[i]
        t_gs = time.perf_counter() - t
        per_step = t_mv + t_p + t_gs
        return per_step * self.iters, {"setup_s": self.setup_s, "matvec_s": t_mv, "oras_s": t_p, "gs_s": t_gs,
                                        "timed_s": 2 * t_mv + t_p * len(self.lus) / self.n_sub + t_gs}


_BLAS_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _oracle_worker(argv, seed, iters_per_col, n_sample_subs, n_samples, barrier, q):
    a = _args(argv)
    healthy, _, parts, part = make_workload(a)
    smp = OracleColumnSample(healthy, part, int(np.prod(parts)), a.overlap, iters_per_col, n_sample_subs, seed=seed,
                             ports=healthy.extra.get("ports"))
    for k in range(n_samples):
        barrier.wait()                 # the processes time their samples side by side
        col_s, det = smp.run()
        q.put((k, seed, col_s, det))


def oracle_throughput(argv, iters_per_col, n_sample_subs, cores=None, n_samples=1, seed0=0):
    """The oracle's column rate on the host's cores: one process per core (spawned, so none
    inherits a CUDA context), each costing its own sampled column; every sample starts after a
    common barrier, so the processes' timed pieces run concurrently.  Returns, per sample, the
    columns/s summed over processes, and the core count and details."""
    import multiprocessing as mp
    cores = cores or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(cores)
    q = ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker,
                      args=(argv, seed0 + k, iters_per_col, n_sample_subs, n_samples, barrier, q))
          for k in range(cores)]
    # one host core per process: the children's BLAS reads its thread count when numpy loads
    saved = {k: os.environ.get(k) for k in _BLAS_THREAD_VARS}
    os.environ.update({k: "1" for k in _BLAS_THREAD_VARS})
    try:
        for p in ps:
            p.start()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    res = [q.get(timeout=3600) for _ in range(cores * n_samples)]
    for p in ps:
        p.join(timeout=120)
    rates = [sum(1.0 / r[2] for r in res if r[0] == k) for k in range(n_samples)]
    det = {"per_process_column_s": sorted(r[2] for r in res if r[0] == 0),
           "setup_s_max": max(r[3]["setup_s"] for r in res), "timed_s_max": max(r[3]["timed_s"] for r in res)}
    return rates, cores, det


# ---------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------
def _setup_leg(a, local, stream):
    """Context, mesh, sources, background-medium preconditioner (profiled), tuned launch shapes
    and the synthetic measurements of one workload."""
    import torch

    from paper_2311_05322_gb300 import mw
    healthy, injured, parts, part = make_workload(a)
    n_sub = int(np.prod(parts))
    freqs = list(healthy.freqs)
    eps0 = np.stack([healthy.eps.real, healthy.eps.imag], 1)
    c = mw.Context(local, stream.cuda_stream)
    setup = {}
    c.set_graphs(a.graphs)
    t = time.perf_counter()
    info = c.set_mesh(healthy.mesh.xyz, healthy.mesh.tets)
    torch.cuda.synchronize()
    setup["mesh_s"] = time.perf_counter() - t
    ports = healthy.extra.get("ports")
    if ports is None:
        c.set_sources(healthy.src_pos, healthy.src_dir)
        hom = np.tile([healthy.eps_bg.real, healthy.eps_bg.imag], (healthy.mesh.n_tet, 1))
    else:
        fv, lab, ps, guide = ports
        c.set_ports(ps.origin, ps.u, ps.v, ps.a, ps.eps_fill, fv, lab)
        hom_c = np.full(healthy.mesh.n_tet, healthy.eps_bg)
        hom_c[guide] = ps.eps_fill[0]
        hom = np.stack([hom_c.real, hom_c.imag], 1)
    # preconditioner of the background medium, reused stale for every eps (as in an inversion)
    c.assemble(freqs, hom, healthy.eps_bg)
    prec = {"bf16": mw.MW_PREC_BF16, "fp32": mw.MW_PREC_FP32, "sparse": mw.MW_PREC_SPARSE,
            "sparse_bf16": mw.MW_PREC_SPARSE_BF16}[a.prec]
    c.profile_enable(1 << mw.MW_K_FACTOR)
    c.set_z_storage(a.z_storage == "bf16")
    t = time.perf_counter()
    c.setup_preconditioner(n_sub, part, a.overlap, prec)
    torch.cuda.synchronize()
    setup["preconditioner_s"] = time.perf_counter() - t
    setup_prof = {k: v for k, v in c.profile_read().items() if v["launches"]}
    c.profile_enable(0)
    t = time.perf_counter()
    tune = c.autotune(a.n_src, mw.MW_MODE_MIXED, 50)      # launch shapes of the timed solves
    setup["autotune_s"] = time.perf_counter() - t
    _, sizes = c.get_partition()
    opts = mw.solve_opts(mode=mw.MW_MODE_MIXED, restart=50, tol=1e-8, inner_tol=a.inner_tol, max_it=2000)
    # synthetic measurements: injured phantom (observed) and empty chamber (normalisation)
    t = time.perf_counter()
    S_empty, _ = c.solve(opts)
    c.assemble(freqs, np.stack([injured.eps.real, injured.eps.imag], 1), injured.eps_bg)
    S_obs, _ = c.solve(opts)
    c.assemble(freqs, eps0, healthy.eps_bg)
    setup["data_s"] = time.perf_counter() - t
    return dict(c=c, healthy=healthy, parts=parts, part=part, n_sub=n_sub, freqs=freqs, eps0=eps0, hom=hom,
                info=info, ports=ports, prec=prec, tune=tune, sizes=sizes, opts=opts, S_empty=S_empty, S_obs=S_obs,
                setup=setup, setup_prof=setup_prof)


def _timed_steps(L, a, local, stream, steps, warmup, world, dist):
    """Device-resident steps (eps, S_obs, S_empty and the gradient in HBM): warm-up, then `steps`
    steps between CUDA events on the library's stream, profiled by kernel class."""
    import torch

    from paper_2311_05322_gb300 import mw
    c = L["c"]
    dev = torch.device("cuda", local)
    eps_d = torch.from_numpy(L["eps0"]).to(dev)
    So_d = torch.from_numpy(L["S_obs"]).to(dev)
    Se_d = torch.from_numpy(L["S_empty"]).to(dev)
    g_d = torch.empty((L["healthy"].mesh.n_tet, 2), dtype=torch.float64, device=dev)

    def step_dev():
        c.assemble_dev(L["freqs"], eps_d, L["healthy"].eps_bg)
        return c.gradient_dev(So_d, Se_d, g_d, a.alpha, L["opts"])

    # the profiler is on during warm-up too, so the restart cycles the timed steps replay (captured
    # with their profiling events) are captured here, outside the timed region
    c.profile_enable((1 << mw.MW_K_NCLASS) - 1)
    for _ in range(warmup):
        step_dev()
    torch.cuda.synchronize()
    c.profile_read()            # discard the warm-up samples
    if world > 1:
        dist.barrier()
    l0 = mw.kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            J = step_dev()
        e1.record(stream)
        torch.cuda.synchronize()
    launches = mw.kernel_launches() - l0
    prof = c.profile_read()
    c.profile_enable(0)
    return e0.elapsed_time(e1) * 1e-3, J, prof, launches, clk.summary()


def _dominant_roofline(prof, ms_step_total, hbm, src, prec, a, L):
    from paper_2311_05322_gb300 import mw
    dom = max(prof, key=lambda k: prof[k]["ms"])
    d = prof[dom]
    achieved = d["bytes"] / (d["ms"] * 1e-3) / 1e9 if d["ms"] > 0 else 0.0
    ratio = oras_traffic_ratio(a.parts) if dom == "oras_apply" and prec == mw.MW_PREC_BF16 and a.cells == "80x80x34" \
        and a.antennas == "dipoles" and a.n_src == 32 else None
    traffic = ratio * d["bytes"] / max(d["launches"], 1) if ratio else None
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "peak_source": src, "traffic": traffic,
            "traffic_note": ("DRAM bytes per algorithmic byte from profiles/oras_apply_traffic_shoulder80x80x34.md "
                             "(ncu, one pass, this workload)") if traffic else None,
            "bytes_per_launch": d["bytes"] / max(d["launches"], 1),
            "avg_launch_ms": d["ms"] / max(d["launches"], 1),
            "share_of_step": d["ms"] / ms_step_total}
    return roof, dom


def nn_leg(local, stream, alu, hbm, n_in=8192, batch=64, samples=1024):
    """One training epoch of the learned initialiser at its real size (8192 inputs, batch 64) on
    seeded random data, profiled by kernel class."""
    from paper_2311_05322_gb300 import inversion, mw
    c = mw.Context(local, stream.cuda_stream)
    rng = np.random.default_rng(21)
    x = rng.normal(size=(samples, n_in)).astype(np.float32)
    t = (0.1 * rng.normal(size=(samples, 2, 32, 32, 32))).astype(np.float32)
    c.nn_init(n_in, inversion.he_init(n_in, 1))
    c.nn_train(x[:batch], t[:batch], batch=batch, epochs=1, lr=1e-4, seed=1)      # warm-up
    c.profile_enable((1 << mw.MW_K_NN_GEMM) | (1 << mw.MW_K_NN_CONV) | (1 << mw.MW_K_NN_OTHER))
    losses, secs = c.nn_train(x, t, batch=batch, epochs=1, lr=1e-4, seed=2)
    prof = c.profile_read()
    c.profile_enable(0)
    c.close()
    return {"config": f"{samples} samples, {n_in} inputs, batch {batch}, one epoch (seeded random data)",
            "train_s": secs, "steps": samples // batch, "classes": rate_classes(prof, hbm, alu)}


def shoulder55_3f_leg(a, local, stream, alu, hbm, src, steps=3, warmup=2):
    """The mixed-precision batched forward/adjoint configuration: 55x55x24 shoulder (525,329
    edges), 64 transmitters x 3 frequencies (0.8 / 1.0 / 1.2 GHz) as one block per frequency,
    BF16 tensor-core ORAS, GMRES-IR to 1e-8."""
    a3 = _args(["--cells", "55x55x24", "--n-src", "64", "--freqs", "0.8e9,1.0e9,1.2e9", "--parts", "11x11x5",
                "--alpha", str(a.alpha), "--z-storage", a.z_storage])
    L = _setup_leg(a3, local, stream)
    sec, J, prof, launches, clocks = _timed_steps(L, a3, local, stream, steps, warmup, 1, None)
    units = 2 * a3.n_src * len(L["freqs"])
    ms = sec * 1e3
    roof, _ = _dominant_roofline(prof, ms, hbm, src, L["prec"], a3, L)
    info, sizes = L["info"], L["sizes"]
    L["c"].close()
    return {"value": units * steps / sec, "unit": UNIT, "ms_per_step": ms / steps, "steps": steps, "warmup": warmup,
            "config": {"workload": f"shoulder phantom 55x55x24 Kuhn cells ({info.n_edge} edges, {info.n_tet} tets), "
                                   f"64 z-dipoles x 3 frequencies, one inversion evaluation (forward+adjoint)",
                       "rhs_solves_per_step": units, "subdomains": L["n_sub"], "n_s_mean": float(sizes.mean()),
                       "n_s_max": int(sizes.max()), "preconditioner_apply": "bf16 tcgen05",
                       "z_storage": a3.z_storage},
            "roofline": roof, "classes": rate_classes(prof, hbm, alu), "gpu_launches": int(launches),
            "clocks": clocks, "setup_s": L["setup"], "J_last": J}


def sparse16_leg(a, local, stream, alu, hbm, src, steps=3, warmup=3):
    """The shoulder-scale configuration with its specified decomposition: 80x80x34 (1,558,914
    edges), 32 dipoles, 16 subdomains of about 132k unknowns with 2 overlap layers, sparse
    multifrontal subdomain solves with their sweeps on the tensor cores, GMRES-IR to 1e-8.  Inner
    cycles at 1e-4: each apply of the exact subdomain solves costs as much as about 20 Gram-Schmidt
    steps, so fewer restarts win (measured over 1e-2 .. 1e-6: 1e-4 takes the fewest Arnoldi
    steps, 102.3 RHS-solves/s at 1e-2 against 107.7 at 1e-4 before the stacked sweeps)."""
    a2 = _args(["--prec", "sparse_bf16", "--parts", "4x4x1", "--overlap", "2", "--alpha", str(a.alpha),
                "--inner-tol", "1e-4"])
    L = _setup_leg(a2, local, stream)
    sec, J, prof, launches, clocks = _timed_steps(L, a2, local, stream, steps, warmup, 1, None)
    units = 2 * a2.n_src * len(L["freqs"])
    ms = sec * 1e3
    roof, _ = _dominant_roofline(prof, ms, hbm, src, L["prec"], a2, L)
    info, sizes = L["info"], L["sizes"]
    L["c"].close()
    return {"value": units * steps / sec, "unit": UNIT, "ms_per_step": ms / steps, "steps": steps, "warmup": warmup,
            "config": {"workload": f"shoulder phantom 80x80x34 Kuhn cells ({info.n_edge} edges), 32 z-dipoles, "
                                   f"one inversion evaluation (forward+adjoint); 16 subdomains, 2 overlap layers",
                       "rhs_solves_per_step": units, "subdomains": L["n_sub"], "n_s_mean": float(sizes.mean()),
                       "n_s_max": int(sizes.max()),
                       "preconditioner_apply": "bf16 tcgen05 multifrontal sweeps", "inner_tol": a2.inner_tol},
            "roofline": roof, "classes": rate_classes(prof, hbm, alu), "gpu_launches": int(launches),
            "clocks": clocks, "setup_s": L["setup"], "J_last": J}


def run_sharded(a, world, rank, local):
    """N > 1 (under torchrun, one process per GPU): one evaluation split by transmitter columns.
    Every rank holds the mesh, matrices and preconditioner; rank r solves its window of the
    columns (mw_forward_cols), the S columns are all-gathered over NCCL, each rank solves its
    adjoints and forms its share of the gradient (mw_gradient_cols), one all-reduce sums the
    shares, and the Tikhonov term is added once.  Strong scaling: the job's columns are fixed."""
    import torch
    import torch.distributed as dist

    from paper_2311_05322_gb300 import mw
    from paper_2311_05322_gb300.sharded import ColumnShardedEvaluation
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    hbm, _, _, src = peaks()
    alu = measured_alu_peaks(torch.device("cuda", local))
    L = _setup_leg(a, local, stream)
    c, healthy, freqs, opts = L["c"], L["healthy"], L["freqs"], L["opts"]
    drv = ColumnShardedEvaluation(dist, a.n_src, len(freqs), device=torch.device("cuda", local))
    eps_h = torch.from_numpy(L["eps0"]).pin_memory().numpy()
    S_obs, S_empty = L["S_obs"], L["S_empty"]
    units = 2 * a.n_src * len(freqs)

    def step():
        c.assemble(freqs, eps_h, healthy.eps_bg)
        return drv.evaluate(lambda j0, nl: c.forward_cols(j0, nl, opts),
                            lambda S, So, Se: c.gradient_cols(S, So, Se, opts), S_obs, S_empty, a.alpha,
                            lambda: c.tikhonov(eps_h))

    c.profile_enable((1 << mw.MW_K_NCLASS) - 1)
    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    c.profile_read()
    dist.barrier()
    l0 = mw.kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0.record(stream)
        for _ in range(a.steps):
            J, g, S = step()
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    launches = mw.kernel_launches() - l0
    prof = c.profile_read()
    c.profile_enable(0)
    value, sec = aggregate(units * a.steps, e0.elapsed_time(e1) * 1e-3, world, dist)
    e2e_value, _ = aggregate(units * a.steps, wall, world, dist)
    ms = sec * 1e3
    roof, _ = _dominant_roofline(prof, ms, hbm, src, L["prec"], a, L)
    roof["classes"] = rate_classes(prof, hbm, alu)
    info = L["info"]
    c.close()
    if rank == 0:
        nS = len(freqs) * a.n_src * a.n_src
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "c64+bf16 inner / c128 outer", "data": "synthetic",
            "config": {"workload": f"shoulder phantom {a.cells} Kuhn cells ({info.n_edge} edges), {a.n_src} z-dipoles "
                                   f"x {len(freqs)} frequencies, one inversion evaluation split by transmitter "
                                   f"columns over {world} GPUs",
                       "parallelism": f"transmitter columns over {world} ranks",
                       "columns_per_rank": drv.nl, "rhs_solves_per_step": units, "subdomains": L["n_sub"],
                       "exchanges": "all_gather of the S columns, all_reduce of the 2T gradient (NCCL)",
                       "l2": "inputs larger than L2 (subdomain inverses and Krylov basis are GBs)"},
            "roofline": roof, "cpu_baseline": None,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": L["eps0"].nbytes + 2 * 16 * nS,
                    "d2h_bytes_per_step": 16 * info.n_tet + 8 + 16 * nS},
            "gpu_launches": int(launches), "clocks": clk.summary(), "setup_s": L["setup"], "J_last": J,
        }
        print(json.dumps(line), flush=True)
    dist.destroy_process_group()


def run_mine(a):
    import torch
    import torch.distributed as dist

    from paper_2311_05322_gb300 import mw

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
        if not a.replicas:
            return run_sharded(a, world, rank, local)
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    hbm, bf16, bf16s, src = peaks()
    alu = measured_alu_peaks(torch.device("cuda", local))

    L = _setup_leg(a, local, stream)
    c, healthy, info, ports, prec, freqs = L["c"], L["healthy"], L["info"], L["ports"], L["prec"], L["freqs"]
    eps0, S_obs, S_empty, opts = L["eps0"], L["S_obs"], L["S_empty"], L["opts"]
    units = 2 * a.n_src * len(freqs)
    sec, J, prof, launches, clocks = _timed_steps(L, a, local, stream, a.steps, a.warmup, world,
                                                  dist if world > 1 else None)
    value, sec = aggregate(units * a.steps, sec, world, dist if world > 1 else None)
    ms = sec * 1e3

    # ---- e2e through the host-buffer API --------------------------------------------------
    eps_h = torch.from_numpy(eps0).pin_memory().numpy()
    So_h = torch.from_numpy(S_obs).pin_memory().numpy()
    Se_h = torch.from_numpy(S_empty).pin_memory().numpy()
    g_h = torch.empty((healthy.mesh.n_tet, 2), dtype=torch.float64).pin_memory().numpy()   # the step's result
    c.assemble(freqs, eps_h, healthy.eps_bg)
    c.gradient(So_h, Se_h, a.alpha, opts, out=g_h)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t = time.perf_counter()
    for _ in range(a.steps):
        c.assemble(freqs, eps_h, healthy.eps_bg)
        Jh, gh = c.gradient(So_h, Se_h, a.alpha, opts, out=g_h)
    torch.cuda.synchronize()
    e2e_value, e2e_s = aggregate(units * a.steps, time.perf_counter() - t, world, dist if world > 1 else None)
    T = healthy.mesh.n_tet
    h2d = eps0.nbytes + S_obs.nbytes + S_empty.nbytes
    d2h = 16 * T + 8

    dev = torch.device("cuda", local)
    n_sub, part = L["n_sub"], L["part"]
    hom = L["hom"]
    # ---- plain FP64 path (FP64 operator, basis and apply, one RHS per Krylov launch) -------
    plain = None
    if ports is not None:
        plain = {"skipped": "dipole-source leg; not run for the waveguide workload"}
    elif a.plain_cols > 0 and rank == 0:
        try:
            c.assemble(freqs, hom, healthy.eps_bg)
            t = time.perf_counter()
            c.setup_preconditioner(n_sub, part, a.overlap,
                                   mw.MW_PREC_FP64 if a.plain_factor == "fp64" else mw.MW_PREC_FP64_FROM_FP32)
            torch.cuda.synchronize()
            ps = time.perf_counter() - t
            c.assemble(freqs, eps0, healthy.eps_bg)
            E = info.n_edge
            rhs = np.zeros((a.plain_cols, E), dtype=np.complex128)
            for j in range(a.plain_cols):
                b = np.zeros(E, dtype=np.complex128)
                b[c.src_edges[j]] = -1j * 2 * np.pi * freqs[0] * 4e-7 * np.pi * c.src_signs[j]
                rhs[j] = b
            b_d = torch.from_numpy(rhs).to(dev)
            x_d = torch.empty_like(b_d)
            po = mw.solve_opts(mode=mw.MW_MODE_FP64, restart=50, batch=1, tol=1e-8, max_it=2000)
            st = c.solve_rhs(a.plain_cols, b_d, x_d, po)
            plain = {"value": a.plain_cols / (st["solve_ms"] * 1e-3), "unit": UNIT, "cols": a.plain_cols,
                     "solve_ms": st["solve_ms"], "arnoldi_steps": st["arnoldi_steps"],
                     "max_relres": st["max_relres"], "preconditioner_setup_s": ps,
                     "note": ("FP64 operator, FP64 Krylov basis, FP64-factorised subdomain inverses applied in "
                              f"FP64 (their factorisation, {ps:.0f} s, is setup), one column per launch"
                              if a.plain_factor == "fp64" else
                              "FP64 operator, FP64 Krylov basis, FP64 apply of FP32-factorised subdomain inverses, "
                              "one column per launch")}
        except Exception as e:  # report, do not hide
            plain = {"error": str(e)}
    # ---- FP64 batched (the same, several columns in one Krylov launch) ----------------------
    fp64_batched = None
    if ports is not None:
        fp64_batched = {"skipped": "dipole-source leg; not run for the waveguide workload"}
    elif a.plain_cols > 0 and a.fp64_batch_cols > 0 and rank == 0 and plain is not None and "error" not in plain:
        try:
            nb = min(a.fp64_batch_cols, a.n_src)
            rhs = np.zeros((nb, info.n_edge), dtype=np.complex128)
            for j in range(nb):
                rhs[j, c.src_edges[j]] = -1j * 2 * np.pi * freqs[0] * 4e-7 * np.pi * c.src_signs[j]
            b_d = torch.from_numpy(rhs).to(dev)
            x_d = torch.empty_like(b_d)
            po = mw.solve_opts(mode=mw.MW_MODE_FP64, restart=50, batch=0, tol=1e-8, max_it=2000)
            st = c.solve_rhs(nb, b_d, x_d, po)
            fp64_batched = {"value": nb / (st["solve_ms"] * 1e-3), "unit": UNIT, "cols": nb,
                            "solve_ms": st["solve_ms"], "arnoldi_steps": st["arnoldi_steps"],
                            "max_relres": st["max_relres"],
                            "note": "as plain_fp64, with the columns in one Krylov launch (batching gain alone)"}
        except Exception as e:
            fp64_batched = {"error": str(e)}
    c.close()

    # ---- roofline of the dominant kernel class, and of every class --------------------------
    roof, dom = _dominant_roofline(prof, ms, hbm, src, prec, a, L)
    roof["classes"] = rate_classes(prof, hbm, alu)
    roof["setup_classes"] = rate_classes(L["setup_prof"], hbm, alu)
    roof["alu_peaks"] = alu
    if prec == mw.MW_PREC_SPARSE and dom == "oras_apply":
        # the sparse sweeps multiply every stored factor entry by all R columns: 8 flop per complex
        # entry and column, FP32 CUDA cores (the factor count follows from the algorithmic bytes)
        d = prof[dom]
        per = d["bytes"] / max(d["launches"], 1)
        fac_entries = (per - 8.0 * a.n_src * (float(L["sizes"].sum()) + info.n_edge)) / 8.0
        flops = 8.0 * fac_entries * a.n_src * d["launches"]
        tf = flops / (d["ms"] * 1e-3) / 1e12
        roof.update({"bound": "fp32", "achieved": tf, "peak": alu["fp32_tflops"], "unit": "TFLOP/s",
                     "frac": tf / alu["fp32_tflops"], "traffic": None, "traffic_note": None,
                     "peak_source": "measured here: " + alu["how"], "factor_entries": fac_entries})

    # ---- extra legs (rank 0 only, each on its own context) -----------------------------------
    legs = {}
    if rank == 0 and world == 1 and not a.no_legs and ports is None and a.cells == "80x80x34" and a.prec == "bf16":
        for name, fn in (("shoulder55_64tx_3f", lambda: shoulder55_3f_leg(a, local, stream, alu, hbm, src)),
                         ("shoulder80_sparse16", lambda: sparse16_leg(a, local, stream, alu, hbm, src)),
                         ("nn_training", lambda: nn_leg(local, stream, alu, hbm))):
            try:
                legs[name] = fn()
            except Exception as e:  # report, do not hide
                legs[name] = {"error": str(e)}
        if a.inversion_leg != "none":
            try:
                legs["time_to_misfit"] = inversion_leg(a.inversion_leg)
            except Exception as e:
                legs["time_to_misfit"] = {"error": str(e)}

    # ---- CPU oracle on the host's cores -------------------------------------------------------
    cpu = None
    if rank == 0 and not a.no_cpu_baseline:
        its = max(1.0, prof["cgs_dots"]["launches"] / max(1, a.steps * 2 * len(freqs)))
        argv = ["--cells", a.cells, "--n-src", str(a.n_src), "--antennas", a.antennas, "--freqs", a.freqs,
                "--parts", a.parts, "--overlap", str(a.overlap)]
        rates, cores, det = oracle_throughput(argv, its, a.cpu_sample_subdomains, cores=a.cpu_cores or None)
        cpu = {"value": rates[0], "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": (f"oracle (numpy/scipy FP64), one process per host core ({cores}), each costing one column: "
                          f"one Arnoldi step on the full workload (FP64 matvec, ORAS sparse-LU solves on "
                          f"{a.cpu_sample_subdomains} random subdomains scaled to {n_sub}, MGS at depth "
                          f"{int(round(min(its, 50) / 2))}) x {its:.1f} Arnoldi steps per column (the GPU solve's "
                          f"count); timed pieces run concurrently after a barrier; value = sum of the processes' "
                          f"column rates"),
               "details": det}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64+bf16 inner / c128 outer" if prec == mw.MW_PREC_BF16 else "c64 inner / c128 outer",
            "data": "synthetic",
            "config": {"workload": f"shoulder phantom {a.cells} Kuhn cells ({info.n_edge} edges, {info.n_tet} tets), "
                                   + (f"{a.n_src} z-dipoles" if ports is None else
                                      f"{a.n_src} TE10 waveguide ports (guides per wall {waveguide_counts(a.n_src)}, "
                                      f"metal walls)")
                                   + f" x {len(freqs)} frequencies, one inversion evaluation (forward+adjoint)",
                       "antennas": a.antennas,
                       "edges": info.n_edge, "nnz": info.nnz, "transmitters": a.n_src, "freqs_hz": freqs,
                       "rhs_solves_per_step": units, "subdomains": n_sub, "overlap": a.overlap,
                       "n_s_mean": float(L["sizes"].mean()), "n_s_max": int(L["sizes"].max()),
                       "solver": "GMRES-IR: FP64 outer residual, FGMRES(50) inner FP32 + ORAS",
                       "cycles": "CUDA graph per restart cycle (conditional nodes)" if a.graphs else "eager",
                       "launch_shapes": {k: L["tune"][k] for k in ("tc_stages", "dots_stages", "update_stages",
                                                                   "spmm_threads")},
                       "preconditioner_apply": {2: "bf16 tcgen05", 1: "fp32 cuda-core",
                                                4: "fp32 multifrontal sweeps",
                                                5: "bf16 tcgen05 multifrontal sweeps"}.get(prec, str(prec)),
                       "tol": 1e-8, "inner_tol": a.inner_tol, "alpha": a.alpha,
                       "z_storage": a.z_storage if prec == mw.MW_PREC_BF16 else "fp32",
                       "l2": "inputs larger than L2 (subdomain inverses and Krylov basis are GBs)"},
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches), "clocks": clocks, "setup_s": L["setup"], "plain_fp64": plain,
            "fp64_batched": fp64_batched,
            "J_last": J,
            **legs,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def inversion_leg(scale):
    """Second metric at reduced scale: time for the plain FP64, mixed, and mixed + learned-start
    inversions to reach the plain FP64 inversion's final misfit."""
    from paper_2311_05322_gb300 import inversion
    r = inversion.run(scale, seed=3, plain=True)
    inv = r["inversion"]
    return {"metric": "inversion time-to-misfit", "unit": "s", "higher_is_better": False, "scale": scale,
            "config": r["config"], "time_to_target_s": {k: v["time_to_target_s"] for k, v in inv.items()},
            "target_J": r["target_J"], "target_rel_band": r["target_rel_band"], "target_from": r["target_from"],
            "J_first_last": {k: [v["J"][0], v["J"][-1]] for k, v in inv.items()},
            "seconds_total": {k: v["seconds"][-1] for k, v in inv.items()},
            "plain_fp64_setup_s": r.get("plain_fp64_setup_s"), "network": r["network"],
            "snr_db": r["cases"][0]["snr_db"], "learned_start_rel_dJ0": r["cases"][0]["learned_start_rel_dJ0"],
            "total_s": r["total_s"]}


# ---------------------------------------------------------------------------------------
# reference arm: the CPU oracle
# ---------------------------------------------------------------------------------------
def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    parts = _dims(a.parts)
    n_sub = int(np.prod(parts))
    # the oracle's own GMRES+ORAS would need minutes per column at this size; each step is the
    # same bounded per-column sample as the GPU arm's cpu_baseline, on every host core, costed at
    # one full GMRES(50) cycle (50 Arnoldi steps) per column, the restart length of the method
    its = 50.0
    argv = ["--cells", a.cells, "--n-src", str(a.n_src), "--antennas", a.antennas, "--freqs", a.freqs,
            "--parts", a.parts, "--overlap", str(a.overlap)]
    rates, cores, det = oracle_throughput(argv, its, a.cpu_sample_subdomains, cores=a.cpu_cores or None,
                                          n_samples=a.warmup + a.steps)
    v = statistics.mean(rates[a.warmup:])
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
                      "steps": a.steps, "warmup": a.warmup, "higher_is_better": True, "data": "synthetic",
                      "config": {"workload": f"shoulder phantom {a.cells}", "antennas": a.antennas,
                                 "subdomains": n_sub},
                      "cpu_baseline": {"kind": "oracle", "cores": cores, "value": v, "unit": UNIT,
                                       "sample": (f"oracle (numpy/scipy FP64), one process per host core ({cores}); "
                                                  "per step each process costs one column: one sampled Arnoldi "
                                                  "step on the full workload x 50 (one GMRES(50) cycle); value = "
                                                  "sum of the processes' column rates, mean over the timed steps"),
                                       "details": det},
                      "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
          flush=True)


def run_inversion(a):
    """Second metric: inversion time-to-misfit (plain FP64 vs mixed vs mixed + learned start)."""
    from paper_2311_05322_gb300 import inversion
    plain = True if a.plain else None
    r = inversion.run(a.inversion, seed=3, plain=plain, tears=a.tears,
                      alphas=[float(x) for x in a.alphas.split(",") if x])
    inv = r["inversion"]
    line = {"metric": "inversion time-to-misfit", "unit": "s", "higher_is_better": False, "n_gpus": 1,
            "value": inv["mixed_learned"]["time_to_target_s"], "data": "synthetic",
            "config": {"workload": f"differential inversion, scale {a.inversion}", **r["config"]},
            "time_to_target_s": {k: v["time_to_target_s"] for k, v in inv.items()},
            "target_J": r["target_J"], "target_from": r["target_from"], "network": r["network"],
            "J": {k: v["J"] for k, v in inv.items()}, "seconds": {k: v["seconds"] for k, v in inv.items()},
            "learned_start_dJ0": r["learned_start_dJ0"], "total_s": r["total_s"],
            "plain_fp64_setup_s": r.get("plain_fp64_setup_s"), "cases": r["cases"], "summary": r["summary"],
            "alpha_sweep": r["alpha_sweep"]}
    print(json.dumps(line), flush=True)


def run_study(a):
    """Third measurement: wall time of the antenna-count design study and its err / ctr rows."""
    from paper_2311_05322_gb300 import design_study
    r = design_study.run(a.study, seed=5)
    secs = [s for row in r["rows"] for s in row["seconds"].values()]
    line = {"metric": "antenna-count study wall time", "unit": "s", "higher_is_better": False, "n_gpus": 1,
            "value": r["total_s"], "data": "synthetic",
            "config": {"workload": f"antenna-count design study, scale {a.study}", **r["config"],
                       "inverse_tets": r["inverse_tets"], "injury_tets": r["injury_tets"]},
            "reconstructions": len(secs), "seconds_per_reconstruction": {"min": min(secs), "max": max(secs)},
            "rows": r["rows"]}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    args = _args()
    if args.study:
        run_study(args)
    elif args.inversion:
        run_inversion(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_mine(args)
