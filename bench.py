#!/usr/bin/env python
"""AIR-GMRES time-to-1e-8 (setup + solve) and V-cycle HBM bandwidth on GB300.

Workload: the statically condensed, block-scaled space-time HDG trace system
of 2D+time advection-diffusion on [0,1]^3 split into 48^3 cubes x 6
tetrahedra, p = 2 (7,934,976 unknowns), rotating velocity
a = (-(y-1/2), x-1/2), nu = 1e-6, manufactured u = sin(pi x) sin(pi y)
cos(2 pi t).  Synthetic and seeded; built on the host before timing.

One step = air_setup (strength, C/F splitting, l-AIR restriction, one-point
interpolation, Galerkin products on every level, coarsest inverse) plus
air_gmres_solve to ||b - A x|| / ||b|| <= 1e-8, with A and b resident in HBM.
It is timed for the FP32 hierarchy inside FP64 flexible GMRES (the reported
value) and for the plain FP64 hierarchy (reported alongside).  The V-cycle
and the SpMV are timed separately for the roofline.

The CPU oracle (oracle/air_oracle.c, one thread) runs the full workload on a
host thread while the GPU legs run, with setup and solve timed separately;
that is the line's cpu_baseline.  --impl reference times the oracle on a
bounded sample of the same workload family (n = 20, 571,200 unknowns) per
step: its setup scaled by the unknown count, its GMRES cost per iteration
scaled by the unknown count and by the oracle's iteration count on the full
workload (tests/golden/oracle_st2d_n48_p2_nu1e-6.json, written by the
committed script beside it).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "AIR-GMRES time-to-1e-8 (setup+solve s) and V-cycle HBM GB/s, FP32-precond vs FP64"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=48)
    ap.add_argument("--p", type=int, default=2)
    ap.add_argument("--nu", type=float, default=1e-6)
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--distance", type=int, default=1, help="l-AIR neighbourhood distance (1 or 2)")
    ap.add_argument("--no-gpu-assembly", action="store_true")
    ap.add_argument("--no-gs", action="store_true", help="skip the forward Gauss-Seidel variant")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched independent-problems leg")
    ap.add_argument("--no-nu2", action="store_true", help="skip the nu = 1e-2 half of the workload")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint workload leg")
    ap.add_argument("--autotune", type=int, default=1, help="time the lanes per row of every level at setup")
    ap.add_argument("--block-size", type=int, default=-1,
                    help="block form of the finest operator: facet block size b (-1: b of the workload, 0: off)")
    ap.add_argument("--falgout-block", type=int, default=8192,
                    help="block size of the Falgout-style splitting variant reported beside the headline (0: off)")
    ap.add_argument("--workers", type=int, default=min(16, os.cpu_count() or 1))
    ap.add_argument("--sample-n", type=int, default=20, help="oracle sample mesh size")
    ap.add_argument("--vcycles", type=int, default=100)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", default="single", choices=["single", "batched", "multirhs", "table2", "largest", "vcycle", "adjoint"],
                    help="batched: 16 independent uneven problems set up and solved at once")
    ap.add_argument("--large-n", type=int, default=56, help="largest workload: cubes per direction")
    ap.add_argument("--adj-n", type=int, default=40, help="adjoint workload: cubes per direction")
    ap.add_argument("--batch-count", type=int, default=16)
    ap.add_argument("--batch-nmin", type=int, default=16)
    ap.add_argument("--batch-nmax", type=int, default=48)
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def block_size(args):
    return (args.p + 1) * (args.p + 2) // 2 if args.block_size < 0 else args.block_size


def workload_config(args):
    n, p = args.n, args.p
    return {"workload": f"st2d_hdg_n{n}_p{p}_rotating_nu{args.nu:g}",
            "mesh": f"{n}^3 cubes x 6 tetrahedra", "p": p, "nu": args.nu, "rtol": args.rtol,
            "unknowns": (12 * n ** 3 - 2 * n * n) * (p + 1) * (p + 2) // 2,
            "theta": 0.25, "distance": args.distance, "relax": "FCF", "restart": 30,
            "finest_storage": f"facet blocks of {block_size(args)}" if block_size(args) else "entries",
            "l2_flush": "inputs larger than L2 (CSR of A is several GB)"}


def make_system(args):
    from sthdg import assemble
    from sthdg.problems import manufactured_2d
    prob = manufactured_2d(n=args.n, p=args.p, nu=args.nu)
    return assemble(prob, workers=args.workers)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.rows, self.proc, self.index = [], None, index

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
                for k, nm in enumerate(names):
                    if r[3 + k].lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------- algorithmic bytes
def vcycle_bytes(H, wbytes, diag_bytes=0):
    """Algorithmic DRAM bytes of one V-cycle (relaxation FCF): each array read
    once per use.

    Per non-coarsest level (n rows, nnz z = z_F + z_C, R with nnz_R entries,
    n_C coarse points, w = value bytes, x = vector element bytes):
      restriction     nnz_R (w+4) + 8 n_C + x n + x n_C
      interpolation   4 n (P's columns) + x n_C + x n
      sweep over a point set S of m_S rows (F, C, F), from one full vector
      into the other: the set's matrix, 4 B of row index for every row (the
      set's rows and the copied rows of the other set), b and 1/a_ii of the
      set, the old vector read and the new one written in full:
                      mat(z_S, m_S) + 4 n + 2 x m_S + 2 x n
    mat(z, m) = z (w+4) in the entry form; a level stored in the block form
    (facet blocks of b) reads (z - m) w + 4 (z - m) / b + x m instead (the
    standalone diagonal one per row, in the vector type).  coarsest: x n_L^2 +
    2 x n_L.  BF16 storage (w = 2) keeps FP32 vectors (x = 4) and adds the FP32
    diagonal (diag_bytes per relaxed row).
    The call takes and returns FP64 vectors: an FP32 or BF16 hierarchy converts
    b into its finest vector and the result back (8 + 4 and 4 + 8 bytes per
    finest row), an FP64 one copies them in and out of its finest buffers
    (16 + 16 bytes per row).
    """
    total = 24 * H.info(0).n if wbytes != 8 else 32 * H.info(0).n
    L = H.levels()
    for l in range(L):
        inf = H.info(l)
        n = inf.n
        x = 4 if wbytes == 2 else wbytes  # vector element bytes
        if inf.coarsest:
            total += x * n * n + 2 * x * n
            continue
        rp = H.export(l, "A.row_ptr")
        cf = H.export(l, "cf").astype(bool)
        rl = np.diff(rp)
        zc = int(rl[cf].sum())
        zf = int(rl[~cf].sum())
        nc = int(cf.sum())
        nf = n - nc
        w = wbytes                       # stored value bytes
        bsz = inf.block_size

        def mat(z, rows):
            if not bsz:
                return z * (w + 4)
            return (z - rows) * w + (z - rows) // bsz * 4 + rows * x

        def sweep(z, m):
            return mat(z, m) + 4 * n + 2 * x * m + 2 * x * n + diag_bytes * m
        total += inf.nnz_r * (w + 4) + 8 * nc + x * n + x * nc
        total += 4 * n + x * nc + x * n
        total += sweep(zf, nf) + sweep(zc, nc) + sweep(zf, nf)
    return total


def vcycle_traffic(alg_bytes):
    """DRAM traffic per V-cycle from the committed ncu capture (profiles/), scaled
    by algorithmic bytes; None when the solve kernels changed since then."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "vcycle_traffic_st2d_n24_p2.json")) as f:
            prof = json.load(f)
        with open(os.path.join(ROOT, "paper_2010_11130_gb300", "csrc", "solve_kernels.cu"), "rb") as f:
            h = hashlib.sha256(f.read()).hexdigest()
        if h != prof["solve_kernels_sha256"]:
            return None
        return float(prof["traffic_per_algorithmic_byte"]) * alg_bytes
    except Exception:
        return None


def median_time(fn, stream, reps, runs=5):
    """Median over `runs` of the CUDA-event time of `reps` calls of fn, per call (s)."""
    import torch
    ts = []
    for _ in range(runs):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / reps / 1e3)
    return float(np.median(ts))


def spmv_bytes(n, nnz):
    return nnz * 12 + (n + 1) * 8 + n * 8 + n * 8


def krylov_spmv_bytes(n, nnz, b):
    """Algorithmic bytes of y = A x with the FP64 copy of A the Krylov solves use:
    block form (facet blocks of b): the off-diagonal blocks' values, one 4 B
    column per block, the standalone diagonal, x read once, y written; entry
    form (b = 0): 12 B per entry plus x and y."""
    if not b:
        return nnz * 12 + 16 * n
    return (nnz - n) * 8 + (nnz - n) // b * 4 + 8 * n + 16 * n


# ------------------------------------------------------------ GPU assembly
def gpu_assembly_leg(args, s, stream):
    """The same trace system assembled, condensed and block-scaled on the GPU
    (air_hdg_assemble), timed with CUDA events (median of 3 after a warm-up),
    and compared with the host-assembled system: pattern identical, values
    per row relative to the row's largest entry."""
    import torch
    from paper_2010_11130_gb300 import hdg
    from sthdg.mesh import build_mesh
    from sthdg.problems import manufactured_2d
    prob = manufactured_2d(n=args.n, p=args.p, nu=args.nu)
    mesh = build_mesh(prob.D, prob.n, reflect=prob.reflect, lower=prob.lower, upper=prob.upper,
                      vertex_map=prob.vertex_map)
    tab = hdg.HdgTables(prob.D, prob.p)
    hm = hdg.HdgMesh.from_mesh(mesh)
    xv, xf, xF = hdg.points(hm, tab)
    xv, xf, xF = xv.cpu().numpy(), xf.cpu().numpy(), xF.cpu().numpy()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    data = hdg.HdgData(prob.nu, 10.0 * prob.p ** 2, dev(prob.velocity(xv)), dev(prob.velocity(xf)),
                       dev(prob.source(xv)), dev(prob.u_initial(xf)), dev(prob.g_dirichlet(xF)))
    del xv, xf, xF
    sysg = hdg.assemble(hm, tab, data)
    del sysg
    ts = []
    for _ in range(3):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sysg = hdg.assemble(hm, tab, data)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
        if len(ts) < 3:
            del sysg
    same = bool(np.array_equal(sysg.A.col.cpu().numpy(), s.col)) and bool(
        np.array_equal(sysg.A.row_ptr.cpu().numpy(), s.row_ptr))
    val = sysg.A.val.cpu().numpy()
    rows = np.repeat(np.arange(s.n), np.diff(s.row_ptr))
    scale = np.zeros(s.n)
    np.maximum.at(scale, rows, np.abs(s.val))
    err = np.zeros(s.n)
    np.maximum.at(err, rows, np.abs(val - s.val))
    rhs_err = float(np.max(np.abs(sysg.rhs.cpu().numpy() - s.rhs)) / np.max(np.abs(s.rhs)))
    return {"s": float(np.median(ts)), "elements": int(mesh.n_elems), "facets": int(mesh.n_facets),
            "kernels": "hdg_element_kernel<3,p> (one warp per element) + facet_kernel (one warp per facet)",
            "pattern_identical": same, "max_row_rel_diff": float(np.max(err / np.maximum(scale, 1e-300))),
            "rhs_rel_diff": rhs_err, "timing": "median of 3 after a warm-up, CUDA events, data resident"}


# ------------------------------------------------------------------ oracle
_SAMPLE = {}


def host_cpu():
    """Model name and core count of the host (lscpu / os.cpu_count)."""
    model = "unknown"
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"model": model, "cores": os.cpu_count()}


def full_oracle_iters(args):
    """The oracle's GMRES iteration count on the full workload, from the record
    written by tests/golden/oracle_full_config.py (None if there is none)."""
    if args.distance != 1:
        return None
    path = os.path.join(ROOT, "tests", "golden", f"oracle_st2d_n{args.n}_p{args.p}_nu{args.nu:g}.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        if rec["unknowns"] == workload_config(args)["unknowns"] and rec["rtol"] == args.rtol:
            return int(rec["iters"])
    except Exception:
        pass
    return None


def oracle_sample(args):
    """CPU oracle (one thread) on a bounded sample of the workload family: the
    same p, nu, velocity and source on an n_s^3 mesh, setup and GMRES to rtol
    timed separately.  The estimate for the full workload scales the setup by
    the unknown count (O(N)) and the GMRES time per iteration by the unknown
    count and by the full workload's iteration count (the oracle's own, from
    its committed record; the sample's count when there is none)."""
    import oracle
    from sthdg import assemble
    from sthdg.problems import manufactured_2d
    oracle.build()
    key = (args.sample_n, args.p, args.nu)
    if key not in _SAMPLE:
        _SAMPLE[key] = assemble(manufactured_2d(n=args.sample_n, p=args.p, nu=args.nu), workers=1)
    s = _SAMPLE[key]
    full_n = workload_config(args)["unknowns"]
    t0 = time.perf_counter()
    H = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, distance=args.distance, max_coarse=1000,
                     copy_levels=False)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, its, rr, ok, _ = oracle.gmres(s.row_ptr, s.col, s.val, H, s.rhs, rtol=args.rtol)
    t_solve = time.perf_counter() - t0
    del H
    scale = full_n / s.n
    its_full = full_oracle_iters(args)
    its_used = its_full if its_full is not None else its
    est_setup = t_setup * scale
    est_solve = t_solve / max(its, 1) * scale * its_used
    return {"value": est_setup + est_solve, "unit": "s", "cores": 1, "kind": "oracle",
            "sample": (f"st2d n={args.sample_n} p={args.p} nu={args.nu:g} ({s.n} unknowns): oracle setup "
                       f"{t_setup:.2f} s, GMRES {t_solve:.2f} s for {its} iterations; full-workload estimate = "
                       f"setup x{scale:.2f} (unknowns) + GMRES per iteration x{scale:.2f} x {its_used} iterations "
                       f"({'the oracle on the full workload, committed record' if its_full else 'the sample'})"),
            "setup_s": est_setup, "solve_s": est_solve, "sample_seconds": t_setup + t_solve,
            "sample_iters": its, "full_iters_used": its_used}


class FullOracle(threading.Thread):
    """The oracle on the full workload, on one host thread (the C calls release
    the GIL), started before the GPU legs and joined after them."""

    def __init__(self, s, args):
        super().__init__(daemon=True)
        self.s, self.args, self.result, self.error, self.x = s, args, None, None, None

    def run(self):
        try:
            import oracle
            oracle.build()
            s = self.s
            t0 = time.perf_counter()
            H = oracle.setup(s.row_ptr, s.col, s.val, theta=0.25, distance=self.args.distance, max_coarse=1000,
                             copy_levels=False)
            t_setup = time.perf_counter() - t0
            t0 = time.perf_counter()
            x, its, rr, ok, _ = oracle.gmres(s.row_ptr, s.col, s.val, H, s.rhs, rtol=self.args.rtol)
            t_solve = time.perf_counter() - t0
            self.x = x
            self.result = {"setup_s": t_setup, "solve_s": t_solve, "iters": its, "relres": rr, "converged": ok,
                           "levels": len(H.sizes())}
        except Exception as e:   # reported in the line, never fatal to the GPU legs
            self.error = repr(e)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample(args)
    t0 = time.perf_counter()
    vals = [oracle_sample(args) for _ in range(args.steps)]
    wall = time.perf_counter() - t0
    v = float(np.median([r["value"] for r in vals]))
    cpu = dict(vals[len(vals) // 2])
    cpu["value"] = v
    cpu["host"] = host_cpu()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * wall / max(1, args.steps),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args), "cpu_baseline": cpu,
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------------- ours
def max_over_ranks(x, dist, device="cuda"):
    """The largest of x over all ranks (x itself without a process group): each
    rank times its own replica, and the job takes as long as the slowest."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_ours(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    # the host-side input build (and its process pool) comes before any CUDA call
    t0 = time.perf_counter()
    s = make_system(args)
    gen_s = time.perf_counter() - t0
    full = None
    if rank == 0 and world == 1 and not args.no_cpu:
        full = FullOracle(s, args)
        full.start()

    import torch
    import paper_2010_11130_gb300 as air
    air.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    A = air.CSR.from_host(s.row_ptr, s.col, s.val, device=f"cuda:{local}")
    b = torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda()
    stream = torch.cuda.current_stream()

    def step(prec):
        H = air.setup(A, theta=0.25, distance=args.distance, precision=prec, block_size=block_size(args),
                      autotune=args.autotune)
        x, info = air.gmres_solve(A, H, b, rtol=args.rtol)
        H.free()
        return info

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    cold = {}

    def timed(prec, warmup, steps):
        for w in range(warmup):
            if w == 0:
                # the first step of a form, cold: graph capture, first loads, pool growth
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                step(prec)
                torch.cuda.synchronize()
                cold[prec] = time.perf_counter() - t0
            else:
                step(prec)
        barrier()
        k0 = air.kernel_launches()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = [step(prec) for _ in range(steps)]
        e1.record(stream)
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1), dist)
        return ms / steps, infos, air.kernel_launches() - k0

    # the reported value: FP32 hierarchy inside FP64 FGMRES, W warm-up + K timed
    # steps; the FP64 and BF16-off-diagonal forms the same
    clocks = ClockSampler(local)
    clocks.start()
    ms32, inf32, launches32 = timed(1, args.warmup, args.steps)
    clk = clocks.stop()
    w_o, k_o = args.warmup, args.steps
    ms64, inf64, _ = timed(0, w_o, k_o)
    ms16, inf16, _ = timed(2, w_o, k_o)

    # V-cycle and SpMV roofline (FP32 hierarchy is the reported form)
    gbs_peak, peak_kind = peaks()
    rl = {}
    kry = {"s": None, "block_size": 0}
    lair_roof = None
    breakdown = {}
    sols = {}
    for prec, key in ((1, "f32"), (0, "f64"), (2, "bf16")):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        H = air.setup(A, theta=0.25, distance=args.distance, precision=prec, block_size=block_size(args),
                      autotune=args.autotune)
        t_setup = time.perf_counter() - t0
        xs = torch.empty_like(b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, inf_s = air.gmres_solve(A, H, b, xs, rtol=args.rtol)
        torch.cuda.synchronize()
        t_solve = time.perf_counter() - t0
        sols[key] = xs.cpu().numpy()
        if key == "f64":
            # the paper's Krylov method on the same hierarchy: BiCGSTAB to the metric's
            # tolerance and to the paper's 1e-12
            bic = {}
            for tol in (args.rtol, 1e-12):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, inf_b = air.bicgstab_solve(A, H, b, torch.empty_like(b), rtol=tol)
                torch.cuda.synchronize()
                bic[f"{tol:g}"] = {"s": time.perf_counter() - t0, "iters": inf_b.iters,
                                   "relres": inf_b.relres, "status": inf_b.status}
        breakdown[key] = {"setup_s": t_setup, "solve_s": t_solve, "iters": inf_s.iters,
                          "setup_phase_ms": H.setup_timings(), "levels": H.levels()}
        vb = vcycle_bytes(H, {1: 4, 0: 8, 2: 2}[prec], diag_bytes=4 if prec == 2 else 0)
        xv = torch.empty_like(b)
        for _ in range(3):
            H.vcycle(b, xv)
        t = median_time(lambda: H.vcycle(b, xv), stream, args.vcycles)
        if key == "f32":
            # the local l-AIR solves: LU of an m x m system, (2/3) m^3 + 2 m^2 flops each
            # (factorisation plus forward and back substitution), m = |N_i| from R's rows
            lf = 0.0
            for l in range(H.levels() - 1):
                m = np.diff(H.export(l, "R.row_ptr")).astype(np.float64) - 1.0
                lf += float(np.sum(2.0 / 3.0 * m ** 3 + 2.0 * m ** 2))
            lair_roof = {"flops": lf, "time_s": H.setup_timings()["lair"] / 1e3}
            # the Krylov solves' matrix product: the hierarchy's FP64 copy of A
            yk = torch.empty_like(b)
            for _ in range(3):
                H.spmv(b, yk)
            kry["s"] = median_time(lambda: H.spmv(b, yk), stream, args.vcycles)
            kry["block_size"] = H.info(0).block_size
        rl[key] = {"bytes": vb, "s": t, "gbs": vb / t / 1e9, "levels": H.levels(),
                   "lanes_per_row": [[H.info(l).lanes_f, H.info(l).lanes_c, H.info(l).lanes_r]
                                     for l in range(H.levels() - 1)],
                   "timing": f"median of 5 runs of {args.vcycles} V-cycles (CUDA-graph replays)"}
        H.free()
    y = torch.empty_like(b)
    for _ in range(3):
        air.spmv(A, b, y)
    t_spmv = median_time(lambda: air.spmv(A, b, y), stream, args.vcycles)
    sb = spmv_bytes(s.n, s.nnz)
    kb = krylov_spmv_bytes(s.n, s.nnz, kry["block_size"])

    # the paper's coarsening as a variant: Falgout-style splitting (blocks of consecutive points)
    falgout = None
    if args.falgout_block > 0:
        def fstep():
            H = air.setup(A, theta=0.25, distance=args.distance, precision=1, falgout_block=args.falgout_block,
                          block_size=block_size(args), autotune=args.autotune)
            x, info = air.gmres_solve(A, H, b, rtol=args.rtol)
            ph = H.setup_timings()
            lv = H.levels()
            H.free()
            return info, ph, lv
        fstep()
        torch.cuda.synchronize()
        fts = []
        for _ in range(max(1, min(args.steps, 3))):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            finfo, fph, flv = fstep()
            e1.record(stream)
            torch.cuda.synchronize()
            fts.append(e0.elapsed_time(e1) / 1e3)
        falgout = {"s": float(np.median(fts)), "iters": finfo.iters, "relres": finfo.relres, "levels": flv,
                   "block": args.falgout_block, "splitting_s": fph["splitting"] / 1e3, "setup_phase_ms": fph,
                   "form": "FP32 hierarchy, FP64 FGMRES; Falgout-style C/F splitting (first pass per block of "
                           "consecutive points, one warp each, then interface rounds)"}

    # the diffusion-significant half of the workload: nu = 1e-2 (GPU-assembled), distance-2 l-AIR,
    # FP32 hierarchy (one warm-up, one timed step) and FP64 hierarchy (one timed step)
    nu2 = None
    if not args.no_nu2 and args.nu != 1e-2:
        from sthdg.problems import manufactured_2d
        A2, b2 = gpu_system(manufactured_2d(n=args.n, p=args.p, nu=1e-2))

        def nstep(prec):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            H = air.setup(A2, theta=0.25, distance=2, precision=prec, block_size=block_size(args),
                          autotune=args.autotune)
            torch.cuda.synchronize()
            tsetup = time.perf_counter() - t0
            t0 = time.perf_counter()
            x, info = air.gmres_solve(A2, H, b2, rtol=args.rtol)
            torch.cuda.synchronize()
            tsolve = time.perf_counter() - t0
            lv = H.levels()
            H.free()
            return {"s": tsetup + tsolve, "setup_s": tsetup, "solve_s": tsolve, "iters": info.iters,
                    "relres": info.relres, "levels": lv}
        nstep(1)
        nu2 = {"f32_precond_fgmres": nstep(1), "f64": nstep(0),
               "form": "nu = 1e-2, distance-2 l-AIR, FGMRES(30) to the metric's tolerance; wall-clock, data "
                       "resident; FP32 after one warm-up step"}

    # the paper's relaxation: forward Gauss-Seidel on F then all points (level-scheduled), one step
    gs = None
    if not args.no_gs:
        def gstep():
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            H = air.setup(A, theta=0.25, distance=args.distance, precision=1, relax="fa",
                          block_size=block_size(args), autotune=args.autotune)
            torch.cuda.synchronize()
            tsetup = time.perf_counter() - t0
            t0 = time.perf_counter()
            x, info = air.gmres_solve(A, H, b, rtol=args.rtol)
            torch.cuda.synchronize()
            tsolve = time.perf_counter() - t0
            vb = torch.empty_like(b)
            tv = median_time(lambda: H.vcycle(b, vb), stream, 10, runs=3)
            H.free()
            return info, tsetup, tsolve, tv
        gstep()
        ginfo, gsetup, gsolve, gvc = gstep()
        gs = {"s": gsetup + gsolve, "setup_s": gsetup, "solve_s": gsolve, "iters": ginfo.iters,
              "relres": ginfo.relres, "vcycle_s": gvc,
              "form": "FP32 hierarchy, FP64 FGMRES, relaxation 'fa' (forward Gauss-Seidel on F then all points, "
                      "level-scheduled); wall-clock after one warm-up step"}

    gpu_asm = None
    if not args.no_gpu_assembly:
        gpu_asm = gpu_assembly_leg(args, s, stream)
        gpu_asm["host_s"] = gen_s
    adjoint = None
    if not args.no_adjoint:
        adjoint = adjoint_leg(args)
    batched = None
    if not args.no_batched:
        batched = batched_leg(args)
        batched["workload"] = f"batched_{args.batch_count}_st2d_n{args.batch_nmin}-{args.batch_nmax}"
        torch.cuda.empty_cache()

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        rp_h = torch.from_numpy(s.row_ptr).pin_memory().numpy()
        ci_h = torch.from_numpy(s.col).pin_memory().numpy()
        v_h = torch.from_numpy(s.val).pin_memory().numpy()
        b_h = torch.from_numpy(np.ascontiguousarray(s.rhs)).pin_memory().numpy()
        x_h = torch.empty(s.n, dtype=torch.float64).pin_memory().numpy()
        Ah = air.CSR(rp_h, ci_h, v_h, s.n)
        torch.cuda.synchronize()
        tt = []
        for _ in range(1):
            t0 = time.perf_counter()
            Hh = air.setup(Ah, theta=0.25, distance=args.distance, precision=1, block_size=block_size(args),
                           autotune=args.autotune)
            _, ih = air.gmres_solve(Ah, Hh, b_h, x_h, rtol=args.rtol)
            Hh.free()
            tt.append(time.perf_counter() - t0)
        h2d = s.row_ptr.nbytes + s.col.nbytes + s.val.nbytes + b_h.nbytes
        e2e = {"value": float(np.mean(tt)), "unit": "s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(x_h.nbytes), "iters": ih.iters, "relres": ih.relres}

    cpu = None
    if full is not None:
        full.join()
        if full.result is not None:
            r = full.result
            hc = host_cpu()
            cpu = {"value": r["setup_s"] + r["solve_s"], "unit": "s", "cores": 1, "kind": "oracle",
                   "sample": (f"the full workload, not sampled: oracle setup {r['setup_s']:.1f} s + GMRES "
                              f"{r['solve_s']:.1f} s ({r['iters']} iterations, relres {r['relres']:.2e}), one "
                              f"host thread of {hc['cores']} ({hc['model']}), run while the GPU legs ran"),
                   "setup_s": r["setup_s"], "solve_s": r["solve_s"], "iters": r["iters"],
                   "relres": r["relres"], "host": hc}
        else:
            cpu = oracle_sample(args)
            cpu["full_run_error"] = full.error
    parity_full = None
    if cpu is not None and "iters" in cpu:
        parity_full = {"oracle_iters": cpu["iters"], "gpu_f64_iters": inf64[-1].iters,
                       "gpu_f64_within_one": abs(inf64[-1].iters - cpu["iters"]) <= 1,
                       "gpu_f32_precond_iters": inf32[-1].iters}
        if full is not None and full.x is not None:
            # final error of every form against the oracle's FP64 solution (all to the same rtol)
            xo = full.x
            no = float(np.linalg.norm(xo))
            parity_full["final_rel_error_vs_oracle"] = {k: float(np.linalg.norm(v - xo)) / no for k, v in sols.items()}
    if rank != 0:
        return
    v32 = rl["f32"]
    line = {
        "metric": METRIC, "value": ms32 / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms32, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 hierarchy / f64 Krylov", "data": "synthetic",
        "config": workload_config(args),
        "variants": {
            "f32_precond_fgmres": {"s": ms32 / 1e3, "iters": inf32[-1].iters, "relres": inf32[-1].relres,
                                   "vcycle_gbs": v32["gbs"]},
            "f64": {"s": ms64 / 1e3, "iters": inf64[-1].iters, "relres": inf64[-1].relres,
                    "vcycle_gbs": rl["f64"]["gbs"], "warmup": w_o, "steps": k_o},
            "bf16_offdiag_precond_fgmres": {"s": ms16 / 1e3, "iters": inf16[-1].iters, "relres": inf16[-1].relres,
                                            "vcycle_gbs": rl["bf16"]["gbs"], "warmup": w_o, "steps": k_o},
            "solve_stage_s": {k: breakdown[k]["solve_s"] for k in breakdown},
            "cold_first_step_s": {{1: "f32", 0: "f64", 2: "bf16"}[p]: t for p, t in cold.items()},
            "falgout_split_f32_precond": falgout,
            "gauss_seidel_fa_f32_precond": gs,
            "batched_independent_problems": batched,
            "nu_1e-2_distance2": nu2,
            "adjoint_mapped_noisy": adjoint},
        "roofline": {"bound": "hbm", "kernel": "V-cycle (FP32 hierarchy, all levels)",
                     "achieved": v32["gbs"], "peak": gbs_peak, "unit": "GB/s",
                     "frac": v32["gbs"] / gbs_peak, "traffic": vcycle_traffic(v32["bytes"]),
                     "algorithmic_bytes": v32["bytes"], "launch_s": v32["s"], "peak_kind": peak_kind},
        "roofline_spmv": {"bound": "hbm",
                          "kernel": (f"bsell_kernel<{kry['block_size']},...,double,double,0> (air_hierarchy_spmv: "
                                     "the FGMRES matrix product, FP64 block layout)") if kry["block_size"] else
                                    "sell_kernel<8,double,double,0> (air_hierarchy_spmv: the FGMRES matrix product)",
                          "achieved": kb / kry["s"] / 1e9, "peak": gbs_peak, "unit": "GB/s",
                          "frac": kb / kry["s"] / 1e9 / gbs_peak, "algorithmic_bytes": kb, "launch_s": kry["s"],
                          "csr_air_spmv": {"kernel": "row_kernel<4,U,double,double,0> (air_spmv: CSR, 4 lanes per row)",
                                           "achieved": sb / t_spmv / 1e9, "frac": sb / t_spmv / 1e9 / gbs_peak,
                                           "algorithmic_bytes": sb, "launch_s": t_spmv}},
        "roofline_lair": None if lair_roof is None else {
            "bound": "fp64 alu (nominal)", "kernel": "lair_solve_kernel (one warp per C point, FP64 LU)",
            "achieved": lair_roof["flops"] / lair_roof["time_s"] / 1e12, "unit": "TFLOP/s", "peak": 1.25,
            "peak_kind": "nominal FP64 rate (no measured FP64 peak)",
            "frac": lair_roof["flops"] / lair_roof["time_s"] / 1e12 / 1.25, "flops": lair_roof["flops"],
            "time_s": lair_roof["time_s"],
            "note": "the l-AIR phase time includes the neighbourhood gathers; 0.4% of the step"},
        "breakdown": breakdown,
        "bicgstab_f64_hierarchy": bic,
        "dominant_kernel": {
            "kernel": "rs5_warp_kernel (sequential first-pass C/F splitting, one warp per level)",
            "bound": "latency (one dependent chain of picks; no HBM or ALU roofline applies)",
            "time_s": breakdown["f32"]["setup_phase_ms"]["splitting"] / 1e3,
            "share_of_step": breakdown["f32"]["setup_phase_ms"]["splitting"] / 1e3 / (ms32 / 1e3)},
        "cpu_baseline": cpu, "parity_full_size": parity_full, "gpu_assembly": gpu_asm, "e2e": e2e, "clocks": clk,
        "gpu_launches": int(launches32),
        "generate_s": gen_s,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def gpu_system(prob):
    """The trace system of a problem assembled, condensed and block-scaled on
    the GPU (air_hdg_assemble): (device CSR, device right-hand side)."""
    import torch
    from paper_2010_11130_gb300 import hdg
    from sthdg.mesh import build_mesh
    mesh = build_mesh(prob.D, prob.n, reflect=prob.reflect, lower=prob.lower, upper=prob.upper,
                      vertex_map=prob.vertex_map)
    tab = hdg.HdgTables(prob.D, prob.p)
    hm = hdg.HdgMesh.from_mesh(mesh)
    xv, xf, xF = hdg.points(hm, tab)
    xv, xf, xF = xv.cpu().numpy(), xf.cpu().numpy(), xF.cpu().numpy()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    data = hdg.HdgData(prob.nu, 10.0 * prob.p ** 2, dev(prob.velocity(xv)), dev(prob.velocity(xf)),
                       dev(prob.source(xv)), dev(prob.u_initial(xf)), dev(prob.g_dirichlet(xF)))
    sysg = hdg.assemble(hm, tab, data)
    return sysg.A, sysg.rhs


def batched_leg(args):
    """Independent uneven problems (seeded recipe of sthdg.problems.batched_problems,
    assembled on the GPU): FP32 hierarchies built with air_setup_batch (level by
    level, each level's local l-AIR solves of all problems in one launch) and
    solved with air_gmres_solve_batch (lockstep rounds, the V-cycles of a round in
    one CUDA graph), against the same calls made one problem at a time.  Parity
    per problem: the batched solution equals the single-problem solution bit for
    bit, with the same iteration count."""
    import torch
    import paper_2010_11130_gb300 as air
    from sthdg.problems import batched_problems
    t0 = time.perf_counter()
    probs, _ = batched_problems(args.batch_count, (args.batch_nmin, args.batch_nmax))
    systems = [gpu_system(p) for p in probs]
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    As = [A for A, _ in systems]
    bs = [b for _, b in systems]
    air.setup(As[int(np.argmin([A.n for A in As]))], precision=1)   # warm-up: module load, memory pools
    torch.cuda.synchronize()

    def clock(fn):
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, time.perf_counter() - t

    l0 = air.kernel_launches()
    (Hs, st), ts_b = clock(lambda: air.setup_batch(As, precision=1))
    assert all(x == 0 for x in st), st
    l1 = air.kernel_launches()
    (xs, infos, st2), tv_b = clock(lambda: air.gmres_solve_batch(As, Hs, bs, rtol=args.rtol))
    assert all(x == 0 for x in st2), st2
    l2 = air.kernel_launches()
    del Hs
    ts_1 = tv_1 = 0.0
    parity = []
    per = []
    launches_1 = [0, 0]
    for A, b, x, inf in zip(As, bs, xs, infos):
        a0 = air.kernel_launches()
        H, t_s = clock(lambda: air.setup(A, precision=1))
        a1 = air.kernel_launches()
        (x1, inf1), t_v = clock(lambda: air.gmres_solve(A, H, b, rtol=args.rtol))
        a2 = air.kernel_launches()
        launches_1[0] += a1 - a0
        launches_1[1] += a2 - a1
        ts_1 += t_s
        tv_1 += t_v
        per.append([round(t_s, 4), round(t_v, 4)])
        parity.append(bool(torch.equal(x, x1)) and inf.iters == inf1.iters)
        del H
    return {"s": ts_b + tv_b, "setup_s": ts_b, "solve_s": tv_b,
            "one_at_a_time_s": ts_1 + tv_1, "one_at_a_time_setup_s": ts_1, "one_at_a_time_solve_s": tv_1,
            "speedup": (ts_1 + tv_1) / (ts_b + tv_b),
            "iters": [int(i.iters) for i in infos], "parity_per_problem_bit_exact": parity,
            "one_at_a_time_per_problem_setup_solve_s": per,
            "launches": {"batched_setup": l1 - l0, "batched_solve": l2 - l1,
                         "one_at_a_time_setup": launches_1[0], "one_at_a_time_solve": launches_1[1]},
            "problems": [{"n": p.n, "p": p.p, "nu": p.nu, "unknowns": int(A.n)} for p, A in zip(probs, As)],
            "unknowns_total": int(sum(A.n for A in As)), "generate_s": gen_s,
            "timing": "wall clock around each call with device synchronisation, data resident"}


def run_batched(args):
    """The batched leg alone, as its own JSON line."""
    import paper_2010_11130_gb300 as air
    air.build()
    r = batched_leg(args)
    out = {"metric": "batched AIR-GMRES time-to-1e-8 over independent problems (setup+solve s)",
           "value": r["s"], "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 1,
           "higher_is_better": False, "dtype": "f32 hierarchy / f64 Krylov", "data": "synthetic",
           "config": {"workload": f"batched_{args.batch_count}_st2d_n{args.batch_nmin}-{args.batch_nmax}"},
           **r}
    print(json.dumps(out))


def run_multirhs(args):
    """32 right-hand sides of the 48^3 system through one FP64 hierarchy: the
    lockstep solve and V-cycle (air_*_multi) against the same work one
    right-hand side at a time."""
    import torch
    import paper_2010_11130_gb300 as air
    air.build()
    s = make_system(args)
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    # FP64 hierarchy for the lockstep solve: BiCGSTAB is not flexible, and with an
    # FP32 V-cycle some columns stagnate short of 1e-8; the FP32 multi V-cycle is
    # timed on its own below
    H = air.setup(A, theta=0.25, distance=1, precision=0)
    H32 = air.setup(A, theta=0.25, distance=1, precision=1)
    k = 32
    rng = np.random.default_rng(2010_11130)
    B = np.empty((s.n, k))
    B[:, 0] = s.rhs
    B[:, 1:] = rng.standard_normal((s.n, k - 1))
    Bd = torch.from_numpy(B).cuda()
    cols = [Bd[:, j].contiguous() for j in range(k)]
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    # V-cycle: k columns at once against k single V-cycles, FP64 and FP32
    def time_vc(Hx, Bm, reps=3):
        X = air.vcycle_multi(Hx, Bm)
        for c in cols[:2]:
            Hx.vcycle(c)
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record(stream)
        for _ in range(reps):
            air.vcycle_multi(Hx, Bm, X)
        e1.record(stream)
        torch.cuda.synchronize()
        t_m = e0.elapsed_time(e1) / reps / 1e3
        x1 = torch.empty_like(cols[0])
        e0.record(stream)
        for c in cols:
            Hx.vcycle(c, x1)
        e1.record(stream)
        torch.cuda.synchronize()
        return t_m, e0.elapsed_time(e1) / 1e3
    t_multi, t_single = time_vc(H, Bd)
    t_multi32, t_single32 = time_vc(H32, Bd.float())
    # lockstep BiCGSTAB to the metric's tolerance against one solve per column
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Xs, infos = air.bicgstab_solve_multi(A, H, Bd, rtol=args.rtol)
    torch.cuda.synchronize()
    t_solve_multi = time.perf_counter() - t0
    t0 = time.perf_counter()
    its = []
    for c in cols:
        its.append(air.bicgstab_solve(A, H, c, rtol=args.rtol)[1].iters)
    torch.cuda.synchronize()
    t_solve_single = time.perf_counter() - t0
    out = {"metric": "32 right-hand sides, AIR-BiCGSTAB to 1e-8 on one FP64 hierarchy (solve s)",
           "value": t_solve_multi, "unit": "s", "n_gpus": 1, "higher_is_better": False, "dtype": "f64",
           "data": "synthetic", "config": {**workload_config(args), "rhs": k,
                                          "rhs_recipe": "column 0 = the manufactured rhs, 31 N(0,1) columns "
                                                        "from default_rng(2010_11130)"},
           "one_at_a_time_s": t_solve_single, "speedup": t_solve_single / t_solve_multi,
           "iters_multi": [i.iters for i in infos], "iters_single": its,
           "vcycle_multi_s": t_multi, "vcycle_single_x32_s": t_single,
           "vcycle_speedup": t_single / t_multi,
           "vcycle_multi_f32_s": t_multi32, "vcycle_single_f32_x32_s": t_single32,
           "vcycle_f32_speedup": t_single32 / t_multi32}
    print(json.dumps(out))


def run_table2(args):
    """The paper's Table 2 study on structured meshes: AIR-preconditioned BiCGSTAB
    iterations to a relative residual of 1e-12 for the rotating Gaussian pulse on its
    time-dependent domain (Section 5.1), over mesh size, p and nu, with the paper's
    strength pair (coarsening 0.2, R 0.3) and the library's default FCF-Jacobi relaxation."""
    import torch
    import paper_2010_11130_gb300 as air
    from sthdg import assemble
    from sthdg.problems import rotating_pulse
    air.build()
    rows = []
    for p, ns in ((1, (8, 16, 32)), (2, (8, 16))):
        for n in ns:
            for nu in (1e-6, 1e-4, 1e-3, 1e-2, 1e-1):
                s = assemble(rotating_pulse(n, p, nu), workers=args.workers)
                A = air.CSR.from_host(s.row_ptr, s.col, s.val)
                b = torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                H = air.setup(A, theta=0.2, theta_r=0.3, distance=1, precision=0, max_iter=5000)
                _, inf = air.bicgstab_solve(A, H, b, rtol=1e-12)
                torch.cuda.synchronize()
                rows.append({"p": p, "n": n, "unknowns": s.n, "nu": nu, "iters": inf.iters,
                             "converged": inf.status == 0, "relres": inf.relres,
                             "setup_solve_s": time.perf_counter() - t0})
                del H, A, b
    print(json.dumps({"metric": "AIR-BiCGSTAB iterations to 1e-12 (Table 2 study)", "unit": "iterations",
                      "data": "synthetic", "rows": rows}))


def run_largest(args):
    """The largest workload: 2D+time on 56^3 cubes x 6 tetrahedra (1,053,696
    tets), p = 3 (21,011,200 unknowns), boundary-layer velocity
    a = (1, 0.5 tanh(20 (x - 1/2))), nu = 1e-5, Gaussian initial pulse, zero
    Dirichlet data.  The trace system is assembled on the GPU (air_hdg_assemble;
    the host assembly of this size takes tens of minutes); then the FP64, FP32
    and BF16-off-diagonal hierarchies each precondition FP64 flexible GMRES to
    1e-10, and one adjoint solve A^T lambda = u (the gradient of 1/2 ||u||^2
    with respect to the right-hand side) runs on the hierarchy of A^T."""
    import torch
    import paper_2010_11130_gb300 as air
    from paper_2010_11130_gb300 import hdg
    from sthdg.mesh import build_mesh
    from sthdg.problems import boundary_layer
    air.build()
    stream = torch.cuda.current_stream()
    prob = boundary_layer(n=args.large_n, p=3, nu=1e-5)
    t0 = time.perf_counter()
    mesh = build_mesh(prob.D, prob.n, reflect=prob.reflect)
    mesh_s = time.perf_counter() - t0
    tab = hdg.HdgTables(3, 3)
    hm = hdg.HdgMesh.from_mesh(mesh)
    t0 = time.perf_counter()
    xv, xf, xF = hdg.points(hm, tab)
    xv, xf, xF = xv.cpu().numpy(), xf.cpu().numpy(), xF.cpu().numpy()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    data = hdg.HdgData(prob.nu, 10.0 * 9, dev(prob.velocity(xv)), dev(prob.velocity(xf)), None,
                       dev(prob.u_initial(xf)), dev(prob.g_dirichlet(xF)))
    del xv, xf, xF
    data_s = time.perf_counter() - t0
    ev = lambda: torch.cuda.Event(enable_timing=True)
    asm_ms = []
    for _ in range(2):
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record(stream)
        sysg = hdg.assemble(hm, tab, data)
        e1.record(stream)
        torch.cuda.synchronize()
        asm_ms.append(e0.elapsed_time(e1))
    A, b, diag = sysg.A, sysg.rhs, sysg.diag
    del data
    torch.cuda.empty_cache()
    out = {"metric": "AIR-FGMRES time-to-1e-10 (setup+solve s), largest workload, per hierarchy precision",
           "unit": "s", "n_gpus": 1, "higher_is_better": False, "data": "synthetic",
           "config": {"workload": f"st2d_hdg_n{args.large_n}_p3_layer_nu1e-05", "mesh": f"{args.large_n}^3 cubes x 6 tetrahedra",
                      "elements": int(mesh.n_elems), "unknowns": int(A.n), "nnz": int(A.nnz), "rtol": 1e-10,
                      "theta": 0.25, "distance": 1, "relax": "FCF", "restart": 30},
           "assembly_gpu_s": [m / 1e3 for m in asm_ms], "mesh_host_s": mesh_s, "data_host_s": data_s}
    res, xs = {}, {}
    for prec, key in ((0, "f64"), (1, "f32"), (2, "bf16")):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        H = air.setup(A, theta=0.25, precision=prec)
        torch.cuda.synchronize()
        ts = time.perf_counter() - t0
        t0 = time.perf_counter()
        x, info = air.gmres_solve(A, H, b, rtol=1e-10)
        torch.cuda.synchronize()
        tv = time.perf_counter() - t0
        res[key] = {"setup_s": ts, "solve_s": tv, "s": ts + tv, "iters": info.iters, "relres": info.relres,
                    "status": info.status, "levels": H.levels(), "setup_phase_ms": H.setup_timings()}
        xs[key] = x
        H.free()
        torch.cuda.empty_cache()
    for key in ("f32", "bf16"):
        res[key]["rel_error_vs_f64"] = float(torch.linalg.norm(xs[key] - xs["f64"]) / torch.linalg.norm(xs["f64"]))
    del xs["f32"], xs["bf16"]
    # the adjoint through the block-scaled similar matrix D_b^{-T} A^T D_b^T (identity diagonal
    # blocks, like A): A^T lam = u  <=>  (D_b^{-T} A^T D_b^T) nu = D_b^{-T} u,  lam = D_b^T nu
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    At = air.transpose_scaled(A, 10, diag)
    Ht = air.setup(At, theta=0.25, precision=1)
    torch.cuda.synchronize()
    ts = time.perf_counter() - t0
    t0 = time.perf_counter()
    g = air.block_diag_apply(10, diag, 3, xs["f64"].contiguous())
    nu_, info = air.gmres_solve(At, Ht, g, rtol=1e-10)
    lam = air.block_diag_apply(10, diag, 1, nu_)
    torch.cuda.synchronize()
    res["adjoint_f32"] = {"form": "D_b^{-T} A^T D_b^T (block-scaled transpose)", "transpose_setup_s": ts,
                          "solve_s": time.perf_counter() - t0, "iters": info.iters, "relres": info.relres,
                          "status": info.status}
    out["results"] = res
    out["value"] = res["f32"]["s"]
    print(json.dumps(out), flush=True)


def run_adjoint(args):
    """The adjoint workload as its own JSON line (adjoint_leg)."""
    import paper_2010_11130_gb300 as air
    air.build()
    r = adjoint_leg(args)
    out = {"metric": "adjoint workload: forward + adjoint AIR-FGMRES to 1e-8 and both gradients (s)",
           "value": r["s"], "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 1, "higher_is_better": False,
           "dtype": "f32 hierarchy / f64 Krylov", "data": "synthetic", "config": r.pop("config"), **r}
    print(json.dumps(out), flush=True)


def adjoint_leg(args):
    """The adjoint workload: 2D+time on the mapped domain x' = x + 0.05 sin(2 pi t)
    sin(pi x) sin(pi y) (y likewise) on --adj-n^3 cubes x 6 tetrahedra, p = 2,
    nu = 1e-4, a piecewise-constant velocity (1, 0.5) + 0.1 N(0, 1) per element
    (sthdg.problems.mapped_noisy).  One step: GPU assembly, forward l-AIR FGMRES
    solve (FP32 hierarchy), adjoint solve A^T lambda = u - u_target on the
    block-scaled transpose with its own hierarchy, the gradient of
    L = 1/2 ||u - u_target||^2 with respect to the right-hand side (lambda) and
    to the element velocities (air_hdg_velocity_gradient).  u_target is the trace
    solution for the noise-free velocity (1, 0.5).  A directional central
    difference of L (h = 1e-6, along an N(0, 1) velocity direction, solves to
    1e-12) checks the velocity gradient at full size."""
    import torch
    import paper_2010_11130_gb300 as air
    from paper_2010_11130_gb300 import hdg
    from sthdg.mesh import build_mesh
    from sthdg.problems import mapped_noisy
    prob = mapped_noisy(args.adj_n, 2, 1e-4)
    t0 = time.perf_counter()
    mesh = build_mesh(prob.D, prob.n, reflect=prob.reflect, vertex_map=prob.vertex_map)
    tab = hdg.HdgTables(3, 2)
    hm = hdg.HdgMesh.from_mesh(mesh)
    xv, xf, xF = hdg.points(hm, tab)
    xv, xf, xF = xv.cpu().numpy(), xf.cpu().numpy(), xF.cpu().numpy()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    src, u0, gd = dev(prob.source(xv)), dev(prob.u_initial(xf)), dev(prob.g_dirichlet(xF))
    gen_s = time.perf_counter() - t0
    b = tab.b
    opts = dict(precision=1, block_size=b, autotune=args.autotune)

    def data(ev):
        evd = dev(ev)
        vv = evd[:, None, :].expand(xv.shape[0], xv.shape[1], 2).contiguous()
        vf = evd[:, None, None, :].expand(xf.shape[0], xf.shape[1], xf.shape[2], 2).contiguous()
        return hdg.HdgData(prob.nu, 10.0 * prob.p ** 2, vv, vf, src, u0, gd)

    def clock(fn):
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, time.perf_counter() - t

    ev0 = prob.elem_velocity.copy()
    ev_mean = np.broadcast_to(np.array([1.0, 0.5]), ev0.shape).copy()
    tsys = hdg.assemble(hm, tab, data(ev_mean))
    Ht = air.setup(tsys.A, **opts)
    target, _ = air.gmres_solve(tsys.A, Ht, tsys.rhs, rtol=1e-12)
    del Ht, tsys

    def loss(ev, rtol):
        sys_ = hdg.assemble(hm, tab, data(ev))
        H = air.setup(sys_.A, **opts)
        u, inf = air.gmres_solve(sys_.A, H, sys_.rhs, rtol=rtol)
        d = u - target
        return 0.5 * float((d * d).sum())

    def step(rtol):
        t = {}
        dat = data(ev0)
        sys_, t["assemble"] = clock(lambda: hdg.assemble(hm, tab, dat))
        S, t["forward_setup"] = clock(lambda: air.AdjointSolver(sys_.A, rtol=rtol, block=(b, sys_.diag), **opts))
        u, t["forward_solve"] = clock(lambda: S.solve(sys_.rhs))
        g = (u - target).contiguous()
        _, t["adjoint_transpose_setup"] = clock(lambda: S.adjoint_hierarchy())
        lam, t["adjoint_solve"] = clock(lambda: S.solve_adjoint(g))
        gv, t["velocity_gradient"] = clock(lambda: hdg.velocity_gradient(hm, tab, dat, sys_, u, lam))
        L = 0.5 * float((g * g).sum())
        return t, L, gv, lam, S.info, S.info_adjoint, sys_.A

    step(args.rtol)                                     # warm-up (module load, pools, graphs)
    t, L, gv, lam, inf_f, inf_a, A = step(args.rtol)
    # full-size check of the velocity gradient at tight tolerances
    _, Lc, gvc, _, _, _, _ = step(1e-12)
    rng = np.random.default_rng(40)
    dirn = rng.standard_normal(ev0.shape)
    h = 1e-6
    fd = (loss(ev0 + h * dirn, 1e-12) - loss(ev0 - h * dirn, 1e-12)) / (2 * h)
    ad = float((gvc.cpu().numpy() * dirn).sum())
    total = sum(t.values())
    return {"s": total,
            "config": {"workload": f"mapped_noisy_n{args.adj_n}_p2_nu1e-4", "unknowns": int(A.n),
                       "elements": int(mesh.n_elems), "rtol": args.rtol, "block_size": b},
            "stages_s": t, "forward_iters": int(inf_f.iters), "adjoint_iters": int(inf_a.iters),
            "loss": L, "grad_f_norm": float(lam.norm()),
            "velocity_gradient_check": {"h": h, "direction": "N(0,1) per element component, default_rng(40)",
                                        "central_difference": fd, "adjoint": ad,
                                        "rel_diff": abs(fd - ad) / max(abs(fd), 1e-300), "solve_rtol": 1e-12},
            "generate_s": gen_s,
            "timing": "wall clock around each stage with device synchronisation, after one warm-up step"}


def run_vcycle(args):
    """V-cycles alone on the workload family (the profiling target): FP32
    hierarchy (block form of the finest operator), 3 warm-up V-cycles, then
    --vcycles timed ones; prints the algorithmic bytes, the time and GB/s."""
    import torch
    import paper_2010_11130_gb300 as air
    air.build()
    s = make_system(args)
    A = air.CSR.from_host(s.row_ptr, s.col, s.val)
    b = torch.from_numpy(np.ascontiguousarray(s.rhs)).cuda()
    H = air.setup(A, theta=0.25, distance=args.distance, precision=1, block_size=block_size(args),
                  autotune=args.autotune)
    vb = vcycle_bytes(H, 4)
    x = torch.empty_like(b)
    for _ in range(3):
        H.vcycle(b, x)
    t = median_time(lambda: H.vcycle(b, x), torch.cuda.current_stream(), args.vcycles, runs=1)
    print(json.dumps({"workload": workload_config(args)["workload"], "vcycle_bytes": vb, "vcycle_s": t,
                      "gbs": vb / t / 1e9, "levels": H.levels(),
                      "level_sizes": [int(H.info(l).n) for l in range(H.levels())],
                      "lanes_per_row": [[H.info(l).lanes_f, H.info(l).lanes_c, H.info(l).lanes_r]
                                        for l in range(H.levels() - 1)]}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "multirhs":
        run_multirhs(args)
    elif args.workload == "table2":
        run_table2(args)
    elif args.workload == "largest":
        run_largest(args)
    elif args.workload == "vcycle":
        run_vcycle(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
