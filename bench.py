#!/usr/bin/env python
"""Time to a 1e-8 relative residual (CE factorization + FP64 PCG) on one GPU.

One step = ce_factorize + pcg_solve of the 2D Poisson 512x512 system (B = 32,
tol 1e-4, 4 levels, J = 4) with the matrix and right-hand side resident in
HBM.  ``--workload poisson2d_batch256`` times instead 256 independent 2D
Poisson systems (sides drawn from {64, 96, 128, 192, 256}) factorized as one
block-diagonal batch and solved by the per-system batched PCG.  The chosen
form (learned ranks with a randomized range finder, FP32 blocks and
compression, FP64 PCG) is the headline value; the plain FP64 form (exact SVD)
is timed beside it, both autotuned and timed alike.  The rank model is trained
on the GPU and the arithmetic peaks are measured before the timed region.
``--impl reference`` times the FP64 CPU oracle on the same workload.  Prints
one JSON line.

    python bench.py [--steps K] [--warmup W] [--impl ours|reference]
"""
import os

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")

import argparse  # noqa: E402
import json  # noqa: E402
import statistics  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import threading  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

METRIC = "time to 1e-8 residual (factor+PCG)"
WORKLOAD = "poisson2d_512_B32"
BATCH = "poisson2d_batch256"
BATCH_SYSTEMS = 256
WARMUP_GRID = 64         # reference arm warm-up: a 64x64 grid of the same kind (untimed)
RTOL = 1e-8


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    p.add_argument("--ranks", default="learned", choices=["learned", "svd"])
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--no-baseline", action="store_true", help="skip the oracle timing")
    p.add_argument("--coloring", type=int, default=1, choices=[1, 2],
                   help="elimination order: 1 distance-2 colours, 2 distance-1 colours")
    return p.parse_args()


# --------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
def max_over_ranks(value, world, device="cpu"):
    """The largest `value` over the ranks of the process group (the slowest
    replica sets a whole-job time); the value itself with one rank."""
    if world <= 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


class Problem:
    """One system, or a batch of independent ones, with its parameters."""

    def __init__(self, name):
        self.name = name
        self.batched = name == BATCH
        self.is3d = name.startswith("poisson3d")
        # super-block cap: 64 rows for the 2D grids (every level stays in the
        # persistent row kernel), none in 3D (the paper's runs of J = 8; the
        # large blocks run the large-row path)
        self.nmax = 0 if self.is3d else 64
        if self.batched:
            self.ws = wl.make_batch(BATCH_SYSTEMS)
            w0 = self.ws[0]
            self.tol, self.levels, self.J = w0.tol, w0.levels, w0.J
            self.B = "16 (sides <= 96) / 32"
            self.desc = (f"{BATCH_SYSTEMS} independent 2D Poisson 5-point systems, sides drawn "
                         f"from {list(wl.BATCH_SIDES)}, Dirichlet")
        else:
            w = wl.make_workload(name)
            self.ws = [w]
            self.tol, self.levels, self.J, self.B, self.desc = w.tol, w.levels, w.J, w.B, w.desc
        self.sizes = [w.A.shape[0] for w in self.ws]
        self.off = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        self.N = int(self.off[-1])
        self.b = np.concatenate([w.b for w in self.ws])

    def host_arrays(self):
        """Host arrays a user hands to the library (CSR, permutation, blocks)."""
        import paper_1603_09133_gb300 as ceg
        if self.batched:
            return ceg.stack_systems([(w.A, w.perm, w.B) for w in self.ws])
        w = self.ws[0]
        A = w.A.tocsr()
        return (np.ascontiguousarray(A.indptr, np.int64), np.ascontiguousarray(A.indices, np.int32),
                np.ascontiguousarray(A.data, np.float64), np.ascontiguousarray(w.perm, np.int32),
                w.B)

    def build(self, arrays):
        import paper_1603_09133_gb300 as ceg
        if self.batched:
            return ceg.csb_build_batched_csr(*arrays)
        rp, ci, va, pm, B = arrays
        import scipy.sparse as sp
        A = sp.csr_matrix((va, ci, rp), shape=(self.N, self.N))
        return ceg.csb_build(A, pm, B)

    def solve(self, csb, F, b, x):
        """PCG to RTOL; returns (max iterations, all converged)."""
        import paper_1603_09133_gb300 as ceg
        if self.batched:
            its, rel, conv = ceg.pcg_solve_batched(csb, F, b, x, RTOL, 1000)
            return int(its.max()), bool(conv.all())
        it, rel, conv = ceg.pcg_solve(csb, F, b, x, RTOL, 1000)
        return it, conv

    def true_relres(self, x):
        return max(float(np.linalg.norm(w.b - w.A @ x[self.off[s]:self.off[s + 1]])
                         / np.linalg.norm(w.b)) for s, w in enumerate(self.ws))


def oracle_solve(w, nmax=64):
    """Oracle factorize + PCG of one workload (seconds, PCG iterations)."""
    from oracle import ce as oce
    t0 = time.perf_counter()
    F = oce.factorize(w.A, w.perm, w.B, w.tol, w.levels, w.J, nmax=nmax)
    res = oce.pcg(w.A, F, w.b, RTOL, 1000)
    t = time.perf_counter() - t0
    assert res.converged
    return t, res.iters


def oracle_step(pb):
    """(seconds for the workload, unknowns timed, PCG iterations, what) of one
    oracle run: the whole workload for a single 2D system; for the batch, one
    64x64 system of it, scaled by N (a whole batch is ~250 s of CPU work); in
    3D the 32^3 grid of the same problem scaled by N (64^3 takes ~20 min in
    the oracle; its block sizes grow faster than N, so this is a lower bound)."""
    if pb.is3d:
        A = wl.poisson3d(32)
        w = wl.Workload("poisson3d_32_B64", A, wl.box_perm((32, 32, 32), (4, 4, 4)), 64, pb.tol, pb.levels,
                        pb.J, wl.rhs(A.shape[0], 0), "3D Poisson 7-point 32^3")
        t, its = oracle_solve(w, nmax=0)
        return t * pb.N / A.shape[0], A.shape[0], its, \
            f"the 32^3 grid of the same problem ({pb.levels} levels), scaled linearly to N={pb.N} (a lower bound)"
    if pb.batched:
        w = next(w for w in pb.ws if w.A.shape[0] == 64 * 64)
        t, its = oracle_solve(w)
        return t * pb.N / w.A.shape[0], w.A.shape[0], its, \
            f"one 64x64 system of the batch ({pb.levels} levels), scaled linearly to N={pb.N}"
    t, its = oracle_solve(pb.ws[0])
    return t, pb.N, its, f"the whole workload ({pb.desc}, {pb.levels} levels), one run, unscaled"


def oracle_warmup(pb):
    """Untimed warm-up of the oracle (imports, allocator): a small grid."""
    from oracle import ce as oce
    A = wl.poisson2d(WARMUP_GRID)
    perm = wl.box_perm((WARMUP_GRID, WARMUP_GRID), (4, 4))
    F = oce.factorize(A, perm, 16, 1e-3, 2, 4, nmax=64)
    oce.pcg(A, F, wl.rhs(A.shape[0], 0), RTOL, 100)


def cpu_baseline(pb):
    t, n, its, what = oracle_step(pb)
    return {"value": t, "unit": "s", "cores": 1, "kind": "oracle",
            "sample": f"FP64 numpy oracle (single-threaded BLAS) on {what}: {n} unknowns, "
                      f"{its} PCG iterations"}


def run_reference(args, rank):
    pb = Problem(args.workload)
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_warmup(pb)
    ts, what = [], ""
    for _ in range(args.steps):
        t, n, its, what = oracle_step(pb)
        ts.append(t)
    v = statistics.mean(ts)
    out = {"metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": args.workload, "N": pb.N, "B": pb.B, "tol": pb.tol,
                      "levels": pb.levels, "J": pb.J},
           "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle",
                            "sample": f"each step: oracle factorize+PCG on {what}; "
                                      f"warm-up steps: a {WARMUP_GRID}x{WARMUP_GRID} grid"},
           "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def committed_traffic(kernel, workload, precision):
    """DRAM traffic per launch of `kernel` from the committed ncu summary
    (profiles/ce_row_kernel_traffic_poisson2d_512.md), if that capture was taken of the
    current kernel source (its SHA-256 is recorded with the numbers); None
    otherwise.  Lines read: `source_sha256: <hex>`, and per captured form
    `traffic: <kernel> <workload> <precision> <bytes per launch>`."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "ce_row_kernel_traffic_poisson2d_512.md")
    src = os.path.join(ROOT, "paper_1603_09133_gb300", "csrc", "row_kernel.cu")
    if not os.path.exists(path):
        return None
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    rec_sha, val = None, None
    for ln in open(path):
        f = ln.strip().strip("`").split()
        if len(f) == 2 and f[0] == "source_sha256:":
            rec_sha = f[1]
        if len(f) == 5 and f[0] == "traffic:" and f[1:4] == [kernel, workload, precision]:
            val = float(f[4])
    if rec_sha != sha or val is None:
        return None
    return {"bytes_per_launch": val,
            "note": "dram__bytes_read.sum + dram__bytes_write.sum per launch, mean over the level "
                    "launches of one factorization (profiles/ce_row_kernel_traffic_poisson2d_512.md)"}


# --------------------------------------------------------------------------
def run_ours(args, rank, world):
    import torch
    import paper_1603_09133_gb300 as ceg
    from paper_1603_09133_gb300 import _lib, build as cebuild

    cebuild.build()
    lib = _lib.load()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    pb = Problem(args.workload)
    N = pb.N
    arrays = pb.host_arrays()
    csb = pb.build(arrays)
    b = torch.as_tensor(pb.b, device=dev)
    x = torch.zeros_like(b)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    model = ceg.trained_rank_model() if args.ranks == "learned" else None
    # measured arithmetic peaks of this GPU (the roofline denominators)
    peaks = {k: ceg.measure_peak(k) for k in ("fp32_fma", "fp64_fma", "tf32_mma", "tf32x3_mma")}
    # row-kernel CTA shape (and learned or exact per level) chosen by
    # measurement for both forms (setup, untimed); in 3D a factorization
    # takes seconds, so the heuristic shapes are kept and only learned or
    # exact compression is chosen per level, from one factorization of each
    tune_ms, tune_ms_plain = np.zeros((2, 4, pb.levels)), np.zeros((2, 4, pb.levels))
    if not pb.is3d:
        tune_ms = ceg.ce_autotune(csb, tol=pb.tol, levels=pb.levels, J=pb.J, precision=args.precision,
                                  rank_model=model, nmax=pb.nmax, coloring=args.coloring)
        tune_ms_plain = ceg.ce_autotune(csb, tol=pb.tol, levels=pb.levels, J=pb.J, precision="fp64",
                                        nmax=pb.nmax, coloring=args.coloring)
    elif model is not None:
        kw = dict(tol=pb.tol, levels=pb.levels, J=pb.J, precision=args.precision, nmax=pb.nmax,
                  coloring=args.coloring)
        Fl = ceg.ce_factorize(csb, rank_model=model, **kw)
        Fe = ceg.ce_factorize(csb, **kw)
        nlv = min(Fl.info.levels_done, Fe.info.levels_done)
        shp = np.array([Fl.info.row_shape[l] if l < nlv else 0 for l in range(16)], np.int32)
        lrn = np.array([int(Fl.info.level_ms[l] <= Fe.info.level_ms[l]) if l < nlv else 0 for l in range(16)],
                       np.int32)
        for l in range(min(nlv, pb.levels)):
            tune_ms[0, shp[l], l] = Fl.info.level_ms[l]
            tune_ms[1, shp[l], l] = Fe.info.level_ms[l]
        csb.set_tuning((nlv, shp, lrn), args.precision, learned=True)
        del Fl, Fe
    tuning = csb.tuning(args.precision, learned=model is not None)

    def step(prec, rm=None):
        F = ceg.ce_factorize(csb, tol=pb.tol, levels=pb.levels, J=pb.J, precision=prec, rank_model=rm,
                             nmax=pb.nmax, coloring=args.coloring)
        it, conv = pb.solve(csb, F, b, x)
        return F, it, conv

    def timed(prec, k, w_, rm=None):
        for _ in range(w_):
            step(prec, rm)
        times, last = [], None
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(dev.index)
        sampler.start()
        l0 = lib.ce_launch_count()
        for _ in range(k):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            last = step(prec, rm)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        launches = (lib.ce_launch_count() - l0) / k
        clocks = sampler.stop()
        if world > 1:
            torch.distributed.barrier()
        return times, last, launches, clocks

    # plain FP64 form with exact SVDs (the comparison), then the chosen form,
    # each autotuned and timed with the same steps, warm-up and clock sampling
    # (in 3D the plain form's exact SVD of blocks of ~700 rows in FP64 takes
    # minutes per factorization and is not timed)
    if pb.is3d:
        t_other, last_other, clocks_other = [float("nan")], (None, None, None), None
    else:
        t_other, last_other, _, clocks_other = timed("fp64", args.steps, args.warmup)
    times, last, launches, clocks = timed(args.precision, args.steps, args.warmup, model)
    F, it, conv = last
    true_rel = pb.true_relres(x.cpu().numpy())
    ms = max_over_ranks(statistics.mean(times), world, dev)

    # roofline of the dominant kernel (the persistent row kernel, one launch
    # per level): algorithmic flops (counted from the actual sizes, ranks,
    # widths and sketch widths) over its CUDA-event time, against the measured
    # FP32 FFMA (FP64: DFMA) rate of this GPU
    # (levels run by the large-row path are reported beside it)
    info = F.info
    nl = info.levels_done
    rk = [l for l in range(nl) if not info.big_rows[l]]
    bg = [l for l in range(nl) if info.big_rows[l]]
    nrk = max(len(rk), 1)
    lms = sum(info.level_ms[l] for l in rk)
    lfl = sum(info.level_flops[l] for l in rk)
    lby = sum(info.level_bytes[l] for l in rk)
    big_levels = None
    if bg:
        bms = sum(info.level_ms[l] for l in bg)
        bfl = sum(info.level_flops[l] for l in bg)
        big_levels = {"levels": bg, "ms_per_step": bms, "algorithmic_flops": bfl,
                      "achieved_tflops": bfl / (bms * 1e-3) / 1e12 if bms > 0 else None}
    pk = "fp32_fma" if args.precision == "fp32" else "fp64_fma"
    peak = peaks[pk]
    achieved = lfl / (lms * 1e-3) / 1e12 if lms > 0 else 0.0
    kname = f"ce_row_kernel<{'float' if args.precision == 'fp32' else 'double'}>"
    traffic = committed_traffic(kname, args.workload, args.precision)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": traffic["bytes_per_launch"] if traffic else None,
                "kernel": kname, "launches_per_step": len(rk),
                "kernel_ms_per_step": lms, "algorithmic_flops_per_launch": lfl / nrk,
                "algorithmic_bytes_per_launch": lby / nrk, "achieved_gbs": lby / (lms * 1e-3) / 1e9 if lms > 0 else 0.0,
                "traffic_note": traffic["note"] if traffic else
                "no ncu capture of this kernel source committed under profiles/",
                "peak_note": f"of measured: ce_measure_peak {pk} on this GPU",
                "measured_peaks_tflops": peaks, "large_row_levels": big_levels}

    # end to end through the public API with host buffers: csb_build from the
    # host CSR (with the tuning measured above set on the new handle), the
    # factorization, H2D of b from pinned memory, PCG, D2H of x
    b_host = torch.as_tensor(pb.b).pin_memory()
    x_host = torch.empty(N, dtype=torch.float64).pin_memory()
    e2e_t = []
    for k in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        csb2 = pb.build(arrays)
        csb2.set_tuning(tuning, args.precision, learned=model is not None)
        F2 = ceg.ce_factorize(csb2, tol=pb.tol, levels=pb.levels, J=pb.J, precision=args.precision,
                              rank_model=model, nmax=pb.nmax, coloring=args.coloring)
        bd = b_host.to(dev, non_blocking=True)
        xd = torch.empty_like(bd)
        pb.solve(csb2, F2, bd, xd)
        x_host.copy_(xd, non_blocking=True)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        F2.close()
        csb2.close()
        if k >= args.warmup:
            e2e_t.append(t1 - t0)
    h2d = sum(a.nbytes for a in arrays if isinstance(a, np.ndarray)) + pb.b.nbytes
    e2e = {"value": max_over_ranks(statistics.mean(e2e_t), world, dev), "unit": "s",
           "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(N * 8)}

    if rank != 0:
        return
    levels_cfg = {"blocks": [info.blocks[l] for l in range(nl)],
                  "colours": [info.colours[l] for l in range(nl)],
                  "max_block": [info.max_block[l] for l in range(nl)],
                  "row_kernel_ms": [round(info.level_ms[l], 3) for l in range(nl)],
                  "row_shape": [info.row_shape[l] for l in range(nl)],
                  "row_learned": [info.row_learned[l] for l in range(nl)],
                  "autotune_ms": np.round(tune_ms, 3).tolist(),
                  "autotune_ms_plain_fp64": np.round(tune_ms_plain, 3).tolist(),
                  "jacobi_capped": [info.jacobi_capped[l] for l in range(nl)],
                  "row_phase_ms": {k: [round(info.row_phase_ms[l][p], 2) for l in range(nl)] for p, k in
                                   enumerate(["wait", "setup", "learned", "R", "jacobi", "transform", "close",
                                              "far", "schur", "sketch_Y", "sketch_QR", "sketch_TSQR"])},
                  "big_rows": [info.big_rows[l] for l in range(nl)],
                  "big_steps_ms": dict(zip(["gather", "sketch", "exact_svd", "UtDU", "chol_inv", "W_Y_far",
                                            "D_Wp", "kept_schur"], [round(v, 2) for v in info.big_ms])),
                  "host_ms": [round(info.host_ms[l], 3) for l in range(nl)],
                  "factor_wall_ms": round(info.total_ms, 3),
                  "coarse_n": info.coarse_n, "coarse_ms": round(info.coarse_ms, 3),
                  "factor_MB": round(info.factor_bytes / 2**20, 1)}
    out = {"metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
           "config": {"workload": args.workload, "desc": pb.desc, "N": int(N), "B": pb.B,
                      "tol": pb.tol, "levels": pb.levels, "J": pb.J,
                      "systems": len(pb.ws),
                      "form": f"{args.ranks} ranks + {args.precision} factor + fp64 PCG",
                      "pcg_iters": it, "final_relres": true_rel,
                      "nmax": pb.nmax,
                      "coloring": {1: "distance-2", 2: "distance-1"}[args.coloring],
                      "plain_fp64_form_s": None if pb.is3d else statistics.mean(t_other) / 1e3,
                      "plain_fp64_form_pcg_iters": last_other[1],
                      "plain_fp64_form_clocks": clocks_other,
                      "plain_fp64_form_timing": "autotuned (exact SVD, FP64), same steps, warm-up, "
                                                "L2 flush and clock sampling as the chosen form",
                      "learned_rows": [info.learned_rows[l] for l in range(info.levels_done)],
                      "fallback_rows": [info.fallback_rows[l] for l in range(info.levels_done)],
                      "rank_model_train_loss": getattr(model, "loss", None),
                      "l2": "256 MB buffer written between timed steps",
                      "parallelism": "replicas" if world > 1 else "single GPU",
                      "levels_detail": levels_cfg},
           "clocks": clocks, "e2e": e2e, "gpu_launches": launches, "roofline": roofline}
    if not args.no_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline(pb)
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group("nccl")
    run_ours(args, rank, world)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
