"""One factorization (and optionally one PCG solve) of a named workload, for
profiler captures of single launches:

    python -m paper_1603_09133_gb300.profile_case --workload poisson2d_256_B32 \
        --precision fp32 [--solve] [--learned] [--shapes 0,1,1,1 --learned-levels 0,1,1,1]

Each level's row kernel is one launch, so ``ncu -k regex:ce_row_kernel -s L -c 1``
on this command captures level L + 1.  Prints the per-level row-kernel times.
"""
import argparse

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="poisson2d_256_B32")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--row-shape", type=int, default=-1)
    ap.add_argument("--solve", action="store_true")
    ap.add_argument("--learned", action="store_true",
                    help="train the rank model and run the learned compression")
    ap.add_argument("--shapes", default=None,
                    help="per-level CTA shapes, e.g. 0,1,1,1 (a tuning as ce_autotune keeps it)")
    ap.add_argument("--learned-levels", default=None,
                    help="per-level learned (1) or exact (0) compression, e.g. 0,1,1,1")
    args = ap.parse_args()
    import torch
    import workloads as wl
    import paper_1603_09133_gb300 as ceg
    w = wl.make_workload(args.workload)
    csb = ceg.csb_build(w.A, w.perm, w.B)
    model = ceg.trained_rank_model() if args.learned else None
    if args.shapes:
        shapes = [int(v) for v in args.shapes.split(",")]
        lrn = [int(v) for v in args.learned_levels.split(",")] if args.learned_levels else [1] * len(shapes)
        csb.set_tuning((len(shapes), shapes + [0] * (16 - len(shapes)), lrn + [0] * (16 - len(lrn))),
                       args.precision, learned=model is not None)
    F = ceg.ce_factorize(csb, tol=w.tol, levels=w.levels, J=w.J, precision=args.precision,
                         row_shape=args.row_shape, rank_model=model)
    nl = F.info.levels_done
    print("row kernel ms per level:", [round(F.info.level_ms[l], 3) for l in range(nl)],
          "shapes:", list(F.info.row_shape[:nl]))
    names = ["wait", "setup", "learned", "R", "jacobi", "transform", "close", "far", "schur", "sketch_Y",
             "sketch_QR", "sketch_TSQR"]
    steps = ["gather", "sketch", "exact_svd", "UtDU", "chol_inv", "W_Y_far", "D_Wp", "kept_schur"]
    if any(F.info.big_rows[l] for l in range(nl)):
        print("large-row levels: steps ms", {k: round(F.info.big_ms[j], 1) for j, k in enumerate(steps)},
              "mean Jacobi sweeps", [round(F.info.jacobi_sweeps[l][0], 2) for l in range(nl) if F.info.big_rows[l]])
    for l in range(nl):
        if F.info.big_rows[l]:
            continue
        ph = [F.info.row_phase_ms[l][p] for p in range(12)]
        tot = sum(ph) or 1.0
        print(f"level {l}: row-phase SM time (ms summed over rows)",
              {k: f"{v:.1f} ({100 * v / tot:.0f}%)" for k, v in zip(names, ph)},
              "Jacobi sweeps (exact, learned):", [round(F.info.jacobi_sweeps[l][k], 2) for k in range(2)])
    if args.solve:
        b = torch.as_tensor(w.b, device="cuda")
        x = torch.zeros_like(b)
        it, rel, conv = ceg.pcg_solve(csb, F, b, x, 1e-8, 500)
        xh = x.cpu().numpy()
        print("PCG iterations", it, "true residual",
              float(np.linalg.norm(w.b - w.A @ xh) / np.linalg.norm(w.b)))
    torch.cuda.synchronize()


if __name__ == "__main__":
    main()
