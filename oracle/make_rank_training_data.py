"""Write the rank-predictor training set from the FP64 oracle's own ranks.

Runs the oracle (only) on training problems that are disjoint from the
measured workloads -- smaller 2D Poisson grids at several tolerances and both
box shapes, and 2D Gaussian-random-field diffusion grids with seeds 1..8 --
and stores, for every block row with a non-empty far row, the features of
``oracle.ce.block_features`` and the target r_i / n_i.

    python -m oracle.make_rank_training_data
writes paper_1603_09133_gb300/models/rank_train.npz.
"""
import os
import sys

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402
from oracle import ce, mlp  # noqa: E402

OUT = os.path.join(ROOT, "paper_1603_09133_gb300", "models", "rank_train.npz")


def problems():
    for n in (64, 128, 256):
        for tol in (1e-3, 1e-4, 1e-5):
            yield f"poisson2d {n} B32 tol {tol}", wl.poisson2d(n), wl.box_perm((n, n), (8, 4)), 32, tol
    for n in (64, 128):
        for tol in (1e-3, 1e-4):
            yield f"poisson2d {n} B16 tol {tol}", wl.poisson2d(n), wl.box_perm((n, n), (4, 4)), 16, tol
    for seed in range(1, 9):
        n = 128 if seed > 4 else 256
        A = wl.diffusion2d(wl.grf2d(n, seed))
        yield f"grf2d {n} seed {seed}", A, wl.box_perm((n, n), (8, 4)), 32, 1e-4


def main():
    Xs, ts, tags = [], [], []
    for name, A, perm, B, tol in problems():
        F = ce.factorize(A, perm, B, tol, 4, 4)
        X, t = mlp.training_set([F])
        Xs.append(X)
        ts.append(t)
        tags += [name] * len(t)
        print(f"{name}: {len(t)} samples, mean r/n {t.mean():.3f}", flush=True)
    X = np.concatenate(Xs).astype(np.float32)
    t = np.concatenate(ts).astype(np.float32)
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    np.savez_compressed(OUT, X=X, t=t, source=np.array(sorted(set(tags))))
    print(f"wrote {OUT}: {X.shape[0]} samples")


if __name__ == "__main__":
    main()
