"""GPU: CE(eps) as a direct solver (Section 4, Table err): x_CE = M^{-1} b from
one factorization and one apply, no Krylov iteration, on the paper's own
problem (3D diffusion, k = diag(x_d^2 + 0.5), f = 1; B = 8 boxes of 2^3,
J = 8, 3 levels, FP64 form), with eta = ||x_CE - x*|| / ||x*|| against the
sparse direct solution x* (SciPy's SuperLU on the CPU).

* N = 8192 (16x16x32), eps = 1e-2, 1e-4, 1e-6, 1e-8: eta on the GPU equals
  the oracle's within 10% (the two factors agree up to rounding and rank
  decisions within rounding of tau); eta falls and the factor grows as eps
  falls.
* N = 65536 (32x32x64, the table's size), on the GPU alone: the same trends,
  printed beside the paper's eta (4.0e-1, 9.1e-3, 1.2e-5, 9.9e-7) and memory
  (553 ... 2671 MB).  The paper's eta are larger because its coarse
  remainder is smaller (its level count is not stated); the trend is the
  claim checked here.
"""
import time

import numpy as np
import pytest

import workloads as wl
from oracle import ce as oce

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EPS = (1e-2, 1e-4, 1e-6, 1e-8)


@pytest.fixture(scope="module")
def ceg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_09133_gb300 import build
    build.build()
    import paper_1603_09133_gb300 as m
    return m


def _reference(A, b):
    import scipy.sparse.linalg as spla
    x = spla.spsolve(A.tocsc(), b)
    assert np.linalg.norm(A @ x - b) <= 1e-10 * np.linalg.norm(b)
    return x


def _direct(ceg, csb, eps, b):
    t0 = time.perf_counter()
    F = ceg.ce_factorize(csb, tol=eps, levels=3, J=8)
    r = torch.as_tensor(b, device="cuda")
    z = torch.empty_like(r)
    ceg.ce_apply(F, r, z)
    torch.cuda.synchronize()
    return z.cpu().numpy(), F, time.perf_counter() - t0


def test_direct_solver_vs_oracle(ceg):
    shape = (16, 16, 32)
    A = wl.diffusion3d_tensor(*shape)
    perm = wl.box_perm(shape, (2, 2, 2))
    b = np.ones(A.shape[0])
    xs = _reference(A, b)
    csb = ceg.csb_build(A, perm, 8)
    eta_g, eta_o, mem = [], [], []
    for eps in EPS:
        x, F, _ = _direct(ceg, csb, eps, b)
        eta_g.append(np.linalg.norm(x - xs) / np.linalg.norm(xs))
        mem.append(F.info.factor_bytes)
        Fo = oce.factorize(A, perm, 8, eps, 3, 8)
        eta_o.append(np.linalg.norm(oce.apply(Fo, b) - xs) / np.linalg.norm(xs))
    print("N = 8192: eta GPU", [f"{e:.2e}" for e in eta_g], "oracle", [f"{e:.2e}" for e in eta_o],
          "factor MB", [round(m / 2 ** 20, 1) for m in mem])
    for eg, eo in zip(eta_g, eta_o):
        assert abs(eg - eo) <= 0.1 * eo, (eg, eo)
    assert all(eta_g[j + 1] < eta_g[j] for j in range(len(EPS) - 1))
    assert all(mem[j + 1] >= mem[j] for j in range(len(EPS) - 1)) and mem[-1] > mem[0]


def test_direct_solver_table_err_size(ceg):
    shape = (32, 32, 64)
    A = wl.diffusion3d_tensor(*shape)
    perm = wl.box_perm(shape, (2, 2, 2))
    b = np.ones(A.shape[0])
    xs = _reference(A, b)
    csb = ceg.csb_build(A, perm, 8)
    rows = []
    for eps in EPS:
        x, F, sec = _direct(ceg, csb, eps, b)
        rows.append((eps, np.linalg.norm(x - xs) / np.linalg.norm(xs), F.info.factor_bytes / 2 ** 20, sec,
                     F.info.coarse_n))
    for eps, eta, mb, sec, nc in rows:
        print(f"N = 65536, eps {eps:.0e}: eta {eta:.2e}, factor {mb:.0f} MB, factorize + apply {sec:.2f} s, "
              f"coarse {nc}")
    print("paper: eta 4.0e-01 9.1e-03 1.2e-05 9.9e-07, memory 553 1348 2494 2671 MB")
    etas = [r[1] for r in rows]
    mem = [r[2] for r in rows]
    assert all(etas[j + 1] < etas[j] for j in range(len(EPS) - 1))
    assert all(mem[j + 1] >= mem[j] for j in range(len(EPS) - 1)) and mem[-1] > mem[0]
