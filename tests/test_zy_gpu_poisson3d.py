"""GPU: the 3D 7-point Laplacian against the FP64 oracle on grids whose levels
fit the row kernel (blocks of at most 64 rows, at most 32 targets and 128 far
blocks per row); levels that outgrow it run the large-row path, covered by
test_gpu_big_rows.py.

Checks the 3D arithmetic of the row kernel: the same distance-2 colouring,
the same ranks (away from the threshold: every oracle singular value here
lies at least 7e-4 relative from tau), the FP64 apply within 1e-10, PCG
iterations within +-1 and a true residual <= 1e-8; the FP32 form (on the grid
whose singular values keep clear of tau by more than FP32 rounding) by its
backward error against the oracle's operator (<= 1e-4).
"""
import numpy as np
import pytest

import workloads as wl
from oracle import ce as oce

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = [
    # grid side, box, levels: 3D boxes of 4^3 (B = 64) and 2^3 (B = 8), J = 8
    (16, (4, 4, 4), 3),
    (16, (2, 2, 2), 3),
]


@pytest.fixture(scope="module")
def ceg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_09133_gb300 import build
    build.build()
    import paper_1603_09133_gb300 as m
    return m


@pytest.fixture(scope="module")
def oracle_factors():
    out = {}
    for n, box, levels in CASES:
        A = wl.poisson3d(n)
        perm = wl.box_perm((n, n, n), box)
        B = int(np.prod(box))
        out[(n, box)] = (A, perm, B, oce.factorize(A, perm, B, 1e-4, levels, 8))
    return out


def _ranks_ok(lev, r_g, rel=1e-5):
    for st in lev.steps:
        if r_g[st.i] == st.r:
            continue
        lo, hi = sorted((r_g[st.i], st.r))
        if not all(k < st.sigma.size and abs(st.sigma[k] - st.tau) <= rel * st.tau for k in range(lo, hi)):
            return False
    return True


def _anorm(A):
    import scipy.sparse.linalg as spla
    return float(spla.eigsh(A, k=1, which="LA", return_eigenvectors=False)[0])


@pytest.mark.parametrize("n,box,levels", CASES)
def test_poisson3d_fp64_matches_oracle(ceg, oracle_factors, n, box, levels):
    A, perm, B, Fo = oracle_factors[(n, box)]
    b = wl.rhs(A.shape[0], 0)
    csb = ceg.csb_build(A, perm, B)
    F = ceg.ce_factorize(csb, tol=1e-4, levels=levels, J=8)
    for l, lev in enumerate(Fo.levels):
        n_g, r_g, c_g, _ = F.level(l)
        assert list(n_g) == list(lev.sizes), l
        assert list(c_g) == list(lev.colour), l
        assert _ranks_ok(lev, r_g), l
    z = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
    ceg.ce_apply(F, torch.as_tensor(b, device="cuda"), z)
    zo = oce.apply(Fo, b)
    err = np.linalg.norm(z.cpu().numpy() - zo) / np.linalg.norm(zo)
    print(f"3D {n}^3 B={B}: apply error {err:.2e}")
    assert err <= 1e-10
    res_o = oce.pcg(A, Fo, b, 1e-8, 500)
    x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
    it, rel, conv = ceg.pcg_solve(csb, F, torch.as_tensor(b, device="cuda"), x, 1e-8, 500)
    true = np.linalg.norm(b - A @ x.cpu().numpy()) / np.linalg.norm(b)
    assert conv and true <= 1e-8 * 1.01 and abs(it - res_o.iters) <= 1, (it, res_o.iters, true)


# FP32 singular values carry errors near 6e-4 tau here; the B = 8 grid has an
# oracle value 1.6e-3 relative from tau, the B = 64 grid none closer than 9.6e-3
@pytest.mark.parametrize("n,box,levels", CASES[:1])
def test_poisson3d_fp32_backward_error(ceg, oracle_factors, n, box, levels):
    A, perm, B, Fo = oracle_factors[(n, box)]
    b = wl.rhs(A.shape[0], 1)
    csb = ceg.csb_build(A, perm, B)
    F = ceg.ce_factorize(csb, tol=1e-4, levels=levels, J=8, precision="fp32")
    z = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
    ceg.ce_apply(F, torch.as_tensor(b, device="cuda"), z)
    zg = z.cpu().numpy()
    eta = np.linalg.norm(b - oce.multiply(Fo, zg)) / (_anorm(A) * np.linalg.norm(zg) + np.linalg.norm(b))
    print(f"3D {n}^3 B={B} fp32: backward error {eta:.2e}")
    assert eta <= 1e-4
    x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
    it, rel, conv = ceg.pcg_solve(csb, F, torch.as_tensor(b, device="cuda"), x, 1e-8, 500)
    true = np.linalg.norm(b - A @ x.cpu().numpy()) / np.linalg.norm(b)
    assert conv and true <= 1e-8 * 1.01
