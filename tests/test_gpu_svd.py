"""GPU: the SVD steps of a large row's compression (Section 2.2: U_i and sigma
of a far row from the R factor of F_i^T) in isolation, through ce_debug_svd:
the QR factorization with column pivoting of R^T, then block one-sided Jacobi
over column blocks of 4, 8, 16 and 32 (every block width the library may
pick), in FP32 and FP64, against numpy's SVD of the same R.

R is the triangular factor of a random tall matrix with prescribed singular
values: graded over six decades, with a cluster of four equal values and an
exact zero (a rank-deficient far row).  With tol = 0 only rounding-level
pairs are skipped, so every singular value must be resolved:
* sigma (column norms of X, sorted) within 20 n u sigma_1 of numpy's;
* V orthogonal to 20 n u;
* R^T R V = V diag(sigma^2) to 50 n u sigma_1^2 (the defining property of the
  left singular vectors of R^T, the U_i of the compression step);
* the Jacobi stops within 20 sweeps.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_09133_gb300 import _lib, build
    build.build()
    return _lib.load()


def _r_factor(n, seed):
    rng = np.random.default_rng(seed)
    sig = 10.0 ** (-6.0 * np.arange(n) / n)
    sig[5:9] = sig[5]          # a cluster of equal singular values
    sig[-1] = 0.0              # rank deficient
    Ql, _ = np.linalg.qr(rng.standard_normal((3 * n, n)))
    Qr, _ = np.linalg.qr(rng.standard_normal((n, n)))
    F = (Ql * sig) @ Qr.T      # 3n x n, singular values sig
    R = np.linalg.qr(F, mode="r")
    return np.triu(R), np.sort(sig)[::-1]


@pytest.mark.parametrize("esize", [4, 8])
@pytest.mark.parametrize("block", [4, 8, 16, 32])
@pytest.mark.parametrize("n", [40, 200])
def test_block_jacobi_svd(lib, esize, block, n):
    dt = torch.float32 if esize == 4 else torch.float64
    u = np.finfo(np.float32 if esize == 4 else np.float64).eps
    R, sig = _r_factor(n, 7 * n + block)
    Rd = torch.as_tensor(R, dtype=dt, device="cuda").contiguous()
    Dd = torch.eye(n, dtype=dt, device="cuda")
    X = torch.empty(n * n, dtype=dt, device="cuda")
    V = torch.empty(n * n, dtype=dt, device="cuda")
    sw = C.c_int(-1)
    st = lib.ce_debug_svd(esize, block, n, C.c_void_p(Rd.data_ptr()), C.c_void_p(Dd.data_ptr()), 0.0,
                          C.c_void_p(X.data_ptr()), C.c_void_p(V.data_ptr()), C.byref(sw), None)
    assert st == 0
    Xh = X.cpu().numpy().astype(np.float64).reshape(n, n).T   # column j of X
    Vh = V.cpu().numpy().astype(np.float64).reshape(n, n).T
    s_g = np.linalg.norm(Xh, axis=0)
    s_np = np.linalg.svd(R.astype(np.float32 if esize == 4 else np.float64).astype(np.float64), compute_uv=False)
    err_s = np.max(np.abs(np.sort(s_g)[::-1] - s_np)) / s_np[0]
    err_o = np.linalg.norm(Vh.T @ Vh - np.eye(n), 2)
    G = R.T @ R
    err_e = np.linalg.norm(G @ Vh - Vh * s_g ** 2, 2) / s_np[0] ** 2
    print(f"esize {esize} block {block} n {n}: sweeps {sw.value}, sigma {err_s:.1e}, orth {err_o:.1e}, "
          f"eig {err_e:.1e}")
    assert err_s <= 20 * n * u, err_s
    assert err_o <= 20 * n * u, err_o
    assert err_e <= 50 * n * u, err_e
    assert 1 <= sw.value <= 20


def test_block_jacobi_rejects_bad_arguments(lib):
    x = torch.zeros(16, dtype=torch.float32, device="cuda")
    p = C.c_void_p(x.data_ptr())
    assert lib.ce_debug_svd(4, 12, 4, p, p, 0.0, p, p, None, None) == 1     # block width (CE_ERR_INVALID_ARG)
    assert lib.ce_debug_svd(2, 8, 4, p, p, 0.0, p, p, None, None) == 1      # element size
    assert lib.ce_debug_svd(4, 8, 0, p, p, 0.0, p, p, None, None) == 1      # n
