"""pcg_solve_noalloc: the PCG for callers that cannot let the library allocate
device memory (a caller-owned memory pool, latency-critical loops, plugins
forbidden to allocate).  Called through the C ABI and checked against
pcg_solve on the same factor, on two calls in a row (the static work array
keeps the previous call's contents, which must not leak into the result).
"""
import ctypes as C

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_09133_gb300 import build
    build.build()
    import paper_1603_09133_gb300 as ceg
    from paper_1603_09133_gb300 import _lib
    return ceg, _lib, _lib.load()


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def test_noalloc_matches_pcg_solve_on_two_calls(env):
    ceg, _lib, lib = env
    w = wl.make_workload("poisson2d_64_B16")
    csb = ceg.csb_build(w.A, w.perm, w.B)
    F = ceg.ce_factorize(csb, tol=w.tol, levels=w.levels, J=w.J)
    b = torch.as_tensor(w.b, device="cuda")
    x_ref = torch.zeros_like(b)
    info_ref = _lib.ce_pcg_info()
    st = lib.pcg_solve(csb.handle, F.handle, _ptr(b), _ptr(x_ref), 1e-8, 200,
                       C.byref(info_ref), _stream())
    torch.cuda.synchronize()
    assert st == _lib.CE_OK and info_ref.converged
    xr = x_ref.cpu().numpy()
    for call in range(2):
        x = torch.full_like(b, float("nan"))
        info = _lib.ce_pcg_info()
        st = lib.pcg_solve_noalloc(csb.handle, F.handle, _ptr(b), _ptr(x), 1e-8, 200,
                                   C.byref(info), _stream())
        torch.cuda.synchronize()
        assert st == _lib.CE_OK, lib.ce_last_error()
        assert info.converged and info.iters == info_ref.iters
        xh = x.cpu().numpy()
        assert np.linalg.norm(xh - xr) / np.linalg.norm(xr) <= 1e-10, call
        true_rel = np.linalg.norm(w.b - w.A @ xh) / np.linalg.norm(w.b)
        assert true_rel <= 1e-8 * 1.01


def test_noalloc_rejects_sizes_beyond_its_limit(env):
    ceg, _lib, lib = env
    n = 264                        # 264^2 = 69696 unknowns > 65536
    A = wl.poisson2d(n)
    perm = wl.box_perm((n, n), (8, 4))
    csb = ceg.csb_build(A, perm, 32)
    F = ceg.ce_factorize(csb, tol=1e-2, levels=2, J=4)
    b = torch.ones(n * n, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    info = _lib.ce_pcg_info()
    st = lib.pcg_solve_noalloc(csb.handle, F.handle, _ptr(b), _ptr(x), 1e-8, 10,
                               C.byref(info), _stream())
    assert st == _lib.CE_ERR_LIMIT
    assert b"65536" in lib.ce_last_error()
