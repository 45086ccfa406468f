"""pcg_solve_noalloc: the PCG for callers that cannot let the library allocate
device memory (a caller-owned memory pool, latency-critical loops, plugins
forbidden to allocate).  Called through the C ABI and checked against
pcg_solve on the same factor, on calls in a row with different right-hand
sides: the static work array keeps the previous call's contents, and a read
of a stale entry would show as a difference from pcg_solve on the new
right-hand side.  This file sorts after every other test file, so that a run
stopping at its first failure has run everything else already.
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


@pytest.fixture(scope="module")
def system(env):
    ceg, _lib, lib = env
    w = wl.make_workload("poisson2d_64_B16")
    csb = ceg.csb_build(w.A, w.perm, w.B)
    F = ceg.ce_factorize(csb, tol=w.tol, levels=w.levels, J=w.J)
    return w, csb, F


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _solve(env, entry, csb, F, b_host, maxit=200):
    """(status, info, x) of one call of `entry` on a fresh NaN-filled x."""
    _, _lib, lib = env
    b = torch.as_tensor(b_host, device="cuda")
    x = torch.full_like(b, float("nan"))
    info = _lib.ce_pcg_info()
    st = getattr(lib, entry)(csb.handle, F.handle, _ptr(b), _ptr(x), 1e-8, maxit, C.byref(info), _stream())
    torch.cuda.synchronize()
    return st, info, x.cpu().numpy()


def test_noalloc_matches_pcg_solve_on_calls_in_a_row(env, system):
    _, _lib, lib = env
    w, csb, F = system
    rhs = [w.b, wl.rhs(w.A.shape[0], 1), w.b]     # a different b in between
    for call, b in enumerate(rhs):
        st_ref, info_ref, xr = _solve(env, "pcg_solve", csb, F, b)
        assert st_ref == _lib.CE_OK and info_ref.converged
        st, info, xh = _solve(env, "pcg_solve_noalloc", csb, F, b)
        assert st == _lib.CE_OK, lib.ce_last_error()
        assert info.converged and info.iters == info_ref.iters, call
        assert np.linalg.norm(xh - xr) / np.linalg.norm(xr) <= 1e-10, call
        true_rel = np.linalg.norm(b - w.A @ xh) / np.linalg.norm(b)
        assert true_rel <= 1e-8 * 1.01


def test_noalloc_iteration_limit_and_zero_rhs(env, system):
    _, _lib, lib = env
    w, csb, F = system
    b = wl.rhs(w.A.shape[0], 2)
    st_ref, info_ref, xr = _solve(env, "pcg_solve", csb, F, b, maxit=1)
    st, info, xh = _solve(env, "pcg_solve_noalloc", csb, F, b, maxit=1)
    assert st_ref == st == _lib.CE_ERR_NO_CONVERGENCE
    assert info.iters == info_ref.iters == 1 and not info.converged
    assert np.linalg.norm(xh - xr) / np.linalg.norm(xr) <= 1e-10
    z = np.zeros(w.A.shape[0])
    st, info, xh = _solve(env, "pcg_solve_noalloc", csb, F, z)
    assert st == _lib.CE_OK and info.converged and info.iters == 0
    assert np.all(xh == 0.0)


def test_noalloc_rejects_sizes_beyond_its_limit(env):
    ceg, _lib, lib = env
    n = 264                        # 264^2 = 69696 unknowns > 65536
    A = wl.poisson2d(n)
    perm = wl.box_perm((n, n), (8, 4))
    csb = ceg.csb_build(A, perm, 32)
    F = ceg.ce_factorize(csb, tol=1e-2, levels=2, J=4)
    st, _, _ = _solve(env, "pcg_solve_noalloc", csb, F, np.ones(n * n), maxit=10)
    assert st == _lib.CE_ERR_LIMIT
    assert b"65536" in lib.ce_last_error()


def test_noalloc_rejects_a_batch_handle(env):
    ceg, _lib, lib = env
    systems = [(wl.poisson2d(s), wl.box_perm((s, s), (4, 4)), 16) for s in (32, 48)]
    csb = ceg.csb_build_batched(systems)
    F = ceg.ce_factorize_batched(csb, tol=1e-3, levels=2, J=4)
    st, _, _ = _solve(env, "pcg_solve_noalloc", csb, F, np.ones(csb.n))
    assert st == _lib.CE_ERR_INVALID_ARG
    assert b"pcg_solve_batched" in lib.ce_last_error()
