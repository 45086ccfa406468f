"""GPU: PCG stopped by its iteration limit.

With maxit below what the preconditioner needs, pcg_solve returns
CE_ERR_NO_CONVERGENCE with converged = 0, iters = maxit and the residual of
the last iterate; that iterate is the oracle's PCG iterate after the same
number of steps (x_0 = 0, the same M), within the FP64 apply tolerance.
(The file sorts after the other GPU tests so that a failure here stops none.)
"""
import ctypes as C

import numpy as np
import pytest

import workloads as wl
from oracle import ce as oce

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ceg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_09133_gb300 import build
    build.build()
    import paper_1603_09133_gb300 as m
    return m


@pytest.mark.parametrize("maxit", [1, 3])
def test_pcg_iteration_limit(ceg, maxit):
    from paper_1603_09133_gb300 import _lib
    lib = _lib.load()
    n = 64
    A = wl.poisson2d(n)
    perm = wl.box_perm((n, n), (4, 4))
    b = wl.rhs(n * n, 2)
    # a weak preconditioner (CE(1): one direction per far row) needs many steps
    Fo = oce.factorize(A, perm, 16, 0.0, 2, 4, tol_mode="fixed", rank=1)
    res_o = oce.pcg(A, Fo, b, 1e-12, maxit)
    assert not res_o.converged
    csb = ceg.csb_build(A, perm, 16)
    F = ceg.ce_factorize(csb, levels=2, J=4, tol_mode="fixed", rank=1)
    x = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    bd = torch.as_tensor(b, device="cuda")
    info = _lib.ce_pcg_info()
    st = lib.pcg_solve(csb.handle, F.handle, C.c_void_p(bd.data_ptr()), C.c_void_p(x.data_ptr()),
                       1e-12, maxit, C.byref(info), None)
    assert st == ceg.CE_ERR_NO_CONVERGENCE
    assert info.converged == 0 and info.iters == maxit
    xg = x.cpu().numpy()
    assert info.relres == pytest.approx(np.linalg.norm(b - A @ xg) / np.linalg.norm(b), rel=1e-8)
    assert np.linalg.norm(xg - res_o.x) / np.linalg.norm(res_o.x) <= 1e-9
