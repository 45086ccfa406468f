"""Failure path of the persistent launches' dependency waits.

A row of the persistent row kernel (ce_factorize) and of the persistent apply
(ce_apply) waits for its lower-colour neighbours before it starts.  Here the
neighbour is never queued, so the wait cannot end; with a 20 ms limit the
kernel must give up, record CE_ERR_CUDA with its reason (5: row kernel, 6:
apply) and the blocked row, and return, leaving the context usable.  No
kernel traps or hangs: the wait is bounded by time and by a poll count.
"""
import ctypes as C
import time

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


@pytest.mark.parametrize("kernel,reason", [(0, 5), (1, 6)])
def test_dependency_wait_expires_and_reports(env, kernel, reason):
    ceg, _lib, lib = env
    status = np.zeros(8, np.int32)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    t0 = time.perf_counter()
    st = lib.ce_debug_wait_expiry(kernel, 20.0, status.ctypes.data_as(_lib.I32P), stream)
    dt = time.perf_counter() - t0
    assert st == _lib.CE_OK, lib.ce_last_error()
    assert status[0] == _lib.CE_ERR_CUDA and status[3] == reason and status[2] == 1, status
    assert dt < 1.5, dt                       # gave up after its short limit
    # the context is still usable: a small factorization and apply
    w = wl.make_workload("poisson2d_64_B16")
    csb = ceg.csb_build(w.A, w.perm, w.B)
    F = ceg.ce_factorize(csb, tol=w.tol, levels=w.levels, J=w.J)
    r = torch.as_tensor(w.b, device="cuda")
    z = torch.empty_like(r)
    ceg.ce_apply(F, r, z)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(z.cpu().numpy()))

