"""GPU: numeric refactorization through csb_update_values.

A csb built for one coefficient field and then given the values of another
field on the same 5-point pattern factorizes exactly as a csb built for the
second field from scratch (the same deterministic kernels on the same
inputs: ranks, colours and the apply agree bit for bit), and matches the FP64
oracle on the second field.  Values that break symmetry are refused on the
host and leave the csb unchanged.
"""
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


def _apply(ceg, F, b):
    z = torch.empty(b.size, dtype=torch.float64, device="cuda")
    ceg.ce_apply(F, torch.as_tensor(b, device="cuda"), z)
    return z.cpu().numpy()


def test_update_values_equals_fresh_build(ceg):
    n = 64
    A1 = wl.diffusion2d(wl.grf2d(n, seed=1))
    A2 = wl.diffusion2d(wl.grf2d(n, seed=2))
    assert np.array_equal(A1.indptr, A2.indptr) and np.array_equal(A1.indices, A2.indices)
    perm = wl.box_perm((n, n), (4, 4))
    b = wl.rhs(n * n, 0)
    csb = ceg.csb_build(A1, perm, 16)
    F1 = ceg.ce_factorize(csb, tol=1e-6, levels=3, J=4)
    z1 = _apply(ceg, F1, b)
    ceg.csb_update_values(csb, A2)
    F2 = ceg.ce_factorize(csb, tol=1e-6, levels=3, J=4)
    fresh = ceg.csb_build(A2, perm, 16)
    Ff = ceg.ce_factorize(fresh, tol=1e-6, levels=3, J=4)
    for l in range(3):
        for a, c in zip(F2.level(l), Ff.level(l)):
            assert np.array_equal(a, c), l
    z2 = _apply(ceg, F2, b)
    assert np.array_equal(z2, _apply(ceg, Ff, b))
    Fo = oce.factorize(A2, perm, 16, 1e-6, 3, 4)
    zo = oce.apply(Fo, b)
    assert np.linalg.norm(z2 - zo) / np.linalg.norm(zo) <= 1e-10
    # the factor made before the update keeps its own values
    assert np.array_equal(_apply(ceg, F1, b), z1)
    assert not np.array_equal(z1, z2)
    # PCG on the updated csb solves the new system
    x = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    it, rel, conv = ceg.pcg_solve(csb, F2, torch.as_tensor(b, device="cuda"), x, 1e-8, 500)
    true = np.linalg.norm(b - A2 @ x.cpu().numpy()) / np.linalg.norm(b)
    assert conv and true <= 1e-8 * 1.01


def test_update_values_rejects_asymmetric(ceg):
    n = 32
    A = wl.poisson2d(n)
    perm = wl.box_perm((n, n), (4, 4))
    csb = ceg.csb_build(A, perm, 16)
    Bad = A.copy().tolil()
    Bad[0, 1] = -0.5
    with pytest.raises(ceg.CEError):
        ceg.csb_update_values(csb, Bad.tocsr())
    F = ceg.ce_factorize(csb, tol=1e-6, levels=2, J=4)
    b = wl.rhs(n * n, 1)
    ref = ceg.ce_factorize(ceg.csb_build(A, perm, 16), tol=1e-6, levels=2, J=4)
    assert np.array_equal(_apply(ceg, F, b), _apply(ceg, ref, b))
