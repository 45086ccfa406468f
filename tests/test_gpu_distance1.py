"""GPU parity of the distance-1 elimination order (ce_opts.coloring = 2)
against the oracle in the same order (order="colour1").

Rows of a colour are never adjacent and share no neighbour of a lower colour,
so no fill block lies between them when they run and neither reads a block
the other writes; they may share close neighbours, whose pairs both Schur
updates add to (atomically on the GPU, in an order fixed by the launch's
timing), so GPU and oracle agree up to the rounding of those sums: colours
bit-exact, ranks equal except within 1e-5 relative of tau, FP64 apply within
1e-10, FP32 backward error <= 1e-4, PCG iterations +-1.  The fewer colours
are the point: the level times of both orders are printed.
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


def _ranks_agree(lev, r_g, rel=1e-5):
    bad = []
    for st in lev.steps:
        if r_g[st.i] == st.r:
            continue
        lo, hi = sorted((r_g[st.i], st.r))
        if not all(k < st.sigma.size and abs(st.sigma[k] - st.tau) <= rel * st.tau for k in range(lo, hi)):
            bad.append((st.i, st.r, int(r_g[st.i])))
    return bad


def _check(ceg, A, perm, B, tol, levels, J, b, precision, nmax=0):
    Fo = oce.factorize(A, perm, B, tol, levels, J, order="colour1", nmax=nmax)
    csb = ceg.csb_build(A, perm, B)
    F = ceg.ce_factorize(csb, tol=tol, levels=levels, J=J, precision=precision, coloring=2, nmax=nmax)
    F2 = ceg.ce_factorize(csb, tol=tol, levels=levels, J=J, precision=precision, coloring=1, nmax=nmax)
    same = True
    for l, lev in enumerate(Fo.levels):
        if not same:
            break
        n_g, r_g, c_g, _ = F.level(l)
        assert list(n_g) == list(lev.sizes) and list(c_g) == list(lev.colour), l
        if precision == "fp64":
            assert _ranks_agree(lev, r_g) == [], l
        same = list(r_g) == list(lev.ranks)
    r = torch.as_tensor(b, device="cuda")
    z = torch.empty_like(r)
    ceg.ce_apply(F, r, z)
    torch.cuda.synchronize()
    zh = z.cpu().numpy()
    if precision == "fp64":
        zo = oce.apply(Fo, b)
        err = np.linalg.norm(zh - zo) / np.linalg.norm(zo)
        assert err <= 1e-10, err
    else:
        import scipy.sparse.linalg as spla
        anorm = float(spla.eigsh(A, k=1, which="LA", return_eigenvectors=False)[0])
        err = np.linalg.norm(b - oce.multiply(Fo, zh)) / (anorm * np.linalg.norm(zh) + np.linalg.norm(b))
        assert err <= 1e-4, err
    x = torch.zeros_like(r)
    it, rel, conv = ceg.pcg_solve(csb, F, r, x, 1e-8, 300)
    torch.cuda.synchronize()
    true = np.linalg.norm(b - A @ x.cpu().numpy()) / np.linalg.norm(b)
    it_o = oce.pcg(A, Fo, b, 1e-8, 300).iters
    nl = F.info.levels_done
    print(f"{precision}: error {err:.2e}, PCG {it} (oracle {it_o}); colours d1 {list(F.info.colours[:nl])} "
          f"d2 {list(F2.info.colours[:nl])}; level ms d1 {[round(F.info.level_ms[l], 2) for l in range(nl)]} "
          f"d2 {[round(F2.info.level_ms[l], 2) for l in range(nl)]}")
    assert conv and true <= 1e-8 * 1.01
    assert abs(it - it_o) <= 1
    return F, F2


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_distance1_small(ceg, precision):
    w = wl.make_workload("poisson2d_64_B16")
    _check(ceg, w.A, w.perm, w.B, w.tol, w.levels, w.J, w.b, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_distance1_512(ceg, precision):
    w = wl.make_workload("poisson2d_512_B32")
    F, F2 = _check(ceg, w.A, w.perm, w.B, w.tol, w.levels, w.J, w.b, precision, nmax=64)
    nl = F.info.levels_done
    assert F.info.colours[0] < F2.info.colours[0]
    assert sum(F.info.colours[:nl]) < sum(F2.info.colours[:nl])


def test_distance1_large_rows_3d(ceg):
    """Large rows of one distance-1 colour share Schur targets: the grouped
    GEMM adds those products atomically (3D 32^3, second level: 64 blocks of
    up to ~260 rows in a 4^3 grid of super-blocks)."""
    A = wl.poisson3d(32)
    perm = wl.box_perm((32, 32, 32), (4, 4, 4))
    F, _ = _check(ceg, A, perm, 64, 1e-4, 2, 8, wl.rhs(A.shape[0], 5), "fp64")
    assert F.info.big_rows[1] == 1
