"""GPU parity of the batched path: many independent systems factorized as one
block-diagonal matrix and solved by the per-system PCG, each system against
the FP64 oracle run on that system alone.

The batch changes nothing in any one system's arithmetic: blocks of different
systems never touch, the greedy colouring of a disjoint union is the union of
the per-system colourings, super-blocks stay inside a system and the coarse
remainder is one dense matrix per system.  So the per-system tolerances of the
single-system parity tests apply unchanged (ranks equal except where an
oracle singular value lies within 1e-5 relative of tau; FP64 apply within
1e-10; PCG iterations within +-1 and a true residual <= 1e-8; FP32 form by
its normwise backward error <= 1e-4).
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


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")


def _slices(ws):
    off = np.concatenate([[0], np.cumsum([w.A.shape[0] for w in ws])]).astype(int)
    return [slice(off[s], off[s + 1]) for s in range(len(ws))]


def _anorm(A):
    import scipy.sparse.linalg as spla
    return float(spla.eigsh(A, k=1, which="LA", return_eigenvectors=False)[0])


def _ranks_ok(lev, r_g, rel=1e-5):
    for st in lev.steps:
        if r_g[st.i] == st.r:
            continue
        lo, hi = sorted((r_g[st.i], st.r))
        if not all(k < st.sigma.size and abs(st.sigma[k] - st.tau) <= rel * st.tau
                   for k in range(lo, hi)):
            return False
    return True


@pytest.fixture(scope="module")
def small_batch():
    # five small systems of three grid sizes (the oracle runs each alone)
    ws = wl.make_batch(5, seed=3, choices=(32, 48, 64), levels=3)
    Fos = [oce.factorize(w.A, w.perm, w.B, w.tol, w.levels, w.J) for w in ws]
    return ws, Fos


def test_batched_fp64_matches_oracle_per_system(ceg, small_batch):
    ws, Fos = small_batch
    csb = ceg.csb_build_batched([(w.A, w.perm, w.B) for w in ws])
    F = ceg.ce_factorize_batched(csb, tol=ws[0].tol, levels=ws[0].levels, J=ws[0].J)
    sl = _slices(ws)
    # level by level: the batch's blocks are the systems' blocks in order
    for l in range(ws[0].levels):
        n_g, r_g, c_g, _ = F.level(l)
        o = 0
        for Fo in Fos:
            lev = Fo.levels[l]
            M = len(lev.sizes)
            assert list(n_g[o:o + M]) == list(lev.sizes)
            assert list(c_g[o:o + M]) == list(lev.colour)
            assert _ranks_ok(lev, r_g[o:o + M])
            o += M
        assert o == len(n_g)
    b = np.concatenate([w.b for w in ws])
    z = torch.empty(b.size, dtype=torch.float64, device="cuda")
    ceg.ce_apply(F, _dev(b), z)
    zg = z.cpu().numpy()
    for s, (w, Fo) in enumerate(zip(ws, Fos)):
        zo = oce.apply(Fo, w.b)
        err = np.linalg.norm(zg[sl[s]] - zo) / np.linalg.norm(zo)
        assert err <= 1e-10, (s, err)
    # per-system PCG against the oracle's PCG on each system
    x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
    its, rel, conv = ceg.pcg_solve_batched(csb, F, _dev(b), x, 1e-8, 500)
    xg = x.cpu().numpy()
    for s, (w, Fo) in enumerate(zip(ws, Fos)):
        res_o = oce.pcg(w.A, Fo, w.b, 1e-8, 500)
        true = np.linalg.norm(w.b - w.A @ xg[sl[s]]) / np.linalg.norm(w.b)
        print(f"system {s} n={w.A.shape[0]}: its {its[s]} (oracle {res_o.iters}), res {true:.2e}")
        assert conv[s]
        assert abs(int(its[s]) - res_o.iters) <= 1, (s, its[s], res_o.iters)
        assert true <= 1e-8 * 1.01
        assert rel[s] <= 1e-8


def test_batched_large_row_path_matches_oracle(ceg, small_batch):
    """Every level of the batch through the large-row path (row_shape 3): it
    walks each level's colours in order although a batch's size buckets
    reorder the rows; the same FP64 bar per system.  Then the autotuner
    (which tries that path as shape 3) on the batch, and a solve with its
    choice."""
    ws, Fos = small_batch
    csb = ceg.csb_build_batched([(w.A, w.perm, w.B) for w in ws])
    F = ceg.ce_factorize_batched(csb, tol=ws[0].tol, levels=ws[0].levels, J=ws[0].J, row_shape=3)
    assert all(F.info.big_rows[l] == 1 for l in range(F.info.levels_done))
    for l in range(ws[0].levels):
        n_g, r_g, c_g, _ = F.level(l)
        o = 0
        for Fo in Fos:
            lev = Fo.levels[l]
            M = len(lev.sizes)
            assert list(n_g[o:o + M]) == list(lev.sizes)
            assert _ranks_ok(lev, r_g[o:o + M])
            o += M
    b = np.concatenate([w.b for w in ws])
    z = torch.empty(b.size, dtype=torch.float64, device="cuda")
    ceg.ce_apply(F, _dev(b), z)
    zg = z.cpu().numpy()
    sl = _slices(ws)
    for s, (w, Fo) in enumerate(zip(ws, Fos)):
        zo = oce.apply(Fo, w.b)
        err = np.linalg.norm(zg[sl[s]] - zo) / np.linalg.norm(zo)
        assert err <= 1e-10, (s, err)
    t = ceg.ce_autotune(csb, tol=ws[0].tol, levels=ws[0].levels, J=ws[0].J)
    assert t.shape[1] == 4 and (t[0, 3] > 0).all()
    F2 = ceg.ce_factorize_batched(csb, tol=ws[0].tol, levels=ws[0].levels, J=ws[0].J)
    x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
    its, rel, conv = ceg.pcg_solve_batched(csb, F2, _dev(b), x, 1e-8, 500)
    assert conv.all()


def test_batched_fp32_learned_backward_error(ceg, small_batch):
    ws, Fos = small_batch
    model = ceg.trained_rank_model(steps=1500)
    csb = ceg.csb_build_batched([(w.A, w.perm, w.B) for w in ws])
    F = ceg.ce_factorize(csb, tol=ws[0].tol, levels=ws[0].levels, J=ws[0].J, precision="fp32",
                         rank_model=model)
    sl = _slices(ws)
    b = np.concatenate([w.b for w in ws])
    z = torch.empty(b.size, dtype=torch.float64, device="cuda")
    ceg.ce_apply(F, _dev(b), z)
    zg = z.cpu().numpy()
    for s, (w, Fo) in enumerate(zip(ws, Fos)):
        zs = zg[sl[s]]
        eta = np.linalg.norm(w.b - oce.multiply(Fo, zs)) / (
            _anorm(w.A) * np.linalg.norm(zs) + np.linalg.norm(w.b))
        assert eta <= 1e-4, (s, eta)
    x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
    its, rel, conv = ceg.pcg_solve_batched(csb, F, _dev(b), x, 1e-8, 500)
    xg = x.cpu().numpy()
    for s, w in enumerate(ws):
        res_o = oce.pcg(w.A, Fos[s], w.b, 1e-8, 500)
        true = np.linalg.norm(w.b - w.A @ xg[sl[s]]) / np.linalg.norm(w.b)
        assert conv[s] and true <= 1e-8 * 1.01, (s, true)
        assert its[s] <= 2 * res_o.iters + 2, (s, its[s], res_o.iters)


def test_batched_pcg_graph_reuse_and_zero_rhs(ceg, small_batch):
    """A second call replays the captured graph and gives the same iterates
    bit for bit; a system with b = 0 stops at once with x = 0 while the others
    iterate; the batch equals the single-system path system by system."""
    ws, _ = small_batch
    csb = ceg.csb_build_batched([(w.A, w.perm, w.B) for w in ws])
    F = ceg.ce_factorize(csb, tol=ws[0].tol, levels=ws[0].levels, J=ws[0].J)
    sl = _slices(ws)
    b = np.concatenate([w.b for w in ws])
    b[sl[2]] = 0.0
    x1 = torch.zeros(b.size, dtype=torch.float64, device="cuda")
    x2 = torch.full((b.size,), 7.0, dtype=torch.float64, device="cuda")
    its1, rel1, conv1 = ceg.pcg_solve_batched(csb, F, _dev(b), x1, 1e-8, 500)
    n0 = ceg.launch_count()
    its2, rel2, conv2 = ceg.pcg_solve_batched(csb, F, _dev(b), x2, 1e-8, 500)
    assert ceg.launch_count() - n0 >= its2.max()          # graph kernels are counted
    assert torch.equal(x1, x2)
    assert list(its1) == list(its2) and np.array_equal(rel1, rel2)
    assert its1[2] == 0 and conv1[2] and rel1[2] == 0.0
    assert float(x1[sl[2]].abs().max()) == 0.0
    for s, w in enumerate(ws):
        if s == 2:
            continue
        c1 = ceg.csb_build(w.A, w.perm, w.B)
        F1 = ceg.ce_factorize(c1, tol=w.tol, levels=w.levels, J=w.J)
        xs = torch.zeros(w.A.shape[0], dtype=torch.float64, device="cuda")
        it, rel, conv = ceg.pcg_solve(c1, F1, _dev(w.b), xs, 1e-8, 500)
        assert conv and abs(it - int(its1[s])) <= 1, (s, it, its1[s])
        d = np.linalg.norm(xs.cpu().numpy() - x1[sl[s]].cpu().numpy()) / np.linalg.norm(xs.cpu().numpy())
        assert d <= 1e-7, (s, d)


def test_batched_invalid_coupling_rejected(ceg):
    """A column outside its system's rows is refused on the host."""
    import scipy.sparse as sp
    ws = wl.make_batch(2, seed=0, choices=(32,))
    A = sp.block_diag([w.A for w in ws], format="lil")
    A[0, ws[0].A.shape[0]] = -0.1
    A[ws[0].A.shape[0], 0] = -0.1
    A = A.tocsr()
    from paper_1603_09133_gb300 import _lib
    import ctypes as C
    lib = _lib.load()
    n0 = ws[0].A.shape[0]
    row_off = np.array([0, n0, 2 * n0], np.int64)
    pm = np.concatenate([ws[0].perm, ws[1].perm + n0]).astype(np.int32)
    Bs = np.array([16, 16], np.int32)
    h = C.c_void_p()
    st = lib.csb_build_batched(2, row_off.ctypes.data_as(_lib.I64P),
                               np.ascontiguousarray(A.indptr, np.int64).ctypes.data_as(_lib.I64P),
                               np.ascontiguousarray(A.indices, np.int32).ctypes.data_as(_lib.I32P),
                               np.ascontiguousarray(A.data, np.float64).ctypes.data_as(_lib.DP),
                               pm.ctypes.data_as(_lib.I32P), Bs.ctypes.data_as(_lib.I32P), C.byref(h))
    assert st == ceg.CE_ERR_INVALID_ARG
    # the batch entry point refuses a handle of one system
    single = ceg.csb_build(ws[0].A, ws[0].perm, 16)
    with pytest.raises(ceg.CEError):
        ceg.ce_factorize_batched(single, tol=1e-4, levels=2)


def test_batched_full_size_256_systems(ceg):
    """256 systems with sides drawn from {64, 96, 128, 192, 256} (7.3M rows),
    learned ranks + FP32 blocks + FP64 PCG: every system reaches a true
    residual <= 1e-8; two sampled systems (one of each block size) are checked
    against the oracle's operator on that system alone."""
    ws = wl.make_batch(256)
    model = ceg.trained_rank_model(steps=1500)
    csb = ceg.csb_build_batched([(w.A, w.perm, w.B) for w in ws])
    F = ceg.ce_factorize(csb, tol=1e-4, levels=4, J=4, precision="fp32", rank_model=model)
    sl = _slices(ws)
    b = np.concatenate([w.b for w in ws])
    x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
    its, rel, conv = ceg.pcg_solve_batched(csb, F, _dev(b), x, 1e-8, 500)
    xg = x.cpu().numpy()
    assert conv.all()
    worst = max(np.linalg.norm(w.b - w.A @ xg[sl[s]]) / np.linalg.norm(w.b) for s, w in enumerate(ws))
    print(f"256 systems: iterations {its.min()}..{its.max()}, worst true residual {worst:.2e}")
    assert worst <= 1e-8 * 1.01
    z = torch.empty(b.size, dtype=torch.float64, device="cuda")
    ceg.ce_apply(F, _dev(b), z)
    zg = z.cpu().numpy()
    picks = [next(s for s, w in enumerate(ws) if w.A.shape[0] == 4096),
             next(s for s, w in enumerate(ws) if w.A.shape[0] == 16384)]
    for s in picks:
        w = ws[s]
        Fo = oce.factorize(w.A, w.perm, w.B, 1e-4, 4, 4)
        zs = zg[sl[s]]
        eta = np.linalg.norm(w.b - oce.multiply(Fo, zs)) / (
            _anorm(w.A) * np.linalg.norm(zs) + np.linalg.norm(w.b))
        print(f"system {s} (n={w.A.shape[0]}): backward error {eta:.2e}")
        assert eta <= 1e-4
