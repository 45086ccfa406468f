"""CPU checks of the C-ABI library: it loads, exports every declared symbol,
validates arguments before any CUDA call, and its host planning (block graph,
distance-2 colouring, squared pattern) matches the oracle's.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as wl
from oracle import ce as oce
from paper_1603_09133_gb300 import _lib, build as cebuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    cebuild.build()
    return _lib.load()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "ce.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b((?:ce|csb|pcg|minres)_\w+)\s*\(", src))
    return names


def test_header_and_binding_agree():
    assert _declared_functions() == set(_lib.SIGNATURES)


def test_library_exports_every_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def _csr_args(A, perm):
    A = sp.csr_matrix(A)
    rp = np.ascontiguousarray(A.indptr, np.int64)
    ci = np.ascontiguousarray(A.indices, np.int32)
    v = np.ascontiguousarray(A.data, np.float64)
    pm = np.ascontiguousarray(perm, np.int32)
    return A.shape[0], rp, ci, v, pm


def _build(lib, A, perm, B):
    n, rp, ci, v, pm = _csr_args(A, perm)
    h = C.c_void_p()
    st = lib.csb_build(n, rp.ctypes.data_as(_lib.I64P), ci.ctypes.data_as(_lib.I32P),
                       v.ctypes.data_as(_lib.DP), pm.ctypes.data_as(_lib.I32P), B, C.byref(h))
    return st, h


def test_csb_build_rejects_bad_input(lib):
    A = wl.poisson2d(8)
    perm = np.arange(64)
    # non-symmetric values
    An = A.tolil()
    An[0, 1] = -2.0
    assert _build(lib, An, perm, 16)[0] == _lib.CE_ERR_INVALID_ARG
    # not a permutation
    bad = perm.copy()
    bad[3] = 5
    assert _build(lib, A, bad, 16)[0] == _lib.CE_ERR_INVALID_ARG
    # block size
    assert _build(lib, A, perm, 0)[0] == _lib.CE_ERR_INVALID_ARG
    # null output
    n, rp, ci, v, pm = _csr_args(A, perm)
    assert lib.csb_build(n, rp.ctypes.data_as(_lib.I64P), ci.ctypes.data_as(_lib.I32P),
                         v.ctypes.data_as(_lib.DP), pm.ctypes.data_as(_lib.I32P), 16,
                         None) == _lib.CE_ERR_INVALID_ARG


def _build_raw(lib, n, rp, ci, v, perm, B):
    h = C.c_void_p()
    pm = np.ascontiguousarray(perm, np.int32)
    return lib.csb_build(n, rp.ctypes.data_as(_lib.I64P), ci.ctypes.data_as(_lib.I32P), v.ctypes.data_as(_lib.DP),
                         pm.ctypes.data_as(_lib.I32P), B, C.byref(h))


def test_symmetry_check_sorted_and_unsorted_rows(lib):
    """csb_build rejects a matrix that is not symmetric, in value or in
    pattern, whether its rows come in ascending column order (searched in
    place) or not (sorted into a copy first); the check runs before any CUDA
    call."""
    A = wl.poisson2d(8).tocsr()
    A.sort_indices()
    n, perm = A.shape[0], np.arange(64)
    rp = np.ascontiguousarray(A.indptr, np.int64)
    ci = np.ascontiguousarray(A.indices, np.int32)
    v = np.ascontiguousarray(A.data, np.float64)
    rng = np.random.default_rng(0)

    def shuffled(ci, v):
        ci2, v2 = ci.copy(), v.copy()
        for a in range(n):
            idx = np.arange(rp[a], rp[a + 1])
            p = rng.permutation(idx)
            ci2[idx], v2[idx] = ci[p], v[p]
        return ci2, v2

    for unsorted in (False, True):
        c0, v0 = shuffled(ci, v) if unsorted else (ci, v)
        # one value changed on one side of the diagonal
        v1 = v0.copy()
        e = next(q for q in range(rp[0], rp[1]) if c0[q] == 1)
        v1[e] = -2.0
        assert _build_raw(lib, n, rp, c0, v1, perm, 16) == _lib.CE_ERR_INVALID_ARG, unsorted
    # a pattern entry (0, 9) without its mirror (9, 0)
    An = A.tolil()
    An[0, 9] = -0.5
    An = An.tocsr()
    An.sort_indices()
    rp2 = np.ascontiguousarray(An.indptr, np.int64)
    assert _build_raw(lib, n, rp2, np.ascontiguousarray(An.indices, np.int32),
                      np.ascontiguousarray(An.data, np.float64), perm, 16) == _lib.CE_ERR_INVALID_ARG


def test_wait_expiry_hook_validates_before_any_cuda_call(lib):
    status = np.zeros(8, np.int32)
    for kernel, ms in ((2, 20.0), (0, 0.0), (0, 5000.0), (1, -1.0)):
        assert lib.ce_debug_wait_expiry(kernel, ms, status.ctypes.data_as(_lib.I32P), None) == \
            _lib.CE_ERR_INVALID_ARG
    assert lib.ce_debug_wait_expiry(0, 20.0, None, None) == _lib.CE_ERR_INVALID_ARG


def test_strerror(lib):
    for s in range(7):
        assert lib.ce_strerror(s)


def _plan(lib, A, perm, B):
    n, rp, ci, v, pm = _csr_args(A, perm)
    M = (n + B - 1) // B
    col = np.zeros(M, np.int32)
    nc = C.c_int()
    npairs = C.c_int64()
    nclose = C.c_int64()
    st = lib.ce_plan_level1(n, rp.ctypes.data_as(_lib.I64P), ci.ctypes.data_as(_lib.I32P),
                            pm.ctypes.data_as(_lib.I32P), B, col.ctypes.data_as(_lib.I32P),
                            C.byref(nc), C.byref(npairs), C.byref(nclose))
    assert st == _lib.CE_OK
    return col, nc.value, npairs.value, nclose.value


@pytest.mark.parametrize("name", ["poisson2d_64_B16", "poisson2d_512_B32", "poisson3d_64_B64"])
def test_host_colouring_matches_oracle(lib, name):
    w = wl.make_workload(name)
    col, nc, npairs, nclose = _plan(lib, w.A, w.perm, w.B)
    S, sizes = oce.initial_blocks(w.A, w.perm, w.B)
    nbr = oce._block_graph(S, len(sizes))
    ocol = np.array(oce.distance2_colouring(nbr))
    assert np.array_equal(col, ocol)
    assert nc == ocol.max() + 1
    assert nclose == len(S)
    # squared pattern: pairs with a common neighbour (or adjacent)
    sq = set()
    for j in range(len(sizes)):
        for a in nbr[j]:
            for b in nbr[j]:
                if a <= b:
                    sq.add((a, b))
    assert npairs == len(sq)


@pytest.mark.parametrize("name", ["poisson2d_64_B16", "poisson2d_512_B32", "poisson3d_64_B64"])
def test_host_colourings_match_oracle(lib, name):
    """The three elimination orders of ce_opts.coloring as the planner makes
    them: natural (block i is colour i), distance 2, and the distance-1 order
    (adjacent blocks differ; neighbours of a block that share a colour lie
    below it), each equal to the oracle's."""
    w = wl.make_workload(name)
    S, sizes = oce.initial_blocks(w.A, w.perm, w.B)
    nbr = oce._block_graph(S, len(sizes))
    A = w.A.tocsr()
    rp = np.ascontiguousarray(A.indptr, np.int64)
    ci = np.ascontiguousarray(A.indices, np.int32)
    pm = np.ascontiguousarray(w.perm, np.int32)
    want = {0: list(range(len(sizes))), 1: oce.distance2_colouring(nbr), 2: oce.distance1_colouring(nbr)}
    for coloring, ocol in want.items():
        col = np.zeros(len(sizes), np.int32)
        nc = C.c_int()
        st = lib.ce_plan_colours(A.shape[0], rp.ctypes.data_as(_lib.I64P), ci.ctypes.data_as(_lib.I32P),
                                 pm.ctypes.data_as(_lib.I32P), w.B, coloring, col.ctypes.data_as(_lib.I32P),
                                 C.byref(nc))
        assert st == _lib.CE_OK
        assert list(col) == list(ocol), coloring
        assert nc.value == max(ocol) + 1
    assert lib.ce_plan_colours(A.shape[0], rp.ctypes.data_as(_lib.I64P), ci.ctypes.data_as(_lib.I32P),
                               pm.ctypes.data_as(_lib.I32P), w.B, 3, None, None) == _lib.CE_ERR_INVALID_ARG


def test_host_plan_ragged_and_natural(lib):
    A = wl.poisson2d(10)
    col, nc, npairs, nclose = _plan(lib, A, np.arange(100), 16)
    assert len(col) == 7
    S, sizes = oce.initial_blocks(A, np.arange(100), 16)
    assert sizes[-1] == 4
    ocol = oce.distance2_colouring(oce._block_graph(S, len(sizes)))
    assert list(col) == ocol


def _groups_c(lib, rank, J, nmax):
    rank = np.ascontiguousarray(rank, np.int32)
    fc = np.zeros(rank.size + 1, np.int32)
    ng = C.c_int()
    st = lib.ce_plan_groups(rank.size, rank.ctypes.data_as(_lib.I32P), J, nmax,
                            fc.ctypes.data_as(_lib.I32P), C.byref(ng))
    assert st == _lib.CE_OK
    return [(int(fc[g]), int(fc[g + 1])) for g in range(ng.value)]


def test_host_groups_match_oracle(lib):
    """The library's super-blocks (Section 2.4, with the 64-row cap) equal the
    oracle's on ragged and random rank vectors, bit for bit."""
    rng = np.random.default_rng(11)
    cases = [([16] * 8, 4, 64), ([16] * 7, 4, 64), ([40, 30, 20, 10, 5], 4, 64),
             ([64, 64, 1, 0, 0], 4, 64), ([0, 0, 0], 8, 0), ([33] * 9, 8, 64)]
    for _ in range(200):
        M = int(rng.integers(1, 40))
        J = int(rng.choice([1, 2, 4, 8]))
        cases.append((list(rng.integers(0, 40, M)), J, int(rng.choice([0, 16, 64, 10 ** 6]))))
    for rank, J, nmax in cases:
        assert _groups_c(lib, rank, J, nmax) == oce._groups(list(rank), J, nmax), (rank, J, nmax)


def test_host_groups_reject_bad_input(lib):
    r = np.array([1, -1, 2], np.int32)
    fc = np.zeros(4, np.int32)
    ng = C.c_int()
    assert lib.ce_plan_groups(3, r.ctypes.data_as(_lib.I32P), 4, 64, fc.ctypes.data_as(_lib.I32P),
                              C.byref(ng)) == _lib.CE_ERR_INVALID_ARG
    r[1] = 1
    assert lib.ce_plan_groups(3, r.ctypes.data_as(_lib.I32P), 0, 64, fc.ctypes.data_as(_lib.I32P),
                              C.byref(ng)) == _lib.CE_ERR_INVALID_ARG


def _deps_c(lib, A, perm, B):
    n, rp, ci, v, pm = _csr_args(A, perm)
    M = (n + B - 1) // B
    ptr = np.zeros(M + 1, np.int64)
    nd = C.c_int64()
    args = (n, rp.ctypes.data_as(_lib.I64P), ci.ctypes.data_as(_lib.I32P), pm.ctypes.data_as(_lib.I32P), B)
    assert lib.ce_plan_level1_deps(*args, ptr.ctypes.data_as(_lib.I64P), None, 0, C.byref(nd)) == _lib.CE_OK
    idx = np.zeros(max(nd.value, 1), np.int32)
    if nd.value:
        assert lib.ce_plan_level1_deps(*args, None, idx.ctypes.data_as(_lib.I32P), nd.value - 1,
                                       None) == _lib.CE_ERR_INVALID_ARG
    assert lib.ce_plan_level1_deps(*args, ptr.ctypes.data_as(_lib.I64P), idx.ctypes.data_as(_lib.I32P),
                                   idx.size, C.byref(nd)) == _lib.CE_OK
    return ptr, idx[:nd.value]


def _random_spd_pattern(n, seed):
    rng = np.random.default_rng(seed)
    R = sp.random(n, n, density=3.0 / n, random_state=rng, format="csr")
    A = (R + R.T + sp.identity(n)).tocsr()
    A.data[:] = 1.0
    return A, rng.permutation(n)


@pytest.mark.parametrize("case", ["poisson2d_64_B16", "poisson2d_512_B32", "poisson3d_64_B64", "random"])
def test_host_row_waits_cover_every_conflict(lib, case):
    """Level 1's persistent launch is race-free: any two rows whose work can
    touch a common block pair (distance <= 2 in the block graph: a shared
    Schur target, or one row's target inside the other's row) have different
    colours, and the later colour waits for the earlier one; no other waits."""
    if case == "random":
        A, perm = _random_spd_pattern(3000, 4)
        B = 16
    else:
        w = wl.make_workload(case)
        A, perm, B = w.A, w.perm, w.B
    n = A.shape[0]
    M = (n + B - 1) // B
    col, _, _, _ = _plan(lib, A, perm, B)
    ptr, idx = _deps_c(lib, A, perm, B)
    # block graph of P A P^T (with the diagonal) and its square, brute force
    iperm = np.empty(n, np.int64)
    iperm[np.asarray(perm)] = np.arange(n)
    Ac = sp.coo_matrix(A)
    G = sp.csr_matrix((np.ones(Ac.nnz), (iperm[Ac.row] // B, iperm[Ac.col] // B)), shape=(M, M))
    G = ((G + sp.identity(M)) > 0).astype(np.int64)
    G2 = sp.coo_matrix((G @ G) > 0)
    conflicts = {(int(i), int(k)) for i, k in zip(G2.row, G2.col) if i != k}
    assert all(col[i] != col[k] for i, k in conflicts)
    want = [set() for _ in range(M)]
    for i, k in conflicts:
        if col[k] < col[i]:
            want[i].add(k)
    got = [set(idx[ptr[i]:ptr[i + 1]].tolist()) for i in range(M)]
    assert all(len(idx[ptr[i]:ptr[i + 1]]) == len(got[i]) for i in range(M))   # no duplicates
    assert got == want


def _next_level_c(lib, A, perm, B, rank, J, nmax):
    n, rp, ci, v, pm = _csr_args(A, perm)
    M = (n + B - 1) // B
    r = np.ascontiguousarray(rank, np.int32)
    nn = np.zeros(M, np.int32)
    col = np.zeros(M, np.int32)
    nM = C.c_int()
    ncl = C.c_int64()
    st = lib.ce_plan_next_level(n, rp.ctypes.data_as(_lib.I64P), ci.ctypes.data_as(_lib.I32P),
                                pm.ctypes.data_as(_lib.I32P), B, r.ctypes.data_as(_lib.I32P), J, nmax,
                                nn.ctypes.data_as(_lib.I32P), col.ctypes.data_as(_lib.I32P), C.byref(nM),
                                C.byref(ncl))
    assert st == _lib.CE_OK
    return nn[:nM.value], col[:nM.value], ncl.value


@pytest.mark.parametrize("kind,n,box,tol,J", [("p2", 64, (4, 4), 1e-3, 4), ("p2", 128, (8, 4), 1e-4, 4),
                                              ("p3", 16, (4, 4, 4), 1e-4, 8), ("grf", 64, (4, 4), 1e-4, 4)])
def test_host_next_level_matches_oracle(lib, kind, n, box, tol, J):
    """Level 2 as the library plans it from level 1 and the oracle's level-1
    ranks (super-blocks capped at 64 rows, sizes, block pattern, colouring)
    equals the oracle's own level 2, bit for bit."""
    if kind == "p3":
        A, perm = wl.poisson3d(n), wl.box_perm((n, n, n), box)
    elif kind == "grf":
        A, perm = wl.diffusion2d(wl.grf2d(n, 3)), wl.box_perm((n, n), box)
    else:
        A, perm = wl.poisson2d(n), wl.box_perm((n, n), box)
    B = int(np.prod(box))
    F = oce.factorize(A, perm, B, tol, 2, J, nmax=64)
    lev1, lev2 = F.levels
    nn, col, ncl = _next_level_c(lib, A, perm, B, lev1.ranks, J, 64)
    assert list(nn) == list(lev2.sizes)
    assert list(col) == list(lev2.colour)
    assert ncl == len(lev2.pairs)


def test_host_next_level_rule_on_random_ranks(lib):
    """The coarsening rule restated by brute force on random ranks: sizes are
    the children's rank sums; a super-block pair exists when a pair of the
    level-1 squared pattern with non-zero ranks on both sides lies inside it,
    and every super-block (an empty one too) keeps its diagonal."""
    rng = np.random.default_rng(5)
    A, perm = wl.poisson2d(64), wl.box_perm((64, 64), (4, 4))
    B, J = 16, 4
    S, sizes = oce.initial_blocks(A, perm, B)
    M = len(sizes)
    nbr = oce._block_graph(S, M)
    sq = set()
    for j in range(M):
        for a in nbr[j]:
            for b in nbr[j]:
                if a <= b:
                    sq.add((a, b))
    for trial in range(5):
        rank = rng.integers(0, B + 1, M)
        rank[rng.random(M) < 0.2] = 0
        for nmax in (64, 10 ** 6):
            groups = oce._groups(list(rank), J, nmax)
            parent = np.empty(M, int)
            for g, (a, b) in enumerate(groups):
                parent[a:b] = g
            want_n = [int(rank[a:b].sum()) for a, b in groups]
            pairs = {(parent[a], parent[b]) for a, b in sq if rank[a] > 0 and rank[b] > 0}
            pairs |= {(g, g) for g in range(len(groups))}
            nn, col, ncl = _next_level_c(lib, A, perm, B, rank, J, nmax)
            assert list(nn) == want_n
            assert ncl == len(pairs)
            g_nbr = [set() for _ in groups]
            for a, b in pairs:
                g_nbr[a].add(b)
                g_nbr[b].add(a)
            for i in range(len(groups)):
                g_nbr[i].add(i)
            assert list(col) == oce.distance2_colouring(g_nbr)


def _work_formula(F, es):
    """Algorithmic work of level 1 from the oracle's own steps: far blocks as
    filled when the row ran, close widths from the W blocks it produced."""
    lev = F.levels[0]
    fl = by = 0.0
    for st in lev.steps:
        i, n, r = st.i, st.n, st.r
        m = n - r

        def wid(k):
            return lev.ranks[k] if lev.colour[k] < lev.colour[i] else lev.sizes[k]
        mF = sum(wid(k) for k in st.far)
        ws = [W.shape[1] for t, W in st.targets if t != i]
        Wc, W2 = sum(ws), sum(w * w for w in ws)
        fl += (2 * mF * n * n + (12 * n ** 3 if mF > 0 else 0) + 4 * n ** 3 + 2 * n * n * Wc + 2 * n * r * mF
               + m ** 3 / 3 + m * m * (r + Wc) + m * ((r + Wc) ** 2 + r * r + W2))
        by += es * (2 * n * n + n * Wc + n * mF + m * m + m * (r + Wc) + r * r + r * Wc + r * mF
                    + (Wc * Wc + W2))
    return fl, by


@pytest.mark.parametrize("kind,n,box,tol", [("p2", 64, (4, 4), 1e-3), ("p2", 96, (8, 4), 1e-4),
                                            ("p3", 16, (4, 4, 4), 1e-4)])
def test_host_work_count_matches_oracle_steps(lib, kind, n, box, tol):
    """The algorithmic flops and bytes behind the roofline (ce_info.level_flops
    / level_bytes) equal the stated per-row formula evaluated on the oracle's
    own level-1 steps: the library's far lists hold exactly the fill present
    when a row runs (no zero blocks counted), its close widths those of the W
    blocks the oracle forms."""
    if kind == "p3":
        A, perm = wl.poisson3d(n), wl.box_perm((n, n, n), box)
    else:
        A, perm = wl.poisson2d(n), wl.box_perm((n, n), box)
    B = int(np.prod(box))
    F = oce.factorize(A, perm, B, tol, 1, 4, nmax=64)
    nn, rp, ci, v, pm = _csr_args(A, perm)
    rk = np.ascontiguousarray(F.levels[0].ranks, np.int32)
    for es in (4, 8):
        fl, by = C.c_double(), C.c_double()
        st = lib.ce_plan_level1_work(nn, rp.ctypes.data_as(_lib.I64P), ci.ctypes.data_as(_lib.I32P),
                                     pm.ctypes.data_as(_lib.I32P), B, rk.ctypes.data_as(_lib.I32P), es,
                                     C.byref(fl), C.byref(by))
        assert st == _lib.CE_OK
        f2, b2 = _work_formula(F, es)
        assert fl.value == pytest.approx(f2, rel=1e-12) and by.value == pytest.approx(b2, rel=1e-12)


def test_host_exports_reject_bad_arguments(lib):
    A, perm = wl.poisson2d(16), wl.box_perm((16, 16), (4, 4))
    n, rp, ci, v, pm = _csr_args(A, perm)
    M = n // 16
    base = (n, rp.ctypes.data_as(_lib.I64P), ci.ctypes.data_as(_lib.I32P), pm.ctypes.data_as(_lib.I32P), 16)
    fl, by = C.c_double(), C.c_double()
    nM, ncl = C.c_int(), C.c_int64()
    out = np.zeros(M, np.int32)
    for bad in (np.full(M, 17, np.int32), np.full(M, -1, np.int32)):      # r_i outside [0, n_i]
        assert lib.ce_plan_level1_work(*base, bad.ctypes.data_as(_lib.I32P), 8, C.byref(fl),
                                       C.byref(by)) == _lib.CE_ERR_INVALID_ARG
        assert lib.ce_plan_next_level(*base, bad.ctypes.data_as(_lib.I32P), 4, 64,
                                      out.ctypes.data_as(_lib.I32P), out.ctypes.data_as(_lib.I32P),
                                      C.byref(nM), C.byref(ncl)) == _lib.CE_ERR_INVALID_ARG
    ok = np.full(M, 4, np.int32)
    assert lib.ce_plan_level1_work(*base, ok.ctypes.data_as(_lib.I32P), 2, C.byref(fl),
                                   C.byref(by)) == _lib.CE_ERR_INVALID_ARG          # element size
    assert lib.ce_plan_next_level(*base, ok.ctypes.data_as(_lib.I32P), 0, 64, None, None, C.byref(nM),
                                  None) == _lib.CE_ERR_INVALID_ARG                    # J
    pm_bad = pm.copy()
    pm_bad[0] = pm_bad[1]                                                             # not a permutation
    nd = C.c_int64()
    assert lib.ce_plan_level1_deps(n, rp.ctypes.data_as(_lib.I64P), ci.ctypes.data_as(_lib.I32P),
                                   pm_bad.ctypes.data_as(_lib.I32P), 16, None, None, 0,
                                   C.byref(nd)) == _lib.CE_ERR_INVALID_ARG
    # valid: level 2 of 16 blocks of rank 4 joined by 4 is 4 blocks of 16 rows
    assert lib.ce_plan_next_level(*base, ok.ctypes.data_as(_lib.I32P), 4, 64, out.ctypes.data_as(_lib.I32P),
                                  None, C.byref(nM), None) == _lib.CE_OK
    assert nM.value == 4 and list(out[:4]) == [16] * 4
