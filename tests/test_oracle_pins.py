"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: the exact
block Cholesky that CE reduces to when nothing is dropped (eq. bl_chol), the
dense Cholesky solve, an independently written block IC(0), the structural
worked example of Section 2, the pattern bounds of Section 2.4 (eq. L, eq.
bsp, Proposition gl), invariances that any correct implementation has, and the
trends of the paper's Tables err / num_it.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import workloads as wl
from oracle import ce

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _minv_dense(F, N):
    return np.stack([ce.apply(F, e) for e in np.eye(N)], axis=1)


def _problem(kind, n, box):
    if kind == "p2":
        A = wl.poisson2d(n)
        perm = wl.box_perm((n, n), box)
    else:
        A = wl.poisson3d(n)
        perm = wl.box_perm((n, n, n), box)
    return A, perm, int(np.prod(box))


# --------------------------------------------------------------------------
# exactness: tol = 0 reduces CE to exact block Cholesky (eq. bl_chol)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kind,n,box,levels,J", [
    ("p2", 16, (4, 4), 2, 4),
    ("p2", 32, (4, 4), 2, 4),
    ("p3", 8, (2, 2, 2), 2, 8),
])
def test_tol0_reproduces_A(kind, n, box, levels, J):
    A, perm, B = _problem(kind, n, box)
    N = A.shape[0]
    F = ce.factorize(A, perm, B, 0.0, levels, J)
    Minv = _minv_dense(F, N)
    M = np.linalg.inv(Minv)
    Ad = A.toarray()
    assert np.linalg.norm(M - Ad) / np.linalg.norm(Ad) < 1e-13
    b = wl.rhs(N, 0)
    x_ref = sla.cho_solve(sla.cho_factor(Ad), b)
    assert np.linalg.norm(ce.apply(F, b) - x_ref) / np.linalg.norm(x_ref) < 1e-12
    res = ce.pcg(A, F, b, 1e-8, 50)
    assert res.converged and res.iters == 1


@pytest.mark.parametrize("kind,n,box,levels,J", [
    ("p2", 32, (4, 4), 2, 4),
    ("p2", 32, (8, 4), 3, 4),
    ("p3", 8, (2, 2, 2), 2, 8),
])
def test_forward_product_tol0_is_A(kind, n, box, levels, J):
    # M x = Q^T L L^T Q x equals A x when nothing is dropped (eq. bl_chol),
    # checked without any inverse
    A, perm, B = _problem(kind, n, box)
    F = ce.factorize(A, perm, B, 0.0, levels, J)
    x = wl.rhs(A.shape[0], 12)
    assert np.linalg.norm(ce.multiply(F, x) - A @ x) / np.linalg.norm(A @ x) < 1e-13


def test_forward_product_inverts_apply():
    w = wl.make_workload("poisson2d_64_B16")
    F = ce.factorize(w.A, w.perm, w.B, 1e-2, w.levels, w.J)
    b = w.b
    assert np.linalg.norm(ce.multiply(F, ce.apply(F, b)) - b) / np.linalg.norm(b) < 1e-12
    # and M approximates A to about the truncation level
    rel = np.linalg.norm(ce.multiply(F, b) - w.A @ b) / np.linalg.norm(w.A @ b)
    assert 0 < rel < 1e-2


def test_levels0_is_dense_cholesky():
    A, perm, B = _problem("p2", 16, (4, 4))
    F = ce.factorize(A, perm, B, 1e-2, 0, 4)
    assert len(F.levels) == 0 and F.coarse_L.shape == (256, 256)
    b = wl.rhs(256, 3)
    x = ce.apply(F, b)
    x_ref = sla.solve(A.toarray(), b, assume_a="pos")
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-13


def test_single_block_is_exact():
    A, perm, _ = _problem("p2", 8, (4, 4))
    F = ce.factorize(A, perm, 64, 1e-2, 2, 4)      # B == N: one block
    st = F.levels[0].steps[0]
    assert st.r == 0 and st.far == []
    b = wl.rhs(64, 1)
    x_ref = sla.solve(A.toarray(), b, assume_a="pos")
    assert np.linalg.norm(ce.apply(F, b) - x_ref) / np.linalg.norm(x_ref) < 1e-13


def test_ragged_last_block_exact():
    # N = 100, B = 16: six blocks of 16 and a last block of 4
    A = wl.poisson2d(10)
    perm = np.arange(100, dtype=np.int32)
    F = ce.factorize(A, perm, 16, 0.0, 2, 2)
    assert F.sizes0 == [16] * 6 + [4]
    b = wl.rhs(100, 2)
    x_ref = sla.solve(A.toarray(), b, assume_a="pos")
    assert np.linalg.norm(ce.apply(F, b) - x_ref) / np.linalg.norm(x_ref) < 1e-12


# --------------------------------------------------------------------------
# eps >= 1 drops every far block: CE is then block IC(0) in the same order
# --------------------------------------------------------------------------
def _block_ic0_minv(A0, sizes, pairs, order):
    """Block incomplete Cholesky with no fill outside ``pairs`` (independent).

    Dense bookkeeping in A_0 coordinates: process blocks in ``order``; the
    pivot block is factorized, the column below scaled, and the Schur update
    applied only where the block pair belongs to the pattern.
    """
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(int)
    sl = [slice(off[j], off[j + 1]) for j in range(len(sizes))]
    pat = set(pairs) | {(k, i) for (i, k) in pairs}
    A = A0.copy()
    N = A.shape[0]
    L = np.zeros((N, N))
    done = set()
    for i in order:
        Lii = np.linalg.cholesky(A[sl[i], sl[i]])
        L[sl[i], sl[i]] = Lii
        nb = [k for k in range(len(sizes)) if (i, k) in pat and k != i and k not in done]
        Lki = {k: sla.solve_triangular(Lii, A[sl[i], sl[k]], lower=True).T for k in nb}
        for k in nb:
            L[sl[k], sl[i]] = Lki[k]
        for k in nb:
            for l in nb:
                if (k, l) in pat:
                    A[sl[k], sl[l]] -= Lki[k] @ Lki[l].T
        done.add(i)
    return L


def test_large_eps_is_block_ic0():
    A, perm, B = _problem("p2", 16, (4, 4))
    F = ce.factorize(A, perm, B, 2.0, 1, 4)
    lev = F.levels[0]
    assert all(r == 0 for r in lev.ranks)
    A0 = A.toarray()[np.ix_(perm, perm)]
    L = _block_ic0_minv(A0, lev.sizes, lev.pairs, lev.order)
    M0 = L @ L.T
    b = wl.rhs(256, 5)
    x_ic = np.empty(256)
    x_ic[perm] = np.linalg.solve(M0, b[perm])
    x = ce.apply(F, b)
    assert np.linalg.norm(x - x_ic) / np.linalg.norm(x_ic) < 1e-12


# --------------------------------------------------------------------------
# per-step properties (Section 2.2): orthogonal U, rank rule, SPD pivots
# --------------------------------------------------------------------------
def test_step_properties_cfg_small():
    w = wl.make_workload("poisson2d_64_B16")
    F = ce.factorize(w.A, w.perm, w.B, w.tol, w.levels, w.J)
    nsteps = 0
    for lev in F.levels:
        assert sorted(st.i for st in lev.steps) == list(range(len(lev.sizes)))
        for st in lev.steps:
            nsteps += 1
            assert np.abs(st.U.T @ st.U - np.eye(st.n)).max() < 1e-13
            if st.sigma.size:
                assert np.all(st.sigma[:st.r] > st.tau)
                assert np.all(st.sigma[st.r:] <= st.tau)
                assert st.tau == pytest.approx(w.tol * st.sigma[0])
            else:
                assert st.r == 0
            if st.n - st.r:
                assert np.all(np.diag(st.Lhat) > 0)
    assert nsteps == sum(len(l.sizes) for l in F.levels)


def test_first_colour_has_no_far_blocks():
    # nothing is eliminated before the first colour: those rows are eliminated
    # whole, as the first block row of Section 2.1
    w = wl.make_workload("poisson2d_64_B16")
    F = ce.factorize(w.A, w.perm, w.B, w.tol, 1, w.J)
    lev = F.levels[0]
    for st in lev.steps:
        if lev.colour[st.i] == 0:
            assert st.far == [] and st.r == 0


def test_distance2_colouring_is_valid():
    A, perm, B = _problem("p2", 32, (4, 4))
    S, sizes = ce.initial_blocks(A, perm, B)
    nbr = ce._block_graph(S, len(sizes))
    col = ce.distance2_colouring(nbr)
    for c in set(col):
        members = [i for i in range(len(sizes)) if col[i] == c]
        seen = set()
        for i in members:
            assert not (nbr[i] & seen)
            seen |= nbr[i]
    # 4-neighbour box grid: a perfect code needs at least 5 colours
    assert max(col) + 1 >= 5


# --------------------------------------------------------------------------
# structural worked example (Section 2, 4 block rows)
# --------------------------------------------------------------------------
def _read_golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, *vals = line.split()
        out[key] = [tuple(int(x) - 1 for x in v.split("-")) for v in vals]
    return out


def test_four_block_worked_example():
    g = _read_golden("four_block_example.txt")
    Bs = 4
    rng = np.random.default_rng(11)
    A = np.zeros((16, 16))
    for (i, k) in g["pattern"]:
        X = rng.standard_normal((Bs, Bs))
        if i == k:
            X = X @ X.T + 4 * Bs * np.eye(Bs)
        A[i * Bs:(i + 1) * Bs, k * Bs:(k + 1) * Bs] = X
        A[k * Bs:(k + 1) * Bs, i * Bs:(i + 1) * Bs] = X.T
    F = ce.factorize(sp.csr_matrix(A), np.arange(16), Bs, 1e-12, 2, J=1, order="natural")
    lev = F.levels[0]
    assert lev.order == [0, 1, 2, 3]
    close = {}
    for (i, k) in g["pattern"]:
        close.setdefault(i, set()).add(k)
        close.setdefault(k, set()).add(i)
    far_seen = set()
    for st in lev.steps:
        # L_1 inherits the block structure of A_0 (eq. L)
        assert {t for t, _ in st.targets} == close[st.i]
        far_seen |= {(min(st.i, k), max(st.i, k)) for k in st.far}
    assert far_seen == set(g["far"])
    # block 1 has no far zone and is eliminated whole
    assert lev.ranks[0] == 0
    nxt = F.levels[1]
    off = {(i, k) for (i, k) in nxt.pairs if i != k and nxt.sizes[i] and nxt.sizes[k]}
    assert off == set(g["remainder_offdiag"])
    x_ref = np.linalg.solve(A, np.ones(16))
    x = ce.apply(F, np.ones(16))
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-8


# --------------------------------------------------------------------------
# pattern bounds (Section 2.4: eq. L, eq. bsp, Proposition gl) and dimensions
# --------------------------------------------------------------------------
def _square_pattern(pairs, M):
    nbr = [set([i]) for i in range(M)]
    for (i, k) in pairs:
        nbr[i].add(k)
        nbr[k].add(i)
    out = set()
    for j in range(M):
        for a in nbr[j]:
            for b in nbr[j]:
                if a <= b:
                    out.add((a, b))
    return out


def test_pattern_bounds_and_dimensions():
    A, perm, B = _problem("p2", 32, (4, 4))
    J = 4
    F = ce.factorize(A, perm, B, 1e-3, 3, J)
    N = A.shape[0]
    eliminated = 0
    for li, lev in enumerate(F.levels):
        M = len(lev.sizes)
        nonempty = {(i, k) for (i, k) in lev.pairs if lev.sizes[i] and lev.sizes[k]}
        bsp = len(nonempty) * 2 - sum(1 for (i, k) in nonempty if i == k)
        nL = sum(1 + len([t for t, W in st.targets if W.size]) for st in lev.steps if st.n - st.r)
        assert nL <= 2 * bsp                                 # eq. L
        if li + 1 < len(F.levels):
            sq = _square_pattern(lev.pairs, M)
            coarse_sq = {(i // J, k // J) for (i, k) in sq}
            nxt = F.levels[li + 1]
            assert set(nxt.pairs) - {(I, I) for I in range(len(nxt.sizes))} <= coarse_sq  # eq. bsp
        eliminated += sum(st.n - st.r for st in lev.steps)
    assert eliminated + F.coarse_L.shape[0] == N               # N = N_L1 + N_A1 + ...


# --------------------------------------------------------------------------
# invariances: U is fixed only up to rotations; order inside a colour is free
# --------------------------------------------------------------------------
def test_basis_rotation_invariance():
    A, perm, B = _problem("p2", 32, (4, 4))
    b = wl.rhs(A.shape[0], 7)
    F1 = ce.factorize(A, perm, B, 1e-3, 2, 4)
    F2 = ce.factorize(A, perm, B, 1e-3, 2, 4, rotate_rng=np.random.default_rng(1))
    assert [l.ranks for l in F1.levels] == [l.ranks for l in F2.levels]
    x1, x2 = ce.apply(F1, b), ce.apply(F2, b)
    assert np.linalg.norm(x1 - x2) / np.linalg.norm(x1) < 1e-12


def test_order_invariance_within_colour():
    A, perm, B = _problem("p2", 32, (4, 4))
    b = wl.rhs(A.shape[0], 8)
    F1 = ce.factorize(A, perm, B, 1e-3, 2, 4)
    F2 = ce.factorize(A, perm, B, 1e-3, 2, 4, shuffle_rng=np.random.default_rng(2))
    assert F1.levels[0].order != F2.levels[0].order
    x1, x2 = ce.apply(F1, b), ce.apply(F2, b)
    assert np.linalg.norm(x1 - x2) / np.linalg.norm(x1) < 1e-12


# --------------------------------------------------------------------------
# trends of the paper's tables (qualitative: other Krylov method and B)
# --------------------------------------------------------------------------
def _factor_words(F):
    # stored factor: L (coarse triangle, every L-hat and W) and Q (every U_i)
    return F.nnz_L + sum(st.n * st.n for lev in F.levels for st in lev.steps)


def test_direct_solve_error_falls_with_eps():
    # Table err (Section 4, CE(eps) as a direct solver): the accuracy eta of the
    # direct solve falls as eps falls while the memory the factor needs grows
    A, perm, B = _problem("p2", 64, (4, 4))
    b = wl.rhs(A.shape[0], 0)
    x_ref = sla.solve(A.toarray(), b, assume_a="pos")
    etas, words = [], []
    for eps in (1e-1, 1e-2, 1e-3, 1e-4):
        F = ce.factorize(A, perm, B, eps, 2, 4)
        x = ce.apply(F, b)
        etas.append(np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref))
        words.append(_factor_words(F))
    assert all(etas[j + 1] < etas[j] for j in range(3)), etas
    assert all(words[j + 1] > words[j] for j in range(3)), words


def test_fixed_rank_is_no_direct_solver():
    # Section 4: CE(r) with r = B/2 is not accurate enough to solve directly,
    # CE(eps) with a small eps is
    A, perm, B = _problem("p2", 64, (4, 4))
    b = wl.rhs(A.shape[0], 0)
    x_ref = sla.solve(A.toarray(), b, assume_a="pos")

    def eta(F):
        return np.linalg.norm(ce.apply(F, b) - x_ref) / np.linalg.norm(x_ref)

    e_r = eta(ce.factorize(A, perm, B, 0.0, 2, 4, tol_mode="fixed", rank=B // 2))
    e_eps = eta(ce.factorize(A, perm, B, 1e-6, 2, 4))
    assert e_r > 1e-3 > 1e-5 > e_eps, (e_r, e_eps)


def test_pcg_iterations_flat_in_N():
    # Table num_it: for fixed eps the iteration count does not grow with N
    its = []
    for n in (32, 64, 128):
        A, perm, B = _problem("p2", n, (4, 4))
        F = ce.factorize(A, perm, B, 1e-3, 2, 4)
        res = ce.pcg(A, F, wl.rhs(A.shape[0], 0), 1e-8, 100)
        assert res.converged
        its.append(res.iters)
    assert max(its) - min(its) <= 2, its
    plain = ce.pcg(wl.poisson2d(128), None, wl.rhs(128 * 128, 0), 1e-8, 2000,
                   precond=lambda r: r)
    assert plain.iters > 5 * max(its)


def test_not_spd_is_reported():
    A = wl.poisson2d(8).toarray()
    A[10, 10] = -5.0
    with pytest.raises(ce.NotSPDError):
        ce.factorize(sp.csr_matrix(A), np.arange(64), 16, 1e-3, 1, 2)


# --------------------------------------------------------------------------
# capped super-blocks: runs of J consecutive blocks join (Section 2.4), a run
# over nmax rows being halved until its parts fit
# --------------------------------------------------------------------------
def test_group_rule_by_hand():
    # sizes 10 20 30 5 | 64 1 1 with J = 4, nmax = 40 (worked by hand): the first
    # run (65 rows) halves into 10 20 | 30 5; the last run (66 rows, 3 blocks)
    # halves into 64 1 | 1, and 64 1 once more into 64 | 1
    assert ce._groups([10, 20, 30, 5, 64, 1, 1], 4, 40) == [(0, 2), (2, 4), (4, 5), (5, 6), (6, 7)]
    # without a cap: plain runs of J
    assert ce._groups([10, 20, 30, 5, 64, 1, 1], 4) == [(0, 4), (4, 7)]
    assert ce._groups([3] * 9, 4, 100) == [(0, 4), (4, 8), (8, 9)]


def test_capped_coarsening_stays_exact():
    # tol = 0 keeps M = A whatever the grouping; super-blocks respect the cap
    A, perm, B = _problem("p2", 32, (4, 4))
    F = ce.factorize(A, perm, B, 0.0, 3, 4, nmax=24)
    for lev in F.levels:
        for g0, g1 in lev.groups:
            sz = sum(lev.ranks[g0:g1])
            assert g1 - g0 <= 4 and (sz <= 24 or g1 - g0 == 1)
    assert any(g1 - g0 < 4 for lev in F.levels for g0, g1 in lev.groups[:-1])   # the cap acted
    x = wl.rhs(A.shape[0], 3)
    Ax = A @ x
    assert np.linalg.norm(ce.multiply(F, x) - Ax) / np.linalg.norm(Ax) < 1e-13
    b = wl.rhs(A.shape[0], 4)
    x_ref = sla.cho_solve(sla.cho_factor(A.toarray()), b)
    assert np.linalg.norm(ce.apply(F, b) - x_ref) / np.linalg.norm(x_ref) < 1e-12


@pytest.mark.slow
def test_paper_experiment_iteration_trends():
    """Table num_it on the paper's own problem (Section 4: -div(k grad u) = 1 on
    [0, 1]^3, k = diag(x_d^2 + 0.5), N = 8192 and 16384 on 16x16x32 and
    16x32x32 grids) with the paper's MINRES to 1e-10.  B = 8 (2^3 boxes) so
    that the table's CE(r), r = 4, is r = B/2; J = 8, 3 levels.  The paper's
    trends: MINRES without a preconditioner needs many more iterations and
    more as N grows; CE(1e-3) needs a handful (4-6 there), flat in N; CE(4)
    needs more than CE(1e-3) and grows mildly (23 -> 25 there)."""
    its = {"none": [], "eps": [], "r": []}
    for shape in [(16, 16, 32), (16, 32, 32)]:
        A = wl.diffusion3d_tensor(*shape)
        perm = wl.box_perm(shape, (2, 2, 2))
        b = np.ones(A.shape[0])
        its["none"].append(ce.minres(A, None, b, 1e-10, 5000, precond=lambda r: r).iters)
        F = ce.factorize(A, perm, 8, 1e-3, 3, 8)
        its["eps"].append(ce.minres(A, F, b, 1e-10, 500).iters)
        F = ce.factorize(A, perm, 8, 0.0, 3, 8, tol_mode="fixed", rank=4)
        its["r"].append(ce.minres(A, F, b, 1e-10, 500).iters)
    none, e, r = its["none"], its["eps"], its["r"]
    assert none[1] > none[0] > 5 * max(r), its
    assert max(e) <= 6 and abs(e[1] - e[0]) <= 1, its
    assert all(r[j] > e[j] for j in range(2)), its
    assert r[0] <= r[1] <= 1.5 * r[0], its


def test_minres_is_the_library_minres():
    """The oracle's MINRES (the Krylov minimisation written out) against
    SciPy's MINRES (the Paige-Saunders recurrence) with the same
    preconditioner and without one: the same iterate after every step."""
    import scipy.sparse.linalg as spla
    w = wl.make_workload("poisson2d_64_B16")
    F = ce.factorize(w.A, w.perm, w.B, w.tol, w.levels, w.J)
    N = w.A.shape[0]
    Mop = spla.LinearOperator((N, N), matvec=lambda v: ce.apply(F, v))
    cases = [(Mop, None, None, 4), (None, None, lambda r: r, 30)]
    for M, Fc, pre, K in cases:
        its = []
        spla.minres(w.A, w.b, rtol=1e-15, maxiter=K, M=M, callback=lambda xk: its.append(xk.copy()))
        assert len(its) >= min(K, 4)
        for k in sorted({1, 2, len(its) // 2, len(its)}):
            res = ce.minres(w.A, F if M is not None else Fc, w.b, 0.0, k, precond=pre)
            assert np.linalg.norm(its[k - 1] - res.x) <= 1e-12 * np.linalg.norm(res.x), k


def test_minres_preconditioned_indefinite_is_the_library_minres():
    """An indefinite symmetric matrix with an SPD (diagonal) preconditioner:
    the oracle's minimisation and SciPy's recurrence give the same iterate
    after every step."""
    import scipy.sparse.linalg as spla
    rng = np.random.default_rng(3)
    n = 80
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([-np.linspace(1, 5, n // 4), np.linspace(0.5, 20, n - n // 4)])
    A = sp.csr_matrix((Q * lam) @ Q.T)
    A = sp.csr_matrix(0.5 * (A + A.T))
    dinv = 1.0 / (1.0 + rng.random(n))
    b = rng.standard_normal(n)
    Mop = spla.LinearOperator((n, n), matvec=lambda v: dinv * v)
    its = []
    spla.minres(A, b, rtol=1e-15, maxiter=25, M=Mop, callback=lambda xk: its.append(xk.copy()))
    for k in (1, 5, 12, len(its)):
        res = ce.minres(A, None, b, 0.0, k, precond=lambda v: dinv * v)
        assert np.linalg.norm(its[k - 1] - res.x) <= 1e-10 * np.linalg.norm(res.x), k


def test_minres_special_cases():
    """Closed forms: with the exact preconditioner C = A^{-1} MINRES ends in one
    step at A^{-1} b; on a symmetric indefinite matrix with d distinct
    eigenvalues (two of them negative) it reaches A^{-1} b in d steps, its
    residual never growing; b = 0 returns x = 0 at once."""
    rng = np.random.default_rng(11)
    A = wl.poisson2d(12).toarray()
    b = rng.standard_normal(144)
    Ainv = np.linalg.inv(A)
    res = ce.minres(sp.csr_matrix(A), None, b, 1e-12, 10, precond=lambda r: Ainv @ r)
    assert res.converged and res.iters == 1
    assert np.linalg.norm(res.x - np.linalg.solve(A, b)) <= 1e-12 * np.linalg.norm(res.x)
    Qm, _ = np.linalg.qr(rng.standard_normal((60, 60)))
    lam = np.repeat([-3.0, -0.5, 1.0, 2.5, 7.0], 12)
    Ai = (Qm * lam) @ Qm.T
    Ai = 0.5 * (Ai + Ai.T)
    bi = rng.standard_normal(60)
    res = ce.minres(sp.csr_matrix(Ai), None, bi, 1e-11, 50, precond=lambda r: r)
    assert res.converged and res.iters <= 5
    assert np.linalg.norm(res.x - np.linalg.solve(Ai, bi)) <= 1e-9 * np.linalg.norm(res.x)
    assert all(h2 <= h1 * (1 + 1e-12) for h1, h2 in zip(res.history, res.history[1:]))
    z = ce.minres(sp.csr_matrix(A), None, np.zeros(144), 1e-10, 10, precond=lambda r: r)
    assert z.converged and z.iters == 0 and not np.any(z.x)


def test_pcg_is_the_library_cg():
    # the oracle's PCG (Section 4 uses a Krylov method around M; this build
    # uses CG) against SciPy's CG with the same preconditioner: the same
    # recurrence, so the same iterates after every number of steps
    import scipy.sparse.linalg as spla
    w = wl.make_workload("poisson2d_64_B16")
    F = ce.factorize(w.A, w.perm, w.B, w.tol, w.levels, w.J)
    N = w.A.shape[0]
    Mop = spla.LinearOperator((N, N), matvec=lambda v: ce.apply(F, v))
    for k in (1, 2, 3):
        xs, _ = spla.cg(w.A, w.b, x0=np.zeros(N), rtol=1e-14, atol=0.0, maxiter=k, M=Mop)
        res = ce.pcg(w.A, F, w.b, 1e-14, k)
        assert np.linalg.norm(xs - res.x) <= 1e-12 * np.linalg.norm(res.x), k
    for k in (1, 5, 20):
        xs, _ = spla.cg(w.A, w.b, x0=np.zeros(N), rtol=1e-14, atol=0.0, maxiter=k)
        res = ce.pcg(w.A, None, w.b, 1e-14, k, precond=lambda r: r)
        assert np.linalg.norm(xs - res.x) <= 1e-12 * np.linalg.norm(res.x), k


@pytest.mark.parametrize("kind", ["poisson2d", "poisson3d"])
def test_dropped_block_is_the_truncated_svd_tail(kind):
    """The compression step of Section 2.2 drops E_i = U_i[:, r:]^T F_i with
    ||E_i||_2 < eps: recomputed from the stored U_i and the far blocks as they
    stood before the step, ||E_i||_2 equals sigma_{r+1}(F_i) (the tail of the
    SVD, so basis and non-basis columns are not swapped) and is at most tau_i,
    while the kept rows U_i[:, :r]^T F_i keep every singular value above tau_i."""
    if kind == "poisson2d":
        w = wl.make_workload("poisson2d_64_B16")
        A, perm, B, tol, levels, J = w.A, w.perm, w.B, w.tol, w.levels, w.J
    else:
        A = wl.poisson3d(16)
        perm = wl.box_perm((16, 16, 16), (4, 4, 4))
        B, tol, levels, J = 64, 1e-4, 2, 8
    F = ce.factorize(A, perm, B, tol, levels, J, record_rows=True)
    checked = 0
    for lev in F.levels:
        for st in lev.steps:
            D, Cs, Fs = st.row
            if not Fs or st.sigma.size == 0:
                continue
            Fi = np.hstack(Fs)
            U, r = st.U, st.r
            assert np.abs(U.T @ U - np.eye(st.n)).max() < 1e-13
            E = U[:, r:].T @ Fi
            e2 = np.linalg.norm(E, 2) if E.size else 0.0
            tail = st.sigma[r] if r < st.sigma.size else 0.0
            assert abs(e2 - tail) <= 1e-12 * st.sigma[0] + 1e-13, (e2, tail)
            assert e2 <= st.tau
            if r > 0:
                kept = np.linalg.svd(U[:, :r].T @ Fi, compute_uv=False)
                assert kept.size == r and kept[-1] > st.tau
            checked += 1
    assert checked > 20


def _fill_aware_valid(nbr, c):
    """Rules of the distance-1 order, checked pair by pair: adjacent blocks
    differ; two neighbours of a block j that share a colour lie below j."""
    for j, nj in enumerate(nbr):
        for a in nj:
            if a == j:
                continue
            if c[a] == c[j]:
                return False
            for b in nj:
                if b != j and b != a and c[a] == c[b] and c[j] < c[a]:
                    return False
    return True


def test_distance1_colouring_is_valid_and_fewer():
    """The distance-1 order's colouring keeps its two rules on the 2D and 3D
    box patterns and on random graphs, and needs fewer colours than distance
    2 on the grids (6 instead of 7 on the 4-neighbour 2D box pattern, 8
    instead of 10 in 3D)."""
    for name, want in [("poisson2d_64_B16", (6, 7)), ("poisson2d_512_B32", (6, 7))]:
        w = wl.make_workload(name)
        S, sizes = ce.initial_blocks(w.A, w.perm, w.B)
        nbr = ce._block_graph(S, len(sizes))
        c1 = ce.distance1_colouring(nbr)
        c2 = ce.distance2_colouring(nbr)
        assert _fill_aware_valid(nbr, c1)
        assert (max(c1) + 1, max(c2) + 1) == want
    A, perm, B = _problem("p3", 16, (4, 4, 4))
    S, sizes = ce.initial_blocks(A, perm, B)
    nbr = ce._block_graph(S, len(sizes))
    c1 = ce.distance1_colouring(nbr)
    assert _fill_aware_valid(nbr, c1)
    assert max(c1) + 1 < max(ce.distance2_colouring(nbr)) + 1
    rng = np.random.default_rng(4)
    for trial in range(20):
        M = 40
        nbr = [{i} for i in range(M)]
        for _ in range(int(rng.integers(20, 120))):
            a, b = rng.integers(0, M, 2)
            nbr[a].add(int(b))
            nbr[b].add(int(a))
        assert _fill_aware_valid(nbr, ce.distance1_colouring(nbr))
    # the plain distance-1 rule (adjacent blocks differ) breaks rule 2 on the
    # 2D grid: a row of the first colour would share fill with another
    w = wl.make_workload("poisson2d_64_B16")
    S, sizes = ce.initial_blocks(w.A, w.perm, w.B)
    nbr = ce._block_graph(S, len(sizes))
    plain = [-1] * len(nbr)
    for i in ce.bfs_order(nbr):
        seen = {plain[j] for j in nbr[i] if j != i}
        plain[i] = min(set(range(len(nbr) + 1)) - seen)
    assert not _fill_aware_valid(nbr, plain)


def test_distance1_order_is_free_inside_a_colour():
    """Rows of one colour of the distance-1 order touch no common block but
    shared Schur targets, whose updates add up: any order inside the colours
    gives the same factor up to rounding (the GPU runs a colour's rows
    concurrently)."""
    w = wl.make_workload("poisson2d_64_B16")
    F1 = ce.factorize(w.A, w.perm, w.B, w.tol, w.levels, w.J, order="colour1")
    F2 = ce.factorize(w.A, w.perm, w.B, w.tol, w.levels, w.J, order="colour1",
                      shuffle_rng=np.random.default_rng(5))
    assert F1.levels[0].order != F2.levels[0].order
    assert [l.ranks for l in F1.levels] == [l.ranks for l in F2.levels]
    x1, x2 = ce.apply(F1, w.b), ce.apply(F2, w.b)
    assert np.linalg.norm(x1 - x2) / np.linalg.norm(x1) < 1e-12


def test_distance1_order_gives_the_same_operator():
    """Rows of a distance-1 colour read nothing another row of the colour
    writes, and their Schur updates of shared pairs add up in either order:
    the factorization in distance-1 colour order equals the distance-2 one up
    to rounding (same ranks on the first level, M^{-1} b to 1e-12 at tol = 0,
    backward error near the truncation level otherwise)."""
    A = wl.poisson2d(32)
    perm = wl.box_perm((32, 32), (4, 4))
    b = wl.rhs(1024, 3)
    F1 = ce.factorize(A, perm, 16, 0.0, 2, 4, order="colour1")
    x = ce.apply(F1, b)
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) < 1e-12
    w = wl.make_workload("poisson2d_64_B16")
    F1 = ce.factorize(w.A, w.perm, w.B, w.tol, w.levels, w.J, order="colour1")
    F2 = ce.factorize(w.A, w.perm, w.B, w.tol, w.levels, w.J)
    it1 = ce.pcg(w.A, F1, w.b, 1e-8, 100).iters
    it2 = ce.pcg(w.A, F2, w.b, 1e-8, 100).iters
    assert abs(it1 - it2) <= 1
