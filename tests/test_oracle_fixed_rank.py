"""Pins of the oracle's CE(r), the fixed-rank strategy of the Section 2.2
remark: r_i = r directions kept per block row, r = B/2 the usual choice.

* r at least the block size keeps every direction that is not rounding noise:
  CE reduces to exact block Cholesky (eq. bl_chol), so M = A and the solve is
  the dense Cholesky solve.
* r = 0 drops every far block: CE(0) is block IC(0) on the level-1 pattern in
  the same order, checked against an independently written block IC(0).
* Every recorded rank is the fixed r, except where F_i has fewer directions
  above rounding noise or where a singular value ties with sigma_r; a cut one
  index off (sigma_{r+1} for sigma_r) fails this on the grids below.
* Memory control (the remark's point): every super-block of the next level
  holds at most J r rows unless a tie widened a child.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle import ce

from test_oracle_pins import _block_ic0_minv, _problem


@pytest.mark.parametrize("kind,n,box,levels,J", [
    ("p2", 16, (4, 4), 2, 4),
    ("p2", 32, (8, 4), 3, 4),
    ("p3", 8, (2, 2, 2), 2, 8),
])
def test_unbounded_rank_is_exact(kind, n, box, levels, J):
    A, perm, B = _problem(kind, n, box)
    F = ce.factorize(A, perm, B, 0.0, levels, J, tol_mode="fixed", rank=10 ** 6)
    x = wl.rhs(A.shape[0], 3)
    assert np.linalg.norm(ce.multiply(F, x) - A @ x) / np.linalg.norm(A @ x) < 1e-13
    Ad = A.toarray()
    b = wl.rhs(A.shape[0], 4)
    x_ref = sla.cho_solve(sla.cho_factor(Ad), b)
    assert np.linalg.norm(ce.apply(F, b) - x_ref) / np.linalg.norm(x_ref) < 1e-12


def test_rank_zero_is_block_ic0():
    A, perm, B = _problem("p2", 16, (4, 4))
    F = ce.factorize(A, perm, B, 0.0, 1, 4, tol_mode="fixed", rank=0)
    lev = F.levels[0]
    assert all(r == 0 for r in lev.ranks)
    A0 = A.toarray()[np.ix_(perm, perm)]
    L = _block_ic0_minv(A0, lev.sizes, lev.pairs, lev.order)
    b = wl.rhs(256, 5)
    x_ic = np.empty(256)
    x_ic[perm] = np.linalg.solve(L @ L.T, b[perm])     # L: triangular in elimination order
    x = ce.apply(F, b)
    assert np.linalg.norm(x - x_ic) / np.linalg.norm(x_ic) < 1e-12


@pytest.mark.parametrize("n,box,r,levels", [(32, (4, 4), 4, 2), (64, (8, 4), 8, 3)])
def test_ranks_are_the_fixed_rank(n, box, r, levels):
    A, perm, B = _problem("p2", n, box)
    F = ce.factorize(A, perm, B, 0.0, levels, 4, tol_mode="fixed", rank=r)
    exact, ties = 0, 0
    for lev in F.levels:
        for st in lev.steps:
            if st.sigma.size == 0:
                assert st.r == 0
                continue
            if st.r < min(r, st.sigma.size):
                # fewer than r kept: what is left is rounding noise
                assert st.sigma[st.r] <= 1e-10 * st.sigma[0]
                continue
            if st.sigma.size <= r:
                assert st.r == int(np.count_nonzero(st.sigma > st.tau))
                continue
            tied = st.sigma[r] >= (1.0 - ce.TIE_REL) * st.sigma[r - 1]
            if tied:
                ties += 1
                assert st.r > r
                assert np.all(st.sigma[r:st.r] >= (1.0 - ce.TIE_REL) * st.sigma[r - 1])
            else:
                exact += 1
                assert st.r == r
    assert exact > 0


@pytest.mark.parametrize("r", [4, 8])
def test_memory_control(r):
    A, perm, B = _problem("p2", 64, (4, 4))
    J = 4
    F = ce.factorize(A, perm, B, 0.0, 3, J, tol_mode="fixed", rank=r)
    for lev in F.levels:
        tied = {st.i for st in lev.steps if st.r > r}
        for g0, g1 in lev.groups:
            rows = sum(lev.ranks[g0:g1])
            if not tied.intersection(range(g0, g1)):
                assert rows <= J * r
    res = ce.pcg(A, F, wl.rhs(A.shape[0], 0), 1e-8, 500)
    assert res.converged


def test_more_rank_is_a_better_preconditioner():
    # CE(r) lacks accuracy control, but a larger r keeps more of every far row
    A, perm, B = _problem("p2", 64, (4, 4))
    b = wl.rhs(A.shape[0], 0)
    its = [ce.pcg(A, ce.factorize(A, perm, B, 0.0, 2, 4, tol_mode="fixed", rank=r), b, 1e-8, 500).iters
           for r in (1, 4, 8)]
    assert its[0] > its[1] > its[2]
