"""FP64 CPU oracle of the compress-and-eliminate (CE) factorization.

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow reference that the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the product library never
does.  It shares no code with the CUDA path: the only common module is
``workloads`` (seeded matrices, permutations, right-hand sides).

It follows the paper (Sushnikova & Oseledets, "Compress and eliminate solver
for symmetric positive definite sparse matrices") step by step, one block row
at a time, with numpy/scipy dense primitives (SVD, Cholesky, triangular solve)
as the library steps:

* ``factorize``      -- Algorithm 1 (CE algorithm), the level loop and the
                        coarse Cholesky of A_K (Section 2.5, Proposition CE_L).
* ``_one_level``     -- Algorithm 2 (one level elimination): for every block
                        row, the compression step of Section 2.2 (eq. rreav and
                        eq. q) and the sub-row elimination of eq. sm_L.
* ``_coarsen``       -- super-blocks of J consecutive blocks, optionally capped
                        at nmax rows (Section 2.4,
                        eq. bsp) that start the next level.
* ``apply``          -- x = Q^T L^{-T} L^{-1} Q b (solve proposition, Sec. 2.5).
* ``multiply``       -- M x = Q^T L L^T Q x (Proposition CE_L), independent
                        of ``apply``.
* ``pcg``            -- preconditioned conjugate gradients with M = Q^T L L^T Q.
* ``minres``         -- preconditioned MINRES (the paper's Krylov method,
                        Section 4) written as its defining minimisation over
                        the Krylov space, not as the short recurrence.

Pins (each function checked against something other than itself; the tests
named are under tests/):

* ``factorize`` / ``_one_level`` / ``apply`` / ``multiply``: tol = 0 (and
  CE(r) with r above every block size) is exact block Cholesky -- M = A and the
  solve is the dense Cholesky solve (test_oracle_pins, test_oracle_fixed_rank);
  levels = 0 is dense Cholesky; eps >= 1 and CE(0) equal an independently
  written block IC(0); the structural worked example of Section 2 (golden
  fixture); per-step orthogonality, rank rule and positive pivots; invariance
  under rotations inside the basis / non-basis subspaces and under reordering
  inside a colour; the trends of Tables err and num_it (the latter on the
  paper's own 3D problem).
* ``distance2_colouring`` / ``bfs_order``: validity of the colouring
  (test_oracle_pins); equality with the library's planner (test_library_cpu).
* ``_groups`` / ``_coarsen``: the grouping rule worked by hand, the capped
  coarsening exact at tol = 0, and the coarsening rule restated by brute force
  (test_library_cpu).
* ``block_features``: against their definitions on the oracle's own steps
  (test_mlp_pins).
* ``pcg``: its iterates equal SciPy's CG with the same preconditioner.
* ``minres``: its iterates equal SciPy's MINRES with the same preconditioner
  (and without one); the exact preconditioner C = A^{-1} converges in one
  step; on a symmetric indefinite matrix with d distinct eigenvalues it
  reaches A^{-1} b in d steps with a non-increasing residual
  (test_oracle_pins).

Readings of points the paper leaves open:

* Rank rule (CE(eps), Section 2.2 remark): the norm of E_i is the spectral
  norm and the tolerance is relative to the far row, tau_i = eps * sigma_1(F_i);
  r_i = #{k : sigma_k > tau_i} (a singular value equal to tau_i is dropped).
  ``tol_mode='abs'`` uses tau_i = eps.  CE(r) (``tol_mode='fixed'``, the
  remark's fixed-rank strategy) keeps r_i = min(r, numerical rank of F_i)
  directions; a singular value within 1e-3 relative of sigma_r is kept with
  it, so a tied cluster (grids are symmetric) is never split and the kept
  subspace is unique.  ``tol == 0`` uses
  tau_i = n_i * eps_64 * sigma_1, which drops only numerically-zero directions.
  In every mode tau_i is at least u * ||D_i||_F (u = unit roundoff of the
  arithmetic, eps_64 here): a far row that is rounding noise of the block row
  (fill that cancelled to roundoff) carries no direction worth keeping.
* Elimination order inside a level: colour-major order of a greedy distance-2
  colouring of the level's block graph, the blocks visited breadth-first from a
  block of least degree (ascending block index inside a colour);
  ``order='colour1'`` uses a colouring that separates only adjacent blocks
  and blocks with an earlier common neighbour, in the same visit order
  (``distance1_colouring``: fewer colours; rows of a colour may share Schur
  targets).  The paper's
  natural order (Algorithm 2) is ``order='natural'``; all are permutations P,
  which the paper leaves free (Section 2).
* Super-blocks: runs of J consecutive blocks (Section 2.4); with ``nmax`` a run
  over nmax rows is halved until its parts fit (they stay aligned with the
  runs).
* Basis first: the columns of U_i are the left singular vectors of F_i in
  descending singular value order; the first r_i are the basis ("compressed")
  dofs, the last n_i - r_i form the eliminated sub-row S_i = [0 I] R_i*.
* Fill bookkeeping: the Schur update of block i allocates every pair of its
  targets {basis of i} U close(i) (so the far pattern is the A^2 pattern,
  Section 2.2); the next level's block graph keeps a pair of super-blocks when
  some child pair with non-empty rows and columns lies inside it.
* A block whose far row is empty (or all zero) gets r_i = 0 and is eliminated
  whole, as in the first block row (Section 2.1).
"""
from __future__ import annotations

import collections
import dataclasses

import os

# The oracle works on many tiny dense matrices; a multi-threaded BLAS spends
# more time waking threads than computing.  Callers that import numpy first
# should set OPENBLAS_NUM_THREADS=1 themselves (tests/conftest.py does).
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")

import numpy as np  # noqa: E402
import scipy.linalg as sla  # noqa: E402
import scipy.sparse as sp  # noqa: E402

EPS64 = np.finfo(np.float64).eps
TIE_REL = 1e-3      # CE(r): singular values within this of sigma_r stay with it


class NotSPDError(RuntimeError):
    """A pivot block D_nn was not positive definite (level, block in args)."""


# --------------------------------------------------------------------------
# block storage: dict of (i, k) -> dense block for i <= k
# --------------------------------------------------------------------------
def _get(S, i, k):
    return S[(i, k)] if i <= k else S[(k, i)].T


def _put(S, i, k, X):
    if i <= k:
        S[(i, k)] = X
    else:
        S[(k, i)] = X.T


def _block_graph(S, M):
    """Adjacency sets of the blocks (pairs present in S), diagonal included."""
    nbr = [set([i]) for i in range(M)]
    for (i, k) in S:
        nbr[i].add(k)
        nbr[k].add(i)
    return nbr


def bfs_order(nbr):
    """Blocks in breadth-first order over the block graph: every component
    starts at its block of least degree (lowest index on ties), neighbours
    are queued in ascending index."""
    M = len(nbr)
    deg = [len(nbr[i]) - (1 if i in nbr[i] else 0) for i in range(M)]
    seen = [False] * M
    order = []
    for root in sorted(range(M), key=lambda i: (deg[i], i)):
        if seen[root]:
            continue
        seen[root] = True
        queue = collections.deque([root])
        while queue:
            i = queue.popleft()
            order.append(i)
            for j in sorted(nbr[i]):
                if not seen[j]:
                    seen[j] = True
                    queue.append(j)
    return order


def distance2_colouring(nbr):
    """Greedy distance-2 colouring, blocks visited in breadth-first order.

    Block i takes the smallest colour not held by any block j != i at graph
    distance 1 or 2 that is already coloured.  Blocks of one colour then have
    disjoint closed neighbourhoods, so their block rows can be compressed and
    eliminated in any order without touching the same pair of blocks.  The
    breadth-first visit sweeps the grid front by front, which reaches the
    minimum on structured grids (9 colours on the 8-neighbour pattern, where
    ascending Morton index needs 12) and so shortens the chain of dependent
    colours of a level.
    """
    M = len(nbr)
    colour = [-1] * M
    for i in bfs_order(nbr):
        seen = set()
        for j in nbr[i]:
            for k in nbr[j]:
                if k != i and colour[k] >= 0:
                    seen.add(colour[k])
        c = 0
        while c in seen:
            c += 1
        colour[i] = c
    return colour


def distance1_colouring(nbr):
    """Greedy colouring for an elimination order whose colours hold adjacent
    blocks apart but let blocks at distance 2 share a colour, in the same
    breadth-first order as ``distance2_colouring``.

    Two rows i, k of one colour must not touch a block that the other's
    compression or elimination changes.  Adjacent rows would (each row holds
    the other's block), and so would rows at distance 2 whose common
    neighbour j ran before them: j's Schur update created the fill block
    (i, k), which both rows would then compress.  Shared close targets are
    harmless (both rows' Schur updates add to them, in either order).  So a
    valid colouring has
      (1) colour[i] != colour[k] for adjacent i, k;
      (2) colour[j] > colour[i] for every block j with two neighbours i, k of
          one colour (the fill between them comes after both ran).
    Block x takes the smallest colour c that keeps (1) and (2) with the blocks
    coloured so far: c is not held by a neighbour; c exceeds every colour held
    by two of x's neighbours (x would be their earlier common neighbour); and c
    is not held by another neighbour k of a neighbour j that holds a colour
    below c (j would be the earlier common neighbour of x and k)."""
    M = len(nbr)
    colour = [-1] * M
    for x in bfs_order(nbr):
        held = [colour[j] for j in nbr[x] if j != x and colour[j] >= 0]
        taken = set(held)
        lowest = 0
        for d in taken:
            if held.count(d) >= 2:
                lowest = max(lowest, d + 1)
        for j in nbr[x]:
            if j == x or colour[j] < 0:
                continue
            for k in nbr[j]:
                if k != x and colour[k] > colour[j]:
                    taken.add(colour[k])
        c = lowest
        while c in taken:
            c += 1
        colour[x] = c
    return colour


# --------------------------------------------------------------------------
# factor records
# --------------------------------------------------------------------------
@dataclasses.dataclass
class BlockStep:
    """One compression + sub-row elimination step (block row i)."""

    i: int
    n: int                 # block size when the row was processed
    r: int                 # kept (basis) rank
    sigma: np.ndarray      # singular values of F_i (descending)
    tau: float             # truncation threshold used
    U: np.ndarray          # n x n orthogonal, basis columns first
    Lhat: np.ndarray       # (n-r) x (n-r) lower Cholesky factor of S_ii
    targets: list          # [(t, W_t)]: t == i is the basis of i, else close t
    far: list              # far blocks whose columns formed F_i (non-empty)
    features: np.ndarray = None  # rank-predictor features (block_features)
    row: tuple = None      # (D_i, [C_ik], [F_ik]) before compression, kept
                           # only with factorize(record_rows=True)


@dataclasses.dataclass
class Level:
    pairs: list            # block pairs (i <= k) of the level-start pattern
    sizes: list            # block sizes at the start of the level
    colour: list
    order: list
    steps: list            # BlockStep in elimination order
    J: int
    ranks: list            # r_i by block index
    groups: list = None    # super-blocks of the next level: child ranges [a, b)


@dataclasses.dataclass
class Factor:
    N: int
    perm: np.ndarray
    sizes0: list           # level-1 block sizes
    levels: list
    coarse_sizes: list     # remainder block sizes (index order)
    coarse_L: np.ndarray   # dense lower Cholesky factor of A_K

    @property
    def nnz_L(self):
        tot = self.coarse_L.shape[0] * (self.coarse_L.shape[0] + 1) // 2
        for lev in self.levels:
            for s in lev.steps:
                m = s.n - s.r
                tot += m * (m + 1) // 2 + sum(m * W.shape[1] for _, W in s.targets)
        return tot


# --------------------------------------------------------------------------
# Algorithm 2: one level of compression and elimination
# --------------------------------------------------------------------------
NFEAT = 11


def _lg(x):
    return np.log10(max(x, 1e-30)) / 10.0


def block_features(level, n, J, D, C_blocks, F_blocks, tol):
    """Cheap features of block row i when it is processed (rank predictor).

    Computed from the row before compression: level, size, Frobenius norms of
    the diagonal block D_i, of the close part C_i and of the far part F_i
    (with the largest and mean far-block norms), the numbers of close and of
    non-empty far blocks, the number of far columns, the mean rank of the J
    children the block was joined from (0 on the first level) and the
    tolerance.  Ratios are taken to ||D_i||_F so the features are scale free.
    """
    dn = np.linalg.norm(D)
    cn = np.sqrt(sum(np.linalg.norm(X) ** 2 for X in C_blocks))
    fb = [np.linalg.norm(X) for X in F_blocks if X.shape[1] > 0]
    fn = np.sqrt(sum(v * v for v in fb))
    mF = sum(X.shape[1] for X in F_blocks)
    fmax = max(fb) if fb else 0.0
    fmean = (sum(fb) / len(fb)) if fb else 0.0
    d = dn if dn > 0 else 1.0
    f = fn if fn > 0 else 1.0
    parent = (n / J) if level > 0 else 0.0
    return np.array([level / 4.0, n / 64.0, _lg(cn / d), _lg(fn / d), _lg(fmax / f),
                     _lg(fmean / f), len(C_blocks) / 8.0, len(fb) / 16.0, parent / 32.0,
                     mF / (16.0 * max(n, 1)), -np.log10(max(tol, 1e-30)) / 8.0])


def _random_orthogonal(rng, k):
    if k == 0:
        return np.zeros((0, 0))
    Qr, Rr = np.linalg.qr(rng.standard_normal((k, k)))
    return Qr * np.sign(np.diag(Rr))


def _one_level(S, sizes, tol, tol_mode, order_mode, level_no,
               rotate_rng=None, shuffle_rng=None, J=4, record_rows=False):
    M = len(sizes)
    size = list(sizes)
    close = _block_graph(S, M)          # level-start pattern = close blocks
    nbr = [set(c) for c in close]       # grows with fill
    if order_mode == "natural":
        colour = [0] * M
        order = list(range(M))
    else:
        colour = distance1_colouring(close) if order_mode == "colour1" else distance2_colouring(close)
        order = sorted(range(M), key=lambda i: (colour[i], i))
        if shuffle_rng is not None:     # self-test: any order inside a colour
            order = []
            for c in range(max(colour) + 1):
                members = [i for i in range(M) if colour[i] == c]
                order += [members[j] for j in shuffle_rng.permutation(len(members))]
    ranks = [0] * M
    steps = []
    for i in order:
        n = size[i]
        # -- compression step (Section 2.2, eq. rreav) ----------------------
        far = sorted(k for k in nbr[i] if k not in close[i] and size[k] > 0)
        Fs = [_get(S, i, k) for k in far]
        Cs = [_get(S, i, k) for k in sorted(close[i] - {i})]
        feats = block_features(level_no, n, J, _get(S, i, i), Cs, Fs, tol)
        row = (_get(S, i, i).copy(), [X.copy() for X in Cs], [X.copy() for X in Fs]) if record_rows else None
        F = np.hstack(Fs) if Fs else np.zeros((n, 0))
        if F.shape[1] == 0 or n == 0 or not np.any(F):
            U = np.eye(n)
            sig = np.zeros(0)
            tau = 0.0
            r = 0
        else:
            U, sig, _ = np.linalg.svd(F, full_matrices=True)
            if tol_mode == "fixed":
                # CE(r): tol carries r; the r leading directions, a cluster
                # tied with sigma_r kept whole, rounding noise never kept
                rk = int(tol)
                tau = n * EPS64 * sig[0]
                if rk == 0:
                    tau = sig[0]
                elif rk < sig.size:
                    tau = max(tau, (1.0 - TIE_REL) * sig[rk - 1])
            elif tol == 0.0:
                tau = n * EPS64 * sig[0]
            elif tol_mode == "abs":
                tau = tol
            else:
                tau = tol * sig[0]
            # rounding floor: singular values at the level of the rounding
            # noise of the block row are never kept
            tau = max(tau, EPS64 * np.linalg.norm(_get(S, i, i)))
            r = int(np.count_nonzero(sig > tau))
        if rotate_rng is not None:      # self-test: U is fixed only up to
            U = U.copy()                # rotations inside basis / non-basis
            U[:, :r] = U[:, :r] @ _random_orthogonal(rotate_rng, r)
            U[:, r:] = U[:, r:] @ _random_orthogonal(rotate_rng, n - r)
        # row and column transform by U_i (eq. q): U^T D U, U^T C, U^T F
        _put(S, i, i, U.T @ _get(S, i, i) @ U)
        for k in nbr[i]:
            if k != i:
                _put(S, i, k, U.T @ _get(S, i, k))
        # -- elimination step (Section 2.2, eq. sm_L) -----------------------
        D = _get(S, i, i)
        targets = [i] + sorted(close[i] - {i})
        Sn = {t: (D[r:, :r] if t == i else _get(S, i, t)[r:, :]) for t in targets}
        Snn = D[r:, r:]
        try:
            Lh = np.linalg.cholesky(Snn) if n - r > 0 else np.zeros((0, 0))
        except np.linalg.LinAlgError as e:
            raise NotSPDError(level_no, i) from e
        if n - r > 0 and not np.all(np.diag(Lh) > 0):
            raise NotSPDError(level_no, i)
        W = {t: sla.solve_triangular(Lh, Sn[t], lower=True) if n - r > 0
             else np.zeros((0, Sn[t].shape[1])) for t in targets}
        # block i keeps its basis rows; the far rows r: (E_i) are dropped and
        # the close rows r: moved into W (they form the eliminated sub-row)
        _put(S, i, i, D[:r, :r])
        for k in nbr[i]:
            if k != i:
                _put(S, i, k, _get(S, i, k)[:r, :])
        size[i] = r
        ranks[i] = r
        # Schur complement on the targets: A(s, t) -= W_s^T W_t
        for a, s in enumerate(targets):
            for t in targets[a:]:
                upd = W[s].T @ W[t]
                key = (min(s, t), max(s, t))
                if key not in S:
                    S[key] = np.zeros((size[key[0]], size[key[1]]))
                    nbr[s].add(t)
                    nbr[t].add(s)
                _put(S, s, t, _get(S, s, t) - (upd if s != t else 0.5 * (upd + upd.T)))
        steps.append(BlockStep(i, n, r, sig, tau, U, Lh,
                               [(t, W[t]) for t in targets], far, feats, row))
    return S, size, colour, order, steps, ranks


def _groups(size, J, nmax=None):
    """Super-blocks as ranges [a, b) of consecutive blocks: runs of J blocks
    join (Section 2.4).  With ``nmax`` (None or 0: no cap), a run whose sizes
    add up to more than nmax rows is halved (first half ceil(len/2) blocks), recursively, until
    every part fits or is a single block, so the parts stay aligned with the
    runs of J (geometric siblings under the box ordering)."""
    M, groups = len(size), []

    def split(a, b):
        if b - a == 1 or nmax is None or nmax <= 0 or sum(size[a:b]) <= nmax:
            groups.append((a, b))
            return
        mid = a + (b - a + 1) // 2
        split(a, mid)
        split(mid, b)

    for a in range(0, M, J):
        split(a, min(a + J, M))
    return groups


def _coarsen(S, size, J, nmax=None):
    """Join consecutive blocks into super-blocks (Section 2.4, eq. bsp).

    Child pairs with an empty side are left out, so a super-block pair exists
    when some child pair with non-empty rows and columns lies inside it.
    Returns the next level's pairs, sizes and the child ranges.
    """
    M = len(size)
    groups = _groups(size, J, nmax)
    Mn = len(groups)
    parent = [0] * M
    for I, (a, b) in enumerate(groups):
        for i in range(a, b):
            parent[i] = I
    off = [0] * M
    nsize = [0] * Mn
    for i in range(M):
        I = parent[i]
        off[i] = nsize[I]
        nsize[I] += size[i]
    T = {}
    for (i, k), X in S.items():
        if size[i] == 0 or size[k] == 0:
            continue
        I, K = parent[i], parent[k]
        if (I, K) not in T:
            T[(I, K)] = np.zeros((nsize[I], nsize[K]))
        T[(I, K)][off[i]:off[i] + size[i], off[k]:off[k] + size[k]] += X
        if I == K and i != k:
            T[(I, K)][off[k]:off[k] + size[k], off[i]:off[i] + size[i]] += X.T
    for I in range(Mn):                 # every super-block keeps its diagonal
        T.setdefault((I, I), np.zeros((nsize[I], nsize[I])))
    return T, nsize, groups


def _dense_from_blocks(S, size):
    off = np.concatenate([[0], np.cumsum(size)]).astype(int)
    A = np.zeros((off[-1], off[-1]))
    for (i, k), X in S.items():
        A[off[i]:off[i + 1], off[k]:off[k + 1]] = X
        if i != k:
            A[off[k]:off[k + 1], off[i]:off[i + 1]] = X.T
    return A


def initial_blocks(A, perm, B):
    """A_0 = P A P^T cut into blocks of B consecutive rows (eq. init_perm).

    The last block is shorter when N is not a multiple of B.
    """
    A = sp.csr_matrix(A)
    N = A.shape[0]
    perm = np.asarray(perm, dtype=np.int64)
    A0 = A[perm][:, perm].tocsr()
    ptr = list(range(0, N, B)) + [N]
    sizes = [ptr[j + 1] - ptr[j] for j in range(len(ptr) - 1)]
    blk = np.repeat(np.arange(len(sizes)), sizes)
    coo = A0.tocoo()
    S = {}
    for rr, cc, v in zip(coo.row, coo.col, coo.data):
        bi, bk = blk[rr], blk[cc]
        if bi > bk:
            continue
        if (bi, bk) not in S:
            S[(bi, bk)] = np.zeros((sizes[bi], sizes[bk]))
        S[(bi, bk)][rr - ptr[bi], cc - ptr[bk]] += v
    # the diagonal pair of every block exists, even if its values are zero
    for j in range(len(sizes)):
        S.setdefault((j, j), np.zeros((sizes[j], sizes[j])))
    return S, sizes


# --------------------------------------------------------------------------
# Algorithm 1: CE factorization
# --------------------------------------------------------------------------
def factorize(A, perm, B, tol, levels, J=4, tol_mode="rel", order="colour",
              rotate_rng=None, shuffle_rng=None, nmax=None, rank=None, record_rows=False):
    """CE factorization A ~= Q^T L L^T Q (Algorithm 1, Proposition CE_L).

    ``levels`` compression-elimination sweeps, each followed by coarsening by
    J; the remainder A_K is factorized by dense Cholesky.  Raises
    :class:`NotSPDError` when a pivot block is not positive definite.

    ``nmax`` caps the super-block size: a run of J consecutive blocks whose
    sizes add up to more than nmax rows is halved (first half ceil(len/2)
    blocks), recursively, until every part fits or is a single block
    (``_groups``).  ``nmax=None`` or 0 (the default) is the paper's rule of
    plain runs of J blocks (Section 2.4).

    ``record_rows`` keeps, for every step, the blocks D_i, C_ik and F_ik of
    its row as they stood before compression (memory grows with the problem;
    for small test cases).

    ``tol_mode='fixed'`` is CE(r) with r = ``rank`` (``tol`` is unused).

    ``rotate_rng`` / ``shuffle_rng`` are self-test hooks: a random rotation of
    each U_i inside its basis and non-basis subspaces, and a random order of
    the blocks inside each colour.  Neither may change M = Q^T L L^T Q.
    """
    N = A.shape[0]
    if tol_mode == "fixed":
        if rank is None or rank < 0:
            raise ValueError("CE(r) needs rank >= 0")
        tol = float(rank)
    S, sizes = initial_blocks(A, perm, B)
    sizes0 = list(sizes)
    recs = []
    for lev in range(levels):
        if len(sizes) == 0:
            break
        sizes_start = list(sizes)
        pairs = sorted(S.keys())
        S, size, colour, order_, steps, ranks = _one_level(
            S, sizes, tol, tol_mode, order, lev, rotate_rng, shuffle_rng, J, record_rows)
        S, sizes, groups = _coarsen(S, size, J, nmax)
        recs.append(Level(pairs, sizes_start, colour, order_, steps, J, ranks, groups))
    Ac = _dense_from_blocks(S, sizes)
    if Ac.shape[0]:
        try:
            Lc = np.linalg.cholesky(Ac)
        except np.linalg.LinAlgError as e:
            raise NotSPDError(levels, -1) from e
    else:
        Lc = np.zeros((0, 0))
    return Factor(N, np.asarray(perm), sizes0, recs, list(sizes), Lc)


# --------------------------------------------------------------------------
# solve: x = Q^T L^{-T} L^{-1} Q b
# --------------------------------------------------------------------------
def _split(v, sizes):
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(int)
    return [v[off[j]:off[j + 1]].copy() for j in range(len(sizes))]


def apply(F: Factor, b):
    """M^{-1} b with M = Q^T L L^T Q (solve proposition, Section 2.5).

    Forward sweep: per level, in elimination order, y_i <- U_i^T y_i, the
    eliminated part solves with L_hat_i and updates its targets; the basis parts
    are joined into super-blocks.  The remainder is solved with the coarse
    Cholesky factor; the backward sweep runs the transposed steps in reverse.
    """
    b = np.asarray(b, dtype=np.float64)
    y = _split(b[F.perm], F.sizes0)
    zs = []
    for lev in F.levels:
        z = {}
        for st in lev.steps:
            i, r = st.i, st.r
            yi = st.U.T @ y[i]
            zi = sla.solve_triangular(st.Lhat, yi[r:], lower=True) if st.n - r else yi[r:]
            y[i] = yi[:r]
            for t, W in st.targets:
                y[t] = y[t] - W.T @ zi
            z[i] = zi
        zs.append(z)
        y = [np.concatenate([y[c] for c in range(g0, g1)]) for g0, g1 in lev.groups]
    yc = np.concatenate(y) if y else np.zeros(0)
    if F.coarse_L.shape[0]:
        xc = sla.solve_triangular(F.coarse_L, yc, lower=True)
        xc = sla.solve_triangular(F.coarse_L.T, xc, lower=False)
    else:
        xc = yc
    sizes_next = F.coarse_sizes
    x = _split(xc, sizes_next)
    for lev, z in zip(reversed(F.levels), reversed(zs)):
        M = len(lev.sizes)
        # split every super-block into its children's basis parts
        xb = [None] * M
        for I, (g0, g1) in enumerate(lev.groups):
            o = 0
            for c in range(g0, g1):
                rc = lev.ranks[c]
                xb[c] = x[I][o:o + rc]
                o += rc
        for st in reversed(lev.steps):
            i, r = st.i, st.r
            rhs = z[i].copy()
            for t, W in st.targets:
                rhs -= W @ xb[t]
            xn = sla.solve_triangular(st.Lhat.T, rhs, lower=False) if st.n - r else rhs
            xb[i] = st.U @ np.concatenate([xb[i], xn])
        x = xb
    out = np.empty_like(b)
    out[F.perm] = np.concatenate(x) if x else np.zeros(0)
    return out


def multiply(F: Factor, x):
    """M x with M = Q^T L L^T Q (the factorization of Proposition CE_L).

    With G the forward sweep of :func:`apply` (M^{-1} = G^T G), M = G^{-1}
    G^{-T}.  G^{-T} runs the steps forward: y_i <- U_i^T y_i, z_i = L_hat_i^T
    y_i[r:] + sum_t W_t y_t, coarse c = L_K^T y_c.  G^{-1} runs them backward:
    y_c = L_K c, then per step y_t += W_t^T z_i, y_i[r:] = L_hat_i z_i,
    y_i <- U_i y_i.  This is an independent check of apply: M (M^{-1} b) = b,
    and with nothing dropped M x = A x.
    """
    x = np.asarray(x, dtype=np.float64)
    # ---- G^{-T} x
    y = _split(x[F.perm], F.sizes0)
    zs = []
    for lev in F.levels:
        z = {}
        for st in lev.steps:
            i, r = st.i, st.r
            yi = st.U.T @ y[i]
            zi = st.Lhat.T @ yi[r:]
            y[i] = yi[:r]
            for t, W in st.targets:
                zi = zi + W @ y[t]
            z[i] = zi
        zs.append(z)
        y = [np.concatenate([y[c] for c in range(g0, g1)]) for g0, g1 in lev.groups]
    yc = np.concatenate(y) if y else np.zeros(0)
    c = F.coarse_L.T @ yc
    # ---- G^{-1} (z, c)
    xc = F.coarse_L @ c
    xs = _split(xc, F.coarse_sizes)
    for lev, z in zip(reversed(F.levels), reversed(zs)):
        M = len(lev.sizes)
        xb = [None] * M
        for I, (g0, g1) in enumerate(lev.groups):
            o = 0
            for ch in range(g0, g1):
                rc = lev.ranks[ch]
                xb[ch] = xs[I][o:o + rc]
                o += rc
        for st in reversed(lev.steps):
            i = st.i
            for t, W in st.targets:
                xb[t] = xb[t] + W.T @ z[i]
            xb[i] = st.U @ np.concatenate([xb[i], st.Lhat @ z[i]])
        xs = xb
    out = np.empty_like(x)
    out[F.perm] = np.concatenate(xs) if xs else np.zeros(0)
    return out


# --------------------------------------------------------------------------
# PCG (replaces the paper's MINRES; M is SPD whenever every pivot is)
# --------------------------------------------------------------------------
@dataclasses.dataclass
class PCGResult:
    x: np.ndarray
    iters: int
    relres: float
    converged: bool
    history: list


def pcg(A, F, b, rtol=1e-8, maxit=1000, precond=None):
    """Preconditioned CG, x0 = 0, stop when ||b - A x||_2 <= rtol ||b||_2.

    ``precond`` defaults to ``apply(F, .)``; pass ``F=None`` and
    ``precond=lambda r: r`` for plain CG.
    """
    A = sp.csr_matrix(A)
    Minv = precond if precond is not None else (lambda v: apply(F, v))
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    r = b.copy()
    bn = np.linalg.norm(b)
    hist = [1.0]
    if bn == 0.0:
        return PCGResult(x, 0, 0.0, True, hist)
    z = Minv(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        Ap = A @ p
        alpha = rz / (p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        rel = np.linalg.norm(r) / bn
        hist.append(rel)
        if rel <= rtol:
            return PCGResult(x, it, rel, True, hist)
        z = Minv(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return PCGResult(x, maxit, hist[-1], False, hist)


def minres(A, F, b, rtol=1e-10, maxit=1000, precond=None):
    """Preconditioned MINRES (Paige and Saunders, 1975), the Krylov method of
    the paper's experiments (Section 4), written as its definition: with
    C = M^{-1} (``apply(F, .)``, or ``precond``), the k-th iterate x_k is the
    vector of the Krylov space K_k(C A, C b) whose residual b - A x has the
    least C-norm ||r||_C = sqrt(r^T C r).  x0 = 0; stops when
    ||b - A x_k||_C <= rtol ||b||_C (the residual computed afresh), or when
    the Krylov space stops growing (then x_k is the solution).

    Each step adds the next Krylov direction to a Euclidean-orthonormal basis
    Q (Gram-Schmidt, done twice), orthonormalises P = A Q in the C-inner
    product (P = Z R, Z^T C Z = I, Gram-Schmidt done twice), and solves the
    least-squares problem in that basis: z = Z^T C b, y = R^{-1} z, x = Q y.
    No short recurrence, so a slip in one would show against the library's.
    """
    A = sp.csr_matrix(A)
    Cop = precond if precond is not None else (lambda v: apply(F, v))
    b = np.asarray(b, dtype=np.float64)
    n = b.size
    x = np.zeros_like(b)
    Cb = Cop(b)
    bC = float(np.sqrt(b @ Cb))
    hist = [1.0]
    if bC == 0.0:
        return PCGResult(x, 0, 0.0, True, hist)
    Q, Z, CZ = [], [], []
    R = np.zeros((0, 0))
    v = Cb.copy()
    for it in range(1, maxit + 1):
        # next direction of K_k(C A, C b), orthogonal to the basis so far
        v0 = np.linalg.norm(v)
        for _ in range(2):
            for q in Q:
                v -= (q @ v) * q
        nv = np.linalg.norm(v)
        if nv <= 1e-14 * v0:           # the Krylov space is invariant
            return PCGResult(x, it - 1, hist[-1], True, hist)
        q = v / nv
        Q.append(q)
        p = A @ q
        w = Cop(p)                     # C A q: also the next Krylov direction
        v = w.copy()
        # C-orthonormalise p against Z (R gains a column)
        col = np.zeros(len(Z) + 1)
        pz, wz = p.copy(), w.copy()
        for _ in range(2):
            for j in range(len(Z)):
                c = CZ[j] @ pz
                col[j] += c
                pz -= c * Z[j]
                wz -= c * CZ[j]
        col[-1] = np.sqrt(pz @ wz)
        Z.append(pz / col[-1])
        CZ.append(wz / col[-1])
        Rn = np.zeros((len(Z), len(Z)))
        Rn[:-1, :-1] = R
        Rn[:, -1] = col
        R = Rn
        z = np.array([cz @ b for cz in CZ])
        y = sla.solve_triangular(R, z)
        x = np.stack(Q, axis=1) @ y
        r = b - A @ x
        rel = float(np.sqrt(max(r @ Cop(r), 0.0))) / bC
        hist.append(rel)
        if rel <= rtol:
            return PCGResult(x, it, rel, True, hist)
    return PCGResult(x, maxit, hist[-1], False, hist)
