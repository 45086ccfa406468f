"""Model problems of the compress-and-eliminate paper, as seeded synthetic inputs.

Everything here is input preparation: matrices in CSR (scipy), the initial
permutation P of eq. (init_perm) and right-hand sides.  The paper fixes the
problem class (A SPD sparse, Section 1) and its experiment (3D diffusion,
Section 4); the configurations below are the 2D/3D Poisson and Gaussian-random-
field diffusion grids the build measures on.

Conventions
-----------
* Grid point (x, y[, z]) has natural index ``x + nx*y (+ nx*ny*z)``.
* Stencils carry no h^2 scaling: 2D Poisson is ``4, -1``, 3D is ``6, -1``;
  Dirichlet boundaries are imposed by omitting the neighbours outside the grid.
* The permutation P groups points into boxes of B points (x fastest inside a
  box) and orders the boxes by their Morton code (bit interleave, x lowest), so
  J = 2^d consecutive boxes are geometric siblings (Proposition "tensor grid",
  Section 2.7).  ``perm[k]`` is the natural index of row k of P A P^T.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp


# --------------------------------------------------------------------------
# matrices
# --------------------------------------------------------------------------
def _stencil_csr(shape, face_coef):
    """Assemble a symmetric FD operator from face coefficients.

    ``face_coef(axis)`` returns an array of the coefficient on the face between
    point p and p+e_axis (shape = grid shape with that axis one shorter), and
    ``face_coef(('bnd', axis, side))`` the coefficient of the Dirichlet face on
    that side (shape = grid shape with that axis of length 1).
    """
    shape = tuple(int(s) for s in shape)
    d = len(shape)
    N = int(np.prod(shape))
    idx = np.arange(N).reshape(shape[::-1]).transpose()  # idx[x, y, (z)]
    diag = np.zeros(shape)
    rows, cols, vals = [], [], []
    for ax in range(d):
        c = face_coef(ax)
        lo = [slice(None)] * d
        hi = [slice(None)] * d
        lo[ax] = slice(0, shape[ax] - 1)
        hi[ax] = slice(1, shape[ax])
        i0 = idx[tuple(lo)].ravel()
        i1 = idx[tuple(hi)].ravel()
        cv = c.ravel()
        rows += [i0, i1]
        cols += [i1, i0]
        vals += [-cv, -cv]
        diag[tuple(lo)] += c
        diag[tuple(hi)] += c
        for side in (0, 1):
            b = face_coef(("bnd", ax, side))
            sl = [slice(None)] * d
            sl[ax] = slice(0, 1) if side == 0 else slice(shape[ax] - 1, shape[ax])
            diag[tuple(sl)] += b
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    A = sp.csr_matrix(
        (np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
        shape=(N, N),
    )
    A.sum_duplicates()
    A.sort_indices()
    return A


def poisson2d(nx: int, ny: int | None = None) -> sp.csr_matrix:
    """5-point Laplacian ``4, -1`` on an nx x ny grid, Dirichlet."""
    ny = nx if ny is None else ny

    def coef(ax):
        if isinstance(ax, tuple):
            _, a, _ = ax
            s = [nx, ny]
            s[a] = 1
            return np.ones(s)
        s = [nx, ny]
        s[ax] -= 1
        return np.ones(s)

    return _stencil_csr((nx, ny), coef)


def poisson3d(nx: int, ny: int | None = None, nz: int | None = None) -> sp.csr_matrix:
    """7-point Laplacian ``6, -1`` on an nx x ny x nz grid, Dirichlet."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz

    def coef(ax):
        s = [nx, ny, nz]
        if isinstance(ax, tuple):
            s[ax[1]] = 1
            return np.ones(s)
        s[ax] -= 1
        return np.ones(s)

    return _stencil_csr((nx, ny, nz), coef)


def diffusion2d(k: np.ndarray) -> sp.csr_matrix:
    """Cell-centred 5-point discretisation of -div(k grad u), Dirichlet.

    ``k[x, y]`` > 0 is the coefficient at each grid point.  An interior face
    takes the harmonic mean of its two points' k; a boundary face takes the
    point's own k.  With k == 1 this is exactly :func:`poisson2d`.
    """
    k = np.asarray(k, dtype=np.float64)
    nx, ny = k.shape

    def coef(ax):
        if isinstance(ax, tuple):
            _, a, side = ax
            sl = [slice(None), slice(None)]
            sl[a] = slice(0, 1) if side == 0 else slice(k.shape[a] - 1, k.shape[a])
            return k[tuple(sl)]
        lo = [slice(None), slice(None)]
        hi = [slice(None), slice(None)]
        lo[ax] = slice(0, k.shape[ax] - 1)
        hi[ax] = slice(1, k.shape[ax])
        a, b = k[tuple(lo)], k[tuple(hi)]
        return 2.0 * a * b / (a + b)

    return _stencil_csr((nx, ny), coef)


def diffusion3d_tensor(nx: int, ny: int, nz: int) -> sp.csr_matrix:
    """7-point discretisation of -div(k grad u) on [0, 1]^3, u = 0 on the
    boundary, with the diagonal tensor k(x) = diag(x_1^2 + 0.5, x_2^2 + 0.5,
    x_3^2 + 0.5) of the paper's experiments (Section 4).

    ``n_d`` equidistant interior nodes per axis, spacing h_d = 1 / (n_d + 1);
    the face between two nodes along axis d carries k_d at the face midpoint
    over h_d^2 (so the operator is the usual second difference, scaled).
    """
    shape = (nx, ny, nz)
    h = [1.0 / (n + 1) for n in shape]

    def coef(ax):
        if isinstance(ax, tuple):
            _, a, side = ax
            xf = 0.5 * h[a] if side == 0 else 1.0 - 0.5 * h[a]
            out = np.empty(tuple(1 if d == a else shape[d] for d in range(3)))
            out[...] = (xf * xf + 0.5) / (h[a] * h[a])
            return out
        xf = (np.arange(1, shape[ax]) + 0.5) * h[ax]      # faces between nodes i and i+1
        c = (xf * xf + 0.5) / (h[ax] * h[ax])
        sh = [1, 1, 1]
        sh[ax] = shape[ax] - 1
        full = [shape[0], shape[1], shape[2]]
        full[ax] = shape[ax] - 1
        return np.broadcast_to(c.reshape(sh), full).copy()

    return _stencil_csr(shape, coef)


def grf2d(n: int, seed: int, corr_frac: float = 1.0 / 32.0, contrast: float = 1.0e4):
    """Coefficient field k = exp(s * g) on an n x n grid.

    g is a zero-mean unit-variance Gaussian random field with squared-
    exponential covariance exp(-|d|^2 / (2 l^2)), l = corr_frac (domain = unit
    square), sampled by circulant embedding on a 2x padded periodic grid.  The
    scale s = ln(contrast) / (max g - min g) makes max k / min k == contrast.
    Returns ``k`` indexed ``k[x, y]``.
    """
    m = 2 * n
    h = 1.0 / n
    ell = corr_frac
    d = np.minimum(np.arange(m), m - np.arange(m)) * h
    cov = np.exp(-(d[:, None] ** 2 + d[None, :] ** 2) / (2.0 * ell * ell))
    lam = np.fft.fft2(cov).real
    lam = np.maximum(lam, 0.0)
    rng = np.random.default_rng(seed)
    xi = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    field = np.fft.fft2(np.sqrt(lam / (m * m)) * xi)
    g = field.real[:n, :n]
    g = g / np.sqrt(cov[0, 0])
    s = math.log(contrast) / float(g.max() - g.min())
    return np.exp(s * g)


# --------------------------------------------------------------------------
# permutation
# --------------------------------------------------------------------------
def _morton(coords: np.ndarray, bits: int) -> np.ndarray:
    """Bit-interleaved key, coordinate 0 in the lowest bit of each group."""
    d = coords.shape[1]
    key = np.zeros(coords.shape[0], dtype=np.int64)
    for b in range(bits):
        for a in range(d):
            key |= ((coords[:, a].astype(np.int64) >> b) & 1) << (b * d + a)
    return key


def box_perm(shape, box) -> np.ndarray:
    """Permutation P: boxes of prod(box) points, boxes in Morton order.

    Requires every grid extent to be a multiple of the box extent, so every
    block of the permuted matrix is exactly one box.
    """
    shape = tuple(int(s) for s in shape)
    box = tuple(int(b) for b in box)
    d = len(shape)
    if any(s % b for s, b in zip(shape, box)):
        raise ValueError("grid extents must be multiples of the box extents")
    nb = [s // b for s, b in zip(shape, box)]
    # all boxes, natural order (x fastest)
    grids = np.meshgrid(*[np.arange(n) for n in nb], indexing="ij")
    bc = np.stack([g.transpose(*reversed(range(d))).ravel() for g in grids], axis=1)
    bits = max(1, int(math.ceil(math.log2(max(nb)))) + 1)
    order = np.argsort(_morton(bc, bits), kind="stable")
    bc = bc[order]
    # points inside a box, x fastest
    inner = np.meshgrid(*[np.arange(b) for b in box], indexing="ij")
    ic = np.stack([g.transpose(*reversed(range(d))).ravel() for g in inner], axis=1)
    pts = bc[:, None, :] * np.array(box)[None, None, :] + ic[None, :, :]
    pts = pts.reshape(-1, d)
    strides = np.cumprod([1] + list(shape[:-1]))
    return (pts * strides[None, :]).sum(axis=1).astype(np.int32)


def rhs(n: int, seed: int) -> np.ndarray:
    """b ~ N(0, 1), FP64, from ``numpy.random.default_rng(seed)``."""
    return np.random.default_rng(seed).standard_normal(n)


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    A: sp.csr_matrix
    perm: np.ndarray
    B: int
    tol: float
    levels: int
    J: int
    b: np.ndarray
    desc: str


WORKLOADS = {
    # name: (kind, grid, box, tol, levels, J, rhs seed)
    "poisson2d_64_B16": ("p2", (64, 64), (4, 4), 1e-3, 2, 4, 0),
    "poisson2d_256_B32": ("p2", (256, 256), (8, 4), 1e-4, 4, 4, 0),
    "poisson2d_512_B32": ("p2", (512, 512), (8, 4), 1e-4, 4, 4, 0),
    "poisson3d_32_B64": ("p3", (32, 32, 32), (4, 4, 4), 1e-4, 4, 8, 0),
    "poisson3d_64_B64": ("p3", (64, 64, 64), (4, 4, 4), 1e-4, 4, 8, 0),
    "grf2d_1024_B32": ("grf", (1024, 1024), (8, 4), 1e-4, 4, 4, 100),
}


def make_workload(name: str, grf_seed: int = 0) -> Workload:
    """Build one named workload (matrix, permutation, parameters, RHS)."""
    kind, grid, box, tol, levels, J, bseed = WORKLOADS[name]
    if kind == "p2":
        A = poisson2d(*grid)
        desc = f"2D Poisson 5-point {grid[0]}x{grid[1]}, Dirichlet"
    elif kind == "p3":
        A = poisson3d(*grid)
        desc = f"3D Poisson 7-point {grid[0]}^3, Dirichlet"
    else:
        A = diffusion2d(grf2d(grid[0], grf_seed))
        desc = f"2D GRF diffusion {grid[0]}x{grid[1]} (k contrast 1e4, seed {grf_seed})"
    perm = box_perm(grid, box)
    B = int(np.prod(box))
    return Workload(name, A, perm, B, tol, levels, J, rhs(A.shape[0], bseed), desc)


# --------------------------------------------------------------------------
# batches of independent systems
# --------------------------------------------------------------------------
BATCH_SIDES = (64, 96, 128, 192, 256)


def make_batch(nsys: int, seed: int = 7, choices=BATCH_SIDES, tol: float = 1e-4,
               levels: int = 4, J: int = 4) -> list:
    """Independent 2D 5-point Poisson systems on square grids whose sides are
    drawn uniformly from ``choices`` (``numpy.random.default_rng(seed)``).

    Grids of side <= 96 use 4x4 boxes (B = 16), larger ones 8x4 boxes
    (B = 32); system s gets the RHS ``rhs(n_s, 1000 + s)``.
    """
    rng = np.random.default_rng(seed)
    sides = rng.choice(np.asarray(choices), size=nsys)
    out = []
    for s, side in enumerate(int(v) for v in sides):
        box = (4, 4) if side <= 96 else (8, 4)
        A = poisson2d(side, side)
        out.append(Workload(f"poisson2d_{side}_sys{s}", A, box_perm((side, side), box),
                            int(np.prod(box)), tol, levels, J,
                            rhs(side * side, 1000 + s),
                            f"2D Poisson 5-point {side}x{side}, Dirichlet (system {s})"))
    return out
