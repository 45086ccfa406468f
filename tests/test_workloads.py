"""Pins of the input generators against closed forms (CPU)."""
import numpy as np

import workloads as wl


def _grid(shape):
    h = [1.0 / (n + 1) for n in shape]
    axes = [np.arange(1, n + 1) * hd for n, hd in zip(shape, h)]
    X = np.meshgrid(*axes, indexing="ij")
    # the generators number points x fastest: flatten in Fortran order
    return [x.ravel(order="F") for x in X]


def test_paper_problem_is_second_order_consistent():
    """diffusion3d_tensor discretises -div(k grad u), k = diag(x_d^2 + 0.5) on
    [0, 1]^3 (Section 4): on u = prod_d sin(pi x_d) its action converges to
    the analytic operator at second order as the grid is refined."""
    errs = []
    for n in (8, 16, 32):
        x = _grid((n, n, n))
        s = [np.sin(np.pi * xd) for xd in x]
        c = [np.cos(np.pi * xd) for xd in x]
        u = s[0] * s[1] * s[2]
        exact = np.zeros_like(u)
        for d in range(3):
            rest = np.prod([s[e] for e in range(3) if e != d], axis=0)
            exact += ((x[d] ** 2 + 0.5) * np.pi ** 2 * s[d] - 2 * x[d] * np.pi * c[d]) * rest
        A = wl.diffusion3d_tensor(n, n, n)
        errs.append(np.abs(A @ u - exact).max() / np.abs(exact).max())
    assert errs[2] < 1e-3
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0, errs


def test_paper_problem_anisotropic_grid_and_spd():
    A = wl.diffusion3d_tensor(4, 6, 8)
    assert A.shape == (192, 192)
    assert abs(A - A.T).max() == 0.0
    assert np.all(np.linalg.eigvalsh(A.toarray()) > 0)
    # constant u: only boundary faces act, so interior rows sum to zero
    rs = np.asarray(A.sum(axis=1)).ravel()
    x = _grid((4, 6, 8))
    interior = np.ones(192, bool)
    for xd, n in zip(x, (4, 6, 8)):
        h = 1.0 / (n + 1)
        interior &= (xd > 1.5 * h) & (xd < 1 - 1.5 * h)
    assert np.abs(rs[interior]).max() < 1e-9 * np.abs(rs).max()


def test_constant_coefficient_diffusion_is_poisson():
    # with k == 1 every face (harmonic mean of 1 and 1) carries 1: the 5-point
    # Laplacian with Dirichlet faces, entry for entry; k scales the operator
    assert abs(wl.diffusion2d(np.ones((12, 9))) - wl.poisson2d(12, 9)).max() == 0.0
    k = np.random.default_rng(0).uniform(0.5, 2.0, (10, 10))
    assert abs(wl.diffusion2d(3.0 * k) - 3.0 * wl.diffusion2d(k)).max() < 1e-12


def test_grf_contrast_and_correlation_length():
    """k = exp(s g): max k / min k is 1e4 exactly, and the normalised
    autocorrelation of log k at one correlation length (n/32 grid steps) is
    that of the squared-exponential covariance, exp(-1/2)."""
    n = 256
    k = wl.grf2d(n, seed=11)
    assert abs(k.max() / k.min() / 1.0e4 - 1) < 1e-12
    g = np.log(k)
    g = g - g.mean()
    lag = n // 32
    rho_x = (g[:-lag, :] * g[lag:, :]).mean() / (g * g).mean()
    rho_y = (g[:, :-lag] * g[:, lag:]).mean() / (g * g).mean()
    assert abs(rho_x - np.exp(-0.5)) < 0.1 and abs(rho_y - np.exp(-0.5)) < 0.1, (rho_x, rho_y)
    assert not np.array_equal(k, wl.grf2d(n, seed=12))


def test_box_perm_boxes_and_morton_siblings():
    """P: a permutation; block b of P A P^T is one geometric box of 8 x 4
    points; the 4 boxes of every run of J = 4 consecutive blocks form a 2 x 2
    square of boxes (Morton siblings, what joining J blocks relies on)."""
    nx, ny, bx, by = 64, 32, 8, 4
    p = wl.box_perm((nx, ny), (bx, by))
    assert np.array_equal(np.sort(p), np.arange(nx * ny))
    x, y = p % nx, p // nx
    B = bx * by
    boxes = []
    for b in range(nx * ny // B):
        xs, ys = x[b * B:(b + 1) * B], y[b * B:(b + 1) * B]
        assert xs.max() - xs.min() == bx - 1 and ys.max() - ys.min() == by - 1
        assert xs.min() % bx == 0 and ys.min() % by == 0
        boxes.append((xs.min() // bx, ys.min() // by))
    for g in range(0, len(boxes), 4):
        q = np.array(boxes[g:g + 4])
        assert q[:, 0].max() - q[:, 0].min() == 1 and q[:, 1].max() - q[:, 1].min() == 1
        assert q[:, 0].min() % 2 == 0 and q[:, 1].min() % 2 == 0
