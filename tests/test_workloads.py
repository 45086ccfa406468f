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
