"""CPU pins of the FP64 rank-predictor reference (oracle/mlp.py): the
analytic gradient against central finite differences, the training set's
features against their definitions on the oracle's own steps."""
import numpy as np
import pytest

import workloads as wl
from oracle import ce, mlp


@pytest.fixture(scope="module")
def data():
    w = wl.make_workload("poisson2d_64_B16")
    F = ce.factorize(w.A, w.perm, w.B, w.tol, w.levels, w.J)
    X, t = mlp.training_set([F])
    return F, X, t


def test_gradient_matches_finite_differences(data):
    _, X, t = data
    rng = np.random.default_rng(3)
    theta = mlp.init(1) + 0.01 * rng.standard_normal(mlp.NPARAM)
    g = mlp.grad(theta, X, t)
    idx = rng.choice(mlp.NPARAM, 60, replace=False)
    h = 1e-6
    for p in idx:
        e = np.zeros(mlp.NPARAM)
        e[p] = h
        fd = (mlp.loss(theta + e, X, t) - mlp.loss(theta - e, X, t)) / (2 * h)
        assert abs(fd - g[p]) <= 1e-6 * max(1.0, abs(g[p])) + 1e-9, (p, fd, g[p])


def test_features_follow_their_definition(data):
    F, X, t = data
    assert X.shape[1] == ce.NFEAT and np.all((t >= 0) & (t <= 1))
    lev = F.levels[0]
    st = next(s for s in lev.steps if s.far)
    x = st.features
    assert x[0] == 0 and x[1] == pytest.approx(st.n / 64)
    assert x[7] == pytest.approx(len(st.far) / 16)
    assert x[10] == pytest.approx(-np.log10(1e-3) / 8)
    assert x[8] == 0            # no parent rank on the first level


def test_training_set_file_matches_oracle_script():
    from paper_1603_09133_gb300 import rank_training_data
    X, t = rank_training_data()
    assert X.shape[1] == ce.NFEAT and X.shape[0] == t.shape[0] > 10000
    assert np.all(np.isfinite(X)) and np.all((t >= 0) & (t <= 1))


def test_features_of_a_hand_made_row():
    """All eleven features of a row whose norms are known by hand:
    D = 2 I_4 (||D||_F = 4), one close block of ones (4 x 2, norm sqrt 8),
    far blocks 3 * ones(4, 1) (norm 6), an empty block (not counted) and
    4 e_1 (norm 4): ||F||_F = sqrt 52, largest 6, mean 5, two far columns."""
    D = 2.0 * np.eye(4)
    C_blocks = [np.ones((4, 2))]
    e1 = np.zeros((4, 1))
    e1[0, 0] = 4.0
    F_blocks = [3.0 * np.ones((4, 1)), np.zeros((4, 0)), e1]
    x = ce.block_features(1, 4, 4, D, C_blocks, F_blocks, 1e-4)
    expect = [
        0.25,                    # level 1 / 4
        4 / 64,                  # n / 64
        -0.0150515,              # log10(sqrt(8)/4)/10 = -log10(2)/20
        0.0255942,               # log10(sqrt(52)/4)/10 = (log10(52)/2 - 2 log10(2))/10
        -0.0079850,              # log10(6/sqrt(52))/10
        -0.0159032,              # log10(5/sqrt(52))/10
        1 / 8,                   # one close block / 8
        2 / 16,                  # two non-empty far blocks / 16
        (4 / 4) / 32,            # parent rank n / J on level 1, / 32
        2 / 64,                  # two far columns / (16 n)
        0.5,                     # -log10(1e-4) / 8
    ]
    assert x.shape == (ce.NFEAT,)
    np.testing.assert_allclose(x, expect, rtol=0, atol=2e-7)


def test_features_are_taken_before_compression():
    """On the oracle's own steps (two levels, recorded rows), the norm
    features equal the norms of the row's blocks as they stood before the
    compression of that row: sums of squares, not norms of transformed
    blocks."""
    w = wl.make_workload("poisson2d_64_B16")
    F = ce.factorize(w.A, w.perm, w.B, w.tol, w.levels, w.J, record_rows=True)
    checked = 0
    for lev in F.levels:
        for st in lev.steps:
            D, Cs, Fs = st.row
            if not Fs:
                continue
            d = np.sqrt(np.sum(D * D))
            c = np.sqrt(sum(np.sum(X * X) for X in Cs))
            norms = [np.sqrt(np.sum(X * X)) for X in Fs if X.shape[1] > 0]
            f = np.sqrt(sum(v * v for v in norms))
            x = st.features
            lg = lambda v: np.log10(max(v, 1e-30)) / 10  # noqa: E731
            np.testing.assert_allclose(
                x[[2, 3, 4, 5, 9]],
                [lg(c / d), lg(f / d), lg(max(norms) / f), lg(np.mean(norms) / f),
                 sum(X.shape[1] for X in Fs) / (16 * st.n)], rtol=1e-12, atol=1e-14)
            assert x[6] == len(Cs) / 8 and x[7] == len(norms) / 16
            checked += 1
    assert checked > 100
