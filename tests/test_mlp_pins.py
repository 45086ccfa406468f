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
