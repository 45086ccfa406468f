"""The benchmarked form against the FP64 oracle, and the learned compression's
inputs against the oracle's.

* The 2D Poisson 512x512 workload (B = 32, tol 1e-4, 4 levels, J = 4) in
  exactly the form bench.py times: the rank model trained on the GPU, the row
  kernel autotuned per level (CTA shape, learned sketch or exact SVD), FP32
  factorization, super-blocks capped at 64 rows (nmax = 64 on both sides).  Its apply is judged by the plain method (the exact-SVD FP64
  oracle): normwise backward error eta = ||b - M_or z|| / (||A|| ||z|| + ||b||)
  with z = M_gpu^{-1} b at most 1e-4, PCG iterations within +-1 of the
  oracle's, true residual <= 1e-8.
* The rank model's eleven features, as the row kernel computes them before
  compressing each row, equal oracle.ce.block_features of the same row: on
  every level reached with identical ranks so far in the exact FP64 form with
  the features recorded (a basis rotation leaves every feature unchanged, so
  only the ranks need agree; rows whose far part is rounding noise, ||F|| <
  1e-12 ||D||, have noise for norms and are compared on the other features),
  and on the first level of the learned form, as the model saw them.
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


@pytest.fixture(scope="module")
def model(ceg):
    return ceg.trained_rank_model()


_ORACLE = {}


def _oracle(name):
    if name not in _ORACLE:
        w = wl.make_workload(name)
        _ORACLE[name] = oce.factorize(w.A, w.perm, w.B, w.tol, w.levels, w.J, nmax=64)   # the bench's cap
    return _ORACLE[name]


def _anorm(A):
    import scipy.sparse.linalg as spla
    return float(spla.eigsh(A, k=1, which="LA", return_eigenvectors=False)[0])


def test_bench_form_512_against_oracle(ceg, model):
    w = wl.make_workload("poisson2d_512_B32")
    csb = ceg.csb_build(w.A, w.perm, w.B)
    ceg.ce_autotune(csb, tol=w.tol, levels=w.levels, J=w.J, precision="fp32", rank_model=model, nmax=64)
    F = ceg.ce_factorize(csb, tol=w.tol, levels=w.levels, J=w.J, precision="fp32", rank_model=model, nmax=64)
    info = F.info
    learned = [info.row_learned[l] for l in range(info.levels_done)]
    acc = [info.learned_rows[l] for l in range(info.levels_done)]
    assert any(learned) and sum(acc) > 0
    Fo = _oracle("poisson2d_512_B32")
    r = torch.as_tensor(w.b, device="cuda")
    z = torch.empty_like(r)
    ceg.ce_apply(F, r, z)
    torch.cuda.synchronize()
    zh = z.cpu().numpy()
    eta = np.linalg.norm(w.b - oce.multiply(Fo, zh)) / (_anorm(w.A) * np.linalg.norm(zh) + np.linalg.norm(w.b))
    res_o = oce.pcg(w.A, Fo, w.b, 1e-8, 500)
    x = torch.zeros_like(r)
    it, rel, conv = ceg.pcg_solve(csb, F, r, x, 1e-8, 500)
    torch.cuda.synchronize()
    xh = x.cpu().numpy()
    true_rel = np.linalg.norm(w.b - w.A @ xh) / np.linalg.norm(w.b)
    print(f"bench form: learned levels {learned}, accepted {acc}, "
          f"fallback {[info.fallback_rows[l] for l in range(info.levels_done)]}, eta {eta:.3e}, "
          f"PCG {it} (oracle {res_o.iters}), true residual {true_rel:.2e}")
    assert eta <= 1e-4, eta
    assert conv and true_rel <= 1e-8 * 1.01
    assert abs(it - res_o.iters) <= 1, (it, res_o.iters)


NOISE = -1.2   # feature 3 = log10(||F|| / ||D||) / 10 below this: the far part is rounding noise


def _compare_features(feat, kw, lev, where, learned):
    n = 0
    for st in lev.steps:
        if st.features[9] == 0:       # no far columns: the features are not computed
            assert not np.any(feat[st.i]) and kw[st.i] == 0
            continue
        idx = [0, 1, 2, 6, 7, 8, 9, 10] if st.features[3] < NOISE else list(range(11))
        np.testing.assert_allclose(feat[st.i][idx], st.features[idx], rtol=2e-5, atol=2e-6,
                                   err_msg=f"{where} block {st.i}")
        n += 1
    if learned:
        assert np.any(kw != 0)        # the sketch ran on this level
    return n


@pytest.mark.parametrize("name", ["poisson2d_64_B16", "poisson2d_512_B32"])
def test_recorded_features_match_oracle(ceg, name):
    w = wl.make_workload(name)
    csb = ceg.csb_build(w.A, w.perm, w.B)
    F = ceg.ce_factorize(csb, tol=w.tol, levels=w.levels, J=w.J, precision="fp64", row_shape=1, nmax=64,
                         record_features=True)
    Fo = _oracle(name)
    compared, levels = 0, 0
    for l, lev in enumerate(Fo.levels):
        n_g, r_g, _, _ = F.level(l)
        assert list(n_g) == list(lev.sizes)
        feat, kw = F.features(l)
        compared += _compare_features(feat, kw, lev, f"level {l}", False)
        levels += 1
        if list(r_g) != list(lev.ranks):
            break                         # later levels start from other blocks
    print(f"{name}: features of {compared} rows on {levels} levels compared")
    assert compared > 0 and levels >= 2


@pytest.mark.parametrize("name", ["poisson2d_64_B16", "poisson2d_512_B32"])
def test_learned_features_first_level(ceg, model, name):
    w = wl.make_workload(name)
    csb = ceg.csb_build(w.A, w.perm, w.B)
    F = ceg.ce_factorize(csb, tol=w.tol, levels=w.levels, J=w.J, precision="fp64", rank_model=model,
                         row_shape=1, nmax=64)
    Fo = _oracle(name)
    feat, kw = F.features(0)
    assert _compare_features(feat, kw, Fo.levels[0], "level 0 (learned)", True) > 0
