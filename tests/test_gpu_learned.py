"""GPU tests of the learned compression: the rank-predictor MLP kernels against
the FP64 CPU reference (oracle/mlp.py), and the learned factorization (MLP
width + randomized range finder + exact-SVD fallback) against the exact one.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import ce as oce
from oracle import mlp

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
def trained(ceg):
    X, t = ceg.rank_training_data()
    rng = np.random.default_rng(0)
    idx = rng.permutation(len(t))
    ntr = int(0.9 * len(t))
    tr, te = idx[:ntr], idx[ntr:]
    model = ceg.RankModel(seed=0)
    loss0 = 0.5 * float(np.mean((model.predict(X[tr]).cpu().numpy() - t[tr]) ** 2))
    loss = model.train(X[tr], t[tr], steps=3000, lr=3e-3)
    return model, X, t, tr, te, loss0, loss


def test_mlp_gradient_matches_cpu_reference(ceg):
    X, t = ceg.rank_training_data()
    Xs, ts = X[:300], t[:300]
    theta = mlp.init(2).astype(np.float32)
    model = ceg.RankModel(seed=1)
    model.set_params(theta)
    g_gpu = model.grad(Xs, ts).cpu().numpy().astype(np.float64)
    g_ref = mlp.grad(theta.astype(np.float64), Xs.astype(np.float64), ts.astype(np.float64))
    rel = np.linalg.norm(g_gpu - g_ref) / np.linalg.norm(g_ref)
    assert rel <= 1e-4, rel


def test_mlp_training_and_fp16_inference(trained):
    model, X, t, tr, te, loss0, loss = trained
    assert loss < 0.25 * loss0, (loss0, loss)
    theta = model.theta.cpu().numpy().astype(np.float64)
    y_ref, _ = mlp.forward(theta, X[te].astype(np.float64))
    y_gpu = model.predict(X[te]).cpu().numpy()
    assert np.max(np.abs(y_gpu - y_ref)) <= 2e-2        # FP16 weights and activations
    mae = np.mean(np.abs(y_gpu - t[te]))
    print(f"held-out MAE of r/n: {mae:.4f}, train loss {loss0:.4f} -> {loss:.5f}")
    assert mae <= 0.06


def _apply(ceg, F, b):
    r = torch.as_tensor(b, device="cuda")
    z = torch.empty_like(r)
    ceg.ce_apply(F, r, z)
    torch.cuda.synchronize()
    return z.cpu().numpy()


def _pcg(ceg, csb, F, A, b):
    x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
    it, rel, conv = ceg.pcg_solve(csb, F, torch.as_tensor(b, device="cuda"), x, 1e-8, 500)
    torch.cuda.synchronize()
    xh = x.cpu().numpy()
    return it, conv, np.linalg.norm(b - A @ xh) / np.linalg.norm(b)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_learned_factorization_small(ceg, trained, precision):
    model = trained[0]
    w = wl.make_workload("poisson2d_64_B16")
    csb = ceg.csb_build(w.A, w.perm, w.B)
    Fe = ceg.ce_factorize(csb, tol=w.tol, levels=w.levels, J=w.J, precision=precision)
    Fl = ceg.ce_factorize(csb, tol=w.tol, levels=w.levels, J=w.J, precision=precision,
                          rank_model=model)
    acc = sum(Fl.info.learned_rows[l] for l in range(Fl.info.levels_done))
    fb = sum(Fl.info.fallback_rows[l] for l in range(Fl.info.levels_done))
    assert acc > 0
    it_e, conv_e, res_e = _pcg(ceg, csb, Fe, w.A, w.b)
    it_l, conv_l, res_l = _pcg(ceg, csb, Fl, w.A, w.b)
    assert conv_l and res_l <= 1e-8 * 1.01
    assert it_l <= it_e + 2, (it_e, it_l)
    # the learned M against the oracle's operator (normwise backward error)
    Fo = oce.factorize(w.A, w.perm, w.B, w.tol, w.levels, w.J)
    z = _apply(ceg, Fl, w.b)
    import scipy.sparse.linalg as spla
    anorm = float(spla.eigsh(w.A, k=1, which="LA", return_eigenvectors=False)[0])
    eta = np.linalg.norm(w.b - oce.multiply(Fo, z)) / (anorm * np.linalg.norm(z) + np.linalg.norm(w.b))
    print(f"{precision}: accepted {acc}, fallback {fb}, PCG {it_e} -> {it_l}, eta {eta:.2e}")
    assert eta <= 1e-4


def test_learned_gain_full_size(ceg, trained):
    """What the trained network gains: 512^2 Poisson, FP32 form, exact SVD vs
    learned widths (same matrix, same tolerance; super-blocks capped at 64 rows
    as in the benchmark, so every level runs the row kernel)."""
    model = trained[0]
    w = wl.make_workload("poisson2d_512_B32")
    csb = ceg.csb_build(w.A, w.perm, w.B)
    res = {}
    for name, rm in (("exact", None), ("learned", model)):
        ceg.ce_factorize(csb, tol=w.tol, levels=w.levels, J=w.J, precision="fp32", rank_model=rm, nmax=64)
        F = ceg.ce_factorize(csb, tol=w.tol, levels=w.levels, J=w.J, precision="fp32", rank_model=rm,
                             nmax=64)
        ms = sum(F.info.level_ms[l] for l in range(F.info.levels_done))
        it, conv, rel = _pcg(ceg, csb, F, w.A, w.b)
        assert conv and rel <= 1e-8 * 1.01
        acc = sum(F.info.learned_rows[l] for l in range(F.info.levels_done))
        fb = sum(F.info.fallback_rows[l] for l in range(F.info.levels_done))
        res[name] = (ms, it, acc, fb)
    print("row-kernel ms / PCG its / accepted / fallback:", res)
    assert res["learned"][2] > res["learned"][3]           # most rows take the sketch
    assert res["learned"][1] <= res["exact"][1] + 1
    assert res["learned"][0] < res["exact"][0]
