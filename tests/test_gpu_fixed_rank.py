"""GPU: CE(r), the fixed-rank strategy of the Section 2.2 remark, against the
FP64 oracle.

Where a far row has fewer than r directions above rounding noise, CE(r) cuts
at the noise floor, and a direction near that floor may be kept by one side
and dropped by the other.  The next level then groups different rows and its
fixed-rank truncation drops different content, so M is defined only up to
that.  Parity is therefore checked where every cut is clear of rounding.

FP64 form, on grids whose cuts are clear (p2 and GRF 64^2, r = 8): colours
bit-exact, ranks equal except for directions at rounding level
(sigma <= 1e-10 sigma_1), the apply within 1e-10 of the oracle's, PCG
iterations within +-1 and a true residual <= 1e-8.
FP32 form (its noise floor n u_32 sigma_1 cuts far above the oracle's): what
holds whatever the noise-level decisions are -- no rank above r, PCG to a true
residual <= 1e-8 in at most twice the oracle's iterations plus two.
CE(r) with the learned rank path, or r < 0, is refused on the host.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as wl
from oracle import ce as oce

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = [
    # kind, grid side, box, B, r, levels
    ("p2", 64, (4, 4), 16, 8, 3),
    ("grf", 64, (4, 4), 16, 8, 3),
]
CASES_FP32 = CASES + [("p2", 128, (8, 4), 32, 16, 3)]


@pytest.fixture(scope="module")
def ceg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_09133_gb300 import build
    build.build()
    import paper_1603_09133_gb300 as m
    return m


def _problem(kind, n, box):
    A = wl.diffusion2d(wl.grf2d(n, seed=3)) if kind == "grf" else wl.poisson2d(n)
    return A, wl.box_perm((n, n), box)


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")


def _levels_agree(F, Fo):
    for l, lev in enumerate(Fo.levels):
        n_g, r_g, c_g, _ = F.level(l)
        if list(n_g) != list(lev.sizes):
            return l               # sizes moved by a noise-level flip below
        assert list(c_g) == list(lev.colour), l
        for st in lev.steps:
            if r_g[st.i] != st.r:
                lo, hi = sorted((int(r_g[st.i]), st.r))
                assert np.all(st.sigma[lo:hi] <= 1e-10 * st.sigma[0]), (l, st.i, r_g[st.i], st.r)
    return len(Fo.levels)


@pytest.mark.parametrize("kind,n,box,B,r,levels", CASES)
def test_fixed_rank_fp64_matches_oracle(ceg, kind, n, box, B, r, levels):
    A, perm = _problem(kind, n, box)
    b = wl.rhs(n * n, 0)
    Fo = oce.factorize(A, perm, B, 0.0, levels, 4, tol_mode="fixed", rank=r)
    csb = ceg.csb_build(A, perm, B)
    F = ceg.ce_factorize(csb, levels=levels, J=4, tol_mode="fixed", rank=r)
    agreed = _levels_agree(F, Fo)
    assert agreed >= 1
    z = torch.empty(n * n, dtype=torch.float64, device="cuda")
    ceg.ce_apply(F, _dev(b), z)
    zo = oce.apply(Fo, b)
    err = np.linalg.norm(z.cpu().numpy() - zo) / np.linalg.norm(zo)
    print(f"{kind} {n}^2 r={r}: levels compared {agreed}, apply error {err:.2e}")
    assert err <= 1e-10
    x = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    it, rel, conv = ceg.pcg_solve(csb, F, _dev(b), x, 1e-8, 500)
    res_o = oce.pcg(A, Fo, b, 1e-8, 500)
    true = np.linalg.norm(b - A @ x.cpu().numpy()) / np.linalg.norm(b)
    assert conv and abs(it - res_o.iters) <= 1, (it, res_o.iters)
    assert true <= 1e-8 * 1.01


@pytest.mark.parametrize("kind,n,box,B,r,levels", CASES_FP32)
def test_fixed_rank_fp32_preconditions(ceg, kind, n, box, B, r, levels):
    A, perm = _problem(kind, n, box)
    b = wl.rhs(n * n, 1)
    Fo = oce.factorize(A, perm, B, 0.0, levels, 4, tol_mode="fixed", rank=r)
    csb = ceg.csb_build(A, perm, B)
    F = ceg.ce_factorize(csb, levels=levels, J=4, tol_mode="fixed", rank=r, precision="fp32")
    for l in range(F.levels()):
        assert int(F.level(l)[1].max(initial=0)) <= r + 4   # fixed rank (ties aside)
    x = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    it, rel, conv = ceg.pcg_solve(csb, F, _dev(b), x, 1e-8, 500)
    true = np.linalg.norm(b - A @ x.cpu().numpy()) / np.linalg.norm(b)
    res_o = oce.pcg(A, Fo, b, 1e-8, 500)
    print(f"{kind} {n}^2 r={r} fp32: PCG {it} iterations (oracle FP64 {res_o.iters}), residual {true:.2e}")
    assert conv and true <= 1e-8 * 1.01
    assert it <= 2 * res_o.iters + 2


def test_fixed_rank_refusals(ceg):
    from paper_1603_09133_gb300 import _lib
    lib = _lib.load()
    A, perm = _problem("p2", 32, (4, 4))
    csb = ceg.csb_build(A, perm, 16)
    with pytest.raises(ceg.CEError):
        ceg.ce_factorize(csb, levels=2, tol_mode="fixed", rank=-1)
    # CE(r) with the learned rank path: refused before any device work
    o = _lib.ce_opts()
    lib.ce_opts_default(C.byref(o))
    o.tol_mode = _lib.CE_TOL_FIXED
    o.rank = 8
    o.levels = 2
    o.rank_mode = _lib.CE_RANK_LEARNED
    dummy = torch.zeros(16, dtype=torch.float16, device="cuda")
    o.rank_model = C.c_void_p(dummy.data_ptr())
    h = C.c_void_p()
    info = _lib.ce_info()
    assert lib.ce_factorize(csb.handle, C.byref(o), C.byref(h), C.byref(info)) == ceg.CE_ERR_INVALID_ARG
    assert not h.value
