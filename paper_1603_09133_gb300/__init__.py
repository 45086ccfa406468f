"""GB300 compress-and-eliminate (CE) solver: Python binding of ``libcegpu.so``.

Same call names as the C ABI (include/ce.h): ``csb_build``, ``ce_factorize``,
``ce_apply``, ``pcg_solve``.  Device vectors are CUDA tensors (torch is used
for device memory and streams only); every step runs in the library's CUDA
kernels.  There is no CPU fallback: without the built library every call
raises.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import (  # noqa: F401
    CE_ERR_CUDA,
    CE_ERR_INVALID_ARG,
    CE_ERR_LIMIT,
    CE_ERR_NO_CONVERGENCE,
    CE_ERR_NOT_SPD,
    CE_ERR_OOM,
    CE_OK,
    CE_PREC_FP32,
    CE_PREC_FP64,
    CE_RANK_LEARNED,
    CE_RANK_SVD,
    CE_TOL_ABS,
    CE_TOL_FIXED,
    CE_TOL_REL,
)


class CEError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = _lib.load()
        msg = lib.ce_strerror(status).decode()
        extra = lib.ce_last_error().decode()
        super().__init__(f"{where}: {msg}" + (f" ({extra})" if extra else ""))
        self.status = status


def _check(status: int, where: str):
    if status != CE_OK:
        raise CEError(status, where)


def _stream_ptr(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _dev_ptr(t, what):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 \
            or not t.is_contiguous():
        raise TypeError(f"{what} must be a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


class CSB:
    """Handle of csb_build: A_0 = P A P^T in blocks of B (device copy + plan)."""

    def __init__(self, handle, n, B, nnz=None):
        self._h = handle
        self.n = n
        self.B = B
        self.nnz = nnz

    @property
    def handle(self):
        return self._h

    def colours(self):
        lib = _lib.load()
        M = lib.csb_blocks(self._h)
        col = np.zeros(M, dtype=np.int32)
        nc = C.c_int(0)
        _check(lib.csb_get_colours(self._h, col.ctypes.data_as(_lib.I32P), C.byref(nc)),
               "csb_get_colours")
        return col, nc.value

    def tuning(self, precision="fp32", learned=True):
        """(levels, shape[16], learned[16]) kept by ce_autotune for a form."""
        lib = _lib.load()
        nl = C.c_int(0)
        shape = np.zeros(16, np.int32)
        lrn = np.zeros(16, np.int32)
        _check(lib.csb_get_tuning(self._h, _prec(precision), int(bool(learned)), C.byref(nl),
                                  shape.ctypes.data_as(_lib.I32P), lrn.ctypes.data_as(_lib.I32P)),
               "csb_get_tuning")
        return nl.value, shape, lrn

    def set_tuning(self, tuning, precision="fp32", learned=True):
        """Apply a tuning from another csb of the same matrix."""
        nl, shape, lrn = tuning
        shape = np.ascontiguousarray(shape, np.int32)
        lrn = np.ascontiguousarray(lrn, np.int32)
        _check(_lib.load().csb_set_tuning(self._h, _prec(precision), int(bool(learned)), int(nl),
                                          shape.ctypes.data_as(_lib.I32P), lrn.ctypes.data_as(_lib.I32P)),
               "csb_set_tuning")

    def close(self):
        if self._h:
            _lib.load().ce_csb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Factor:
    """Handle of ce_factorize (factor L, Q on the device)."""

    def __init__(self, handle, info, csb):
        self._h = handle
        self.info = info
        self._csb = csb       # keeps the permutation alive

    @property
    def handle(self):
        return self._h

    def levels(self):
        return _lib.load().ce_factor_levels(self._h)

    def level(self, l):
        """Per-block arrays of level l: n, rank, colour, tau."""
        lib = _lib.load()
        M = lib.ce_factor_level_size(self._h, l)
        n = np.zeros(M, np.int32)
        r = np.zeros(M, np.int32)
        col = np.zeros(M, np.int32)
        tau = np.zeros(M, np.float64)
        _check(lib.ce_factor_get_level(self._h, l, n.ctypes.data_as(_lib.I32P),
                                       r.ctypes.data_as(_lib.I32P), col.ctypes.data_as(_lib.I32P),
                                       tau.ctypes.data_as(_lib.DP)), "ce_factor_get_level")
        return n, r, col, tau

    def features(self, l):
        """What the learned compression saw on level l: the rank model's
        features (M_l x nfeat, zeros where the model did not run) and the
        sketch width per block (k accepted, -k rejected, 0 none)."""
        lib = _lib.load()
        M = lib.ce_factor_level_size(self._h, l)
        feat = np.zeros((M, lib.ce_mlp_nfeatures()), np.float32)
        kw = np.zeros(M, np.int32)
        _check(lib.ce_factor_get_features(self._h, l, feat.ctypes.data_as(C.c_void_p),
                                          kw.ctypes.data_as(_lib.I32P)), "ce_factor_get_features")
        return feat, kw

    def sigma(self, l):
        """Singular values of every F_i of level l, concatenated (n_i each)."""
        lib = _lib.load()
        n, _, _, _ = self.level(l)
        s = np.zeros(int(n.sum()), np.float64)
        _check(lib.ce_factor_get_sigma(self._h, l, s.ctypes.data_as(_lib.DP)), "ce_factor_get_sigma")
        return s

    def close(self):
        if self._h:
            _lib.load().ce_factor_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


PEAK_KINDS = {"fp32_fma": 0, "fp64_fma": 1, "tf32_mma": 2, "tf32x3_mma": 3}


def measure_peak(kind: str, stream=None) -> float:
    """Measured rate (TFLOP/s) of one execution unit of the current GPU:
    'fp32_fma', 'fp64_fma', 'tf32_mma' or 'tf32x3_mma' (ce_measure_peak)."""
    out = C.c_double(0.0)
    _check(_lib.load().ce_measure_peak(PEAK_KINDS[kind], C.byref(out), _stream_ptr(stream)),
           "ce_measure_peak")
    return out.value


def launch_count() -> int:
    """Kernels this library has launched in the process (graph replays
    count every kernel node)."""
    return int(_lib.load().ce_launch_count())


def csb_build(A, perm, B: int) -> CSB:
    """A (scipy sparse, symmetric), perm[k] = original index of row k, block B."""
    import scipy.sparse as sp
    lib = _lib.load()
    A = sp.csr_matrix(A)
    n = A.shape[0]
    rowptr = np.ascontiguousarray(A.indptr, dtype=np.int64)
    col = np.ascontiguousarray(A.indices, dtype=np.int32)
    val = np.ascontiguousarray(A.data, dtype=np.float64)
    pm = np.ascontiguousarray(perm, dtype=np.int32)
    if pm.shape != (n,):
        raise ValueError("perm must have one entry per row")
    h = C.c_void_p()
    _check(lib.csb_build(n, rowptr.ctypes.data_as(_lib.I64P), col.ctypes.data_as(_lib.I32P),
                         val.ctypes.data_as(_lib.DP), pm.ctypes.data_as(_lib.I32P), int(B),
                         C.byref(h)), "csb_build")
    return CSB(h, n, int(B), int(A.nnz))


def csb_update_values(csb: CSB, A, stream=None):
    """New values for the csb's pattern (A: scipy sparse with the same CSR
    pattern as the matrix given to csb_build); the next ce_factorize reuses
    all symbolic work."""
    import scipy.sparse as sp
    lib = _lib.load()
    A = sp.csr_matrix(A)
    if A.shape != (csb.n, csb.n) or csb.nnz is None or A.nnz != csb.nnz:
        raise ValueError("A must have the shape and number of stored entries of the csb's matrix")
    val = np.ascontiguousarray(A.data, dtype=np.float64)
    _check(lib.csb_update_values(csb.handle, val.ctypes.data_as(_lib.DP), _stream_ptr(stream)),
           "csb_update_values")


def stack_systems(systems):
    """Stacked CSR arrays of independent systems [(A, perm, B), ...] in the
    layout csb_build_batched_csr takes: (row_off, rowptr, col, val, perm, Bs)."""
    import scipy.sparse as sp
    mats = [sp.csr_matrix(A) for A, _, _ in systems]
    row_off = np.zeros(len(mats) + 1, np.int64)
    row_off[1:] = np.cumsum([m.shape[0] for m in mats])
    S = sp.block_diag(mats, format="csr")
    pm = np.concatenate([np.asarray(p, np.int64) + row_off[s]
                         for s, (_, p, _) in enumerate(systems)]).astype(np.int32)
    return (row_off, np.ascontiguousarray(S.indptr, dtype=np.int64),
            np.ascontiguousarray(S.indices, dtype=np.int32),
            np.ascontiguousarray(S.data, dtype=np.float64), pm,
            np.asarray([B for _, _, B in systems], np.int32))


def csb_build_batched_csr(row_off, rowptr, col, val, perm, Bs) -> CSB:
    """csb_build_batched on stacked host arrays (see stack_systems)."""
    lib = _lib.load()
    row_off = np.ascontiguousarray(row_off, np.int64)
    rowptr = np.ascontiguousarray(rowptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    val = np.ascontiguousarray(val, np.float64)
    perm = np.ascontiguousarray(perm, np.int32)
    Bs = np.ascontiguousarray(Bs, np.int32)
    h = C.c_void_p()
    _check(lib.csb_build_batched(len(row_off) - 1, row_off.ctypes.data_as(_lib.I64P),
                                 rowptr.ctypes.data_as(_lib.I64P), col.ctypes.data_as(_lib.I32P),
                                 val.ctypes.data_as(_lib.DP), perm.ctypes.data_as(_lib.I32P),
                                 Bs.ctypes.data_as(_lib.I32P), C.byref(h)), "csb_build_batched")
    csb = CSB(h, int(row_off[-1]), int(Bs[0]), int(rowptr[-1]))
    csb.row_off = row_off
    return csb


def csb_build_batched(systems) -> CSB:
    """Many independent systems [(A, perm, B), ...] as one block-diagonal
    batch; rows are stacked in the order given."""
    return csb_build_batched_csr(*stack_systems(systems))


_TOL_MODES = {"rel": CE_TOL_REL, "abs": CE_TOL_ABS, "fixed": CE_TOL_FIXED}


def _prec(precision):
    if precision not in ("fp64", "fp32"):
        raise ValueError("precision must be 'fp64' or 'fp32'")
    return CE_PREC_FP64 if precision == "fp64" else CE_PREC_FP32


_ENGINES = {"tc": 0, "cuda": 1, "tc_bf16_schur": 2}


def _opts(tol, levels, J, precision, tol_mode, coloring, stream, rank_model, oversample, seed,
          row_shape, rank=16, nmax=0, record_features=False, gemm_engine="tc"):
    lib = _lib.load()
    o = _lib.ce_opts()
    lib.ce_opts_default(C.byref(o))
    o.tol = float(tol)
    if tol_mode not in _TOL_MODES:
        raise ValueError(f"tol_mode must be one of {sorted(_TOL_MODES)}")
    o.tol_mode = _TOL_MODES[tol_mode]
    o.rank = int(rank)
    o.levels = int(levels)
    o.J = int(J)
    o.precision = CE_PREC_FP64 if precision == "fp64" else CE_PREC_FP32
    # True / 1: distance-2 colours, 2: distance-1 colours, False / 0: natural order
    o.coloring = 2 if coloring == 2 else (1 if coloring else 0)
    o.stream = _stream_ptr(stream)
    if rank_model is not None:
        o.rank_mode = CE_RANK_LEARNED
        o.rank_model = C.c_void_p(rank_model.model.data_ptr())
        o.oversample = int(oversample)
        o.seed = int(seed)
    o.row_shape = int(row_shape)
    o.nmax = int(nmax)
    o.record_features = 1 if record_features else 0
    if gemm_engine not in _ENGINES:
        raise ValueError(f"gemm_engine must be one of {sorted(_ENGINES)}")
    o.gemm_engine = _ENGINES[gemm_engine]
    return o


def ce_autotune(csb: CSB, tol=1e-4, levels=4, J=4, precision="fp64", tol_mode="rel",
                coloring=True, stream=None, rank_model=None, oversample=8, seed=0, nmax=0):
    """Time every row-kernel CTA shape per level, and the large-row path as
    shape 3 (and, with a rank model, learned compression against the exact
    SVD), and keep the fastest in the csb; returns the
    [learned/exact][shape][level] times (ms) as a 2 x 4 x levels array (the
    exact half is zero without a rank model)."""
    lib = _lib.load()
    o = _opts(tol, levels, J, precision, tol_mode, coloring, stream, rank_model, oversample, seed, -1,
              nmax=nmax)
    t = np.zeros(2 * 4 * 16, np.float64)
    _check(lib.ce_autotune(csb.handle, C.byref(o), t.ctypes.data_as(_lib.DP)), "ce_autotune")
    return t.reshape(2, 4, 16)[:, :, :levels]


def ce_factorize(csb: CSB, tol=1e-4, levels=4, J=4, precision="fp64", tol_mode="rel",
                 coloring=True, stream=None, rank_model=None, oversample=8, seed=0,
                 row_shape=-1, batched=False, rank=16, nmax=0, record_features=False,
                 gemm_engine="tc") -> Factor:
    """Algorithm 1 on the device; returns the factor (raises CEError).

    ``rank_model`` (a :class:`RankModel`) switches the compression step to the
    learned rank + randomized range finder with exact-SVD fallback.
    ``tol_mode="fixed"`` is CE(r) with r = ``rank`` (``tol`` unused).
    ``nmax`` > 0 caps the super-blocks at nmax rows (runs of J halved until
    they fit); 0 is the paper's plain runs of J.  ``record_features`` keeps the
    rank model's features of every row (Factor.features), also without a
    model.  ``gemm_engine`` picks the engine of the large-row products in the
    FP32 form: "tc" (tensor cores, three split-BF16 products), "cuda" (FP32 on
    the CUDA cores) or "tc_bf16_schur" (one BF16 product for the Schur updates).
    """
    lib = _lib.load()
    o = _opts(tol, levels, J, precision, tol_mode, coloring, stream, rank_model, oversample, seed,
              row_shape, rank, nmax, record_features, gemm_engine)
    info = _lib.ce_info()
    h = C.c_void_p()
    entry = lib.ce_factorize_batched if batched else lib.ce_factorize
    st = entry(csb.handle, C.byref(o), C.byref(h), C.byref(info))
    if st != CE_OK:
        where = "ce_factorize"
        if st == CE_ERR_NOT_SPD:
            why = {1: f"pivot {info.err_pivot} = {info.err_value:.3e}",
                   2: "non-finite singular values"}.get(info.err_reason, "")
            where += f" (level {info.err_level}, block {info.err_block}; {why})"
        err = CEError(st, where)
        err.info = info
        raise err
    return Factor(h, info, csb)


def ce_factorize_batched(csb: CSB, **kw) -> Factor:
    """ce_factorize through the batch entry point (the handle must come from
    csb_build_batched)."""
    return ce_factorize(csb, batched=True, **kw)


def ce_apply(F: Factor, r, z, stream=None):
    """z = M^{-1} r on the device (r, z: float64 CUDA tensors, may alias)."""
    lib = _lib.load()
    _check(lib.ce_apply(F.handle, _dev_ptr(r, "r"), _dev_ptr(z, "z"), _stream_ptr(stream)),
           "ce_apply")
    return z


def pcg_solve(csb: CSB, F: Factor, b, x, rtol=1e-8, maxit=1000, stream=None, check=True):
    """FP64 PCG on the device; returns (iters, relres, converged)."""
    lib = _lib.load()
    info = _lib.ce_pcg_info()
    st = lib.pcg_solve(csb.handle, F.handle, _dev_ptr(b, "b"), _dev_ptr(x, "x"), float(rtol),
                       int(maxit), C.byref(info), _stream_ptr(stream))
    if check and st not in (CE_OK, CE_ERR_NO_CONVERGENCE):
        raise CEError(st, "pcg_solve")
    return info.iters, info.relres, bool(info.converged)


def minres_solve(csb: CSB, F: Factor, b, x, rtol=1e-10, maxit=1000, stream=None, check=True):
    """FP64 preconditioned MINRES on the device (the Krylov method of the
    paper's Section 4); returns (iters, relres, converged) with relres the
    preconditioned residual norm over ||b||_{M^{-1}}."""
    lib = _lib.load()
    info = _lib.ce_pcg_info()
    st = lib.minres_solve(csb.handle, F.handle, _dev_ptr(b, "b"), _dev_ptr(x, "x"), float(rtol),
                          int(maxit), C.byref(info), _stream_ptr(stream))
    if check and st not in (CE_OK, CE_ERR_NO_CONVERGENCE):
        raise CEError(st, "minres_solve")
    return info.iters, info.relres, bool(info.converged)


def pcg_solve_batched(csb: CSB, F: Factor, b, x, rtol=1e-8, maxit=1000, stream=None, check=True):
    """Per-system FP64 PCG of a batch; returns (iters, relres, converged)
    as numpy arrays with one entry per system."""
    lib = _lib.load()
    ns = len(csb.row_off) - 1
    its = np.zeros(ns, np.int32)
    rel = np.zeros(ns, np.float64)
    conv = np.zeros(ns, np.int32)
    info = _lib.ce_pcg_info()
    st = lib.pcg_solve_batched(csb.handle, F.handle, _dev_ptr(b, "b"), _dev_ptr(x, "x"), float(rtol),
                               int(maxit), its.ctypes.data_as(_lib.I32P), rel.ctypes.data_as(_lib.DP),
                               conv.ctypes.data_as(_lib.I32P), C.byref(info), _stream_ptr(stream))
    if check and st not in (CE_OK, CE_ERR_NO_CONVERGENCE):
        raise CEError(st, "pcg_solve_batched")
    return its, rel, conv.astype(bool)


class RankModel:
    """The rank-predictor MLP on the device: FP32 parameters + FP16 model."""

    def __init__(self, seed=0, device="cuda"):
        import torch
        lib = _lib.load()
        self.nparams = lib.ce_mlp_nparams()
        self.nfeatures = lib.ce_mlp_nfeatures()
        self.theta = torch.empty(self.nparams, dtype=torch.float32, device=device)
        self.model = torch.empty(self.nparams, dtype=torch.float16, device=device)
        _check(lib.ce_mlp_init(C.c_void_p(self.theta.data_ptr()), int(seed), _stream_ptr(None)),
               "ce_mlp_init")
        self.pack()

    def set_params(self, theta):
        import torch
        self.theta.copy_(torch.as_tensor(np.asarray(theta, dtype=np.float32)))
        self.pack()

    def pack(self):
        _check(_lib.load().ce_mlp_pack(C.c_void_p(self.theta.data_ptr()),
                                       C.c_void_p(self.model.data_ptr()), _stream_ptr(None)),
               "ce_mlp_pack")

    def grad(self, X, t):
        """Full-batch gradient of 0.5 mean (y - t)^2 (FP32, device)."""
        import torch
        Xd = torch.as_tensor(np.ascontiguousarray(X, np.float32), device=self.theta.device)
        td = torch.as_tensor(np.ascontiguousarray(t, np.float32), device=self.theta.device)
        g = torch.empty_like(self.theta)
        _check(_lib.load().ce_mlp_grad(C.c_void_p(Xd.data_ptr()), C.c_void_p(td.data_ptr()),
                                       Xd.shape[0], C.c_void_p(self.theta.data_ptr()),
                                       C.c_void_p(g.data_ptr()), _stream_ptr(None)), "ce_mlp_grad")
        return g

    def train(self, X, t, steps=2000, lr=3e-3):
        """Adam on the full batch; returns the final loss of the FP16 model."""
        import torch
        Xd = torch.as_tensor(np.ascontiguousarray(X, np.float32), device=self.theta.device)
        td = torch.as_tensor(np.ascontiguousarray(t, np.float32), device=self.theta.device)
        loss = C.c_double(0.0)
        _check(_lib.load().ce_mlp_train(C.c_void_p(Xd.data_ptr()), C.c_void_p(td.data_ptr()),
                                        Xd.shape[0], C.c_void_p(self.theta.data_ptr()), int(steps),
                                        float(lr), C.byref(loss), _stream_ptr(None)), "ce_mlp_train")
        self.pack()
        return loss.value

    def predict(self, X):
        """FP16 inference (the code the compression step runs)."""
        import torch
        Xd = torch.as_tensor(np.ascontiguousarray(X, np.float32), device=self.theta.device)
        out = torch.empty(Xd.shape[0], dtype=torch.float32, device=self.theta.device)
        _check(_lib.load().ce_mlp_predict(C.c_void_p(Xd.data_ptr()), Xd.shape[0],
                                          C.c_void_p(self.model.data_ptr()),
                                          C.c_void_p(out.data_ptr()), _stream_ptr(None)),
               "ce_mlp_predict")
        return out


def rank_training_data():
    """(features, r/n) training set written from the oracle's ranks."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "models", "rank_train.npz")
    d = np.load(path)
    return d["X"], d["t"]


def trained_rank_model(steps=3000, lr=3e-3, seed=0):
    """Rank model trained on the GPU on the stored training set."""
    X, t = rank_training_data()
    m = RankModel(seed=seed)
    m.loss = m.train(X, t, steps=steps, lr=lr)
    return m
