"""The library's grouped GEMM engines (used by the large-row path for the
transforms, the triangular products and the Schur updates of Algorithm 2 on
big blocks) against an FP64 product, through the C ABI (ce_debug_gemm), on
ragged shapes spanning several 128 x 128 tiles and 64-deep K blocks, every
operand layout, and alpha / beta accumulation.

Each entry of C = alpha op(A) op(B) + beta C is checked against the
elementwise bound |err| <= gamma (|alpha| |A| |B| + |beta| |C0|) with gamma
from the arithmetic: CUDA cores FP32 K u32 + u32, FP64 K u64 + u64; tensor
cores with FP32 operands split into BF16 hi + lo and three products
(hi*hi + hi*lo + lo*hi): the dropped lo*lo and the split's residual are
below 2^-15 of each term, plus FP32 accumulation; one BF16 product: two
BF16 roundings, 2^-7.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_09133_gb300 import _lib, build
    build.build()
    return _lib, _lib.load()


U32 = 2.0 ** -24
U64 = 2.0 ** -53
GAMMA = {0: lambda K: 2 * K * U32 + U32, 3: lambda K: 2 * K * U64 + U64,
         1: lambda K: 2.0 ** -15 + 2 * K * U32, 2: lambda K: 2.0 ** -7 + 2 * K * U32}


def _run(lib, engine, M, N, K, ta, tb, tc, alpha, beta, seed):
    _lib, L = lib
    rng = np.random.default_rng(seed)
    dt = np.float64 if engine == 3 else np.float32
    A = rng.standard_normal((K, M) if ta else (M, K)).astype(dt)
    B = rng.standard_normal((N, K) if tb else (K, N)).astype(dt)
    C0 = rng.standard_normal((N, M) if tc else (M, N)).astype(dt)
    dA, dB, dC = (torch.as_tensor(x, device="cuda") for x in (A, B, C0))
    st = L.ce_debug_gemm(engine, M, N, K, C.c_void_p(dA.data_ptr()), A.shape[1], ta, C.c_void_p(dB.data_ptr()),
                         B.shape[1], tb, C.c_void_p(dC.data_ptr()), C0.shape[1], tc, alpha, beta,
                         C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == _lib.CE_OK, L.ce_last_error()
    Ad = A.astype(np.float64).T if ta else A.astype(np.float64)
    Bd = B.astype(np.float64).T if tb else B.astype(np.float64)
    C0d = C0.astype(np.float64).T if tc else C0.astype(np.float64)
    ref = alpha * (Ad @ Bd) + beta * C0d
    bound = GAMMA[engine](K) * (abs(alpha) * (np.abs(Ad) @ np.abs(Bd)) + abs(beta) * np.abs(C0d))
    got = dC.cpu().numpy().astype(np.float64)
    got = got.T if tc else got
    err = np.abs(got - ref)
    worst = float(np.max(err / np.maximum(bound, 1e-300)))
    return worst, float(np.max(err))


SHAPES = [(200, 150, 97), (128, 128, 64), (33, 300, 700), (257, 129, 1), (5, 7, 3), (390, 260, 259)]


@pytest.mark.parametrize("engine", [0, 1, 2, 3])
@pytest.mark.parametrize("M,N,K", SHAPES)
def test_gemm_engine(lib, engine, M, N, K):
    for case, (ta, tb, tc) in enumerate([(0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 1, 1), (0, 0, 1)]):
        for alpha, beta in ((1.0, 0.0), (-1.0, 1.0)):
            worst, emax = _run(lib, engine, M, N, K, ta, tb, tc, alpha, beta, seed=case)
            assert worst <= 1.0, (engine, M, N, K, ta, tb, tc, alpha, beta, worst, emax)


def test_tensor_core_split_is_fp32_class(lib):
    """Three split-BF16 products are far more accurate than one."""
    w3, e3 = _run(lib, 1, 256, 256, 512, 0, 0, 0, 1.0, 0.0, seed=7)
    w1, e1 = _run(lib, 2, 256, 256, 512, 0, 0, 0, 1.0, 0.0, seed=7)
    print(f"max abs error: 3 passes {e3:.3e}, 1 pass {e1:.3e}")
    assert e3 < e1 / 50
