// Grouped GEMM on the 5th-generation tensor cores (tcgen05) for the FP32 form
// of the large-row path: C = alpha op(A) op(B) + beta op(Cin) for a list of
// independent products (the per-row transforms, the TRSM products and the
// Schur updates A(p, q) -= W_p^T W_q of Algorithm 2 on big blocks).
//
// Operands are FP32 in global memory with arbitrary layouts.  Each distinct
// operand ("panel") is packed once per launch into two BF16 planes, x = hi +
// lo with hi = bf16(x) and lo = bf16(x - hi), K-major (row = output row or
// column, K contiguous), zero beyond K.  One 2D tensor map covers both planes;
// TMA (cp.async.bulk.tensor, 128-byte swizzle) stages 128 x 64 tiles into a
// 3-stage shared-memory ring tracked by mbarriers; one thread issues
// tcgen05.mma (kind::f16, BF16 x BF16, FP32 accumulate, M = N = 128, K = 16
// per instruction) into a 128-column TMEM accumulator: hi*hi + hi*lo + lo*hi
// per K step (the dropped lo*lo term is ~2^-16 of the product), then the four
// warps read the accumulator back with tcgen05.ld and apply alpha / beta.
// With `passes` = 1 only hi*hi runs (plain BF16 products with FP32
// accumulation).
//
// Every mbarrier wait is bounded (time and polls): on expiry the kernel sets
// the error word and returns after releasing its TMEM.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "kernels.h"

namespace ce {

namespace {

constexpr int TM = 128, TN = 128, TK = 64, STAGES = 3;
constexpr int PLANE_A = TM * TK * 2;  // bytes of one 128 x 64 BF16 tile
constexpr int PLANE_B = TN * TK * 2;
constexpr int STAGE = 2 * PLANE_A + 2 * PLANE_B;
constexpr int TC_THREADS = 128;
constexpr int TC_SMEM = STAGES * STAGE + 1024;  // + alignment slack (1024-byte swizzle atoms)
constexpr unsigned long long kTcWaitNs = 1000000000ull;  // an mbarrier wait gives up after 1 s

struct TcTask {
  int a_row, b_row;   // first row of the A / B panel in the hi plane
  int M, N, kb;       // output size, K blocks of 64
  int tile0;
  int ldc, ldcin, tc, tcin, atomic;
  float alpha, beta;
  void* C;
  const void* Cin;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait for the phase with the given parity; false (and the error
// word set) when it did not complete in time or another role gave up
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, volatile int* abort_flag) {
  const unsigned long long t0 = gtimer();
  for (int it = 0; it < (1 << 22); ++it) {
    if (mbar_try(bar, parity)) return true;
    if (*abort_flag) return false;
    if ((it & 63) == 63 && gtimer() - t0 > kTcWaitNs) break;
  }
  *abort_flag = 1;
  atomicExch(err, 1);
  return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), version 1 (bit 46)
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// instruction descriptor of kind::f16: D F32, A and B BF16, both K-major, N, M
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap map, const TcTask* __restrict__ tasks, int ntasks,
                   int lo_rows, int passes, int* err) {
  extern __shared__ unsigned char tc_smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], acc_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_task;
  __shared__ volatile int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  if (tid == 0) {
    int lo = 0, hi = ntasks - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tasks[mid].tile0 <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    s_task = lo;
    s_abort = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    mbar_init(smem_u32(&acc_bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(TN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const TcTask tk = tasks[s_task];
  const int tl = blockIdx.x - tk.tile0, tn = (tk.N + TN - 1) / TN;
  const int m0 = (tl / tn) * TM, n0 = (tl % tn) * TN;
  const uint32_t dtm = tmem_base;
  const int nkb = tk.kb;
  if (warp == 0 && lane == 0) {
    // producer: TMA of the hi and lo tiles of A and B for each K block
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES;
      if (kb >= STAGES && !mbar_wait(smem_u32(&empty_bar[s]), ((kb / STAGES) - 1) & 1, err, &s_abort)) break;
      unsigned char* st = base + s * STAGE;
      const uint32_t fb = smem_u32(&full_bar[s]);
      mbar_expect_tx(fb, STAGE);
      const int x = kb * TK;
      tma_load_2d(smem_u32(st), &map, x, tk.a_row + m0, fb);
      tma_load_2d(smem_u32(st + PLANE_A), &map, x, lo_rows + tk.a_row + m0, fb);
      tma_load_2d(smem_u32(st + 2 * PLANE_A), &map, x, tk.b_row + n0, fb);
      tma_load_2d(smem_u32(st + 2 * PLANE_A + PLANE_B), &map, x, lo_rows + tk.b_row + n0, fb);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    bool ok = true;
    for (int kb = 0; kb < nkb && ok; ++kb) {
      const int s = kb % STAGES;
      if (!mbar_wait(smem_u32(&full_bar[s]), (kb / STAGES) & 1, err, &s_abort)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      unsigned char* st = base + s * STAGE;
      const uint64_t ahi = sdesc(smem_u32(st)), alo = sdesc(smem_u32(st + PLANE_A));
      const uint64_t bhi = sdesc(smem_u32(st + 2 * PLANE_A)), blo = sdesc(smem_u32(st + 2 * PLANE_A + PLANE_B));
#pragma unroll
      for (int kk = 0; kk < TK / 16; ++kk) {
        const uint64_t adv = (uint64_t)((kk * 32) >> 4);  // 16 BF16 = 32 bytes along K
        mma_bf16(dtm, ahi + adv, bhi + adv, (kb > 0 || kk > 0) ? 1u : 0u);
        if (passes > 1) {
          mma_bf16(dtm, ahi + adv, blo + adv, 1u);
          mma_bf16(dtm, alo + adv, bhi + adv, 1u);
        }
      }
      mma_commit(smem_u32(&empty_bar[s]));   // the stage is free once these MMAs complete
    }
    if (ok) mma_commit(smem_u32(&acc_bar));   // the accumulator is complete
  }
  // epilogue: warp w holds rows 32 w .. 32 w + 31 of the tile (TMEM lanes)
  __syncwarp();
  // warp-uniform: tcgen05.ld is executed by whole warps only
  const bool have = __all_sync(0xffffffffu, mbar_wait(smem_u32(&acc_bar), 0, err, &s_abort));
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (have) {
    const int m = m0 + warp * 32 + lane;
    float* C = static_cast<float*>(tk.C);
    const float* Cin = static_cast<const float*>(tk.Cin);
    for (int c0 = 0; c0 < TN; c0 += 16) {
      float v[16];
      tmem_ld16(dtm + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (m < tk.M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = n0 + c0 + j;
          if (n < tk.N) {
            float o = tk.alpha * v[j];
            float* dst = tk.tc ? &C[(int64_t)n * tk.ldc + m] : &C[(int64_t)m * tk.ldc + n];
            if (tk.atomic) {
              atomicAdd(dst, o);
            } else {
              if (tk.beta != 0.f)
                o += tk.beta * (tk.tcin ? Cin[(int64_t)n * tk.ldcin + m] : Cin[(int64_t)m * tk.ldcin + n]);
              *dst = o;
            }
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(dtm), "r"(TN) : "memory");
  }
}

// one operand panel: rows x K elements, element (row, k) at
// src[trans ? k * ld + row : row * ld + k], packed at hi-plane row `row0`
struct Panel {
  const float* src;
  int ld, trans, rows, K;
  int row0;
};

__global__ void pack_panels_kernel(const Panel* panels, int npanels, int KP, int lo_rows, __nv_bfloat16* pk) {
  const Panel p = panels[blockIdx.y];
  const int64_t total = (int64_t)p.rows * p.K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int row, k;
    if (p.trans) {  // rows contiguous in the source: read along rows
      k = static_cast<int>(e / p.rows);
      row = static_cast<int>(e - (int64_t)k * p.rows);
    } else {
      row = static_cast<int>(e / p.K);
      k = static_cast<int>(e - (int64_t)row * p.K);
    }
    const float x = p.trans ? p.src[(int64_t)k * p.ld + row] : p.src[(int64_t)row * p.ld + k];
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    const int64_t o = (int64_t)(p.row0 + row) * KP + k;
    pk[o] = h;
    pk[o + (int64_t)lo_rows * KP] = l;
  }
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  }
  return fn;
}

}  // namespace

cudaError_t launch_gemm_tc(const std::vector<GemmTask>& tasks_in, int passes, int* err, cudaStream_t s) {
  // panels (distinct operand views) and the task list
  std::map<std::tuple<const void*, int, int, int, int>, int> index;
  std::vector<Panel> panels;
  int rows = 0, KP = 64;
  auto panel = [&](const void* src, int ld, int trans, int R, int K) {
    const auto key = std::make_tuple(src, ld, trans, R, K);
    auto it = index.find(key);
    if (it != index.end()) return panels[it->second].row0;
    Panel p{static_cast<const float*>(src), ld, trans, R, K, rows};
    rows += R;
    KP = std::max(KP, (K + TK - 1) / TK * TK);
    index.emplace(key, static_cast<int>(panels.size()));
    panels.push_back(p);
    return p.row0;
  };
  std::vector<TcTask> tasks;
  int tiles = 0;
  for (const GemmTask& t : tasks_in) {
    if (t.M <= 0 || t.N <= 0 || t.K <= 0) continue;
    TcTask u{};
    u.a_row = panel(t.A, t.lda, t.ta, t.M, t.K);
    u.b_row = panel(t.B, t.ldb, t.tb ? 0 : 1, t.N, t.K);
    u.M = t.M;
    u.N = t.N;
    u.kb = (t.K + TK - 1) / TK;
    u.tile0 = tiles;
    u.ldc = t.ldc;
    u.ldcin = t.ldcin;
    u.tc = t.tc;
    u.tcin = t.tcin;
    u.atomic = t.atomic;
    u.alpha = t.alpha;
    u.beta = t.beta;
    u.C = t.C;
    u.Cin = t.Cin;
    tiles += ((t.M + TM - 1) / TM) * ((t.N + TN - 1) / TN);
    tasks.push_back(u);
  }
  if (tasks.empty()) return cudaSuccess;
  EncodeFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int64_t elems = (int64_t)2 * rows * KP;
  __nv_bfloat16* pk = nullptr;
  Panel* dpanels = nullptr;
  TcTask* dtasks = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&pk), elems * 2, s);
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&dpanels), panels.size() * sizeof(Panel), s);
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&dtasks), tasks.size() * sizeof(TcTask), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(pk, 0, elems * 2, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dpanels, panels.data(), panels.size() * sizeof(Panel), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dtasks, tasks.data(), tasks.size() * sizeof(TcTask), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    int maxpe = 1;
    for (const Panel& p : panels) maxpe = std::max<int64_t>(maxpe, (int64_t)p.rows * p.K);
    const int gx = std::min(64, std::max(1, (maxpe + 255) / 256));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    pack_panels_kernel<<<dim3(gx, static_cast<unsigned>(panels.size())), 256, 0, s>>>(dpanels,
                                                                                      (int)panels.size(), KP,
                                                                                      rows, pk);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    const cuuint64_t dims[2] = {(cuuint64_t)KP, (cuuint64_t)(2 * rows)};
    const cuuint64_t strides[1] = {(cuuint64_t)KP * 2};
    const cuuint32_t box[2] = {TK, TM};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, pk, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      e = cudaErrorInvalidValue;
    } else {
      g_launches.fetch_add(1, std::memory_order_relaxed);
      tc_gemm_kernel<<<tiles, TC_THREADS, TC_SMEM, s>>>(map, dtasks, (int)tasks.size(), rows, passes, err);
      e = cudaGetLastError();
    }
  }
  cudaFreeAsync(pk, s);
  cudaFreeAsync(dpanels, s);
  cudaFreeAsync(dtasks, s);
  return e;
}

}  // namespace ce
