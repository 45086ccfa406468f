/*
 * ce.h -- C ABI of the GB300 compress-and-eliminate (CE) solver.
 *
 * The library computes the approximate factorization A ~= Q^T L L^T Q of a
 * sparse symmetric positive definite matrix A (Sushnikova & Oseledets,
 * "Compress and eliminate solver for symmetric positive definite sparse
 * matrices": problem statement Ax = b of Section 1, Algorithms 1-2 of
 * Section 2.6, factorization statement Proposition CE_L) on one CUDA GPU, and
 * uses it as the preconditioner of an FP64 conjugate-gradient solve.
 *
 * Conventions shared by every entry point
 *   - Every call returns a ce_status; no C++ exception crosses this boundary.
 *   - Pointers named *_dev are CUDA device pointers; every other pointer is a
 *     host pointer.  The caller owns all arrays it passes; the library copies
 *     what it keeps.  Handles (ce_csb, ce_factor) are owned by the library
 *     until the matching *_destroy call.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device work is ordered on that stream.
 *   - There is no CPU fallback: if the CUDA runtime fails, CE_ERR_CUDA is
 *     returned and ce_last_error() holds the CUDA error text.
 *   - Indices are 0-based.  The matrix is given in CSR with both triangles.
 */
#ifndef CE_H
#define CE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ce_csb ce_csb;       /* blocked matrix + symbolic plan (opaque) */
typedef struct ce_factor ce_factor; /* factor L, Q on the device (opaque)       */

typedef enum {
  CE_OK = 0,
  CE_ERR_INVALID_ARG = 1,   /* bad size, pointer, permutation, block size   */
  CE_ERR_NOT_SPD = 2,       /* a pivot block was not positive definite      */
  CE_ERR_NO_CONVERGENCE = 3,/* PCG reached maxit                            */
  CE_ERR_OOM = 4,           /* device allocation failed                     */
  CE_ERR_CUDA = 5,          /* CUDA runtime / launch error                  */
  CE_ERR_LIMIT = 6          /* a block exceeded a compiled size limit       */
} ce_status;

/* Truncation rule of the compression step (Section 2.2, eq. rreav and the
 * CE(eps) remark): r_i = #{k : sigma_k(F_i) > tau_i}. */
enum {
  CE_TOL_REL = 0,  /* tau_i = tol * sigma_1(F_i); tol == 0: n_i*eps*sigma_1 */
  CE_TOL_ABS = 1,  /* tau_i = tol                                           */
  CE_TOL_FIXED = 2 /* CE(r) of the Section 2.2 remark: r_i = min(r, numerical
                      rank of F_i), r = ce_opts.rank; singular values within
                      1e-3 relative of sigma_r are kept with it (a tied
                      cluster is kept whole, so the kept subspace is unique).
                      tol is ignored; not with CE_RANK_LEARNED               */
};

/* How the compression step finds U_i and r_i. */
enum {
  CE_RANK_SVD = 0,     /* exact: Householder R of F_i^T + one-sided Jacobi SVD     */
  CE_RANK_LEARNED = 1  /* MLP-predicted width r_hat, randomized range finder of
                          width r_hat + oversample, a-posteriori check, exact SVD
                          for rows that fail it                                    */
};

/* Arithmetic of the factorization. */
enum {
  CE_PREC_FP64 = 0, /* blocks, compression and elimination in FP64       */
  CE_PREC_FP32 = 1  /* FP32 blocks and compression; coarse level in FP64 */
};

typedef struct {
  double tol;      /* eps of CE(eps)                                     */
  int tol_mode;    /* CE_TOL_REL / CE_TOL_ABS / CE_TOL_FIXED             */
  int levels;      /* K, number of compress-and-eliminate sweeps         */
  int J;           /* super-block size: J consecutive blocks join        */
  int precision;   /* CE_PREC_*                                          */
  int coloring;    /* elimination order within a level: 1 (default)
                      colour-major order of a distance-2 colouring (rows
                      of a colour touch disjoint block pairs); 2 of a
                      colouring whose colours hold adjacent blocks apart
                      and let two blocks share a neighbour only if its
                      colour is higher (no fill block between two rows of
                      a colour; fewer colours; rows of a colour may share
                      Schur targets, updated atomically, so sums of shared
                      targets are order-dependent at the rounding level);
                      0 natural order                                     */
  void* stream;    /* cudaStream_t for all device work                   */
  int rank_mode;   /* CE_RANK_SVD (default) / CE_RANK_LEARNED; on levels
                      run by the large-row path the learned form (FP32)
                      sketches each row with width 72, doubled after a
                      rejection up to min(512, 3n/4), before the exact
                      SVD                                                 */
  const void* rank_model; /* device, ce_mlp_nparams() FP16 values from
                             ce_mlp_pack (CE_RANK_LEARNED only)          */
  int oversample;  /* p, sketch columns beyond r_hat (default 8)         */
  uint64_t seed;   /* key of the sketch's counter-based Gaussians        */
  int row_shape;   /* CTA shape of the row kernel: -1 (default) the csb's
                      autotuned choice per level (ce_autotune), else a
                      heuristic; 0: 256 threads, 72 KB shared memory;
                      1: 512 threads, all shared memory; 2: 128 threads,
                      40 KB; 3: the large-row path instead of the row
                      kernel (per colour, batched kernels that spread
                      each row over the whole GPU: fewer, wider launches
                      pay off on levels with few rows per colour)       */
  int rank;        /* r of CE(r) (CE_TOL_FIXED only; >= 0, default 16)    */
  int nmax;        /* super-block cap: a run of J blocks whose sizes add up
                      to more than nmax rows is halved until its parts fit
                      (0, the default: plain runs of J blocks, the paper's
                      rule of Section 2.4)                                 */
  int record_features; /* 1: every row with far columns records the rank
                      model's features (ce_factor_get_features), also on
                      levels that run the exact SVD (default 0)           */
  int gemm_engine; /* products of the large-row path in the FP32 form:
                      0 (default) tensor cores, FP32 operands split into
                      BF16 hi + lo, three products, FP32 accumulation;
                      1 CUDA cores (FP32 FMA); 2 as 0, but the Schur
                      updates W_p^T W_q with one BF16 product (FP32
                      accumulate).  The FP64 form uses the CUDA cores.     */
} ce_opts;

typedef struct {
  int levels_done;     /* sweeps actually run                             */
  int err_level;       /* for CE_ERR_NOT_SPD: level (K = coarse) ...      */
  int err_block;       /* ... and block index (-1 = coarse)               */
  int err_reason;      /* 1: pivot <= 0 (index err_pivot, value err_value);
                          2: non-finite singular values of F_i;
                          5: a row's wait for its neighbours timed out
                          (CE_ERR_CUDA; never expected);
                          CE_ERR_LIMIT: 3 a block over 1536 rows, 4 a
                          row with over 63 close blocks, 8 a colour of a
                          large-row level with over 65535 rows
                          (err_pivot: the size or count)                 */
  int err_pivot;
  double err_value;
  int coarse_n;        /* size of the dense remainder A_K                 */
  int64_t factor_bytes;/* device bytes held by the factor                 */
  int blocks[16];      /* M_l, number of blocks per level (first 16)      */
  int colours[16];     /* colours per level (first 16)                    */
  int max_block[16];   /* largest block per level (first 16)              */
  /* measurement, per level: device time of the row-kernel launches (CUDA
   * events on `stream`), and the algorithmic flops / bytes of those
   * launches counted from the actual sizes, ranks and widths */
  double level_ms[16];
  double level_flops[16];
  double level_bytes[16];
  double coarse_ms;    /* dense assembly + Cholesky of A_K               */
  int learned_rows[16];  /* CE_RANK_LEARNED: rows whose sketch was accepted */
  int fallback_rows[16]; /* ... and rows sent to the exact SVD             */
  double host_ms[16];  /* host time of level l while the GPU waits: its
                          metadata upload, then the planning of level l+1
                          (coarsening, pattern, colouring, reassembly)    */
  double total_ms;     /* wall time of the whole call                     */
  int row_shape[16];   /* CTA shape the row kernel used per level         */
  int row_learned[16]; /* 1: level l ran the learned compression            */
  int spec_miss[16];   /* blocks of level l whose r_l = 0 or r_l > 0 the
                          speculative planning of level l+1 guessed wrong
                          (0: the pattern planned during the GPU work is
                          kept; otherwise it is planned again)            */
  int big_rows[16];    /* 1: level l ran the large-row path (blocks over 64
                          rows, or over 32 close / 128 far blocks)        */
  double big_ms[8];    /* device time of the large-row levels by step
                          (CUDA events, summed over their colours): gather
                          of F_i^T, randomized range finder (learned form),
                          exact SVD (TSQR + Jacobi), U^T D U, Cholesky and
                          inverse, W_b / Y_p / far rows, D_i and W_p,
                          kept rows and Schur updates                      */
  int jacobi_capped[16]; /* rows of level l whose Jacobi SVD stopped at its
                          sweep cap (40 sweeps) with a pair still above the
                          orthogonality threshold; their singular values
                          and vectors are used as they stand             */
  double row_phase_ms[16][12]; /* row-kernel levels: SM time of each row
                          phase summed over the level's rows (ms at the
                          maximum SM clock; divide by the resident CTAs to
                          compare with level_ms): 0 wait for the lower-
                          colour neighbourhood, 1 setup (norms, far-row
                          layout), 2 learned sketch: features, MLP, Jacobi
                          on its k x k factor, completion of U, 3 R of
                          F_i^T, 4 Jacobi SVD, 5 transform, Cholesky,
                          L_hat^{-1}, W_b, 6 close rows, 7 far rows,
                          8 Schur updates, 9 sketch Y = F_i Omega, 10 its
                          Householder QR and explicit Q, 11 its TSQR of
                          F_i^T Q                                         */
  double jacobi_sweeps[16][2]; /* row-kernel levels: mean Jacobi sweeps per
                          row of the exact SVD [0] and of the learned
                          sketch's k x k factor [1] (0: none ran)         */
} ce_info;

typedef struct {
  int iters;           /* PCG iterations run                              */
  double relres;       /* ||b - A x||_2 / ||b||_2 at exit (recursive r)   */
  int converged;       /* 1 if relres <= rtol                             */
} ce_pcg_info;

/* Defaults: tol 1e-4, CE_TOL_REL, levels 4, J 4, FP64, colouring on,
 * CE_RANK_SVD, oversample 8, seed 0, row_shape -1 (autotuned, else a
 * heuristic), rank 16, nmax 0 (no super-block cap), record_features 0,
 * gemm_engine 0. */
void ce_opts_default(ce_opts* o);

/*
 * csb_build -- A_0 = P A P^T in compressed sparse block form (Section 2,
 * eq. init_perm and the CSB storage of Section 2.1).
 *   n        number of rows of A (> 0)
 *   rowptr   host, n+1 entries, CSR row pointers of A (both triangles)
 *   col      host, rowptr[n] column indices
 *   val      host, rowptr[n] values; A must be symmetric
 *   perm     host, n entries: perm[k] = original index of row k of P A P^T
 *   B        block size (> 0): blocks are consecutive runs of B rows of
 *            P A P^T; the last block is shorter when B does not divide n
 *   out      receives the handle
 * Copies the matrix to the device (CSR for the CG products and the block
 * pattern of level 1), keeps a host copy of the pattern (for
 * csb_update_values) and plans level 1 on the host (block graph, A^2
 * pattern, distance-2 colouring).  CE_ERR_INVALID_ARG if perm is not a
 * permutation, an index is out of range or A is not symmetric.
 */
ce_status csb_build(int64_t n, const int64_t* rowptr, const int32_t* col,
                    const double* val, const int32_t* perm, int32_t B,
                    ce_csb** out);

/*
 * csb_update_values -- new values for the same pattern (numeric
 * refactorization): replaces the values of A in place, so the next
 * ce_factorize skips all symbolic work (pattern, colouring, level-1 plan).
 *   val     host, nnz values in the order of the CSR given to csb_build;
 *           the matrix must stay symmetric (checked: CE_ERR_INVALID_ARG)
 *   stream  cudaStream_t of the copy; the call returns after it completes.
 *           No work that reads A (ce_factorize, pcg_solve) may run on
 *           another stream meanwhile.
 * Factors made before the call stay valid and unchanged (they hold their
 * own values).
 * Not part of the paper (a usage pattern of repeated solves).
 */
ce_status csb_update_values(ce_csb* A, const double* val, void* stream);

/*
 * csb_build_batched -- many independent SPD systems as one block-diagonal
 * matrix, so that each level's launches cover the block rows of all of them
 * (the independent-set batching of Section 2.3 applied across systems; the
 * paper factors one system at a time).
 *   nsys     number of systems (> 0)
 *   row_off  host, nsys+1 entries: system s owns rows and columns
 *            [row_off[s], row_off[s+1]) of the stacked matrix; row_off[0] = 0
 *   rowptr, col, val   host CSR of the stacked matrix (both triangles)
 *   perm     host: the stacked permutation; for every system perm maps its
 *            own rows to its own rows
 *   B        host, nsys entries: block size of each system (> 0)
 *   out      receives the handle
 * Blocks never straddle two systems, super-blocks are formed within one
 * system (J consecutive blocks of that system), and the coarse remainder is
 * one dense matrix per system, so ce_factorize on the result gives, system
 * by system, the factor of that system alone.  CE_ERR_INVALID_ARG also if a
 * column or a permuted index leaves its system.
 */
ce_status csb_build_batched(int nsys, const int64_t* row_off,
                            const int64_t* rowptr, const int32_t* col,
                            const double* val, const int32_t* perm,
                            const int32_t* B, ce_csb** out);

/*
 * ce_factorize_batched -- ce_factorize for a handle from csb_build_batched
 * (the same call; the name states the intent): every system of the batch is
 * factorized as if alone, all systems sharing each level's launches.
 * CE_ERR_INVALID_ARG if A was not built by csb_build_batched.
 */
ce_status ce_factorize_batched(const ce_csb* A, const ce_opts* o,
                               ce_factor** out, ce_info* info);

/*
 * ce_factorize -- Algorithm 1 (CE algorithm): `levels` sweeps of Algorithm 2
 * (one level elimination: per block row the compression of the far blocks
 * F_i by an SVD truncated at tau_i, the row/column transform by U_i and the
 * Cholesky elimination of the non-basis sub-row S_i, eq. sm_L), each followed
 * by joining J consecutive blocks into super-blocks (eq. bsp); then the dense
 * Cholesky of the remainder A_K.  The block rows of a level run in one
 * persistent launch in the colour-major order of a distance-2 colouring: a
 * row starts once every row of a lower colour within distance 2 of it has
 * finished (ce_plan_level1_deps lists these waits for level 1), which gives
 * the same arithmetic as one launch per colour.
 *   A     handle from csb_build (not modified)
 *   o     options (NULL = defaults)
 *   out   receives the factor
 *   info  optional, filled on success and on CE_ERR_NOT_SPD
 * Levels whose blocks outgrow the persistent row kernel (more than 64 rows,
 * more than 32 close or 128 far blocks; 3D super-blocks) run the large-row
 * path: one colour at a time, the steps of its rows as batched kernels with
 * the row matrices in global memory (GEMM-shaped products on a grouped GEMM),
 * synchronizing the stream once per colour.  Otherwise the stream is
 * synchronized once per level (the next level's layout depends on the
 * ranks).  CE_ERR_LIMIT if a block grows beyond 1536 rows or a row has more
 * than 63 close blocks.  The factor uses device memory of A (the permutation
 * and the level-1 plan): destroy the factor before A.
 */
ce_status ce_factorize(const ce_csb* A, const ce_opts* o, ce_factor** out,
                       ce_info* info);

/*
 * ce_factorize_simple -- csb_build + ce_factorize with the paper's inputs
 * (A, P, B, eps, K) and default J, FP64, relative tolerance.  The csb handle
 * is kept inside the factor and released with it.
 */
ce_status ce_factorize_simple(int64_t n, const int64_t* rowptr,
                              const int32_t* col, const double* val,
                              const int32_t* perm, int32_t B, double tol,
                              int levels, ce_factor** out);

/*
 * ce_autotune -- choose, per level and by measurement, the row kernel's CTA
 * shape and (with o->rank_mode = CE_RANK_LEARNED) whether the learned
 * compression or the exact SVD runs: factorizes A with every combination
 * (options o, row_shape ignored), times every level's launch with CUDA
 * events, and keeps the fastest per level in A (the default -- learned
 * compression, heuristic shape -- unless another is more than 3 % faster).
 * Later ce_factorize calls with row_shape = -1 and the same precision and
 * rank mode use it.  A shape only changes how a row's work is spread over
 * threads (and the rounding of in-row reductions); the exact SVD instead of
 * the learned sketch on a level gives ranks at least as tight under the same
 * tolerance.
 * Shape 3 (the large-row path) is one of the candidates.
 *   level_ms  optional host array of 2 x 4 x 16 doubles:
 *             [learned, exact][shape][level] times (ms)
 * Not part of the paper (launch configuration of this implementation).
 */
ce_status ce_autotune(ce_csb* A, const ce_opts* o, double* level_ms);

/*
 * csb_get_tuning / csb_set_tuning -- the choices ce_autotune keeps in a csb
 * for one precision (CE_PREC_*) and rank mode (CE_RANK_*), host-only: the
 * number of tuned levels, and per level (16 entries each) the row kernel's CTA
 * shape (0..3, see ce_opts.row_shape) and whether the learned compression runs (1) or the exact SVD
 * (0).  A tuning measured on one csb can be set on another csb of the same
 * matrix (e.g. one rebuilt from host arrays) so that it runs the same
 * schedule.  CE_ERR_INVALID_ARG on a bad precision, mode, count or value.
 * Not part of the paper (launch configuration of this implementation).
 */
ce_status csb_get_tuning(const ce_csb* A, int precision, int rank_mode, int* levels, int32_t* shape,
                         int32_t* learned);
ce_status csb_set_tuning(ce_csb* A, int precision, int rank_mode, int levels, const int32_t* shape,
                         const int32_t* learned);

/*
 * ce_apply -- z = M^{-1} r = Q^T L^{-T} L^{-1} Q r (solve proposition of
 * Section 2.5).  r_dev and z_dev are device arrays of n doubles in the
 * original ordering of A; they may alias.  All work is queued on `stream`
 * with no host synchronization (on a batch handle pcg_solve_batched replays
 * it from a captured CUDA graph; a single system's coarse solve is a
 * cooperative launch).
 * The apply's scheduling state (queue counters, per-row flags, an epoch)
 * lives in the factor: calls on one factor must not overlap on the GPU
 * (issue them on one stream, or serialize them); different factors are
 * independent.
 */
ce_status ce_apply(const ce_factor* F, const double* r_dev, double* z_dev,
                   void* stream);

/*
 * pcg_solve -- preconditioned conjugate gradients in FP64 with M = Q^T L L^T Q
 * (the paper's experiments use MINRES, Section 4, which minres_solve runs;
 * CG is valid here because A and M are SPD).
 * x0 = 0; stops when ||r||_2 <= rtol ||b||_2 or after maxit iterations.
 *   b_dev, x_dev  device arrays of n doubles (original ordering)
 *   info          optional
 * Reads the residual norm to the host once per iteration.  Applies F, so
 * it must not overlap other work on F (see ce_apply).
 * CE_ERR_NO_CONVERGENCE if maxit is reached (x_dev holds the last iterate).
 */
ce_status pcg_solve(const ce_csb* A, const ce_factor* F, const double* b_dev,
                    double* x_dev, double rtol, int maxit, ce_pcg_info* info,
                    void* stream);

/*
 * minres_solve -- preconditioned MINRES in FP64 with M = Q^T L L^T Q, the
 * Krylov method of the paper's experiments (Section 4): the Lanczos process
 * preconditioned by M, the QR factorization of its tridiagonal matrix kept
 * by Givens rotations, and the iterate updated along the directions w of
 * Paige and Saunders (1975).  x0 = 0; stops when the preconditioned
 * residual norm ||r||_{M^{-1}} (the recurrence's phibar) is <= rtol times
 * ||b||_{M^{-1}}, when the Krylov space is exhausted, or after maxit
 * iterations.  M must be SPD (a factor from ce_factorize is); A only
 * symmetric.
 *   b_dev, x_dev  device arrays of n doubles (original ordering)
 *   info          optional: iterations, the final phibar / ||b||_{M^{-1}}
 *                 (relres), converged
 * One system per call: a batch handle is rejected with CE_ERR_INVALID_ARG.
 * Allocates six work vectors (stream-ordered) and frees them on return;
 * reads two dot products to the host per iteration.  Applies F, so it must
 * not overlap other work on F (see ce_apply).  CE_ERR_NOT_SPD if a
 * preconditioned inner product r^T M^{-1} r is negative or not finite;
 * CE_ERR_NO_CONVERGENCE if maxit is reached (x_dev holds the last iterate).
 */
ce_status minres_solve(const ce_csb* A, const ce_factor* F, const double* b_dev,
                       double* x_dev, double rtol, int maxit, ce_pcg_info* info,
                       void* stream);

/*
 * pcg_solve_batched -- pcg_solve for a batch from csb_build_batched: one CG
 * recurrence per system (its own step lengths, residual norm and stopping
 * test ||r_s|| <= rtol ||b_s||); a converged system is frozen while the
 * others iterate.  One iteration of all systems is captured once into a CUDA
 * graph (kept in the factor together with its work vectors and reused by the
 * next call with the same matrix handle; calls on one factor must not
 * overlap) and replayed; the host reads the count of unconverged systems one
 * iteration behind the GPU.
 *   b_dev, x_dev  device arrays of n doubles (stacked original orderings)
 *   iters, relres, converged   optional host arrays of nsys entries
 *   info          optional: maximum iterations and residual, all converged
 * pcg_solve on a batch handle calls this with the per-system arrays NULL.
 * CE_ERR_NO_CONVERGENCE if some system reached maxit.
 */
ce_status pcg_solve_batched(const ce_csb* A, const ce_factor* F,
                            const double* b_dev, double* x_dev, double rtol,
                            int maxit, int32_t* iters, double* relres,
                            int32_t* converged, ce_pcg_info* info,
                            void* stream);

/*
 * pcg_solve_noalloc -- the FP64 PCG of pcg_solve for one system (same
 * arguments, same arithmetic, same results as pcg_solve on a handle from
 * csb_build), for callers that cannot let a library allocate device memory:
 * applications whose GPU memory is reserved up front by their own pool
 * allocator, latency-critical loops that cannot afford the implicit device
 * synchronization of cudaMalloc/cudaFree, and plugins whose host application
 * forbids allocation.  The paper has no counterpart; it is a deployment
 * variant of pcg_solve.
 *   - Allocates nothing: the work vectors live in one static device array
 *     (4 x 65536 doubles plus reduction partials, about 2 MiB) that every GPU
 *     loading the library holds until the process exits.
 *   - n > 65536 is rejected with CE_ERR_LIMIT (ce_last_error() says why).
 *   - A batch handle (csb_build_batched with more than one system) is
 *     rejected with CE_ERR_INVALID_ARG: pcg_solve runs one CG recurrence per
 *     system there, and the static array holds one recurrence.
 *   - Every call looks the array's device address up (cudaGetSymbolAddress,
 *     which allocates nothing) with the caller's device current, so it stays
 *     valid across a cudaDeviceReset; make the first call on a device before
 *     any stream capture (that lookup may load the module).
 *   - All calls share the array and it keeps the last call's contents; calls
 *     whose work overlaps on the GPU (other streams, other host threads) race
 *     on it and must be serialized by the caller.
 */
ce_status pcg_solve_noalloc(const ce_csb* A, const ce_factor* F,
                            const double* b_dev, double* x_dev, double rtol,
                            int maxit, ce_pcg_info* info, void* stream);

/* Release a handle (NULL is ignored). */
void ce_csb_destroy(ce_csb* A);
void ce_factor_destroy(ce_factor* F);

/*
 * Rank predictor for the compression step.  The paper always runs a full
 * SVD there; its conclusion names a cheaper rank-revealing factorization as
 * the way to cut the time spent in it (Section 6).
 * A 3-layer MLP (ce_mlp_nfeatures() -> 64 -> 64 -> 1, ReLU, sigmoid) maps the
 * per-row features of the compression step to r_i / n_i.  Parameters are a
 * flat FP32 device array of ce_mlp_nparams() values: W1 (64 x nfeat,
 * row-major), b1 (64), W2 (64 x 64), b2 (64), w3 (64), b3 (1).
 *   ce_mlp_init     He-normal weights from a counter-based generator, zero
 *                   biases
 *   ce_mlp_grad     full-batch gradient of 0.5 mean (y - t)^2 (deterministic)
 *   ce_mlp_train    `steps` Adam steps (lr) on the full batch; allocates its
 *                   optimizer state; *loss_out (host, optional) = final loss
 *   ce_mlp_pack     FP32 parameters -> FP16 model for ce_opts.rank_model
 *   ce_mlp_predict  FP16 inference, out[s] = prediction for row s of X
 * X is ns x nfeat row-major (device), t has ns targets (device).
 */
int ce_mlp_nparams(void);
int ce_mlp_nfeatures(void);
ce_status ce_mlp_init(float* theta_dev, uint64_t seed, void* stream);
ce_status ce_mlp_grad(const float* X_dev, const float* t_dev, int ns,
                      const float* theta_dev, float* grad_dev, void* stream);
ce_status ce_mlp_train(const float* X_dev, const float* t_dev, int ns,
                       float* theta_dev, int steps, float lr, double* loss_out,
                       void* stream);
ce_status ce_mlp_pack(const float* theta_dev, void* model_dev, void* stream);
ce_status ce_mlp_predict(const float* X_dev, int ns, const void* model_dev,
                         float* out_dev, void* stream);

/* Number of kernels the library has launched so far (process-wide). */
int64_t ce_launch_count(void);

/*
 * ce_measure_peak -- measured arithmetic rate of one execution unit of the
 * current device, the denominator of a roofline fraction (not part of the
 * paper).  A kernel that keeps the unit busy on every SM (independent chains,
 * full occupancy) runs a few milliseconds, three times after one warm-up; the
 * best rate is returned in TFLOP/s (an FMA counts 2 flops).
 *   kind  0: FP32 FFMA; 1: FP64 DFMA; 2: TF32 mma.sync m16n8k8 with FP32
 *         accumulate; 3: the 3xTF32 product of the row kernel (operands split
 *         into TF32 hi + lo, three MMAs counted as one product)
 * Allocates and frees a few KB on `stream`; synchronizes it.
 */
ce_status ce_measure_peak(int kind, double* tflops, void* stream);

/* Static text of a status code; text of the last CUDA failure (per thread). */
const char* ce_strerror(ce_status s);
const char* ce_last_error(void);

/*
 * Introspection of a factor (host copies; for tests and reports).
 *   ce_factor_levels       number of sweeps stored
 *   ce_factor_level_size   M_l (blocks) of level l
 *   ce_factor_get_level    per block of level l, each array host, M_l
 *                          entries (any may be NULL): block size n_i,
 *                          rank r_i, colour, and tau_i (double)
 *   ce_factor_get_sigma    singular values of F_i for every block of level
 *                          l, concatenated in block order (sum of n_i
 *                          doubles; zeros where F_i had fewer columns)
 */
int ce_factor_levels(const ce_factor* F);
/*
 * ce_factor_get_features -- what the learned compression saw on level l, per
 * block (host copies):
 *   feat  M_l x ce_mlp_nfeatures() floats, row-major (may be NULL): the rank
 *         model's input features of block i (zeros where the model did not
 *         run: exact levels, rows without far blocks)
 *   kw    M_l ints (may be NULL): sketch width k of the randomized range
 *         finder, k > 0 accepted, -k rejected and sent to the exact SVD,
 *         0 no sketch
 */
ce_status ce_factor_get_features(const ce_factor* F, int level, float* feat, int32_t* kw);
int ce_factor_level_size(const ce_factor* F, int level);
ce_status ce_factor_get_level(const ce_factor* F, int level, int32_t* n,
                              int32_t* rank, int32_t* colour, double* tau);
ce_status ce_factor_get_sigma(const ce_factor* F, int level, double* sigma);

/*
 * ce_plan_level1 -- host-only symbolic analysis of level 1 (no CUDA call):
 * the block graph of P A P^T with blocks of B rows, its greedy distance-2
 * colouring (blocks visited breadth-first from a block of least degree,
 * ascending neighbours; smallest colour free within distance 2), and the
 * number of block pairs of the
 * squared pattern (close + far pairs, Section 2.2).  Arguments as csb_build
 * (values are not needed).
 *   colour    host, ceil(n/B) entries, may be NULL
 *   ncolours  may be NULL
 *   npairs    pairs (i <= k) of the squared pattern, may be NULL
 *   nclose    pairs (i <= k) of the block pattern of P A P^T, may be NULL
 */
ce_status ce_plan_level1(int64_t n, const int64_t* rowptr, const int32_t* col,
                         const int32_t* perm, int32_t B, int32_t* colour,
                         int* ncolours, int64_t* npairs, int64_t* nclose);

/*
 * ce_plan_colours -- host-only (no CUDA call): level 1's elimination order
 * as ce_factorize plans it for ce_opts.coloring (0 natural: block i is colour
 * i; 1 distance 2; 2 the order whose colours separate adjacent blocks and
 * blocks with a common neighbour of a lower colour, see ce_opts.coloring).
 * Arguments as ce_plan_level1; colour (host, ceil(n/B) entries) and ncolours
 * may be NULL.  CE_ERR_INVALID_ARG as ce_plan_level1 or for another coloring.
 */
ce_status ce_plan_colours(int64_t n, const int64_t* rowptr, const int32_t* col,
                          const int32_t* perm, int32_t B, int coloring,
                          int32_t* colour, int* ncolours);

/*
 * ce_plan_level1_deps -- host-only (no CUDA call): the waits of level 1's
 * persistent row launch.  The rows of one colour are independent (the
 * distance-2 colouring makes each colour an independent set in the sense of
 * Section 2.3); row i waits for every row k of a lower colour with (i, k) in
 * the squared pattern, i.e. within distance 2 in the block graph, which
 * covers every row whose Schur update writes a pair that row i reads or
 * writes.  Arguments as ce_plan_level1.
 *   dep_ptr  host, M + 1 offsets (may be NULL)
 *   dep_idx  host, cap entries (may be NULL): the rows k of row i are
 *            dep_idx[dep_ptr[i] .. dep_ptr[i+1])
 *   ndeps    total number of waits (may be NULL)
 * CE_ERR_INVALID_ARG as ce_plan_level1, or when dep_idx is given with
 * cap < *ndeps (call once with dep_idx = NULL to size it).
 */
ce_status ce_plan_level1_deps(int64_t n, const int64_t* rowptr, const int32_t* col,
                              const int32_t* perm, int32_t B, int64_t* dep_ptr,
                              int32_t* dep_idx, int64_t cap, int64_t* ndeps);

/*
 * ce_plan_next_level -- host-only (no CUDA call): the symbolic plan of level
 * 2 that ce_factorize derives from level 1 and its ranks (Section 2.4, eq.
 * bsp): super-blocks as ce_plan_groups forms them, sizes = sums of the
 * children's ranks, a pair of super-blocks kept when some pair of the level-1
 * squared pattern with non-empty ranks on both sides lies inside it, and the
 * distance-2 colouring of that pattern.  Arguments as ce_plan_level1, plus
 *   rank         host, ceil(n/B) entries, 0 <= r_i <= n_i (level-1 ranks)
 *   J, nmax      as ce_plan_groups (0: no cap)
 *   next_n       host, room for ceil(n/B) entries (may be NULL): sizes
 *   next_colour  host, room for ceil(n/B) entries (may be NULL)
 *   next_M       number of level-2 blocks
 *   next_nclose  pairs (I <= K) of the level-2 block pattern (may be NULL)
 */
ce_status ce_plan_next_level(int64_t n, const int64_t* rowptr, const int32_t* col,
                             const int32_t* perm, int32_t B, const int32_t* rank, int J,
                             int nmax, int32_t* next_n, int32_t* next_colour, int* next_M,
                             int64_t* next_nclose);

/*
 * ce_plan_level1_work -- host-only (no CUDA call): the algorithmic work of
 * level 1's row kernel, as ce_info.level_flops / level_bytes count it, for
 * given level-1 ranks.  Per block row (n, r, m = n - r, far columns mF and
 * close columns Wc as they stand when the row runs: rows of an earlier colour
 * keep only their r columns): 2 mF n^2 (R of F^T) + 12 n^3 (SVD of R, when
 * mF > 0) + 4 n^3 + 2 n^2 Wc + 2 n r mF (transforms) + m^3/3 + m^2 (r + Wc)
 * (Cholesky, TRSM) + m ((r + Wc)^2 + r^2 + sum w^2) (Schur) flops, and the
 * bytes of the pairs read and written and of the factor written.
 *   rank   host, ceil(n/B) entries, 0 <= r_i <= n_i
 *   esize  4 (FP32 form) or 8 (FP64 form)
 *   flops, bytes  receive the totals
 */
ce_status ce_plan_level1_work(int64_t n, const int64_t* rowptr, const int32_t* col,
                              const int32_t* perm, int32_t B, const int32_t* rank,
                              int esize, double* flops, double* bytes);

/*
 * ce_plan_groups -- host-only (no CUDA call): the super-blocks that
 * ce_factorize forms from one level's blocks (Section 2.4).  Runs of J
 * consecutive blocks join; with nmax > 0 a run whose ranks add up to more
 * than nmax rows is halved, first half ceil(len/2) blocks, recursively, until
 * every part fits or is one block (ce_factorize: ce_opts.nmax; 0 = no cap).
 *   M            blocks of the level
 *   rank         host, M kept sizes r_i (>= 0)
 *   first_child  host, room for M + 1 entries: super-block I holds blocks
 *                [first_child[I], first_child[I + 1])
 *   ngroups      number of super-blocks
 * CE_ERR_INVALID_ARG for M < 1, J < 1, nmax < 0, a negative rank or a NULL
 * pointer.
 */
ce_status ce_plan_groups(int M, const int32_t* rank, int J, int nmax, int32_t* first_child, int* ngroups);

/*
 * ce_debug_wait_expiry -- test of the failure path of the persistent
 * launches' dependency waits (no counterpart in the paper).  Builds a level of
 * two coupled 4-row blocks on the device and queues only the second, whose
 * wait for the first (kernel 0: the row kernel of ce_factorize, reason 5;
 * kernel 1: the forward apply of ce_apply, reason 6) can never be satisfied,
 * with the wait limited to limit_ms (0 < limit_ms <= 2000; the library's own
 * limit is 2 s).  The kernel gives up, records CE_ERR_CUDA with its reason and
 * returns; the context stays usable.
 *   status_out  host, 8 ints: the kernel's status words [code, level, block,
 *               reason, ...]
 * Returns CE_OK when the launch itself worked (whatever the kernel recorded).
 */
ce_status ce_debug_wait_expiry(int kernel, double limit_ms, int32_t* status_out, void* stream);

/*
 * ce_debug_gemm -- one product C = alpha op(A) op(B) + beta C through one of
 * the library's GEMM engines (for tests; not part of the paper):
 *   engine 0: CUDA cores, FP32; 3: CUDA cores, FP64; 1: tensor cores
 *   (tcgen05, FP32 operands split into BF16 hi + lo, three products
 *   hi*hi + hi*lo + lo*hi, FP32 accumulation); 2: tensor cores, one BF16
 *   product (hi*hi).  Engines 0-2 take FP32 arrays, engine 3 FP64.
 *   A_dev  M x K (ta = 0, element (m, k) at A[m lda + k]) or K x M (ta = 1)
 *   B_dev  K x N (tb = 0) or N x K (tb = 1, element (k, n) at B[n ldb + k])
 *   C_dev  M x N (tc = 0) or N x M (tc = 1), read when beta != 0
 * Synchronizes the stream.  CE_ERR_CUDA if a tensor-core pipeline wait expired.
 */
ce_status ce_debug_gemm(int engine, int M, int N, int K, const void* A_dev, int lda, int ta, const void* B_dev,
                        int ldb, int tb, void* C_dev, int ldc, int tc, double alpha, double beta, void* stream);

/*
 * ce_debug_svd -- the SVD steps of the compression of a large row (Section
 * 2.2: U_i and sigma of a far row through the R factor of F_i^T) on one
 * n x n upper triangular R, for tests: the QR factorization with column
 * pivoting of R^T (R^T P = Q3 R3), then block one-sided Jacobi with column
 * blocks of `block` (4, 8, 16 or 32) on X = R3^T, rotations accumulated into
 * V = Q3.  On return the columns of X are the left singular vectors of R^T
 * scaled by the singular values (in no particular order) and V holds the
 * unit vectors: R^T R V = V diag(||X_j||^2) up to rounding.
 *   esize   4 (FP32) or 8 (FP64) for every array
 *   R_dev   n x n row-major (zero below the diagonal), not modified
 *   D_dev   n x n: ||D||_F sets the rounding floor of the pair-skipping rule
 *   tol     eps of the rule (0: only rounding-level pairs are skipped)
 *   X_dev, V_dev  n x n each, column-major (column j at j n)
 *   sweeps  optional host int: sweeps run
 * Synchronizes the stream.  CE_ERR_INVALID_ARG for another esize or block,
 * n outside 1..1536, or when 4 block n values do not fit in shared memory.
 * Not part of the paper's interface.
 */
ce_status ce_debug_svd(int esize, int block, int n, const void* R_dev, const void* D_dev, double tol, void* X_dev,
                       void* V_dev, int* sweeps, void* stream);

/* Level-1 plan of a csb handle: blocks, colours, colour of every block. */
int csb_blocks(const ce_csb* A);
ce_status csb_get_colours(const ce_csb* A, int32_t* colour, int* ncolours);

#ifdef __cplusplus
}
#endif
#endif /* CE_H */
