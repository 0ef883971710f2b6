/*
 * ozdmrg.h -- C ABI of libozdmrg: Ozaki-scheme emulated FP64 products and the block-sparse
 * two-site effective-Hamiltonian product of ab initio DMRG, on sm_103a (GB300).
 *
 * Method (arXiv 2510.04795):
 *   - section "Theory of emulated FP64 arithmetic": C = A B by (1) fixed point with one exponent
 *     shared per row of A and per column of B, (2) S slices of 8 bits, (3) all kept slice-pair
 *     products in low precision, (4) accumulation at high precision and conversion back to FP64;
 *     products in the less significant ("lower-triangular") part of the S x S grid are skipped;
 *   - section "Numerical procedure": S slices hold 8S-1 mantissa bits plus the sign
 *     (S = ceildiv(bits+1, 8));
 *   - section "Theory of TNS/DMRG regarding error analysis": the DMRG update diagonalises the
 *     effective Hamiltonian with a Krylov solver, whose matrix-vector product is built from binary
 *     tensor contractions done as matrix multiplications.
 *
 * Conventions for every entry point:
 *   - matrices are row-major FP64 unless stated; `ld*` is the row stride in elements;
 *   - pointers named d_* are DEVICE pointers owned by the caller; the library never frees them;
 *   - work is enqueued on the given CUDA stream and returns before it completes (asynchronous);
 *     device-side faults of the inputs (NaN/Inf, timeouts of bounded waits) are latched in the
 *     context and reported by oz_status(), which synchronises the stream;
 *   - every call returns an int status (OZ_OK or one of the codes below); oz_last_error() gives a
 *     thread-local message for the last failing call.  No C++ exception crosses the ABI.
 *
 * Numerics of the emulation (readings where the paper is silent):
 *   e_i  = smallest integer with max_k |a_ik| <= (127/128) 2^e_i  (0 for an all-zero row);
 *   X_ik = RN_even(a_ik 2^(8S-1-e_i)), an integer; slices d_1..d_S = its balanced base-256 digits,
 *          each in [-128, 127] (INT8), X = sum_t d_t 256^(S-t);
 *   level s <= S uses d_1..d_s and the pairs t + u <= s + 1 (s(s+1)/2 products);
 *   C_ij = RN_even(2^(e_i+e_j-2(8S-1)) * sum_{t+u<=s+1} 256^(2S-t-u) P_tu[i][j]) -- the exact
 *          integer sum rounded ONCE, so the result is bit-identical to the exact definition and
 *          independent of tiling and summation order.
 */
#ifndef OZDMRG_H
#define OZDMRG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define OZ_OK 0
#define OZ_EINVAL 1        /* an argument is out of range (message in oz_last_error) */
#define OZ_ENONFINITE 2    /* an input held NaN or Inf: outputs are unspecified */
#define OZ_ENOCONV 3       /* an iterative solver reached its iteration limit */
#define OZ_EVARIATIONAL 4  /* an energy fell below the previous one by more than the tolerance */
#define OZ_ETIMEOUT 5      /* a bounded device-side wait gave up; outputs are unspecified */
#define OZ_ECUDA 6         /* a CUDA runtime or library call failed */
#define OZ_ENOMEM 7        /* device memory could not be allocated */

/* precision / dispatch of a product */
#define OZ_MODE_EAGER 0    /* every product emulated (the paper's eager mode) */
#define OZ_MODE_NATIVE 1   /* native FP64 (cuBLAS DGEMM, emulation off) on the same task list */
#define OZ_MODE_PERFORMANT 2 /* ozaki_gemm only: the faster of the two for the shape (paper's performant mode) */

typedef struct oz_prec {
  int slices; /* S: digits stored per value, 1..9 */
  int level;  /* s: digits used, 1..S; 0 means s = S.  Level 9 runs each tile in two passes (nine
                 diagonal accumulators exceed TMEM) and accepts reductions k <= 130048, where the
                 exact 96-bit sums cannot overflow; levels up to 8 accept k <= 1048576 */
  int mode;   /* OZ_MODE_EAGER or OZ_MODE_NATIVE (OZ_MODE_PERFORMANT: ozaki_gemm only) */
  int tile;   /* H_eff handles: OZ_TILE_AUTO (0), OZ_TILE_CTA (128 x 64 tiles, one CTA each) or
                 OZ_TILE_PAIR (256 x 64 tiles on a CTA pair: one MMA issuer for two SMs); AUTO
                 takes OZ_TILE_CTA, the faster of the two on GB300 (OZ_EINVAL for OZ_TILE_PAIR on a
                 device without clusters of two).  Results are identical.  Other entry points
                 ignore it. */
} oz_prec;
#define OZ_TILE_AUTO 0
#define OZ_TILE_CTA 1
#define OZ_TILE_PAIR 2

typedef void* oz_stream_t; /* a cudaStream_t (0 = legacy default stream) */

typedef struct oz_ctx_s oz_ctx;
typedef struct oz_heff_s oz_heff;

/* ------------------------------------------------------------------------------------------
 * Context: one per device.  Owns a grow-only device workspace for ozaki_gemm and the
 * device-side error latch.  oz_ctx_create makes `device` current on the calling thread.
 * ------------------------------------------------------------------------------------------ */
int oz_ctx_create(oz_ctx** out, int device);
int oz_ctx_destroy(oz_ctx* ctx);
const char* oz_last_error(void);
/* Synchronises `stream` and returns (then clears) the latched device status:
 * OZ_ENONFINITE if a sliced input held NaN/Inf, OZ_ETIMEOUT if a bounded wait gave up. */
int oz_status(oz_ctx* ctx, oz_stream_t stream);

/* ------------------------------------------------------------------------------------------
 * ozaki_gemm: C = alpha * (A B) + beta * C with the emulated product of the header comment
 * (paper, section "Theory of emulated FP64 arithmetic").
 *   A: m x k (lda >= k), B: k x n (ldb >= n), C: m x n (ldc >= n); all device, row-major.
 *   alpha*c and beta*C are each rounded to FP64 and then added (no fused multiply-add).
 *   prec->mode == OZ_MODE_NATIVE runs cuBLAS DGEMM instead.
 *   prec->mode == OZ_MODE_PERFORMANT (paper, section "Numerical procedure": emulation only where it
 *   pays off) runs whichever of the two was faster for this shape class: the first call whose
 *   (ceil log2 m, ceil log2 n, ceil log2 k, S, s) is new times both paths on the caller's A and B
 *   into a scratch C (synchronising the stream, allocating m x n doubles), caches the winner in the
 *   context and then runs it; later calls of the class run the cached choice.  The result is that
 *   of the chosen path (bit-exact emulation or cuBLAS DGEMM).  Not for use under stream capture.
 * Errors: OZ_EINVAL for negative sizes, short leading dimensions, slices outside 1..9, a level
 * outside 1..S, or k above the level's limit (1048576; 130048 at level 9).  May grow the context workspace (cudaMalloc, synchronous): call it once
 * outside stream capture before capturing.
 * ------------------------------------------------------------------------------------------ */
int ozaki_gemm(oz_ctx* ctx, int m, int n, int k, double alpha, const double* d_A, int lda, const double* d_B,
               int ldb, double beta, double* d_C, int ldc, const oz_prec* prec, oz_stream_t stream);
/* The choice OZ_MODE_PERFORMANT made for the shape class of (m, n, k) at prec's S and level:
 * *mode = OZ_MODE_EAGER or OZ_MODE_NATIVE, or -1 if no call of that class has been timed yet;
 * ms (2 floats, may be null) receives the timed emulated and native durations. */
int oz_performant_choice(oz_ctx* ctx, int m, int n, int k, const oz_prec* prec, int* mode, float* ms);

/* ------------------------------------------------------------------------------------------
 * ozaki_gemm_noalloc: the same emulated product as ozaki_gemm (bit-identical results) for callers
 * that cannot allocate device memory: code running under a host framework that owns the device's
 * memory pool, callers inside a region that must not synchronise the device (cudaMalloc and
 * cudaFree do), or deployments that fix their memory footprint in advance.  The paper has no
 * counterpart; it is an interface of this library.
 *   - No context is needed and nothing is allocated: the scratch (digit planes, exponents, row
 *     maxima, status words) is one statically sized device array of 64 MiB (plus 256 bytes) that
 *     every GPU loading this library holds until the process exits.
 *   - A product is rejected with OZ_EINVAL when its scratch would exceed 64 MiB (about
 *     S * 2 * (m_pad k_pad + n_pad k_pad) bytes, m padded to 128, n to 64, k to 16), when
 *     k > 1048576, or for the argument errors of ozaki_gemm.  Errors are reported by the return
 *     code only (oz_last_error is not updated).  Device-side conditions are not reported at
 *     all: with a NaN/Inf input, or when a kernel's bounded wait gives up (about 2 s), the call
 *     still returns OZ_OK and C is unspecified.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress) and
 *     caches it; make that first call before any stream capture.
 *   - All calls share the array and it keeps the last call's contents; the parts that must start
 *     at zero are cleared on the stream by each call.  Calls whose execution overlaps on the GPU
 *     (different streams, or concurrent host threads) race on the array: serialise them.
 * Arguments as ozaki_gemm; slices S in 1..9, level in 1..S (0 = S).
 * ------------------------------------------------------------------------------------------ */
int ozaki_gemm_noalloc(int m, int n, int k, double alpha, const double* d_A, int lda, const double* d_B, int ldb,
                       double beta, double* d_C, int ldc, int slices, int level, oz_stream_t stream);

/* ------------------------------------------------------------------------------------------
 * Verification entry points for the slicing and the slice products (same kernels as ozaki_gemm).
 * ozaki_slice: shared exponents (d_exps[rows]) and digits (d_digits[t][i][j], S x rows x cols,
 *   int8, t = 0 is the most significant) of the rows of A (rows x cols, lda).
 * ozaki_slice_products: every slice product P_tu = A^t B^u (A sliced by rows, B by columns):
 *   d_P[(t*S+u)*m*n + i*n + j] = sum_k dA_t[i][k] dB_u[k][j] as an exact integer in FP64,
 *   for all t, u < S (the full grid), computed by the tcgen05 kernel at level 1.
 * ------------------------------------------------------------------------------------------ */
int ozaki_slice(oz_ctx* ctx, int rows, int cols, const double* d_A, int lda, int slices, int8_t* d_digits,
                int* d_exps, oz_stream_t stream);
int ozaki_slice_products(oz_ctx* ctx, int m, int n, int k, const double* d_A, int lda, const double* d_B, int ldb,
                         int slices, double* d_P, oz_stream_t stream);

/* ------------------------------------------------------------------------------------------
 * Block-sparse two-site H_eff (paper, section "Theory of TNS/DMRG ...": the Krylov update of the
 * two-site tensor and binary contractions as matrix products).
 *
 * psi is stored as sector blocks q = 0..nsec-1, block q of shape m[q] x n[q] (left enlarged
 * sector x complementary right sector), row-major, concatenated in q order (offset of block q =
 * sum_{p<q} m[p] n[p]).  A task adds  coef * L (m[dst] x m[src]) psi[src] R^T  to Y[dst], with
 * R of shape n[dst] x n[src]; L and R are row-major device blocks owned by the caller.
 *
 * heff_apply computes, for every source sector, one emulated product of the stacked L blocks with
 * psi[src] (the intermediate T, rounded once per element), and for every target sector one
 * emulated product of the concatenated T blocks with the stacked (coef R)^T blocks.
 * ------------------------------------------------------------------------------------------ */
typedef struct oz_task {
  int src, dst;
  double coef;
  const double* d_L; /* m[dst] x m[src] */
  const double* d_R; /* n[dst] x n[src] */
} oz_task;

/* Builds the handle: slices every L and coef*R once (they may be freed afterwards in EAGER mode;
 * NATIVE mode keeps stacked FP64 copies), allocates scratch, tables and a CUDA graph.
 * Synchronous.  Errors: OZ_EINVAL (sector index out of range, non-positive dims), OZ_ENOMEM,
 * OZ_ENONFINITE (an operator block held NaN/Inf). */
int oz_heff_create(oz_ctx* ctx, int nsec, const int* m, const int* n, int ntask, const oz_task* tasks,
                   const oz_prec* prec, oz_heff** out);
int oz_heff_destroy(oz_heff* h);
/* New operator values for the same structure (paper, section "Theory of TNS/DMRG regarding error
 * analysis": the operators change every time the environments are rebuilt, the sector structure
 * with them only when the bond dimension does).  tasks: ntask entries with the same (src, dst) as
 * at oz_heff_create, in the same order; coef, d_L and d_R may change (device pointers, read during
 * the call only).  Re-slices the operators into the handle's planes (emulated) or re-copies them
 * (native), and rebuilds the diagonal and the selector's operator statistics; allocations, tile
 * schedules, per-sector levels and the captured graph are kept.  The next product is bit-identical
 * to that of a handle created from the new tasks.  Synchronous (waits for products in flight).
 * Errors: OZ_EINVAL (count or sectors differ, null pointer), OZ_ENONFINITE (NaN/Inf in a block; the
 * handle's operators are then undefined until a successful update). */
int oz_heff_update_ops(oz_heff* h, int ntask, const oz_task* tasks);
/* d_y = H_eff d_psi (flat block vectors of length sum m[q] n[q]; d_y must not alias d_psi). */
int heff_apply(oz_heff* h, const double* d_psi, double* d_y, oz_stream_t stream);
/* End-to-end form of heff_apply on HOST vectors: copies psi_host to the device, applies H_eff,
 * copies the result to y_host, all enqueued on `stream` (page-locked host memory makes the copies
 * asynchronous; pageable memory works but serialises them). */
int heff_apply_host(oz_heff* h, const double* psi_host, double* y_host, oz_stream_t stream);
/* Device durations (ms) of the stages of the last heff_apply / heff_apply_host of an EAGER handle,
 * from CUDA events recorded on its stream: [0] slicing of psi, [1] stage-1 GEMM launch,
 * [2] slicing of the intermediate, [3] stage-2 GEMM launch.  Waits for that product to finish. */
int oz_heff_stage_times(oz_heff* h, float* ms4);
/* Device ms (ms2[0] rowmax pass, ms2[1] digit pass; CUDA events) and algorithmic bytes of the last
 * operator slicing of an emulated handle (oz_heff_create or oz_heff_update_ops): bytes2[0] = 8 per
 * operator element read by the row-maximum pass; bytes2[1] = 8 per element read plus 2S per
 * element of the 8 x 8-padded digit tiles written.  Zeros for a native handle.  Either pointer may
 * be null. */
int oz_heff_ops_times(const oz_heff* h, float* ms2, long long* bytes2);
/* Sizes and bookkeeping of the handle. */
typedef struct oz_heff_info {
  long long dim;          /* length of psi */
  long long flops;        /* FP64 flops of one native product: sum over tasks of 2(m'mn + m'nn') */
  long long carrier_flops;/* tensor-core flops of one emulated product (padded tiles included) */
  long long bytes_ops;    /* device bytes held for the operators */
  long long bytes_scratch;/* device bytes of per-product scratch */
  long long gemm1_tiles, gemm2_tiles;
  int slices, level, mode;
  int tile;               /* OZ_TILE_CTA or OZ_TILE_PAIR: the GEMM tiles of the products */
  int units;              /* persistent units of the GEMM launches: CTAs, or CTA pairs */
  int epilogue1, epilogue2;/* epilogue layout of the stage-1 / stage-2 GEMM launches: 0 = 16 warps
                              owning 16 columns each (short tiles), 1 = 8 owners of 32 columns with
                              TMEM lane quarter 1 handed over by a loader warp, which keeps the MMA
                              issuer's scheduler partition free (long tiles: 48 k-blocks or more on
                              average); identical results.  Set once the handle has run its first
                              product (or by oz_heff_set_epilogue), 0 before */
} oz_heff_info;
int oz_heff_info_get(const oz_heff* h, oz_heff_info* out);
/* Epilogue layout of the stage-1 / stage-2 GEMM launches of an emulated handle (see
 * oz_heff_info.epilogue1/2): 0, 1, or -1 for the automatic choice from the tile lengths.  Results
 * are identical; re-captures the handle's graph (synchronises the device).  OZ_EINVAL for other
 * values, native handles, or layout 1 on a CTA-pair handle. */
int oz_heff_set_epilogue(oz_heff* h, int e1, int e2);
/* Per-block precision dial (emulated handles): s1[q] = slice level of the stage-1 product of
 * source sector q, s2[q] = level of the stage-2 product of target sector q (arrays of nsec ints;
 * null = the handle's level).  Each level must lie in 1..the handle's level s; the operator and
 * psi digits stay S deep and a product at level t uses digits 1..t and the pairs t+u <= t+1 of
 * the header comment.  Takes effect for the next product (the problem tables are rewritten in
 * place; synchronises the device).  info.carrier_flops follows the levels. */
int oz_heff_set_levels(oz_heff* h, const int* s1, const int* s2);
int oz_heff_get_levels(const oz_heff* h, int* s1, int* s2);
/* Schedule autotuner of the grouped persistent launches (emulated handles): times every schedule
 * of the stage tile lists over the persistent CTAs -- 0: longest first onto the least loaded CTA,
 * each CTA's tiles in descending cost; 1: the same, ascending; 2: strided (CTA b takes tiles b,
 * b + #CTAs, ... of the k-descending list) -- with `reps` products of d_psi each (after one
 * warm-up product), and keeps the fastest per stage.  sched (2 ints, may be null) receives the
 * choice for stage 1 and 2; ms (6 floats, may be null) the best stage-1 / stage-2 time of each
 * schedule.  Synchronous.  Results do not depend on the schedule. */
int oz_heff_autotune(oz_heff* h, const double* d_psi, int reps, int* sched, float* ms, oz_stream_t stream);

/* ------------------------------------------------------------------------------------------
 * Term sharding over several GPUs (paper, section "Numerical procedure" and the timing discussion:
 * the sweeps run on one multi-GPU node; how the effective-Hamiltonian work is divided is not
 * described, so the natural split of the task sum is used).  Each rank builds an H_eff handle from
 * the tasks it owns (oz_heff_create with that subset), computes its partial Y with heff_apply,
 * exchanges the partial vectors (a collective of the caller's framework) and sums them with
 * oz_reduce_ordered.  The stage-2 exponents are shared by the tasks of a target sector on one
 * handle, so the sharded sum equals the single-handle product within the emulation's accuracy,
 * not bit for bit.
 * oz_heff_partition: HOST function (no GPU needed).  owner[t] in 0..world-1 for every task t of
 *   the structure (m[nsec], n[nsec], src[ntask], dst[ntask]): tasks in descending order of FP64
 *   flop cost 2 m[dst] m[src] n[src] + 2 m[dst] n[src] n[dst] (equal costs in task order), each
 *   onto the rank with the least cost so far (ties to the lower rank).  Deterministic: every rank
 *   computes the same table.  OZ_EINVAL: world < 1, sector out of range, null pointers.
 * oz_reduce_ordered: d_out[i] = ((p_0[i] + p_1[i]) + p_2[i]) + ... in FP64 on `stream`, one
 *   rounding per addition in part order (a result independent of arrival order).  d_parts is a
 *   HOST array of nparts (1..64) DEVICE pointers of length len; d_out may alias d_parts[0].
 *   OZ_EINVAL on bad arguments, OZ_ECUDA on a launch failure.
 * ------------------------------------------------------------------------------------------ */
int oz_heff_partition(int nsec, const int* m, const int* n, int ntask, const int* src, const int* dst, int world,
                      int* owner);
int oz_reduce_ordered(const double* const* d_parts, int nparts, long long len, double* d_out, oz_stream_t stream);
/* The term-sharded product on ONE GPU, for structures whose operator digit planes do not fit in
 * device memory at once (oz_heff_create fails with OZ_ENOMEM): the tasks are split into `chunks`
 * groups by oz_heff_partition (world = chunks); for each group in turn a handle is built (its
 * operators sliced), its partial product computed and the handle destroyed; the partial vectors
 * are summed in group order as in oz_reduce_ordered.  d_y (dim doubles, dim = sum_q m[q] n[q])
 * then holds exactly what the sharded product over `chunks` ranks reduces to.  Every call slices
 * every operator again; peak device memory is one group's handle plus one partial vector.  prec
 * as for oz_heff_create; chunks = 1 is one handle's product.  Synchronises the stream.  Errors:
 * those of oz_heff_create and heff_apply (OZ_ENOMEM when even one group does not fit),
 * OZ_EINVAL for chunks < 1. */
int oz_heff_apply_streamed(oz_ctx* ctx, int nsec, const int* m, const int* n, int ntask, const oz_task* tasks,
                           const oz_prec* prec, int chunks, const double* d_psi, double* d_y, oz_stream_t stream);

/* ------------------------------------------------------------------------------------------
 * Slice-level selection per block (the precision dial of sections "Theory of emulated FP64
 * arithmetic" and "Numerical procedure"; the paper's library picks the slice count per GEMM).
 *
 * Features of one product (OZ_NFEAT floats): for A (rows) then B (columns), the fractions of
 * elements whose exponent lies 0, 1, 2-3, 4-7, 8-15, 16-31, 32-63, >= 64 below the largest of
 * their row/column, and the fraction of zeros (9 + 9); then log2(K)/16 and log2(M N)/32.
 * oz_heff_problem_features: features of every stage-1 product (feat1, row q = source sector q)
 *   and stage-2 product (feat2, row q = target sector q) for psi (rows of sectors without a
 *   product are zero); runs one product at the handle's level.  Host arrays of nsec x OZ_NFEAT.
 * oz_heff_problem_errors: true relative Frobenius errors of every product at `level` against the
 *   handle's own level (stage 1 with stage 2 at the full level and vice versa); err = -1 where a
 *   sector has no product.  Host arrays of nsec.  Levels are restored afterwards.
 * oz_heff_select_levels: picks and sets per-product levels with the smallest carrier flops it can
 *   reach greedily while the predicted error of each stage output, sum_q (10^(pred_q + margin)
 *   |out_q|)^2, stays within (budget |out| / sqrt 2)^2 (norms from one product at the full level;
 *   `budget` is a relative Frobenius error, `margin` a safety in decades).  selector:
 *   OZ_SELECT_FIXED (the handle's level), OZ_SELECT_ANALYTIC (error 2^(gA + gB - 8 s + 3) from
 *   the effective exponent gaps), OZ_SELECT_LEARNED (`net`, OZ_NFEAT inputs, outputs = log10
 *   error at levels 3..8).  Levels below 3 are never picked.  A handle at level 9 (the fixed
 *   fallback) starts there with its error counted as zero and is lowered from 9 to 8 like any
 *   other step.  Writes the levels to s1/s2 (may be null).
 * ------------------------------------------------------------------------------------------ */
#define OZ_NFEAT 20
#define OZ_SELECT_FIXED 0
#define OZ_SELECT_ANALYTIC 1
#define OZ_SELECT_LEARNED 2
typedef struct oz_mlp_s oz_mlp;
int oz_heff_problem_features(oz_heff* h, const double* d_psi, float* feat1, float* feat2, oz_stream_t stream);
int oz_heff_problem_errors(oz_heff* h, const double* d_psi, int level, double* err1, double* err2,
                           oz_stream_t stream);
int oz_heff_select_levels(oz_heff* h, const double* d_psi, int selector, double budget, oz_mlp* net, double margin,
                          int* s1, int* s2, oz_stream_t stream);

/* ------------------------------------------------------------------------------------------
 * Selector network: a two-hidden-layer tanh MLP in FP32, trained on the device by its own
 * forward, backward and Adam kernels.  H1 = tanh(X W1 + b1), H2 = tanh(H1 W2 + b2),
 * Y = H2 W3 + b3; loss = sum(M (Y - T)^2) / max(1, sum M) (M masks missing targets).  Parameters
 * flattened as W1 (nin x nh, row-major), b1, W2, b2, W3, b3; Xavier-uniform init from `seed`.
 * Device matrices are row-major FP32 (X: rows x nin; Y, T, M: rows x nout).
 * oz_mlp_gradient: loss and gradient over all rows (host_grad: param_count floats, may be null).
 * oz_mlp_train: epochs of Adam (b1 0.9, b2 0.999, eps 1e-8) over shuffled minibatches of
 *   `batch` rows (a partial last batch is skipped); final_loss (may be null) = loss over all rows.
 * ------------------------------------------------------------------------------------------ */
int oz_mlp_create(int nin, int nhidden, int nout, unsigned long long seed, oz_mlp** out);
int oz_mlp_destroy(oz_mlp* net);
int oz_mlp_param_count(const oz_mlp* net);
int oz_mlp_nin(const oz_mlp* net);
int oz_mlp_nout(const oz_mlp* net);
int oz_mlp_get_params(const oz_mlp* net, float* host);
int oz_mlp_set_params(oz_mlp* net, const float* host);
int oz_mlp_forward(oz_mlp* net, const float* d_X, int rows, float* d_Y, oz_stream_t stream);
int oz_mlp_gradient(oz_mlp* net, const float* d_X, const float* d_T, const float* d_M, int rows, float* loss,
                    float* host_grad, oz_stream_t stream);
int oz_mlp_train(oz_mlp* net, const float* d_X, const float* d_T, const float* d_M, int rows, int epochs, int batch,
                 float lr, unsigned long long seed, float* final_loss, oz_stream_t stream);

/* Diagonal of H_eff (length dim) into d_diag: sum over the tasks with src == dst of
 * coef L[i][i] R[j][j] at element (src, i, j) -- the Davidson preconditioner.  Built from the FP64
 * operator blocks during oz_heff_create (an exact function of them, independent of the emulation). */
int oz_heff_diag(const oz_heff* h, double* d_diag, oz_stream_t stream);

/* ------------------------------------------------------------------------------------------
 * Davidson eigensolver for the lowest eigenpair of H_eff (paper, section "Theory of TNS/DMRG
 * regarding error analysis": the two-site update solves the eigenproblem of H_eff with a Krylov
 * method; section "Numerical procedure": stop at a residual threshold).  Iteration:
 *   G = V^T W symmetrised, (theta, y) = lowest eigenpair of G, x = V y, r = W y - theta x;
 *   converged when |r|_2 <= tol; otherwise d = r / (theta - diag H_eff) (|theta - diag| floored
 *   at 1e-12, sign kept), restart to the two lowest Ritz vectors when V holds max_sub vectors,
 *   orthogonalise d against V twice (classical Gram-Schmidt), normalise, append, W += H_eff d.
 * Every step runs on the device in FP64 except the H_eff products (emulated or native as the handle
 * says).  The state owns 2 (max_sub + 3) + 1 device vectors of length dim.  The handle must outlive
 * the state.  Each davidson_step synchronises `stream` twice (it returns theta and |r|).
 * ------------------------------------------------------------------------------------------ */
typedef struct oz_davidson_s oz_davidson;
/* max_sub in 3..32; tol > 0.  Errors: OZ_EINVAL, OZ_ENOMEM. */
int oz_davidson_create(oz_heff* h, int max_sub, double tol, oz_davidson** out);
int oz_davidson_destroy(oz_davidson* d);
/* V = [x0 / |x0|], W = [H_eff V_0].  OZ_EINVAL if x0 has zero or non-finite norm. */
int davidson_start(oz_davidson* d, const double* d_x0, oz_stream_t stream);
/* One iteration: writes the Ritz value and residual norm of the current subspace; sets
 * *converged = 1 (and expands nothing) when |r| <= tol, else expands the subspace by one vector.
 * OZ_ENOCONV if the correction vanished after orthogonalisation (norm < 1e-14); OZ_ENONFINITE if
 * theta or |r| is not finite. */
int davidson_step(oz_davidson* d, double* theta, double* resid, int* converged, oz_stream_t stream);
/* The normalised Ritz vector of the last davidson_step into d_x (length dim). */
int davidson_ritz(oz_davidson* d, double* d_x, oz_stream_t stream);
/* Whole solve with max_sub = 24: d_psi is the start vector on entry and the normalised Ritz vector
 * on exit; *energy = last Ritz value, *iters = iterations.  OZ_ENOCONV when max_iter iterations did
 * not converge (d_psi and *energy then hold the last iterate).  The projected matrix of each
 * iteration is the previous one bordered by one row and column, so its Jacobi solve starts from
 * the previous eigenvectors (Davidson and Lanczos; restarts solve from scratch). */
int davidson_solve(oz_heff* h, double* d_psi, double tol, int max_iter, double* energy, int* iters,
                   oz_stream_t stream);
/* Lanczos alternative to davidson_solve (paper, section "Theory of TNS/DMRG ...": the Krylov
 * solver of the two-site update, Lanczos in most of the paper's runs): Krylov vectors with full
 * reorthogonalisation (classical Gram-Schmidt twice), the lowest eigenpair of the tridiagonal
 * matrix by the one-CTA Jacobi solver, explicit restart from the Ritz vector every `krylov`
 * vectors (2..31).  Converged when the residual estimate beta_j |y_j| <= eps ("Numerical
 * procedure": Krylov threshold epsilon).  d_psi: start vector in, normalised Ritz vector out;
 * *energy = Ritz value, *iters = products.  OZ_ENOCONV when max_iter products (or an invariant
 * subspace) end the run first; psi and energy then hold the last Ritz pair. */
int lanczos_solve(oz_heff* h, double* d_psi, double eps, int max_iter, int krylov, double* energy, int* iters,
                  oz_stream_t stream);
/* Verification entry point of the projected eigensolver (one-CTA cyclic Jacobi, FP64): eigenvalues
 * of the symmetric m x m matrix d_G (row-major, ldg; m in 1..32) ascending into d_w[m] and the
 * eigenvectors as the columns of d_V (row-major m x m, ldv).  Synchronous.  OZ_ENOCONV if 60 sweeps
 * did not bring the off-diagonal mass below 1e-32 of the total. */
int oz_symeig_small(const double* d_G, int m, int ldg, double* d_w, double* d_V, int ldv, oz_stream_t stream);

/* ------------------------------------------------------------------------------------------
 * Matrix product operator of the ab initio Hamiltonian (host code, no GPU needed)
 *   H = sum_{pq,s} h_pq a+_{ps} a_{qs} + 1/2 sum_{pqrs,s,t} (pq|rs) a+_{ps} a+_{rt} a_{st} a_{qs}
 * on L spatial orbitals, one site per orbital (local states |0>, |up>, |down>, |up down>),
 * Jordan-Wigner order orbital-major, up before down.  It defines the renormalised operators of the
 * two-site sweep (paper, section "Theory of TNS/DMRG ...": the effective Hamiltonian of the
 * two-site update; the paper leaves the operator construction to the cited DMRG literature).
 *   h1: L x L, eri: L^4 chemist-notation (pq|rs) at index ((p L + q) L + r) L + s; HOST FP64.
 * oz_mpo_bond_dims: chi[b + 1] = number of MPO states on bond b = -1..L-1 (chi has L + 1 entries).
 * oz_mpo_dense: the MPO contracted to the dense 4^L x 4^L matrix (row-major, basis index
 *   sum_p s_p 4^p), for L in 2..4 -- a verification entry point.
 * ------------------------------------------------------------------------------------------ */
int oz_mpo_bond_dims(const double* h1, const double* eri, int L, int* chi);
int oz_mpo_dense(const double* h1, const double* eri, int L, double* out);

/* ------------------------------------------------------------------------------------------
 * Two-site DMRG sweep (paper, section "Theory of TNS/DMRG regarding error analysis": sweep the
 * chain; at every bond find the lowest eigenpair of the effective Hamiltonian of the two-site
 * tensor with a Krylov method, truncate it with an SVD of the two-site tensor and renormalise the
 * block operators; the energy approaches the exact ground state from above).
 *   - U(1) x U(1) symmetry (electron number, 2 Sz); the environments are the MPO's partial sums
 *     on every block, so H_eff = sum_w L_w (x) R_w is a task list of heff_apply (emulated or
 *     native FP64 as `prec` says); its lowest eigenpair comes from davidson_solve (tolerance
 *     davidson_tol on |r|_2, at most 1000 iterations), started from the previous bond's solution
 *     carried to this bond (oz_dmrg_set_prediction), or else from a counter-based generator keyed
 *     by `seed` and the step number.
 *   - Start: every right block holds the single state of the reference determinant (orbitals
 *     filled from 0 with (N + 2Sz)/2 up and (N - 2Sz)/2 down electrons).
 *   - A sweep is bonds 0..L-2 left to right, then L-2..0 right to left; every bond but the last of
 *     a half-sweep truncates the enlarged block: all of it when it has at most D states, otherwise
 *     the largest eigenvalues (> 1e-14, at most D, never cutting through a group of equal values)
 *     of the reduced density matrix of each sector (FP64 on the device).
 *   - h1 (L x L) and eri (L^4, chemist) are HOST arrays as for oz_mpo_bond_dims.
 * Limits: a density-matrix sector may hold at most 1024 states (OZ_EINVAL otherwise; sectors of
 * more than 112 states are diagonalised in global instead of shared memory).
 * A bond whose Davidson run stops short of its tolerance keeps its best Ritz pair and is marked
 * in oz_dmrg_step.converged.  Errors: OZ_EINVAL (arguments, limits), OZ_ENOCONV (density-matrix
 * Jacobi did not converge), OZ_ENONFINITE, OZ_ECUDA, OZ_ENOMEM.  Synchronous; uses its own stream
 * on the context's device.
 * ------------------------------------------------------------------------------------------ */
typedef struct oz_dmrg_s oz_dmrg;
typedef struct oz_dmrg_step {
  int sweep;         /* 0-based sweep */
  int dir;           /* 0 = left to right, 1 = right to left */
  int bond;          /* i: the two sites are i and i + 1 */
  int dim;           /* length of the two-site vector */
  int nterm;         /* MPO states on the bond: terms w of H_eff */
  int ntask;         /* sector tasks of H_eff */
  int iters;         /* Davidson iterations */
  int converged;     /* 1 if the eigensolver met its tolerance (0: best Ritz pair kept, sweep continued) */
  int kept;          /* states of the new block (0: no truncation at this bond) */
  double energy;     /* lowest Ritz value */
  double discarded;  /* sum of the discarded density-matrix eigenvalues */
  double energy_fp64;  /* with the FP64 check: psi^T H_eff psi in native FP64 (else = energy) */
  int nonvariational;  /* with the FP64 check: 1 if energy < energy_fp64 - 1e-8 Eh */
  int predicted;       /* 1 if the eigensolver started from the previous bond's transformed solution */
  int rotated;         /* 1 if the truncation chose states (density-matrix eigenvectors) and
                          renormalised the operators; 0 if the whole enlarged block was kept */
} oz_dmrg_step;
int oz_dmrg_create(oz_ctx* ctx, const double* h1, const double* eri, int L, int nelec, int twosz, int D,
                   const oz_prec* prec, double davidson_tol, unsigned long long seed, oz_dmrg** out);
int oz_dmrg_destroy(oz_dmrg* d);
/* Start vectors of the two-site eigensolver (on by default): the previous bond's solution carried
 * to this bond -- the same vector at a turning point (unchanged problem), otherwise the truncated
 * side rotated into the new block (U^T psi or psi U) and the other block's states expanded over
 * (site x block) with the kept vectors that made that block in the previous sweep.  Where no
 * prediction applies (the first pass over the reference blocks) or its squared norm is below 1e-6, a
 * seeded random vector is used, as with on = 0.  Converged energies do not depend on the start. */
int oz_dmrg_set_prediction(oz_dmrg* d, int on);
/* Runs nsweeps more sweeps; energies (if not null) receives 2 (L - 1) nsweeps Ritz values in
 * bond order. */
int oz_dmrg_run(oz_dmrg* d, int nsweeps, double* energies);
/* Per-bond record of every step run so far (*n = count; up to cap entries copied). */
int oz_dmrg_steps(const oz_dmrg* d, oz_dmrg_step* out, int cap, int* n);
/* Verification entry point: builds H_eff of `bond` from the current environments; *dim = length
 * of its two-site vector; patterns (if not null, length *dim) = determinant occupation pattern of
 * every basis state (bit 2p = orbital p up, bit 2p + 1 down; -1 once a block was rotated by a
 * truncation); if d_psi and d_y are not null, d_y = H_eff d_psi (device vectors).  Call first
 * with null pointers to learn *dim. */
int oz_dmrg_bond_heff(oz_dmrg* d, int bond, const double* d_psi, double* d_y, long long* patterns,
                      long long* dim, oz_stream_t stream);
/* Precision of the renormalisation products E' = U^T O U of the sweep (paper, section
 * "Theory of TNS/DMRG ...": the renormalisation is the other GEMM-heavy subroutine of the sweep).
 * Default OZ_MODE_NATIVE (FP64 on the device); OZ_MODE_EAGER runs both passes of every bond as
 * grouped emulated products with prec->slices digits at prec->level. */
int oz_dmrg_set_renorm_prec(oz_dmrg* d, const oz_prec* prec);
/* Precision of the reduced density matrices psi psi^T (psi^T psi on the right) that the
 * truncation diagonalises (paper, section "Theory of TNS/DMRG ...": the truncation subroutine).
 * Default OZ_MODE_NATIVE; OZ_MODE_EAGER forms them as grouped emulated products.  The Jacobi
 * eigensolver itself stays FP64. */
int oz_dmrg_set_rdm_prec(oz_dmrg* d, const oz_prec* prec);
/* Eigensolver of the two-site update: OZ_SOLVER_DAVIDSON (default; tol on |r|_2) or
 * OZ_SOLVER_LANCZOS (tol = the Krylov threshold epsilon on beta_j |y_j|; Krylov dimension 30);
 * at most 1000 products per bond.  check_fp64 = 1 re-evaluates every Ritz vector of an emulated
 * sweep with the bond's FP64 H_eff (oz_dmrg_step.energy_fp64) and flags Ritz values below it
 * (oz_dmrg_step.nonvariational). */
#define OZ_SOLVER_DAVIDSON 0
#define OZ_SOLVER_LANCZOS 1
int oz_dmrg_set_solver(oz_dmrg* d, int solver, double tol, int check_fp64);
/* Verification entry points for the emulated renormalisation and density matrices (the same
 * passages as oz_dmrg_set_renorm_prec and oz_dmrg_set_rdm_prec).  oz_dmrg_set_trace(d, stride)
 * clears the record and, for stride > 0, copies products 0, stride, 2 stride, ... of every
 * emulated batch that the sweep runs from then on (each truncating bond runs one batch per
 * renormalisation pass and one of density matrices) to host memory: operands and result.
 * stride = 0 stops recording.  The copies synchronise the sweep's stream; use it on small systems.
 * oz_dmrg_trace(d, i, info, A, B, C, n): *n (if not null) = number of records; for i >= 0,
 * info[0..6] = kind (0: T = O U, the first renormalisation pass of an MPO state and sector; 1:
 * E = U^T T, the second pass; 2: a density matrix psi psi^T or psi^T psi of one sector), step
 * (index of the oz_dmrg_steps entry of the bond), M, N, K, slices, level; A (M x K) and B (K x N)
 * receive the operands as multiplied (op(A), op(B)) and C (M x N) the emulated result, all
 * row-major HOST arrays that the caller sizes from info (pass null to skip).  i < 0 only sets *n.
 * OZ_EINVAL: null handle, negative stride, i out of range. */
int oz_dmrg_set_trace(oz_dmrg* d, int stride);
int oz_dmrg_trace(const oz_dmrg* d, long long i, int* info, double* A, double* B, double* C, long long* n);
/* One-shot form: create, run nsweeps, destroy. */
int dmrg_sweep(oz_ctx* ctx, const double* h1, const double* eri, int L, int nelec, int twosz, int D, int nsweeps,
               const oz_prec* prec, double davidson_tol, unsigned long long seed, double* energies);

#ifdef __cplusplus
}
#endif
#endif /* OZDMRG_H */
