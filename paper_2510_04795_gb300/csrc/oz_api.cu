// C ABI of libozdmrg: contexts, ozaki_gemm, verification entries and the H_eff handle.
// Host orchestration only; every step of a product runs in the kernels of oz_slice.cu and
// oz_gemm.cu (or cuBLAS DGEMM in OZ_MODE_NATIVE).
#include <cublas_v2.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ozdmrg.h"
#include "oz_gemm.cuh"
#include "oz_handles.cuh"
#include "oz_internal.cuh"
#include "oz_slice.cuh"

using oz::GemmProblem;
using oz::GemmTile;
using oz::SliceSeg;

namespace {
thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
int cuda_fail(cudaError_t e, const char* where) {
  return fail(e == cudaErrorMemoryAllocation ? OZ_ENOMEM : OZ_ECUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}
#define OZ_CU(call)                                   \
  do {                                                \
    cudaError_t _e = (call);                          \
    if (_e != cudaSuccess) return cuda_fail(_e, #call); \
  } while (0)

inline long long cdiv(long long a, long long b) { return (a + b - 1) / b; }
inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int check_prec(const oz_prec* p, int* S, int* s, int* mode) {
  if (!p) return fail(OZ_EINVAL, "prec is null");
  if (p->slices < 1 || p->slices > 9) return fail(OZ_EINVAL, "slices must be in 1..9");
  int lvl = p->level == 0 ? p->slices : p->level;
  if (lvl < 1 || lvl > p->slices || lvl > oz::MAX_LEVEL) return fail(OZ_EINVAL, "level must be in 1..S");
  if (p->mode != OZ_MODE_EAGER && p->mode != OZ_MODE_NATIVE) return fail(OZ_EINVAL, "unknown mode");
  *S = p->slices;
  *s = lvl;
  *mode = p->mode;
  return OZ_OK;
}

__global__ void scale_kernel(double* C, int m, int n, int ldc, double beta) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)m * n) return;
  int i = (int)(idx / n), j = (int)(idx % n);
  double* c = C + (long long)i * ldc + j;
  *c = beta == 0.0 ? 0.0 : __dmul_rn(beta, *c);
}
__global__ void fill_int_kernel(int* p, long long n, int v) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < n) p[idx] = v;
}
}  // namespace


extern "C" const char* oz_last_error(void) { return g_err.c_str(); }

extern "C" int oz_ctx_create(oz_ctx** out, int device) {
  if (!out) return fail(OZ_EINVAL, "out is null");
  *out = nullptr;
  OZ_CU(cudaSetDevice(device));
  cudaDeviceProp prop;
  OZ_CU(cudaGetDeviceProperties(&prop, device));
  if (prop.major != 10 || prop.minor != 3)
    return fail(OZ_EINVAL, "libozdmrg is built for sm_103a (GB300); found sm_" + std::to_string(prop.major) +
                               std::to_string(prop.minor));
  oz_ctx* c = new oz_ctx_s();
  c->device = device;
  c->nsm = prop.multiProcessorCount;
  cudaError_t e = cudaMalloc(&c->d_flags, 16);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "cudaMalloc flags");
  }
  cudaMemset(c->d_flags, 0, 16);
  if (cublasCreate(&c->cublas) != CUBLAS_STATUS_SUCCESS) {
    cudaFree(c->d_flags);
    delete c;
    return fail(OZ_ECUDA, "cublasCreate failed");
  }
  // native FP64 comparator: default math (no fixed-point emulation)
  cublasSetMathMode(c->cublas, CUBLAS_DEFAULT_MATH);
  *out = c;
  return OZ_OK;
}

extern "C" int oz_ctx_destroy(oz_ctx* c) {
  if (!c) return OZ_OK;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  if (c->cublas) cublasDestroy(c->cublas);
  if (c->ws) cudaFree(c->ws);
  if (c->d_flags) cudaFree(c->d_flags);
  delete c;
  return OZ_OK;
}

extern "C" int oz_status(oz_ctx* c, oz_stream_t stream) {
  if (!c) return fail(OZ_EINVAL, "ctx is null");
  OZ_CU(cudaStreamSynchronize((cudaStream_t)stream));
  int f[4];
  OZ_CU(cudaMemcpy(f, c->d_flags, 16, cudaMemcpyDeviceToHost));
  OZ_CU(cudaMemset(c->d_flags, 0, 16));
  if (f[1]) return fail(OZ_ETIMEOUT, "a bounded device wait gave up (kernel aborted)");
  if (f[0]) return fail(OZ_ENONFINITE, "an input held NaN or Inf");
  return OZ_OK;
}

// --------------------------------------------------------------------------------------------
// dense products
// --------------------------------------------------------------------------------------------
namespace {
struct DenseOperands {
  __half* dA;
  __half* dB;
  unsigned long long* mx;
  int* ex;
  int nkb, nrbA, nrbB, mpad, npad;
};

// Workspace layout and slicing of A (rows) and B (columns) for one product.
int slice_pair(oz_ctx* c, int m, int n, int k, const double* A, int lda, const double* B, int ldb, int S,
               DenseOperands& o, cudaStream_t st) {
  o.nkb = (int)cdiv(k, oz::KB);
  o.nrbA = (int)cdiv(m, oz::TILE_M);
  o.nrbB = (int)cdiv(n, oz::BN);
  o.mpad = o.nrbA * oz::TILE_M;
  o.npad = o.nrbB * oz::BN;
  size_t bA = (size_t)o.nrbA * o.nkb * S * oz::TILE_M * oz::KB * 2;
  size_t bB = (size_t)o.nrbB * o.nkb * S * oz::BN * oz::KB * 2;
  size_t bM = (size_t)(o.mpad + o.npad) * 8;
  size_t bE = (size_t)(o.mpad + o.npad) * 4;
  size_t need = align256(bA) + align256(bB) + align256(bM) + align256(bE) + 256;
  int rc = c->reserve(need);
  if (rc) return rc;
  char* p = c->ws;
  o.dA = (__half*)p;
  p += align256(bA);
  o.dB = (__half*)p;
  p += align256(bB);
  o.mx = (unsigned long long*)p;
  p += align256(bM);
  o.ex = (int*)p;
  OZ_CU(cudaMemsetAsync(o.mx, 0, bM, st));
  oz::SegPack pk{};
  SliceSeg& a = pk.seg[0];
  a.src = A; a.ld = lda; a.rows = m; a.cols = k; a.prows = o.mpad; a.pcols = o.nkb * oz::KB;
  a.r0 = 0; a.k0 = 0; a.trans = 0; a.S = S; a.scale = 1.0; a.dst = o.dA; a.TR = oz::TILE_M; a.nkb = o.nkb;
  a.rowmax = o.mx; a.rowexp = o.ex; a.unit0 = 0; a.unit0m = 0;
  SliceSeg& b = pk.seg[1];
  b.src = B; b.ld = ldb; b.rows = n; b.cols = k; b.prows = o.npad; b.pcols = o.nkb * oz::KB;
  b.r0 = 0; b.k0 = 0; b.trans = 1; b.S = S; b.scale = 1.0; b.dst = o.dB; b.TR = oz::BN; b.nkb = o.nkb;
  b.rowmax = o.mx + o.mpad; b.rowexp = o.ex + o.mpad;
  b.unit0 = oz::digit_units(a.prows, a.pcols);
  b.unit0m = oz::rowmax_units(a.rows, a.cols, a.trans);
  const int nseg = B ? 2 : 1;
  long long um = b.unit0m + (B ? oz::rowmax_units(b.rows, b.cols, b.trans) : 0);
  long long ud = b.unit0 + (B ? oz::digit_units(b.prows, b.pcols) : 0);
  OZ_CU(oz::launch_rowmax(nullptr, &pk, nseg, um, c->d_flags, st));
  OZ_CU(oz::launch_digits(nullptr, &pk, nseg, ud, S, st));
  return OZ_OK;
}
}  // namespace

namespace {
int ceil_log2(int x) {
  int r = 0;
  while ((1ll << r) < (long long)x) ++r;
  return r;
}
// shape class of the performant dispatch
unsigned long long perf_key(int m, int n, int k, int S, int s) {
  return ((unsigned long long)ceil_log2(std::max(m, 1)) << 32) | ((unsigned long long)ceil_log2(std::max(n, 1)) << 24) |
         ((unsigned long long)ceil_log2(std::max(k, 1)) << 16) | ((unsigned long long)S << 8) | (unsigned long long)s;
}
}  // namespace

extern "C" int oz_performant_choice(oz_ctx* c, int m, int n, int k, const oz_prec* prec, int* mode, float* ms) {
  if (!c || !prec || !mode) return fail(OZ_EINVAL, "null argument");
  oz_prec q = *prec;
  q.mode = OZ_MODE_EAGER;
  int S, s, md;
  if (int rc = check_prec(&q, &S, &s, &md)) return rc;
  auto it = c->perf.find(perf_key(m, n, k, S, s));
  *mode = it == c->perf.end() ? -1 : it->second.mode;
  if (ms) {
    ms[0] = it == c->perf.end() ? 0.f : it->second.ms_emu;
    ms[1] = it == c->perf.end() ? 0.f : it->second.ms_nat;
  }
  return OZ_OK;
}

extern "C" int ozaki_gemm(oz_ctx* c, int m, int n, int k, double alpha, const double* A, int lda, const double* B,
                          int ldb, double beta, double* C, int ldc, const oz_prec* prec, oz_stream_t stream) {
  if (!c) return fail(OZ_EINVAL, "ctx is null");
  if (prec && prec->mode == OZ_MODE_PERFORMANT) {
    // the paper's performant mode: emulate only where it is faster, decided per shape class by
    // timing both paths once (into a scratch C, so that beta * C is not disturbed)
    oz_prec q = *prec;
    q.mode = OZ_MODE_EAGER;
    int S, s, md;
    if (int rc = check_prec(&q, &S, &s, &md)) return rc;
    if (m > 0 && n > 0 && k > 0 && k <= oz::max_k_of_level(s) && lda >= k && ldb >= n && ldc >= n) {
      const unsigned long long key = perf_key(m, n, k, S, s);
      auto it = c->perf.find(key);
      if (it == c->perf.end()) {
        cudaStream_t st = (cudaStream_t)stream;
        double* tmp = nullptr;
        OZ_CU(cudaMalloc(&tmp, (size_t)m * n * 8));
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float t[2] = {0.f, 0.f};
        int rc = OZ_OK;
        for (int path = 0; path < 2 && rc == OZ_OK; ++path) {
          oz_prec r = q;
          r.mode = path == 0 ? OZ_MODE_EAGER : OZ_MODE_NATIVE;
          // one untimed run (workspace growth, library warm-up), one timed run
          rc = ozaki_gemm(c, m, n, k, 1.0, A, lda, B, ldb, 0.0, tmp, n, &r, stream);
          if (rc == OZ_OK) {
            cudaEventRecord(e0, st);
            rc = ozaki_gemm(c, m, n, k, 1.0, A, lda, B, ldb, 0.0, tmp, n, &r, stream);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&t[path], e0, e1);
          }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaFree(tmp);
        if (rc != OZ_OK) return rc;
        it = c->perf.emplace(key, oz_ctx_s::PerfChoice{t[0] <= t[1] ? OZ_MODE_EAGER : OZ_MODE_NATIVE, t[0], t[1]}).first;
      }
      q.mode = it->second.mode;
    }
    return ozaki_gemm(c, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, &q, stream);
  }
  int S, s, mode;
  if (int rc = check_prec(prec, &S, &s, &mode)) return rc;
  if (m < 0 || n < 0 || k < 0) return fail(OZ_EINVAL, "negative size");
  if (lda < std::max(k, 1) || ldb < std::max(n, 1) || ldc < std::max(n, 1)) return fail(OZ_EINVAL, "leading dimension too small");
  if (m == 0 || n == 0) return OZ_OK;
  if (k > oz::max_k_of_level(s))
    return fail(OZ_EINVAL, s >= oz::SPLIT_LEVEL ? "k exceeds the exact-accumulation limit of level 9 (130048)"
                                                : "k exceeds the exact-accumulation limit (1048576)");
  cudaStream_t st = (cudaStream_t)stream;
  if (k == 0) {
    scale_kernel<<<(unsigned)cdiv((long long)m * n, 256), 256, 0, st>>>(C, m, n, ldc, beta);
    OZ_CU(cudaGetLastError());
    return OZ_OK;
  }
  if (mode == OZ_MODE_NATIVE) {
    cublasSetStream(c->cublas, st);
    // row-major C = A B  <=>  column-major C^T = B^T A^T
    if (cublasDgemm(c->cublas, CUBLAS_OP_N, CUBLAS_OP_N, n, m, k, &alpha, B, ldb, A, lda, &beta, C, ldc) !=
        CUBLAS_STATUS_SUCCESS)
      return fail(OZ_ECUDA, "cublasDgemm failed");
    return OZ_OK;
  }
  DenseOperands o;
  if (int rc = slice_pair(c, m, n, k, A, lda, B, ldb, S, o, st)) return rc;
  GemmProblem P{};
  P.A = o.dA; P.B = o.dB; P.ea = o.ex; P.eb = o.ex + o.mpad;
  P.M = m; P.N = n; P.nkb = o.nkb; P.SA = S; P.SB = S; P.s = s;
  P.mode = oz::OUT_DENSE; P.C = C; P.ldc = ldc; P.alpha = alpha; P.beta = beta;
  int ntiles = o.nrbA * o.nrbB;
  OZ_CU(oz::launch_gemm(nullptr, nullptr, ntiles, c->nsm, &P, 0, c->d_flags + 1, st, nullptr, false,
                        oz::gemm_handover_for(o.nkb)));
  return OZ_OK;
}

extern "C" int ozaki_slice(oz_ctx* c, int rows, int cols, const double* A, int lda, int slices, int8_t* digits,
                           int* exps, oz_stream_t stream) {
  if (!c) return fail(OZ_EINVAL, "ctx is null");
  if (rows <= 0 || cols <= 0 || lda < cols) return fail(OZ_EINVAL, "bad sizes");
  if (slices < 1 || slices > 9) return fail(OZ_EINVAL, "slices must be in 1..9");
  cudaStream_t st = (cudaStream_t)stream;
  DenseOperands o;
  if (int rc = slice_pair(c, rows, 1, cols, A, lda, nullptr, 1, slices, o, st)) return rc;
  OZ_CU(oz::launch_untile(o.dA, oz::TILE_M, o.nkb, slices, rows, cols, digits, st));
  OZ_CU(cudaMemcpyAsync(exps, o.ex, (size_t)rows * 4, cudaMemcpyDeviceToDevice, st));
  return OZ_OK;
}

extern "C" int ozaki_slice_products(oz_ctx* c, int m, int n, int k, const double* A, int lda, const double* B,
                                    int ldb, int slices, double* Pout, oz_stream_t stream) {
  if (!c) return fail(OZ_EINVAL, "ctx is null");
  if (m <= 0 || n <= 0 || k <= 0 || lda < k || ldb < n) return fail(OZ_EINVAL, "bad sizes");
  if (slices < 1 || slices > 9) return fail(OZ_EINVAL, "slices must be in 1..9");
  cudaStream_t st = (cudaStream_t)stream;
  const int S = slices;
  DenseOperands o;
  if (int rc = slice_pair(c, m, n, k, A, lda, B, ldb, S, o, st)) return rc;
  // unit exponents (7 + 7 - 8 - 6 = 0): the epilogue then returns the integer P_tu itself
  int* sevens = nullptr;
  {
    size_t used = (size_t)((char*)(o.ex + o.mpad + o.npad) - c->ws);
    size_t need = align256(used) + align256((size_t)std::max(o.mpad, o.npad) * 4);
    if (need > c->ws_bytes) return fail(OZ_ENOMEM, "workspace too small for slice products");
    sevens = (int*)(c->ws + align256(used));
    long long ne = std::max(o.mpad, o.npad);
    fill_int_kernel<<<(unsigned)cdiv(ne, 256), 256, 0, st>>>(sevens, ne, 7);
    OZ_CU(cudaGetLastError());
  }
  for (int t = 0; t < S; ++t)
    for (int u = 0; u < S; ++u) {
      GemmProblem P{};
      P.A = o.dA + (size_t)t * oz::TILE_M * oz::KB;
      P.B = o.dB + (size_t)u * oz::BN * oz::KB;
      P.ea = sevens; P.eb = sevens;
      P.M = m; P.N = n; P.nkb = o.nkb; P.SA = S; P.SB = S; P.s = 1;
      P.mode = oz::OUT_DENSE; P.C = Pout + (size_t)(t * S + u) * m * n; P.ldc = n; P.alpha = 1.0; P.beta = 0.0;
      OZ_CU(oz::launch_gemm(nullptr, nullptr, o.nrbA * o.nrbB, c->nsm, &P, 0, c->d_flags + 1, st));
    }
  return OZ_OK;
}

// --------------------------------------------------------------------------------------------
// H_eff handle
// --------------------------------------------------------------------------------------------

namespace {
__global__ void scatter_rows_kernel(const double* __restrict__ T, const long long* __restrict__ rowinfo,
                                    double* __restrict__ stage) {
  // one block per row: rowinfo[2r] = source offset in T, rowinfo[2r+1] = destination offset | (ncols << 40)
  long long r = blockIdx.x;
  long long src = rowinfo[2 * r], d = rowinfo[2 * r + 1];
  int nc = (int)(d >> 40);
  long long dst = d & ((1ll << 40) - 1);
  for (int j = threadIdx.x; j < nc; j += blockDim.x) stage[dst + j] = T[src + j];
}
}  // namespace

int oz_heff_s::enqueue(cudaStream_t st, bool capturing) {
  const unsigned evf = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (mode == OZ_MODE_EAGER) {
    // events are recorded as graph nodes when captured (external record), plain records otherwise
    OZ_CU(cudaEventRecordWithFlags(ev[0], st, evf));
    if (bytes_mB1) OZ_CU(cudaMemsetAsync(mB1, 0, bytes_mB1, st));
    if (bytes_mA2) OZ_CU(cudaMemsetAsync(mA2, 0, bytes_mA2, st));
    OZ_CU(oz::launch_rowmax(dSegPsi, nullptr, nsegPsi, uPsiM, ctx->d_flags, st, dCtaPsiM));
    OZ_CU(oz::launch_digits(dSegPsi, nullptr, nsegPsi, uPsiD, S, st, dCtaPsiD));
    OZ_CU(cudaEventRecordWithFlags(ev[1], st, evf));
    OZ_CU(oz::launch_gemm(dP1, dT1, nt1, units, nullptr, s, ctx->d_flags + 1, st, dF1, pair, ho1));
    OZ_CU(cudaEventRecordWithFlags(ev[2], st, evf));
    OZ_CU(oz::launch_digits(dSegA2, nullptr, nsegA2, uA2D, S, st, dCtaA2D));
    if (zero_y) OZ_CU(cudaMemsetAsync(dY, 0, (size_t)dim * 8, st));
    OZ_CU(cudaEventRecordWithFlags(ev[3], st, evf));
    OZ_CU(oz::launch_gemm(dP2, dT2, nt2, units, nullptr, s, ctx->d_flags + 1, st, dF2, pair, ho2));
    OZ_CU(cudaEventRecordWithFlags(ev[4], st, evf));
    return OZ_OK;
  }
  // native FP64: one DGEMM per source sector, scatter into the concatenated layout, one per target
  cublasSetStream(ctx->cublas, st);
  const double one = 1.0, zero = 0.0;
  for (const auto& g : nat1) {
    // T (rows x n[q]) = A1 (rows x m[q]) psi[q] (m[q] x n[q]), row-major
    int nq = n[g.q];
    if (cublasDgemm(ctx->cublas, CUBLAS_OP_N, CUBLAS_OP_N, nq, g.rows, g.kdim, &one, dPsi + psioff[g.q], nq,
                    nA1 + g.a1off, g.kdim, &zero, nT + g.toff, nq) != CUBLAS_STATUS_SUCCESS)
      return fail(OZ_ECUDA, "cublasDgemm (stage 1)");
  }
  if (nTrows > 0) {
    scatter_rows_kernel<<<(unsigned)nTrows, 128, 0, st>>>(nT, dScatter, dStage);
    OZ_CU(cudaGetLastError());
  }
  if (zero_y) OZ_CU(cudaMemsetAsync(dY, 0, (size_t)dim * 8, st));
  for (const auto& g : nat2) {
    // Y[q] (m x n') = Stage (m x ld2) B2T^T, B2T: n' x ld2 row-major
    int mq = m[g.q], nq = n[g.q];
    if (cublasDgemm(ctx->cublas, CUBLAS_OP_T, CUBLAS_OP_N, nq, mq, g.ld2, &one, nB2 + g.b2off, g.ld2,
                    dStage + g.stoff, g.ld2, &zero, dY + psioff[g.q], nq) != CUBLAS_STATUS_SUCCESS)
      return fail(OZ_ECUDA, "cublasDgemm (stage 2)");
  }
  return OZ_OK;
}

namespace {
// Tensor-core flops of one emulated product (padded tiles included) at the given levels.
long long carrier_flops_of(int nsec, const int* m, const int* n, const std::vector<int>& rows1,
                           const std::vector<int>& nkb1, const std::vector<int>& nkb2,
                           const std::vector<std::vector<int>>& bysrc, const std::vector<std::vector<int>>& bydst,
                           const std::vector<int>& lev1, const std::vector<int>& lev2, const std::vector<char>& swap2,
                           int TM) {
  long long f = 0;
  for (int q = 0; q < nsec; ++q) {
    const long long P1 = (long long)lev1[q] * (lev1[q] + 1) / 2, P2 = (long long)lev2[q] * (lev2[q] + 1) / 2;
    if (!bysrc[q].empty())
      f += P1 * 2 * (cdiv(rows1[q], TM) * TM) * (cdiv(n[q], oz::BN) * oz::BN) *
           ((long long)nkb1[q] * oz::KB);
    if (!bydst[q].empty()) {
      const long long r2 = swap2[q] ? n[q] : m[q], c2 = swap2[q] ? m[q] : n[q];
      f += P2 * 2 * (cdiv(r2, TM) * TM) * (cdiv(c2, oz::BN) * oz::BN) * ((long long)nkb2[q] * oz::KB);
    }
  }
  return f;
}

__global__ void copy_block_kernel(const double* __restrict__ src, int rows, int cols, long long lds, double scale,
                                  double* __restrict__ dst, long long ldd) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)rows * cols) return;
  int i = (int)(idx / cols), j = (int)(idx % cols);
  double v = src[(long long)i * lds + j];
  dst[(long long)i * ldd + j] = scale != 1.0 ? __dmul_rn(v, scale) : v;
}
}  // namespace

namespace {
// Native path: copy every L block into the stacked stage-1 A operand and every c*R block into the
// stacked stage-2 B^T operand (the handle's layout; asynchronous on the legacy stream).
void native_copy_ops(const oz_heff_s* h, const oz_task* tasks) {
  for (int t = 0; t < h->ntask; ++t) {
    const oz_task& tk = tasks[t];
    const int q = tk.src, d = tk.dst;
    long long rows = h->m[d], cols = h->m[q];
    copy_block_kernel<<<(unsigned)cdiv(rows * cols, 256), 256>>>(tk.d_L, (int)rows, (int)cols, cols, 1.0,
                                                                h->nA1 + h->a1o[q] + h->rowin1[t] * h->m[q], h->m[q]);
    rows = h->n[d];
    cols = h->n[q];
    copy_block_kernel<<<(unsigned)cdiv(rows * cols, 256), 256>>>(tk.d_R, (int)rows, (int)cols, cols, tk.coef,
                                                                h->nB2 + h->b2o[d] + h->offk[t], h->ld2[d]);
  }
}

// Emulated path: slice every L block into the stacked stage-1 A planes and every c*R block into the
// stacked stage-2 B^T planes (row maxima, shared exponents, S digits), synchronously.
int slice_ops(oz_heff_s* h, const oz_task* tasks) {
  const int S = h->S;
  const std::vector<int>& m = h->m;
  const std::vector<int>& n = h->n;
  std::vector<SliceSeg> lops, rops;
  lops.reserve((size_t)h->ntask);
  rops.reserve((size_t)h->ntask);
  for (int q = 0; q < h->nsec; ++q)
    for (int t : h->bysrc[q]) {
      const oz_task& tk = tasks[t];
      SliceSeg g{};
      g.src = tk.d_L; g.ld = m[q]; g.rows = m[tk.dst]; g.cols = m[q]; g.prows = g.rows; g.pcols = g.cols;
      g.r0 = (int)h->rowin1[t]; g.k0 = 0; g.trans = 0; g.S = S; g.scale = 1.0;
      g.dst = h->dA1 + h->A1off[q]; g.TR = oz::TILE_M; g.nkb = h->nkb1[q];
      g.rowmax = h->mA1 + h->A1row[q]; g.rowexp = h->eA1 + h->A1row[q];
      lops.push_back(g);
    }
  for (int q = 0; q < h->nsec; ++q)
    for (int t : h->bydst[q]) {
      const oz_task& tk = tasks[t];
      SliceSeg g{};
      g.src = tk.d_R; g.ld = n[tk.src]; g.rows = n[q]; g.cols = n[tk.src]; g.prows = g.rows; g.pcols = g.cols;
      g.r0 = 0; g.k0 = (int)h->offk[t]; g.trans = 0; g.S = S; g.scale = tk.coef;
      g.dst = h->dB2 + h->B2off[q]; g.TR = h->swap2[q] ? oz::TILE_M : oz::BN; g.nkb = h->nkb2[q];
      g.half_major = h->pair && !h->swap2[q] ? 1 : 0;
      g.rowmax = h->mB2 + h->B2row[q]; g.rowexp = h->eB2 + h->B2row[q];
      rops.push_back(g);
    }
  // The c*R segments take one FP64 multiply per element, which the FP64 pipe executes far below the
  // memory rate; the L segments are pure streaming.  Merging the two lists by element count keeps
  // both kinds in every wave of CTAs, so the multiplies overlap the L segments' memory traffic.
  std::vector<SliceSeg> ops;
  ops.reserve(lops.size() + rops.size());
  {
    size_t il = 0, ir = 0;
    long long el = 0, er = 0;
    while (il < lops.size() || ir < rops.size()) {
      const bool takel = ir == rops.size() || (il < lops.size() && el <= er);
      SliceSeg& g = takel ? lops[il++] : rops[ir++];
      (takel ? el : er) += (long long)g.rows * g.cols;
      ops.push_back(g);
    }
  }
  long long um = 0, ud = 0;
  for (SliceSeg& g : ops) {
    g.unit0 = ud;
    g.unit0m = um;
    ud += oz::digit_units(g.prows, g.pcols);
    um += oz::rowmax_units(g.rows, g.cols, g.trans);
  }
  if (ops.empty()) return OZ_OK;
  oz_ctx* c = h->ctx;
  OZ_CU(cudaMemset(h->mA1, 0, (size_t)h->A1row[h->nsec] * 8));
  OZ_CU(cudaMemset(h->mB2, 0, (size_t)h->B2row[h->nsec] * 8));
  SliceSeg* dops;
  OZ_CU(cudaMalloc(&dops, ops.size() * sizeof(SliceSeg)));
  cudaMemcpy(dops, ops.data(), ops.size() * sizeof(SliceSeg), cudaMemcpyHostToDevice);
  const std::vector<int> tm = oz::rowmax_cta_table(ops, um), td = oz::digits_cta_table(ops, ud);
  int *dtm = nullptr, *dtd = nullptr;
  cudaError_t ea = cudaMalloc(&dtm, tm.size() * sizeof(int));
  if (ea == cudaSuccess) ea = cudaMalloc(&dtd, td.size() * sizeof(int));
  if (ea != cudaSuccess) {
    cudaFree(dops);
    cudaFree(dtm);
    return oz::cuda_fail(ea, "operator slicing tables");
  }
  cudaMemcpy(dtm, tm.data(), tm.size() * sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(dtd, td.data(), td.size() * sizeof(int), cudaMemcpyHostToDevice);
  // algorithmic bytes: the rowmax pass reads every operator element once; the digit pass reads it
  // again and writes S FP16 digits per element of the 8 x 8-padded segment
  long long brm = 0, bdg = 0;
  for (const SliceSeg& g : ops) {
    brm += 8ll * g.rows * g.cols;
    bdg += 8ll * g.rows * g.cols + 2ll * S * ((g.prows + 7) / 8 * 8) * ((g.pcols + 7) / 8 * 8);
  }
  cudaEvent_t t0 = nullptr, t1 = nullptr, t2 = nullptr;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  cudaEventCreate(&t2);
  cudaEventRecord(t0, 0);
  cudaError_t e1 = oz::launch_rowmax(dops, nullptr, (int)ops.size(), um, c->d_flags, 0, dtm);
  cudaEventRecord(t1, 0);
  cudaError_t e2 = oz::launch_digits(dops, nullptr, (int)ops.size(), ud, S, 0, dtd);
  cudaEventRecord(t2, 0);
  cudaError_t e3 = cudaDeviceSynchronize();
  cudaFree(dops);
  cudaFree(dtm);
  cudaFree(dtd);
  h->ops_ms[0] = h->ops_ms[1] = 0.f;
  if (e3 == cudaSuccess) {
    cudaEventElapsedTime(&h->ops_ms[0], t0, t1);
    cudaEventElapsedTime(&h->ops_ms[1], t1, t2);
  }
  h->ops_bytes[0] = brm;
  h->ops_bytes[1] = bdg;
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  cudaEventDestroy(t2);
  if (e1 != cudaSuccess) return oz::cuda_fail(e1, "operator rowmax");
  if (e2 != cudaSuccess) return oz::cuda_fail(e2, "operator digits");
  if (e3 != cudaSuccess) return oz::cuda_fail(e3, "operator slicing");
  int f[4];
  cudaMemcpy(f, c->d_flags, 16, cudaMemcpyDeviceToHost);
  if (f[0]) {
    cudaMemset(c->d_flags, 0, 16);
    return fail(OZ_ENONFINITE, "an operator block held NaN or Inf");
  }
  return OZ_OK;
}
}  // namespace

extern "C" int oz_heff_create(oz_ctx* c, int nsec, const int* m, const int* n, int ntask, const oz_task* tasks,
                              const oz_prec* prec, oz_heff** out) {
  if (!out) return fail(OZ_EINVAL, "out is null");
  *out = nullptr;
  if (!c) return fail(OZ_EINVAL, "ctx is null");
  int S, s, mode;
  if (int rc = check_prec(prec, &S, &s, &mode)) return rc;
  if (nsec <= 0 || ntask < 0 || !m || !n || (ntask > 0 && !tasks)) return fail(OZ_EINVAL, "bad structure");
  for (int q = 0; q < nsec; ++q)
    if (m[q] <= 0 || n[q] <= 0) return fail(OZ_EINVAL, "sector dims must be positive");
  for (int t = 0; t < ntask; ++t) {
    if (tasks[t].src < 0 || tasks[t].src >= nsec || tasks[t].dst < 0 || tasks[t].dst >= nsec)
      return fail(OZ_EINVAL, "task sector out of range");
    if (!tasks[t].d_L || !tasks[t].d_R) return fail(OZ_EINVAL, "task block pointer is null");
  }
  if (prec->tile < OZ_TILE_AUTO || prec->tile > OZ_TILE_PAIR) return fail(OZ_EINVAL, "unknown tile choice");
  OZ_CU(cudaSetDevice(c->device));
  // products on CTA pairs on request (emulated handles only); OZ_TILE_AUTO takes one CTA per tile,
  // which measured faster on GB300 for both stages of the 300-block workload
  int pair_units = 0;
  if (mode == OZ_MODE_EAGER && prec->tile == OZ_TILE_PAIR) pair_units = oz::gemm_pair_units(c->nsm);
  if (prec->tile == OZ_TILE_PAIR && pair_units <= 0) return fail(OZ_EINVAL, "this device runs no CTA pairs");
  oz_heff* h = new oz_heff_s();
  h->ctx = c;
  h->pair = pair_units > 0;
  h->units = h->pair ? pair_units : c->nsm;
  h->nsec = nsec;
  h->ntask = ntask;
  h->S = S;
  h->s = s;
  h->mode = mode;
  h->m.assign(m, m + nsec);
  h->n.assign(n, n + nsec);
  h->lev1.assign(nsec, s);
  h->lev2.assign(nsec, s);
  h->psioff.assign(nsec + 1, 0);
  for (int q = 0; q < nsec; ++q) h->psioff[q + 1] = h->psioff[q] + (long long)m[q] * n[q];
  h->dim = h->psioff[nsec];
  auto bail = [&](int rc) {
    oz_heff_destroy(h);
    return rc;
  };
  // longest reduction of one emulated product at this level (native products: the common limit)
  const long long kmax = mode == OZ_MODE_EAGER ? oz::max_k_of_level(s) : oz::MAX_K;
  if (int rc = h->alloc(&h->dDiag, (size_t)h->dim * 8)) return bail(rc);
  if (int rc = oz::build_heff_diag(nsec, m, n, h->psioff.data(), ntask, tasks, h->dDiag)) return bail(rc);

  std::vector<std::vector<int>> bysrc(nsec), bydst(nsec);
  for (int t = 0; t < ntask; ++t) {
    bysrc[tasks[t].src].push_back(t);
    bydst[tasks[t].dst].push_back(t);
    const long long mp = m[tasks[t].dst], mm = m[tasks[t].src], nn = n[tasks[t].src], nq = n[tasks[t].dst];
    h->flops += 2 * (mp * mm * nn + mp * nn * nq);
  }
  for (int q = 0; q < nsec; ++q)
    if (bydst[q].empty()) h->zero_y = true;

  // ---- layout of stage 1 (per source sector) and stage 2 (per target sector)
  std::vector<int> rows1(nsec, 0), nkb1(nsec), nkb2(nsec), ld2(nsec);
  std::vector<long long> offk(ntask, 0), rowin1(ntask, 0);
  for (int q = 0; q < nsec; ++q) {
    for (int t : bysrc[q]) {
      rowin1[t] = rows1[q];
      rows1[q] += m[tasks[t].dst];
    }
    if (m[q] > kmax) return bail(fail(OZ_EINVAL, "a sector dimension exceeds the level-9 reduction limit (130048)"));
    nkb1[q] = (int)cdiv(m[q], oz::KB);
    long long k2 = 0;
    for (int t : bydst[q]) {
      offk[t] = k2;
      k2 += cdiv(n[tasks[t].src], 8) * 8;
    }
    if (k2 > kmax)
      return bail(fail(OZ_EINVAL, kmax < oz::MAX_K
                                      ? "a target sector's concatenated reduction exceeds 130048, the level-9 limit"
                                      : "a target sector's concatenated reduction exceeds 1048576"));
    nkb2[q] = (int)cdiv(std::max(k2, 1ll), oz::KB);
    ld2[q] = nkb2[q] * oz::KB;
  }
  std::vector<long long> stoff(nsec + 1, 0);
  for (int q = 0; q < nsec; ++q) stoff[q + 1] = stoff[q] + (long long)m[q] * ld2[q];
  const long long A1tile = (long long)oz::TILE_M * oz::KB, Btile = (long long)oz::BN * oz::KB;
  std::vector<long long> A1off(nsec + 1, 0), B1off(nsec + 1, 0), A2off(nsec + 1, 0), B2off(nsec + 1, 0);
  std::vector<long long> A1row(nsec + 1, 0), B1row(nsec + 1, 0), A2row(nsec + 1, 0), B2row(nsec + 1, 0);
  // rows of a tile's M side: 128, or 256 on a CTA pair (the orientation of stage 2 weighs the
  // padding of that tile)
  const int TMt = h->pair ? 2 * oz::TILE_M : oz::TILE_M;
  auto a_tiles = [&](long long rows) { return cdiv(rows, oz::TILE_M); };
  h->swap2.assign(nsec, 0);
  for (int q = 0; q < nsec; ++q)
    h->swap2[q] = cdiv(n[q], TMt) * TMt * cdiv(m[q], oz::BN) * oz::BN < cdiv(m[q], TMt) * TMt * cdiv(n[q], oz::BN) * oz::BN;
  for (int q = 0; q < nsec; ++q) {
    long long nrbA1 = a_tiles(rows1[q]), nrbB1 = cdiv(n[q], oz::BN);
    // stage 2: T (m[q] rows) and the (cR) stack (n[q] rows) take the 128- and 64-row sides of the
    // tile, or the other way round when the handle computes this sector transposed
    const long long trA2 = h->swap2[q] ? oz::BN : oz::TILE_M, trB2 = h->swap2[q] ? oz::TILE_M : oz::BN;
    long long nrbA2 = h->swap2[q] ? cdiv(m[q], trA2) : a_tiles(m[q]);
    long long nrbB2 = h->swap2[q] ? a_tiles(n[q]) : cdiv(n[q], trB2);
    A1off[q + 1] = A1off[q] + nrbA1 * nkb1[q] * S * A1tile;
    B1off[q + 1] = B1off[q] + nrbB1 * nkb1[q] * S * Btile;
    A2off[q + 1] = A2off[q] + nrbA2 * nkb2[q] * S * trA2 * oz::KB;
    B2off[q + 1] = B2off[q] + nrbB2 * nkb2[q] * S * trB2 * oz::KB;
    A1row[q + 1] = A1row[q] + nrbA1 * oz::TILE_M;
    B1row[q + 1] = B1row[q] + nrbB1 * oz::BN;
    A2row[q + 1] = A2row[q] + nrbA2 * trA2;
    B2row[q + 1] = B2row[q] + nrbB2 * trB2;
  }
  h->carrier_flops = carrier_flops_of(nsec, m, n, rows1, nkb1, nkb2, bysrc, bydst, h->lev1, h->lev2, h->swap2, TMt);

  int rc;
  h->bytes_scratch = (long long)stoff[nsec] * 8 + 2 * h->dim * 8;

  h->bysrc = std::move(bysrc);
  h->bydst = std::move(bydst);
  h->rows1 = rows1; h->nkb1 = nkb1; h->nkb2 = nkb2; h->ld2 = ld2;
  h->offk = offk; h->rowin1 = rowin1; h->stoff = stoff;
  h->A1off = A1off; h->B1off = B1off; h->A2off = A2off; h->B2off = B2off;
  h->A1row = A1row; h->B1row = B1row; h->A2row = A2row; h->B2row = B2row;
  h->tsrc.resize(ntask); h->tdst.resize(ntask);
  for (int t = 0; t < ntask; ++t) { h->tsrc[t] = tasks[t].src; h->tdst[t] = tasks[t].dst; }

  if (mode == OZ_MODE_NATIVE) {
    if ((rc = h->alloc(&h->dPsi, (size_t)h->dim * 8))) return bail(rc);
    if ((rc = h->alloc(&h->dY, (size_t)h->dim * 8))) return bail(rc);
    if ((rc = h->alloc(&h->dStage, (size_t)stoff[nsec] * 8))) return bail(rc);
    OZ_CU(cudaMemset(h->dStage, 0, (size_t)stoff[nsec] * 8));
    // stacked FP64 copies: A1 (per source: rows1 x m[q]) and B2T (per target: n[q] x ld2, zero padded)
    std::vector<long long>& a1o = h->a1o;
    std::vector<long long>& b2o = h->b2o;
    std::vector<long long> to(nsec + 1, 0);
    a1o.assign(nsec + 1, 0);
    b2o.assign(nsec + 1, 0);
    for (int q = 0; q < nsec; ++q) {
      a1o[q + 1] = a1o[q] + (long long)rows1[q] * m[q];
      b2o[q + 1] = b2o[q] + (long long)n[q] * ld2[q];
      to[q + 1] = to[q] + (long long)rows1[q] * n[q];
    }
    if ((rc = h->alloc(&h->nA1, (size_t)a1o[nsec] * 8))) return bail(rc);
    if ((rc = h->alloc(&h->nB2, (size_t)b2o[nsec] * 8))) return bail(rc);
    if ((rc = h->alloc(&h->nT, (size_t)to[nsec] * 8))) return bail(rc);
    OZ_CU(cudaMemset(h->nB2, 0, (size_t)b2o[nsec] * 8));
    h->bytes_ops = (a1o[nsec] + b2o[nsec]) * 8;
    h->bytes_scratch += to[nsec] * 8;
    native_copy_ops(h, tasks);
    OZ_CU(cudaGetLastError());
    std::vector<long long> sc;
    sc.reserve(2 * (size_t)to[nsec]);
    for (int q = 0; q < nsec; ++q) {
      if (h->bysrc[q].empty()) continue;
      h->nat1.push_back({a1o[q], to[q], rows1[q], m[q], q});
      for (int t : h->bysrc[q]) {
        int d = tasks[t].dst;
        for (int i = 0; i < m[d]; ++i) {
          long long srcoff = to[q] + (rowin1[t] + i) * n[q];
          long long dstoff = stoff[d] + (long long)i * ld2[d] + offk[t];
          sc.push_back(srcoff);
          sc.push_back(dstoff | ((long long)n[q] << 40));
        }
      }
    }
    h->nTrows = (long long)sc.size() / 2;
    if ((rc = h->alloc(&h->dScatter, sc.size() * 8))) return bail(rc);
    OZ_CU(cudaMemcpy(h->dScatter, sc.data(), sc.size() * 8, cudaMemcpyHostToDevice));
    for (int q = 0; q < nsec; ++q)
      if (!h->bydst[q].empty()) h->nat2.push_back({stoff[q], b2o[q], q, ld2[q]});
    OZ_CU(cudaDeviceSynchronize());
  } else {
    // ---- device buffers of the emulated path
    size_t bA1 = A1off[nsec] * 2, bB1 = B1off[nsec] * 2, bA2 = A2off[nsec] * 2, bB2 = B2off[nsec] * 2;
    if ((rc = h->alloc(&h->dA1, bA1))) return bail(rc);
    if ((rc = h->alloc(&h->dB2, bB2))) return bail(rc);
    OZ_CU(cudaMemset(h->dA1, 0, bA1));
    OZ_CU(cudaMemset(h->dB2, 0, bB2));
    h->bytes_ops = (long long)(bA1 + bB2);
    h->bytes_scratch += (long long)(bB1 + bA2);
    if ((rc = h->alloc(&h->eA1, A1row[nsec] * 4))) return bail(rc);
    if ((rc = h->alloc(&h->eB2, B2row[nsec] * 4))) return bail(rc);
    if ((rc = h->alloc(&h->mA1, A1row[nsec] * 8))) return bail(rc);
    if ((rc = h->alloc(&h->mB2, B2row[nsec] * 8))) return bail(rc);
    // ---- operator slicing (once): L blocks into A1, coef*R blocks into B2T
    if ((rc = slice_ops(h, tasks))) return bail(rc);
  }
  for (auto& e : h->ev) OZ_CU(cudaEventCreate(&e));
  if (mode == OZ_MODE_NATIVE) h->prepared = true;
  else if (int rc2 = oz::heff_operator_hist(h, tasks)) return bail(rc2);
  *out = h;
  return OZ_OK;
}


extern "C" int oz_heff_update_ops(oz_heff* h, int ntask, const oz_task* tasks) {
  if (!h) return fail(OZ_EINVAL, "handle is null");
  if (ntask != h->ntask || (ntask > 0 && !tasks)) return fail(OZ_EINVAL, "task count differs from the handle's");
  for (int t = 0; t < ntask; ++t) {
    if (tasks[t].src != h->tsrc[t] || tasks[t].dst != h->tdst[t])
      return fail(OZ_EINVAL, "task sectors differ from the handle's");
    if (!tasks[t].d_L || !tasks[t].d_R) return fail(OZ_EINVAL, "task block pointer is null");
  }
  OZ_CU(cudaSetDevice(h->ctx->device));
  OZ_CU(cudaDeviceSynchronize());  // products in flight still read the old operators
  if (int rc = oz::build_heff_diag(h->nsec, h->m.data(), h->n.data(), h->psioff.data(), ntask, tasks, h->dDiag))
    return rc;
  if (h->mode == OZ_MODE_NATIVE) {
    native_copy_ops(h, tasks);
    OZ_CU(cudaGetLastError());
    OZ_CU(cudaDeviceSynchronize());
    return OZ_OK;
  }
  if (int rc = slice_ops(h, tasks)) return rc;
  return oz::heff_operator_hist(h, tasks);
}

// Per-product buffers, tables, slicing segments and the CUDA graph of the emulated path.  Done on
// the first product so that the caller can free its FP64 operator blocks after oz_heff_create.
int oz_heff_s::prepare() {
  if (prepared) return OZ_OK;
  int rc;
  const int nsec = this->nsec;
  oz_ctx* c = ctx;
  const std::vector<int>& m = this->m;
  const std::vector<int>& n = this->n;
  const int S = this->S, s = this->s, mode = this->mode;
  (void)mode;
  int* eA1 = this->eA1;
  int* eB2 = this->eB2;
  (void)c;
  if ((rc = alloc(&dPsi, (size_t)dim * 8))) return rc;
  if ((rc = alloc(&dY, (size_t)dim * 8))) return rc;
  if ((rc = alloc(&dStage, (size_t)stoff[nsec] * 8))) return rc;
  OZ_CU(cudaMemset(dStage, 0, (size_t)stoff[nsec] * 8));
  size_t bB1 = B1off[nsec] * 2, bA2 = A2off[nsec] * 2;
  if ((rc = alloc(&dB1, bB1))) return rc;
  if ((rc = alloc(&dA2, bA2))) return rc;
  OZ_CU(cudaMemset(dB1, 0, bB1));
  OZ_CU(cudaMemset(dA2, 0, bA2));
  if ((rc = alloc(&eB1, B1row[nsec] * 4))) return rc;
  if ((rc = alloc(&eA2, A2row[nsec] * 4))) return rc;
  bytes_mB1 = B1row[nsec] * 8;
  bytes_mA2 = A2row[nsec] * 8;
  if ((rc = alloc(&mB1, bytes_mB1))) return rc;
  if ((rc = alloc(&mA2, bytes_mA2))) return rc;
  {
    // ---- row tables of stage 1 (stacked L rows -> concatenated T layout of stage 2)
    std::vector<long long> rowdst(A1row[nsec], 0);
    std::vector<int> rowslot(A1row[nsec], 0);
    for (int q = 0; q < nsec; ++q)
      for (int t : bysrc[q]) {
        int d = tdst[t];
        for (int i = 0; i < m[d]; ++i) {
          long long r = A1row[q] + rowin1[t] + i;
          rowdst[r] = stoff[d] + (long long)i * ld2[d] + offk[t];
          rowslot[r] = (int)(A2row[d] + i);
        }
      }
    long long* dRowdst;
    int* dRowslot;
    if ((rc = this->alloc(&dRowdst, rowdst.size() * 8))) return rc;
    if ((rc = this->alloc(&dRowslot, rowslot.size() * 4))) return rc;
    OZ_CU(cudaMemcpy(dRowdst, rowdst.data(), rowdst.size() * 8, cudaMemcpyHostToDevice));
    OZ_CU(cudaMemcpy(dRowslot, rowslot.data(), rowslot.size() * 4, cudaMemcpyHostToDevice));

    // ---- problems and tiles (larger k first; n-blocks of one m-block adjacent for L2 reuse)
    std::vector<GemmProblem> p1, p2;
    std::vector<int> ord1, ord2;
    for (int q = 0; q < nsec; ++q) {
      if (!bysrc[q].empty()) {
        GemmProblem P{};
        P.A = this->dA1 + A1off[q]; P.B = this->dB1 + B1off[q]; P.ea = eA1 + A1row[q]; P.eb = this->eB1 + B1row[q];
        P.M = rows1[q]; P.N = n[q]; P.nkb = nkb1[q]; P.SA = S; P.SB = S; P.s = s;
        P.mode = oz::OUT_ROWTABLE; P.C = this->dStage; P.ldc = 0;
        P.rowdst = dRowdst + A1row[q]; P.rowslot = dRowslot + A1row[q]; P.rowmax = this->mA2;
        P.alpha = 1.0; P.beta = 0.0;
        P.s = lev1[q];
        p1.push_back(P);
        this->p1sec.push_back(q);
      }
      if (!bydst[q].empty()) {
        GemmProblem P{};
        if (!swap2[q]) {
          P.A = this->dA2 + A2off[q]; P.B = this->dB2 + B2off[q]; P.ea = this->eA2 + A2row[q]; P.eb = eB2 + B2row[q];
          P.M = m[q]; P.N = n[q]; P.mode = oz::OUT_DENSE;
        } else {  // Y^T = (cR stack) T^T: identical elements (the rounding of each is unchanged)
          P.A = this->dB2 + B2off[q]; P.B = this->dA2 + A2off[q]; P.ea = eB2 + B2row[q]; P.eb = this->eA2 + A2row[q];
          P.M = n[q]; P.N = m[q]; P.mode = oz::OUT_DENSE_T;
        }
        P.nkb = nkb2[q]; P.SA = S; P.SB = S; P.s = s;
        P.C = this->dY + this->psioff[q]; P.ldc = n[q];
        P.alpha = 1.0; P.beta = 0.0;
        P.s = lev2[q];
        p2.push_back(P);
        this->p2sec.push_back(q);
      }
    }
    const int TMt = this->pair ? 2 * oz::TILE_M : oz::TILE_M;  // tile rows: one CTA, or a CTA pair
    auto make_tiles = [TMt](const std::vector<GemmProblem>& ps) {
      std::vector<int> ord(ps.size());
      for (size_t i = 0; i < ps.size(); ++i) ord[i] = (int)i;
      std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return ps[a].nkb > ps[b].nkb; });
      std::vector<GemmTile> tl;
      for (int pi : ord) {
        int nrb = (int)cdiv(ps[pi].M, TMt), nnb = (int)cdiv(ps[pi].N, oz::BN);
        for (int mb = 0; mb < nrb; ++mb)
          for (int nb = 0; nb < nnb; ++nb) tl.push_back({pi, mb, nb, 0});
      }
      return tl;
    };
    this->hp1 = p1;
    this->hp2 = p2;
    std::vector<GemmTile> t1 = make_tiles(p1), t2 = make_tiles(p2);
    this->nt1 = (int)t1.size();
    this->nt2 = (int)t2.size();
    // epilogue layout per stage from the average tile length (CTA pairs: the 16-owner layout)
    auto kb_per_tile = [](const std::vector<GemmProblem>& ps, const std::vector<GemmTile>& tl) {
      double kb = 0.0;
      for (const GemmTile& t : tl) kb += ps[t.prob].nkb;
      return tl.empty() ? 0.0 : kb / (double)tl.size();
    };
    this->ho1 = this->ho1_auto = !this->pair && oz::gemm_handover_for(kb_per_tile(p1, t1));
    this->ho2 = this->ho2_auto = !this->pair && oz::gemm_handover_for(kb_per_tile(p2, t2));
    this->bt1 = t1;
    this->bt2 = t2;
    if ((rc = this->alloc(&this->dF1, (size_t)(c->nsm + 1) * 4))) return rc;
    if ((rc = this->alloc(&this->dF2, (size_t)(c->nsm + 1) * 4))) return rc;
    if ((rc = this->alloc(&this->dP1, std::max<size_t>(1, p1.size()) * sizeof(GemmProblem)))) return rc;
    if ((rc = this->alloc(&this->dP2, std::max<size_t>(1, p2.size()) * sizeof(GemmProblem)))) return rc;
    if ((rc = this->alloc(&this->dT1, std::max<size_t>(1, t1.size()) * sizeof(GemmTile)))) return rc;
    if ((rc = this->alloc(&this->dT2, std::max<size_t>(1, t2.size()) * sizeof(GemmTile)))) return rc;
    if (!p1.empty()) OZ_CU(cudaMemcpy(this->dP1, p1.data(), p1.size() * sizeof(GemmProblem), cudaMemcpyHostToDevice));
    if (!p2.empty()) OZ_CU(cudaMemcpy(this->dP2, p2.data(), p2.size() * sizeof(GemmProblem), cudaMemcpyHostToDevice));
    if ((rc = this->balance())) return rc;

    // ---- per-product slicing segments: psi (B of stage 1) and the concatenated T (A of stage 2)
    std::vector<SliceSeg> sp, sa;
    long long pm = 0, pd = 0, ad = 0;
    for (int q = 0; q < nsec; ++q) {
      if (bysrc[q].empty()) continue;
      SliceSeg g{};
      g.src = this->dPsi + this->psioff[q]; g.ld = n[q]; g.rows = n[q]; g.cols = m[q]; g.prows = g.rows; g.pcols = g.cols;
      g.r0 = 0; g.k0 = 0; g.trans = 1; g.S = S; g.scale = 1.0;
      g.dst = this->dB1 + B1off[q]; g.TR = oz::BN; g.nkb = nkb1[q]; g.half_major = this->pair ? 1 : 0;
      g.rowmax = this->mB1 + B1row[q]; g.rowexp = this->eB1 + B1row[q];
      g.unit0 = pd; g.unit0m = pm;
      pd += oz::digit_units(g.prows, g.pcols);
      pm += oz::rowmax_units(g.rows, g.cols, g.trans);
      sp.push_back(g);
    }
    for (int q = 0; q < nsec; ++q) {
      if (bydst[q].empty()) continue;
      SliceSeg g{};
      g.src = this->dStage + stoff[q]; g.ld = ld2[q]; g.rows = m[q]; g.cols = ld2[q]; g.prows = g.rows;
      g.pcols = g.cols; g.r0 = 0; g.k0 = 0; g.trans = 0; g.S = S; g.scale = 1.0;
      g.dst = this->dA2 + A2off[q]; g.TR = swap2[q] ? oz::BN : oz::TILE_M; g.nkb = nkb2[q];
      g.half_major = this->pair && swap2[q] ? 1 : 0;
      g.rowmax = this->mA2 + A2row[q]; g.rowexp = this->eA2 + A2row[q];
      g.unit0 = ad; g.unit0m = 0;
      ad += oz::digit_units(g.prows, g.pcols);
      sa.push_back(g);
    }
    this->nsegPsi = (int)sp.size();
    this->nsegA2 = (int)sa.size();
    this->uPsiM = pm;
    this->uPsiD = pd;
    this->uA2D = ad;
    if ((rc = this->alloc(&this->dSegPsi, std::max<size_t>(1, sp.size()) * sizeof(SliceSeg)))) return rc;
    if ((rc = this->alloc(&this->dSegA2, std::max<size_t>(1, sa.size()) * sizeof(SliceSeg)))) return rc;
    if (!sp.empty()) OZ_CU(cudaMemcpy(this->dSegPsi, sp.data(), sp.size() * sizeof(SliceSeg), cudaMemcpyHostToDevice));
    if (!sa.empty()) OZ_CU(cudaMemcpy(this->dSegA2, sa.data(), sa.size() * sizeof(SliceSeg), cudaMemcpyHostToDevice));
    // CTA -> first segment tables of the three per-product slicing launches
    auto upload_table = [&](const std::vector<int>& t, int** dst) -> int {
      if (int r = this->alloc(dst, std::max<size_t>(1, t.size()) * sizeof(int))) return r;
      if (!t.empty()) OZ_CU(cudaMemcpy(*dst, t.data(), t.size() * sizeof(int), cudaMemcpyHostToDevice));
      return OZ_OK;
    };
    if (!sp.empty()) {
      if ((rc = upload_table(oz::rowmax_cta_table(sp, pm), &this->dCtaPsiM))) return rc;
      if ((rc = upload_table(oz::digits_cta_table(sp, pd), &this->dCtaPsiD))) return rc;
    }
    if (!sa.empty() && (rc = upload_table(oz::digits_cta_table(sa, ad), &this->dCtaA2D))) return rc;
  
  }
  // ---- CUDA graph of one product (psi and y are the handle's own buffers)
  OZ_CU(cudaStreamCreateWithFlags(&this->cap, cudaStreamNonBlocking));
  if (mode == OZ_MODE_EAGER && (rc = this->capture())) return rc;
  prepared = true;
  return OZ_OK;
}

// (Re)captures the graph of one product with the current launch configuration.
int oz_heff_s::capture() {
  if (exec) {
    cudaGraphExecDestroy(exec);
    exec = nullptr;
  }
  // warm launch outside capture sets kernel attributes once (on a zero psi: no stale NaN patterns)
  OZ_CU(cudaMemset(this->dPsi, 0, (size_t)this->dim * 8));
  if (int rc = this->enqueue(this->cap)) return rc;
  OZ_CU(cudaStreamSynchronize(this->cap));
  cudaGraph_t g;
  OZ_CU(cudaStreamBeginCapture(this->cap, cudaStreamCaptureModeThreadLocal));
  const int rc = this->enqueue(this->cap, true);
  cudaError_t e = cudaStreamEndCapture(this->cap, &g);
  if (rc) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&this->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  return OZ_OK;
}

extern "C" int oz_heff_set_epilogue(oz_heff* h, int e1, int e2) {
  if (!h) return fail(OZ_EINVAL, "handle is null");
  if (h->mode != OZ_MODE_EAGER) return fail(OZ_EINVAL, "epilogue layouts exist for emulated handles only");
  if (e1 < -1 || e1 > 1 || e2 < -1 || e2 > 1) return fail(OZ_EINVAL, "layouts are -1 (automatic), 0 or 1");
  if (int rc = h->prepare()) return rc;
  if (h->pair && (e1 == 1 || e2 == 1)) return fail(OZ_EINVAL, "CTA-pair handles use layout 0");
  const bool n1 = e1 < 0 ? h->ho1_auto : e1 == 1, n2 = e2 < 0 ? h->ho2_auto : e2 == 1;
  if (n1 == h->ho1 && n2 == h->ho2) return OZ_OK;
  OZ_CU(cudaDeviceSynchronize());
  h->ho1 = n1;
  h->ho2 = n2;
  return h->capture();
}

extern "C" int oz_heff_destroy(oz_heff* h) {
  if (!h) return OZ_OK;
  cudaSetDevice(h->ctx->device);
  cudaDeviceSynchronize();
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->cap) cudaStreamDestroy(h->cap);
  for (auto& e : h->ev)
    if (e) cudaEventDestroy(e);
  for (void* p : h->allocs) cudaFree(p);
  delete h;
  return OZ_OK;
}

extern "C" int heff_apply(oz_heff* h, const double* psi, double* y, oz_stream_t stream) {
  if (!h) return fail(OZ_EINVAL, "handle is null");
  if (!psi || !y) return fail(OZ_EINVAL, "null vector");
  if (psi == y) return fail(OZ_EINVAL, "y must not alias psi");
  cudaStream_t st = (cudaStream_t)stream;
  if (int rc = h->prepare()) return rc;
  OZ_CU(cudaMemcpyAsync(h->dPsi, psi, (size_t)h->dim * 8, cudaMemcpyDeviceToDevice, st));
  if (h->exec) {
    OZ_CU(cudaGraphLaunch(h->exec, st));
  } else if (int rc = h->enqueue(st)) {
    return rc;
  }
  OZ_CU(cudaMemcpyAsync(y, h->dY, (size_t)h->dim * 8, cudaMemcpyDeviceToDevice, st));
  return OZ_OK;
}

extern "C" int heff_apply_host(oz_heff* h, const double* psi_host, double* y_host, oz_stream_t stream) {
  if (!h) return fail(OZ_EINVAL, "handle is null");
  if (!psi_host || !y_host) return fail(OZ_EINVAL, "null vector");
  cudaStream_t st = (cudaStream_t)stream;
  if (int rc = h->prepare()) return rc;
  OZ_CU(cudaMemcpyAsync(h->dPsi, psi_host, (size_t)h->dim * 8, cudaMemcpyHostToDevice, st));
  if (h->exec) {
    OZ_CU(cudaGraphLaunch(h->exec, st));
  } else if (int rc = h->enqueue(st)) {
    return rc;
  }
  OZ_CU(cudaMemcpyAsync(y_host, h->dY, (size_t)h->dim * 8, cudaMemcpyDeviceToHost, st));
  return OZ_OK;
}

extern "C" int oz_heff_ops_times(const oz_heff* h, float* ms2, long long* bytes2) {
  if (!h) return fail(OZ_EINVAL, "null handle");
  if (ms2) {
    ms2[0] = h->ops_ms[0];
    ms2[1] = h->ops_ms[1];
  }
  if (bytes2) {
    bytes2[0] = h->ops_bytes[0];
    bytes2[1] = h->ops_bytes[1];
  }
  return OZ_OK;
}

extern "C" int oz_heff_stage_times(oz_heff* h, float* ms) {
  if (!h || !ms) return fail(OZ_EINVAL, "null argument");
  if (h->mode != OZ_MODE_EAGER) return fail(OZ_EINVAL, "stage times exist for the emulated path only");
  OZ_CU(cudaEventSynchronize(h->ev[4]));
  for (int i = 0; i < 4; ++i) OZ_CU(cudaEventElapsedTime(&ms[i], h->ev[i], h->ev[i + 1]));
  return OZ_OK;
}

extern "C" int oz_heff_info_get(const oz_heff* h, oz_heff_info* o) {
  if (!h || !o) return fail(OZ_EINVAL, "null argument");
  o->dim = h->dim;
  o->flops = h->flops;
  o->carrier_flops = h->carrier_flops;
  o->bytes_ops = h->bytes_ops;
  o->bytes_scratch = h->bytes_scratch;
  o->gemm1_tiles = h->nt1;
  o->gemm2_tiles = h->nt2;
  o->slices = h->S;
  o->level = h->s;
  o->mode = h->mode;
  o->tile = h->pair ? OZ_TILE_PAIR : OZ_TILE_CTA;
  o->units = h->units;
  o->epilogue1 = h->ho1 ? 1 : 0;
  o->epilogue2 = h->ho2 ? 1 : 0;
  return OZ_OK;
}

// ---- library-internal hooks (oz_internal.cuh)
namespace oz {
int api_fail(int code, const std::string& msg) { return fail(code, msg); }
int ctx_device(const oz_ctx* c) { return c->device; }
long long heff_dim(const oz_heff* h) { return h->dim; }
int heff_device(const oz_heff* h) { return h->ctx->device; }
int heff_nsm(const oz_heff* h) { return h->ctx->nsm; }
oz_ctx* heff_ctx(const oz_heff* h) { return h->ctx; }
const double* heff_diag_ptr(const oz_heff* h) { return h->dDiag; }
}  // namespace oz

extern "C" int oz_heff_diag(const oz_heff* h, double* d_diag, oz_stream_t stream) {
  if (!h || !d_diag) return fail(OZ_EINVAL, "null argument");
  OZ_CU(cudaMemcpyAsync(d_diag, h->dDiag, (size_t)h->dim * 8, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return OZ_OK;
}

int oz_heff_s::set_levels(const int* s1, const int* s2) {
  if (mode != OZ_MODE_EAGER) return fail(OZ_EINVAL, "slice levels exist for the emulated path only");
  for (int q = 0; q < nsec; ++q) {
    const int a = s1 ? s1[q] : s, b = s2 ? s2[q] : s;
    if (a < 1 || a > s || b < 1 || b > s)
      return fail(OZ_EINVAL, "per-sector levels must be in 1..the handle's level (" + std::to_string(s) + ")");
  }
  if (int rc = prepare()) return rc;
  for (int q = 0; q < nsec; ++q) {
    lev1[q] = s1 ? s1[q] : s;
    lev2[q] = s2 ? s2[q] : s;
  }
  for (size_t i = 0; i < hp1.size(); ++i) hp1[i].s = lev1[p1sec[i]];
  for (size_t i = 0; i < hp2.size(); ++i) hp2[i].s = lev2[p2sec[i]];
  // the captured graph reads the problem tables from device memory: rewriting them is enough
  OZ_CU(cudaDeviceSynchronize());
  if (!hp1.empty()) OZ_CU(cudaMemcpy(dP1, hp1.data(), hp1.size() * sizeof(GemmProblem), cudaMemcpyHostToDevice));
  if (!hp2.empty()) OZ_CU(cudaMemcpy(dP2, hp2.data(), hp2.size() * sizeof(GemmProblem), cudaMemcpyHostToDevice));
  if (int rc = balance()) return rc;
  carrier_flops = carrier_flops_of(nsec, m.data(), n.data(), rows1, nkb1, nkb2, bysrc, bydst, lev1, lev2, swap2,
                                   pair ? 2 * oz::TILE_M : oz::TILE_M);
  return OZ_OK;
}

extern "C" int oz_heff_set_levels(oz_heff* h, const int* s1, const int* s2) {
  if (!h) return fail(OZ_EINVAL, "handle is null");
  return h->set_levels(s1, s2);
}

extern "C" int oz_heff_get_levels(const oz_heff* h, int* s1, int* s2) {
  if (!h) return fail(OZ_EINVAL, "handle is null");
  for (int q = 0; q < h->nsec; ++q) {
    if (s1) s1[q] = h->lev1[q];
    if (s2) s2[q] = h->lev2[q];
  }
  return OZ_OK;
}

int oz_heff_s::balance() {
  // tiles of each stage onto the persistent CTAs by cost at the current levels (the problem tables
  // on the device already hold those levels); same sizes, so the captured graph stays valid
  std::vector<int> f1, f2;
  ht1 = bt1;
  ht2 = bt2;
  oz::schedule_tiles(hp1, ht1, units, sched1, f1);
  oz::schedule_tiles(hp2, ht2, units, sched2, f2);
  if (!ht1.empty()) OZ_CU(cudaMemcpy(dT1, ht1.data(), ht1.size() * sizeof(GemmTile), cudaMemcpyHostToDevice));
  if (!ht2.empty()) OZ_CU(cudaMemcpy(dT2, ht2.data(), ht2.size() * sizeof(GemmTile), cudaMemcpyHostToDevice));
  OZ_CU(cudaMemcpy(dF1, f1.data(), f1.size() * 4, cudaMemcpyHostToDevice));
  OZ_CU(cudaMemcpy(dF2, f2.data(), f2.size() * 4, cudaMemcpyHostToDevice));
  return OZ_OK;
}

extern "C" int oz_heff_autotune(oz_heff* h, const double* d_psi, int reps, int* sched, float* ms,
                                oz_stream_t stream) {
  if (!h || !d_psi) return fail(OZ_EINVAL, "null argument");
  if (h->mode != OZ_MODE_EAGER) return fail(OZ_EINVAL, "the autotuner schedules emulated handles only");
  if (reps < 1) return fail(OZ_EINVAL, "reps must be positive");
  cudaStream_t st = (cudaStream_t)stream;
  if (int rc = h->prepare()) return rc;
  // every schedule of both stages in turn; each product's stage times come from its events
  OZ_CU(cudaMemcpyAsync(h->dPsi, d_psi, (size_t)h->dim * 8, cudaMemcpyDeviceToDevice, st));
  float best[2] = {3.4e38f, 3.4e38f};
  int pick[2] = {h->sched1, h->sched2};
  for (int c = 0; c < oz::SCHED_COUNT; ++c) {
    h->sched1 = c;
    h->sched2 = c;
    if (int rc = h->balance()) return rc;
    float t[2] = {3.4e38f, 3.4e38f};
    for (int r = 0; r <= reps; ++r) {  // first product warms the new tables
      OZ_CU(cudaGraphLaunch(h->exec, st));
      OZ_CU(cudaStreamSynchronize(st));
      float m4[4];
      if (int rc = oz_heff_stage_times(h, m4)) return rc;
      if (r > 0) {
        t[0] = std::min(t[0], m4[1]);
        t[1] = std::min(t[1], m4[3]);
      }
    }
    if (ms) {
      ms[2 * c] = t[0];
      ms[2 * c + 1] = t[1];
    }
    for (int k = 0; k < 2; ++k)
      if (t[k] < best[k]) {
        best[k] = t[k];
        pick[k] = c;
      }
  }
  h->sched1 = pick[0];
  h->sched2 = pick[1];
  if (int rc = h->balance()) return rc;
  if (sched) {
    sched[0] = pick[0];
    sched[1] = pick[1];
  }
  return OZ_OK;
}

namespace oz {
int emulated_batch(oz_ctx* c, const std::vector<EmuJob>& jobs, int S, int s, cudaStream_t st) {
  if (jobs.empty()) return OZ_OK;
  // layout: digit planes of every A and every B, row maxima and exponents, then the tables
  std::vector<SliceSeg> segs;
  std::vector<GemmProblem> probs;
  std::vector<GemmTile> tiles;
  std::vector<long long> offA, offB, rowA, rowB;
  long long dA = 0, dB = 0, rA = 0, rB = 0;
  for (const EmuJob& j : jobs) {
    if (j.M <= 0 || j.N <= 0 || j.K <= 0 || j.K > oz::max_k_of_level(s)) return fail(OZ_EINVAL, "emulated batch: bad sizes");
    const long long nkb = cdiv(j.K, KB), nrbA = cdiv(j.M, TILE_M), nrbB = cdiv(j.N, BN);
    offA.push_back(dA);
    offB.push_back(dB);
    rowA.push_back(rA);
    rowB.push_back(rB);
    dA += nrbA * nkb * S * TILE_M * KB;
    dB += nrbB * nkb * S * BN * KB;
    rA += nrbA * TILE_M;
    rB += nrbB * BN;
  }
  const size_t bA = (size_t)dA * 2, bB = (size_t)dB * 2, bM = (size_t)(rA + rB) * 8, bE = (size_t)(rA + rB) * 4;
  const size_t n = jobs.size();
  const size_t bS = 2 * n * sizeof(SliceSeg), bP = n * sizeof(GemmProblem);
  long long ntile = 0;
  for (const EmuJob& j : jobs) ntile += cdiv(j.M, TILE_M) * cdiv(j.N, BN);
  const size_t bT = (size_t)ntile * sizeof(GemmTile);
  // the CTA -> first segment tables need the unit prefixes: count them first
  long long umt = 0, udt = 0;
  for (const EmuJob& j : jobs) {
    const int nkb = (int)cdiv(j.K, KB);
    umt += rowmax_units(j.M, j.K, j.transA) + rowmax_units(j.N, j.K, j.transB ? 0 : 1);
    udt += digit_units((int)(cdiv(j.M, TILE_M) * TILE_M), nkb * KB) + digit_units((int)(cdiv(j.N, BN) * BN), nkb * KB);
  }
  const size_t bCm = (size_t)((umt + 255) / 256 + 1) * sizeof(int), bCd = (size_t)((udt + 31) / 32 + 1) * sizeof(int);
  const size_t need = align256(bA) + align256(bB) + align256(bM) + align256(bE) + align256(bS) + align256(bP) +
                      align256(bT) + align256(bCm) + align256(bCd) + 256;
  if (int rc = c->reserve(need)) return rc;
  char* p = c->ws;
  __half* hA = (__half*)p;
  p += align256(bA);
  __half* hB = (__half*)p;
  p += align256(bB);
  unsigned long long* mx = (unsigned long long*)p;
  p += align256(bM);
  int* ex = (int*)p;
  p += align256(bE);
  SliceSeg* dSeg = (SliceSeg*)p;
  p += align256(bS);
  GemmProblem* dProb = (GemmProblem*)p;
  p += align256(bP);
  GemmTile* dTile = (GemmTile*)p;
  p += align256(bT);
  int* dCm = (int*)p;
  p += align256(bCm);
  int* dCd = (int*)p;
  long long um = 0, ud = 0;
  for (size_t i = 0; i < n; ++i) {
    const EmuJob& j = jobs[i];
    const int nkb = (int)cdiv(j.K, KB);
    SliceSeg a{};
    a.src = j.A; a.ld = j.lda; a.rows = j.M; a.cols = j.K; a.prows = (int)(cdiv(j.M, TILE_M) * TILE_M);
    a.pcols = nkb * KB; a.r0 = 0; a.k0 = 0; a.trans = j.transA; a.S = S; a.scale = 1.0; a.dst = hA + offA[i];
    a.TR = TILE_M; a.nkb = nkb; a.rowmax = mx + rowA[i]; a.rowexp = ex + rowA[i]; a.unit0 = ud; a.unit0m = um;
    ud += digit_units(a.prows, a.pcols);
    um += rowmax_units(a.rows, a.cols, a.trans);
    SliceSeg b{};
    b.src = j.B; b.ld = j.ldb; b.rows = j.N; b.cols = j.K; b.prows = (int)(cdiv(j.N, BN) * BN); b.pcols = nkb * KB;
    b.r0 = 0; b.k0 = 0; b.trans = j.transB ? 0 : 1; b.S = S; b.scale = 1.0; b.dst = hB + offB[i]; b.TR = BN;
    b.nkb = nkb;
    b.rowmax = mx + rA + rowB[i]; b.rowexp = ex + rA + rowB[i]; b.unit0 = ud; b.unit0m = um;
    ud += digit_units(b.prows, b.pcols);
    um += rowmax_units(b.rows, b.cols, b.trans);
    segs.push_back(a);
    segs.push_back(b);
    GemmProblem P{};
    P.A = a.dst; P.B = b.dst; P.ea = a.rowexp; P.eb = b.rowexp; P.M = j.M; P.N = j.N; P.nkb = nkb;
    P.SA = S; P.SB = S; P.s = s; P.mode = OUT_DENSE; P.C = j.C; P.ldc = j.ldc; P.alpha = 1.0; P.beta = 0.0;
    probs.push_back(P);
    for (int mb = 0; mb < (int)cdiv(j.M, TILE_M); ++mb)
      for (int nb = 0; nb < (int)cdiv(j.N, BN); ++nb) tiles.push_back({(int)i, mb, nb, 0});
  }
  OZ_CU(cudaMemsetAsync(mx, 0, bM, st));
  OZ_CU(cudaMemcpyAsync(dSeg, segs.data(), bS, cudaMemcpyHostToDevice, st));
  OZ_CU(cudaMemcpyAsync(dProb, probs.data(), bP, cudaMemcpyHostToDevice, st));
  OZ_CU(cudaMemcpyAsync(dTile, tiles.data(), bT, cudaMemcpyHostToDevice, st));
  const std::vector<int> tcm = rowmax_cta_table(segs, um), tcd = digits_cta_table(segs, ud);
  if (um != umt || ud != udt || tcm.size() * sizeof(int) > bCm || tcd.size() * sizeof(int) > bCd)
    return fail(OZ_EINVAL, "emulated batch: inconsistent slicing units");
  OZ_CU(cudaMemcpyAsync(dCm, tcm.data(), tcm.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  OZ_CU(cudaMemcpyAsync(dCd, tcd.data(), tcd.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  OZ_CU(launch_rowmax(dSeg, nullptr, (int)segs.size(), um, c->d_flags, st, dCm));
  OZ_CU(launch_digits(dSeg, nullptr, (int)segs.size(), ud, S, st, dCd));
  OZ_CU(launch_gemm(dProb, dTile, (int)tiles.size(), c->nsm, nullptr, s, c->d_flags + 1, st));
  // the host tables above are read by the copies: wait before they go out of scope
  OZ_CU(cudaStreamSynchronize(st));
  return OZ_OK;
}
}  // namespace oz
