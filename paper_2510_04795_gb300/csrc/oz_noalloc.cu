// ozaki_gemm_noalloc: the emulated product of ozaki_gemm for callers that must not allocate device
// memory (see include/ozdmrg.h).  Its scratch -- digit planes, shared exponents, row maxima and the
// device status words -- is one file-scope __device__ array of fixed size that every GPU loading
// this library holds until the process exits.  Host code never passes the array's name to a
// kernel (on the host it names a host-side stand-in); it passes the device address obtained once
// per device with cudaGetSymbolAddress.
#include <cstring>
#include <mutex>
#include <string>

#include "ozdmrg.h"
#include "oz_gemm.cuh"
#include "oz_slice.cuh"

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)64 << 20;  // 64 MiB
constexpr int MAX_DEVICES = 64;

// 64 MiB of scratch plus 16 bytes of status words (kernels latch NaN/Inf and timeouts there; this
// entry point does not report them).
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES + 256];

std::mutex g_mu;
unsigned char* g_scratch_ptr[MAX_DEVICES] = {nullptr};
int g_nsm[MAX_DEVICES] = {0};
// this entry point reports its errors through the returned status code only
int fail(int code, const std::string&) { return code; }

inline long long cdiv(long long a, long long b) { return (a + b - 1) / b; }
inline size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

__global__ void noalloc_scale(double* C, int m, int n, int ldc, double beta) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)m * n) return;
  const int i = (int)(idx / n), j = (int)(idx % n);
  double* c = C + (long long)i * ldc + j;
  *c = beta == 0.0 ? 0.0 : __dmul_rn(beta, *c);
}

// Per-device set-up: the device address of the scratch array (and the SM count), once per device.
int setup(int dev, unsigned char** base, int* nsm) {
  if (dev < 0 || dev >= MAX_DEVICES) return fail(OZ_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return fail(OZ_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    int sm = 0;
    e = cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(OZ_ECUDA, std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    g_nsm[dev] = sm;
  }
  *base = g_scratch_ptr[dev];
  *nsm = g_nsm[dev];
  return OZ_OK;
}

}  // namespace

extern "C" int ozaki_gemm_noalloc(int m, int n, int k, double alpha, const double* A, int lda, const double* B,
                                  int ldb, double beta, double* C, int ldc, int slices, int level,
                                  oz_stream_t stream) {
  if (slices < 1 || slices > 9) return fail(OZ_EINVAL, "slices must be in 1..9");
  const int s = level == 0 ? slices : level;
  if (s < 1 || s > slices || s > oz::MAX_LEVEL) return fail(OZ_EINVAL, "level must be in 1..S");
  if (m < 0 || n < 0 || k < 0) return fail(OZ_EINVAL, "negative size");
  if (lda < (k > 1 ? k : 1) || ldb < (n > 1 ? n : 1) || ldc < (n > 1 ? n : 1))
    return fail(OZ_EINVAL, "leading dimension too small");
  if (k > oz::max_k_of_level(s))
    return fail(OZ_EINVAL, s >= oz::SPLIT_LEVEL ? "k exceeds the exact-accumulation limit of level 9 (130048)"
                                                : "k exceeds the exact-accumulation limit (1048576)");
  if (m == 0 || n == 0) return OZ_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(OZ_ECUDA, "cudaGetDevice failed");
  unsigned char* base = nullptr;
  int nsm = 0;
  if (int rc = setup(dev, &base, &nsm)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int* flags = reinterpret_cast<int*>(base + NOALLOC_SCRATCH_BYTES);
  if (k == 0) {
    noalloc_scale<<<(unsigned)cdiv((long long)m * n, 256), 256, 0, st>>>(C, m, n, ldc, beta);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? OZ_OK : fail(OZ_ECUDA, cudaGetErrorString(e));
  }
  // scratch layout (same operand format as ozaki_gemm)
  const int S = slices;
  const int nkb = (int)cdiv(k, oz::KB), nrbA = (int)cdiv(m, oz::TILE_M), nrbB = (int)cdiv(n, oz::BN);
  const int mpad = nrbA * oz::TILE_M, npad = nrbB * oz::BN;
  const size_t bA = (size_t)nrbA * nkb * S * oz::TILE_M * oz::KB * 2;
  const size_t bB = (size_t)nrbB * nkb * S * oz::BN * oz::KB * 2;
  const size_t bM = (size_t)(mpad + npad) * 8, bE = (size_t)(mpad + npad) * 4;
  const size_t need = a256(bA) + a256(bB) + a256(bM) + a256(bE);
  if (need > NOALLOC_SCRATCH_BYTES)
    return fail(OZ_EINVAL, "problem needs " + std::to_string(need) + " bytes of scratch; the allocation-free entry "
                           "point holds 67108864");
  unsigned char* p = base;
  __half* dA = reinterpret_cast<__half*>(p);
  p += a256(bA);
  __half* dB = reinterpret_cast<__half*>(p);
  p += a256(bB);
  unsigned long long* mx = reinterpret_cast<unsigned long long*>(p);
  p += a256(bM);
  int* ex = reinterpret_cast<int*>(p);
  // the row maxima accumulate with atomicMax: they must start at zero on every call
  cudaError_t e = cudaMemsetAsync(mx, 0, bM, st);
  if (e != cudaSuccess) return fail(OZ_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  oz::SegPack pk{};
  oz::SliceSeg& a = pk.seg[0];
  a.src = A; a.ld = lda; a.rows = m; a.cols = k; a.prows = mpad; a.pcols = nkb * oz::KB;
  a.r0 = 0; a.k0 = 0; a.trans = 0; a.S = S; a.scale = 1.0; a.dst = dA; a.TR = oz::TILE_M; a.nkb = nkb;
  a.rowmax = mx; a.rowexp = ex; a.unit0 = 0; a.unit0m = 0;
  oz::SliceSeg& b = pk.seg[1];
  b.src = B; b.ld = ldb; b.rows = n; b.cols = k; b.prows = npad; b.pcols = nkb * oz::KB;
  b.r0 = 0; b.k0 = 0; b.trans = 1; b.S = S; b.scale = 1.0; b.dst = dB; b.TR = oz::BN; b.nkb = nkb;
  b.rowmax = mx + mpad; b.rowexp = ex + mpad;
  b.unit0 = oz::digit_units(a.prows, a.pcols);
  b.unit0m = oz::rowmax_units(a.rows, a.cols, a.trans);
  const long long um = b.unit0m + oz::rowmax_units(b.rows, b.cols, b.trans);
  const long long ud = b.unit0 + oz::digit_units(b.prows, b.pcols);
  if ((e = oz::launch_rowmax(nullptr, &pk, 2, um, flags, st)) != cudaSuccess) return fail(OZ_ECUDA, cudaGetErrorString(e));
  if ((e = oz::launch_digits(nullptr, &pk, 2, ud, S, st)) != cudaSuccess) return fail(OZ_ECUDA, cudaGetErrorString(e));
  oz::GemmProblem P{};
  P.A = dA; P.B = dB; P.ea = ex; P.eb = ex + mpad;
  P.M = m; P.N = n; P.nkb = nkb; P.SA = S; P.SB = S; P.s = s;
  P.mode = oz::OUT_DENSE; P.C = C; P.ldc = ldc; P.alpha = alpha; P.beta = beta;
  if ((e = oz::launch_gemm(nullptr, nullptr, nrbA * nrbB, nsm, &P, 0, flags + 1, st)) != cudaSuccess)
    return fail(OZ_ECUDA, cudaGetErrorString(e));
  return OZ_OK;
}
