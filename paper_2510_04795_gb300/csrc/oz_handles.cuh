// Definitions of the context and H_eff handles, shared by the library's translation units
// (not part of the C ABI).
#pragma once
#include <cublas_v2.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "ozdmrg.h"
#include "oz_gemm.cuh"
#include "oz_internal.cuh"
#include "oz_slice.cuh"

namespace oz {
inline int cuda_fail(cudaError_t e, const char* where) {
  return api_fail(e == cudaErrorMemoryAllocation ? OZ_ENOMEM : OZ_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
}  // namespace oz

struct oz_ctx_s {
  int device = 0;
  int nsm = 0;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  int* d_flags = nullptr;  // [0] non-finite input, [1] kernel timeout/abort
  cublasHandle_t cublas = nullptr;
  // performant dispatch of ozaki_gemm: shape class -> (chosen mode, emulated ms, native ms)
  struct PerfChoice { int mode; float ms_emu, ms_nat; };
  std::map<unsigned long long, PerfChoice> perf;

  // bump allocation inside the workspace (grown with cudaMalloc when too small)
  int reserve(size_t bytes) {
    if (bytes <= ws_bytes) return OZ_OK;
    if (ws) {
      cudaDeviceSynchronize();
      cudaFree(ws);
      ws = nullptr;
      ws_bytes = 0;
    }
    size_t b = std::max(bytes, (size_t)64 << 20);
    cudaError_t e = cudaMalloc(&ws, b);
    if (e != cudaSuccess) return oz::cuda_fail(e, "workspace cudaMalloc");
    ws_bytes = b;
    return OZ_OK;
  }
};

struct oz_heff_s {
  oz_ctx* ctx = nullptr;
  int nsec = 0, ntask = 0, S = 7, s = 7, mode = OZ_MODE_EAGER;
  std::vector<int> m, n;
  std::vector<long long> psioff;
  long long dim = 0, flops = 0, carrier_flops = 0, bytes_ops = 0, bytes_scratch = 0;
  std::vector<void*> allocs;

  // emulated path
  __half *dA1 = nullptr, *dB1 = nullptr, *dA2 = nullptr, *dB2 = nullptr;
  double* dStage = nullptr;
  int *eB1 = nullptr, *eA2 = nullptr;
  unsigned long long *mB1 = nullptr, *mA2 = nullptr;
  size_t bytes_mB1 = 0, bytes_mA2 = 0;
  oz::GemmProblem *dP1 = nullptr, *dP2 = nullptr;
  oz::GemmTile *dT1 = nullptr, *dT2 = nullptr;
  int nt1 = 0, nt2 = 0;
  oz::SliceSeg *dSegPsi = nullptr, *dSegA2 = nullptr;
  int *dCtaPsiM = nullptr, *dCtaPsiD = nullptr, *dCtaA2D = nullptr;  // CTA -> first segment tables
  int nsegPsi = 0, nsegA2 = 0;
  long long uPsiM = 0, uPsiD = 0, uA2D = 0;
  bool zero_y = false;

  // native path (stacked FP64 copies)
  double *nA1 = nullptr, *nB2 = nullptr, *nT = nullptr;
  struct NatG1 { long long a1off, toff; int rows, kdim, q; };
  struct NatG2 { long long stoff, b2off; int q, ld2; };
  std::vector<NatG1> nat1;
  std::vector<NatG2> nat2;
  long long* dScatter = nullptr;  // per stacked T row: destination offset in the staging buffer
  long long nTrows = 0;

  double *dPsi = nullptr, *dY = nullptr;
  double* dDiag = nullptr;  // diagonal of H_eff (Davidson preconditioner)
  bool prepared = false;
  // layout kept for the lazy per-product setup of the emulated path
  std::vector<std::vector<int>> bysrc, bydst;
  std::vector<int> rows1, nkb1, nkb2, ld2, tsrc, tdst;
  std::vector<long long> offk, rowin1, stoff, A1off, B1off, A2off, B2off, A1row, B1row, A2row, B2row;
  int* eA1 = nullptr;
  int* eB2 = nullptr;
  unsigned long long *mA1 = nullptr, *mB2 = nullptr;  // row maxima of the stacked operators
  std::vector<long long> a1o, b2o;                    // native path: offsets of the stacked FP64 copies
  // problems of the two stages (host copies), the sector of each, and per-sector slice levels
  std::vector<oz::GemmProblem> hp1, hp2;
  std::vector<oz::GemmTile> bt1, bt2;  // tile lists of the two stages in creation order
  std::vector<oz::GemmTile> ht1, ht2;  // the same, scheduled over the CTAs (uploaded)
  int *dF1 = nullptr, *dF2 = nullptr;  // per-CTA first tile of each stage (nsm + 1 entries)
  int sched1 = 0, sched2 = 0;          // schedule of each stage (oz::SCHED_*), set by the autotuner
  bool ho1 = false, ho2 = false;  // epilogue layouts of the two GEMM launches (hand-over of lane quarter 1)
  bool ho1_auto = false, ho2_auto = false;  // the layouts chosen from the tile lengths
  bool pair = false;                   // products on CTA pairs (256 x 64 tiles)
  int units = 0;                       // persistent units of the GEMM launches: CTAs, or CTA pairs
  int balance();                       // (re)assigns the tiles to CTAs for the current levels
  std::vector<int> p1sec, p2sec;
  std::vector<int> lev1, lev2;  // per source sector (stage 1), per target sector (stage 2)
  // stage-2 orientation per target sector: 1 = computed as Y^T = (cR stack) T^T, so that the
  // smaller of m[q], n[q] takes the 64-row side of the tile (less padding)
  std::vector<char> swap2;
  // exponent-gap histograms of the operators (9 bins per sector): stage-1 A, stage-2 B
  std::vector<unsigned long long> histA1, histB2;
  int set_levels(const int* s1, const int* s2);
  int prepare();
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // stage boundaries of the last product
  float ops_ms[2] = {0.f, 0.f};          // last operator slicing: rowmax pass, digit pass (device ms)
  long long ops_bytes[2] = {0, 0};       // their algorithmic bytes (read + written)

  template <class T>
  int alloc(T** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 256;
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e != cudaSuccess) return oz::cuda_fail(e, "cudaMalloc");
    allocs.push_back((void*)*p);
    return OZ_OK;
  }
  int enqueue(cudaStream_t st, bool capturing = false);
  int capture();
};
