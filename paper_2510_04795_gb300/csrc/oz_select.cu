// Per-block slice levels for the H_eff products (the precision dial of the paper's sections
// "Theory of emulated FP64 arithmetic" and "Numerical procedure": the slice count trades accuracy
// for time; the library's automatic mode picks it per GEMM).
//
// Every stacked product of an H_eff handle (stage 1 per source sector, stage 2 per target sector)
// is described by operand statistics: for each operand, the histogram of the exponent gaps
// between every element and the largest element of its row (A) or column (B) -- the quantity that
// decides how many 8-bit slices an element needs before its leading bits enter the shared
// fixed-point frame -- plus the reduction length and the output size.  A selector maps these
// features to the predicted log10 relative error of the product at every level 3..8; per stage,
// levels are then lowered greedily -- the largest carrier-flop saving per predicted squared error
// first -- while the predicted error of the stage output, sum_q (err_q |out_q|)^2, stays within
// (budget |out| / sqrt 2)^2 (the norms from one product at the full level).
// Selectors: fixed (the handle's level), analytic (error ~ 2^(gA + gB - 8 s + 3) from the mean
// gaps) and learned (the MLP of oz_mlp.cu).  The harvest entry point measures the true relative
// errors per product and level on the device, which is what the network is trained on.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "ozdmrg.h"
#include "oz_handles.cuh"
#include "oz_internal.cuh"

namespace {

constexpr int NBIN = 9;  // gap bins 0, 1, 2-3, 4-7, 8-15, 16-31, 32-63, >= 64, and exact zeros
constexpr int NF = OZ_NFEAT;
constexpr int LMIN = 3;  // lowest level a selector picks
constexpr int LPRED = 8; // highest level with a predicted error; a handle at level 9 (the fixed
                         // fallback) starts there with its error counted as zero

struct HistSeg {
  const double* p;
  long long ld;
  int rows, cols;  // histogram rows: the row (or with trans, the column) whose maximum sets the gap
  int trans;
};

__device__ __forceinline__ int gap_bin(int g) {
  if (g <= 0) return 0;
  if (g == 1) return 1;
  if (g < 4) return 2;
  if (g < 8) return 3;
  if (g < 16) return 4;
  if (g < 32) return 5;
  if (g < 64) return 6;
  return 7;
}

// One CTA per segment, one warp per histogram row: exponent of the row maximum, then the bin of
// every element's exponent gap.  Counts per segment into cnt[seg * NBIN + bin].
__global__ void gap_hist_kernel(const HistSeg* __restrict__ segs, unsigned long long* __restrict__ cnt) {
  __shared__ unsigned int h[NBIN];
  const HistSeg S = segs[blockIdx.x];
  if (threadIdx.x < NBIN) h[threadIdx.x] = 0;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int r = warp; r < S.rows; r += nw) {
    auto at = [&](int c) { return S.trans ? S.p[(long long)c * S.ld + r] : S.p[(long long)r * S.ld + c]; };
    double mx = 0.0;
    for (int c = lane; c < S.cols; c += 32) mx = fmax(mx, fabs(at(c)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int er = mx > 0.0 ? ilogb(mx) : 0;
    for (int c = lane; c < S.cols; c += 32) {
      const double x = fabs(at(c));
      atomicAdd(&h[x == 0.0 ? NBIN - 1 : gap_bin(er - ilogb(x))], 1u);
    }
  }
  __syncthreads();
  if (threadIdx.x < NBIN) cnt[(long long)blockIdx.x * NBIN + threadIdx.x] = h[threadIdx.x];
}

struct NormSeg {
  const double* x;
  const double* ref;  // null: only |x|^2
  long long ld;
  int rows, cols;
};

// Per segment: out[2 s] = sum (x - ref)^2, out[2 s + 1] = sum ref^2 (or x^2 without ref).
__global__ void seg_norm_kernel(const NormSeg* __restrict__ segs, double* __restrict__ out) {
  __shared__ double sa[256], sb[256];
  const NormSeg S = segs[blockIdx.x];
  double a = 0.0, b = 0.0;
  for (long long idx = threadIdx.x; idx < (long long)S.rows * S.cols; idx += blockDim.x) {
    const long long r = idx / S.cols, c = idx % S.cols;
    const double x = S.x[r * S.ld + c];
    const double y = S.ref ? S.ref[r * S.ld + c] : x;
    a = fma(x - y, x - y, a);
    b = fma(y, y, b);
  }
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sa[threadIdx.x] += sa[threadIdx.x + w];
      sb[threadIdx.x] += sb[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[2 * blockIdx.x] = sa[0];
    out[2 * blockIdx.x + 1] = sb[0];
  }
}

#define SE_CU(call)                                                                 \
  do {                                                                              \
    cudaError_t _e = (call);                                                        \
    if (_e != cudaSuccess)                                                          \
      return oz::api_fail(_e == cudaErrorMemoryAllocation ? OZ_ENOMEM : OZ_ECUDA,   \
                          std::string(#call) + ": " + cudaGetErrorString(_e));      \
  } while (0)

template <class T>
struct DVec {
  T* p = nullptr;
  DVec() = default;
  DVec(const DVec&) = delete;
  DVec& operator=(const DVec&) = delete;
  ~DVec() {
    if (p) cudaFree(p);
  }
  int alloc(size_t n) {
    if (p) cudaFree(p);
    p = nullptr;
    SE_CU(cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)));
    return OZ_OK;
  }
};

// counts of every segment (host), one launch
int hist_segments(const std::vector<HistSeg>& segs, std::vector<unsigned long long>* cnt, cudaStream_t st) {
  cnt->assign(segs.size() * NBIN, 0ull);
  if (segs.empty()) return OZ_OK;
  DVec<HistSeg> ds;
  DVec<unsigned long long> dc;
  if (int rc = ds.alloc(segs.size())) return rc;
  if (int rc = dc.alloc(segs.size() * NBIN)) return rc;
  SE_CU(cudaMemcpyAsync(ds.p, segs.data(), segs.size() * sizeof(HistSeg), cudaMemcpyHostToDevice, st));
  gap_hist_kernel<<<(unsigned)segs.size(), 256, 0, st>>>(ds.p, dc.p);
  SE_CU(cudaGetLastError());
  SE_CU(cudaMemcpyAsync(cnt->data(), dc.p, segs.size() * NBIN * 8, cudaMemcpyDeviceToHost, st));
  SE_CU(cudaStreamSynchronize(st));
  return OZ_OK;
}

int norm_segments(const std::vector<NormSeg>& segs, std::vector<double>* out, cudaStream_t st) {
  out->assign(segs.size() * 2, 0.0);
  if (segs.empty()) return OZ_OK;
  DVec<NormSeg> ds;
  DVec<double> dd;
  if (int rc = ds.alloc(segs.size())) return rc;
  if (int rc = dd.alloc(segs.size() * 2)) return rc;
  SE_CU(cudaMemcpyAsync(ds.p, segs.data(), segs.size() * sizeof(NormSeg), cudaMemcpyHostToDevice, st));
  seg_norm_kernel<<<(unsigned)segs.size(), 256, 0, st>>>(ds.p, dd.p);
  SE_CU(cudaGetLastError());
  SE_CU(cudaMemcpyAsync(out->data(), dd.p, segs.size() * 16, cudaMemcpyDeviceToHost, st));
  SE_CU(cudaStreamSynchronize(st));
  return OZ_OK;
}

// Segments of the stage-1 output of source q (rows of T in the stage-2 layout) and of the
// stage-2 output of target q (Y[q]); ref_* (optional) are buffers of the same layout.
void out_segments(const oz_heff* h, const double* T, const double* refT, const double* Y, const double* refY,
                  std::vector<NormSeg>* segs, std::vector<int>* owner, bool stage1) {
  for (int q = 0; q < h->nsec; ++q) {
    if (stage1) {
      for (int t : h->bysrc[q]) {
        const int d = h->tdst[t];
        const long long off = h->stoff[d] + h->offk[t];
        segs->push_back({T + off, refT ? refT + off : nullptr, h->ld2[d], h->m[d], h->n[q]});
        owner->push_back(q);
      }
    } else if (!h->bydst[q].empty()) {
      const long long off = h->psioff[q];
      segs->push_back({Y + off, refY ? refY + off : nullptr, h->n[q], h->m[q], h->n[q]});
      owner->push_back(q);
    }
  }
}

int product(oz_heff* h, const double* d_psi, cudaStream_t st) {
  if (int rc = h->prepare()) return rc;
  SE_CU(cudaMemcpyAsync(h->dPsi, d_psi, (size_t)h->dim * 8, cudaMemcpyDeviceToDevice, st));
  SE_CU(cudaGraphLaunch(h->exec, st));
  SE_CU(cudaStreamSynchronize(st));
  return OZ_OK;
}

void features_from_counts(const unsigned long long* a, const unsigned long long* b, double K, double MN, float* f) {
  double na = 0.0, nb = 0.0;
  for (int i = 0; i < NBIN; ++i) {
    na += (double)a[i];
    nb += (double)b[i];
  }
  for (int i = 0; i < NBIN; ++i) {
    f[i] = na > 0 ? (float)(a[i] / na) : 0.0f;
    f[NBIN + i] = nb > 0 ? (float)(b[i] / nb) : 0.0f;
  }
  f[2 * NBIN] = (float)(std::log2(std::max(K, 1.0)) / 16.0);
  f[2 * NBIN + 1] = (float)(std::log2(std::max(MN, 1.0)) / 32.0);
}

// Effective gap (bits) of an operand from its histogram: -log2 of the RMS of 2^-gap over its
// nonzero elements, with each bin at its midpoint.
double effective_gap(const float* f) {
  const double mid[NBIN - 1] = {0.0, 1.0, 2.5, 5.5, 11.5, 23.5, 47.5, 80.0};
  double s = 0.0, w = 0.0;
  for (int i = 0; i < NBIN - 1; ++i) {
    s += f[i] * std::exp2(-2.0 * mid[i]);
    w += f[i];
  }
  if (w <= 0.0 || s <= 0.0) return 0.0;
  return -0.5 * std::log2(s / w);
}

// Features of every product of h for psi: a product at the handle's level gives T.
int problem_features(oz_heff* h, const double* d_psi, std::vector<float>* f1, std::vector<float>* f2,
                     cudaStream_t st) {
  const int nsec = h->nsec;
  f1->assign((size_t)nsec * NF, 0.0f);
  f2->assign((size_t)nsec * NF, 0.0f);
  if (int rc = product(h, d_psi, st)) return rc;
  std::vector<HistSeg> segs;
  std::vector<int> kind, sec;  // kind 0: psi of stage-1 source q, 1: T of stage-2 target q
  for (int q = 0; q < nsec; ++q) {
    if (!h->bysrc[q].empty()) {
      segs.push_back({h->dPsi + h->psioff[q], h->n[q], h->n[q], h->m[q], 1});  // columns of psi[q]
      kind.push_back(0);
      sec.push_back(q);
    }
    if (!h->bydst[q].empty()) {
      segs.push_back({h->dStage + h->stoff[q], h->ld2[q], h->m[q], h->ld2[q], 0});  // rows of T
      kind.push_back(1);
      sec.push_back(q);
    }
  }
  std::vector<unsigned long long> cnt;
  if (int rc = hist_segments(segs, &cnt, st)) return rc;
  for (size_t i = 0; i < segs.size(); ++i) {
    const int q = sec[i];
    if (kind[i] == 0)
      features_from_counts(&h->histA1[(size_t)q * NBIN], &cnt[i * NBIN], (double)h->m[q],
                           (double)h->rows1[q] * h->n[q], &(*f1)[(size_t)q * NF]);
    else
      features_from_counts(&cnt[i * NBIN], &h->histB2[(size_t)q * NBIN], (double)h->ld2[q],
                           (double)h->m[q] * h->n[q], &(*f2)[(size_t)q * NF]);
  }
  return OZ_OK;
}

}  // namespace

namespace oz {
// Operator histograms of an H_eff handle (stage-1 A = stacked L, rows; stage-2 B = stacked
// (cR)^T, one row of R per output column, gap taken within each task's block), from the FP64
// blocks while oz_heff_create still has them.
int heff_operator_hist(oz_heff* h, const oz_task* tasks) {
  const int nsec = h->nsec;
  std::vector<HistSeg> segs;
  std::vector<int> kind, sec;
  for (int q = 0; q < nsec; ++q)
    for (int t : h->bysrc[q]) {
      segs.push_back({tasks[t].d_L, h->m[q], h->m[tasks[t].dst], h->m[q], 0});
      kind.push_back(0);
      sec.push_back(q);
    }
  for (int q = 0; q < nsec; ++q)
    for (int t : h->bydst[q]) {
      segs.push_back({tasks[t].d_R, h->n[tasks[t].src], h->n[q], h->n[tasks[t].src], 0});
      kind.push_back(1);
      sec.push_back(q);
    }
  std::vector<unsigned long long> cnt;
  if (int rc = hist_segments(segs, &cnt, 0)) return rc;
  h->histA1.assign((size_t)nsec * NBIN, 0ull);
  h->histB2.assign((size_t)nsec * NBIN, 0ull);
  for (size_t i = 0; i < segs.size(); ++i) {
    auto& dst = kind[i] == 0 ? h->histA1 : h->histB2;
    for (int b = 0; b < NBIN; ++b) dst[(size_t)sec[i] * NBIN + b] += cnt[i * NBIN + b];
  }
  return OZ_OK;
}
}  // namespace oz

extern "C" int oz_heff_problem_features(oz_heff* h, const double* d_psi, float* feat1, float* feat2,
                                        oz_stream_t stream) {
  if (!h || !d_psi || !feat1 || !feat2) return oz::api_fail(OZ_EINVAL, "null argument");
  if (h->mode != OZ_MODE_EAGER) return oz::api_fail(OZ_EINVAL, "features exist for emulated handles only");
  std::vector<float> f1, f2;
  if (int rc = problem_features(h, d_psi, &f1, &f2, (cudaStream_t)stream)) return rc;
  std::copy(f1.begin(), f1.end(), feat1);
  std::copy(f2.begin(), f2.end(), feat2);
  return OZ_OK;
}

extern "C" int oz_heff_problem_errors(oz_heff* h, const double* d_psi, int level, double* err1, double* err2,
                                      oz_stream_t stream) {
  if (!h || !d_psi || !err1 || !err2) return oz::api_fail(OZ_EINVAL, "null argument");
  if (h->mode != OZ_MODE_EAGER) return oz::api_fail(OZ_EINVAL, "errors exist for emulated handles only");
  if (level < 1 || level > h->s) return oz::api_fail(OZ_EINVAL, "level must be in 1..the handle's level");
  cudaStream_t st = (cudaStream_t)stream;
  const int nsec = h->nsec;
  std::vector<int> save1 = h->lev1, save2 = h->lev2, full(nsec, h->s), low(nsec, level);
  if (int rc = h->set_levels(full.data(), full.data())) return rc;
  if (int rc = product(h, d_psi, st)) return rc;
  DVec<double> refT, refY;
  const size_t nT = (size_t)h->stoff[nsec], nY = (size_t)h->dim;
  if (int rc = refT.alloc(nT)) return rc;
  if (int rc = refY.alloc(nY)) return rc;
  SE_CU(cudaMemcpyAsync(refT.p, h->dStage, nT * 8, cudaMemcpyDeviceToDevice, st));
  SE_CU(cudaMemcpyAsync(refY.p, h->dY, nY * 8, cudaMemcpyDeviceToDevice, st));
  for (int stage = 1; stage <= 2; ++stage) {
    if (int rc = h->set_levels(stage == 1 ? low.data() : full.data(), stage == 1 ? full.data() : low.data()))
      return rc;
    if (int rc = product(h, d_psi, st)) return rc;
    std::vector<NormSeg> segs;
    std::vector<int> owner;
    out_segments(h, h->dStage, refT.p, h->dY, refY.p, &segs, &owner, stage == 1);
    std::vector<double> nr;
    if (int rc = norm_segments(segs, &nr, st)) return rc;
    std::vector<double> num(nsec, 0.0), den(nsec, 0.0);
    for (size_t i = 0; i < segs.size(); ++i) {
      num[owner[i]] += nr[2 * i];
      den[owner[i]] += nr[2 * i + 1];
    }
    double* out = stage == 1 ? err1 : err2;
    for (int q = 0; q < nsec; ++q) out[q] = den[q] > 0.0 ? std::sqrt(num[q] / den[q]) : -1.0;
  }
  return h->set_levels(save1.data(), save2.data());
}

extern "C" int oz_heff_select_levels(oz_heff* h, const double* d_psi, int selector, double budget, oz_mlp* net,
                                     double margin, int* s1, int* s2, oz_stream_t stream) {
  if (!h || !d_psi) return oz::api_fail(OZ_EINVAL, "null argument");
  if (h->mode != OZ_MODE_EAGER) return oz::api_fail(OZ_EINVAL, "levels exist for emulated handles only");
  if (selector < OZ_SELECT_FIXED || selector > OZ_SELECT_LEARNED) return oz::api_fail(OZ_EINVAL, "unknown selector");
  if (!(budget > 0.0)) return oz::api_fail(OZ_EINVAL, "budget must be positive");
  if (selector == OZ_SELECT_LEARNED && (!net || oz_mlp_nin(net) != NF || oz_mlp_nout(net) < LPRED - LMIN + 1))
    return oz::api_fail(OZ_EINVAL, "the learned selector needs a network with OZ_NFEAT inputs and 6 outputs");
  cudaStream_t st = (cudaStream_t)stream;
  const int nsec = h->nsec, smax = h->s;
  std::vector<int> full(nsec, smax), l1(nsec, smax), l2(nsec, smax);
  if (selector != OZ_SELECT_FIXED) {
    if (int rc = h->set_levels(full.data(), full.data())) return rc;
    std::vector<float> f1, f2;
    if (int rc = problem_features(h, d_psi, &f1, &f2, st)) return rc;  // T and Y of the full level stay
    // output norms per product and in total
    std::vector<NormSeg> segs;
    std::vector<int> owner;
    out_segments(h, h->dStage, nullptr, h->dY, nullptr, &segs, &owner, true);
    const size_t n1 = segs.size();
    out_segments(h, h->dStage, nullptr, h->dY, nullptr, &segs, &owner, false);
    std::vector<double> nr;
    if (int rc = norm_segments(segs, &nr, st)) return rc;
    std::vector<double> o1(nsec, 0.0), o2(nsec, 0.0);
    double t1 = 0.0, t2 = 0.0;
    for (size_t i = 0; i < segs.size(); ++i) {
      if (i < n1) {
        o1[owner[i]] += nr[2 * i + 1];
        t1 += nr[2 * i + 1];
      } else {
        o2[owner[i]] += nr[2 * i + 1];
        t2 += nr[2 * i + 1];
      }
    }
    // predicted log10 errors for levels LMIN..LPRED
    const int nl = LPRED - LMIN + 1;
    std::vector<float> pred((size_t)2 * nsec * nl, 0.0f);
    if (selector == OZ_SELECT_ANALYTIC) {
      for (int stage = 0; stage < 2; ++stage)
        for (int q = 0; q < nsec; ++q) {
          const float* f = &(stage == 0 ? f1 : f2)[(size_t)q * NF];
          const double g = effective_gap(f) + effective_gap(f + NBIN);
          for (int k = 0; k < nl; ++k)
            pred[((size_t)stage * nsec + q) * nl + k] = (float)((g - 8.0 * (LMIN + k) + 3.0) * std::log10(2.0));
        }
    } else {
      std::vector<float> X((size_t)2 * nsec * NF);
      std::copy(f1.begin(), f1.end(), X.begin());
      std::copy(f2.begin(), f2.end(), X.begin() + (size_t)nsec * NF);
      DVec<float> dX, dY;
      const int no = oz_mlp_nout(net);
      if (int rc = dX.alloc(X.size())) return rc;
      if (int rc = dY.alloc((size_t)2 * nsec * no)) return rc;
      SE_CU(cudaMemcpyAsync(dX.p, X.data(), X.size() * 4, cudaMemcpyHostToDevice, st));
      if (int rc = oz_mlp_forward(net, dX.p, 2 * nsec, dY.p, stream)) return rc;
      std::vector<float> Y((size_t)2 * nsec * no);
      SE_CU(cudaMemcpyAsync(Y.data(), dY.p, Y.size() * 4, cudaMemcpyDeviceToHost, st));
      SE_CU(cudaStreamSynchronize(st));
      for (int r = 0; r < 2 * nsec; ++r)
        for (int k = 0; k < nl; ++k) pred[(size_t)r * nl + k] = Y[(size_t)r * no + k];
    }
    // Per stage, lower levels greedily (largest carrier flops saved per predicted squared error
    // added) while sum_q (10^(pred_q + margin) |out_q|)^2 stays within (budget |out| / sqrt 2)^2.
    for (int stage = 0; stage < 2; ++stage) {
      std::vector<int>& lev = stage == 0 ? l1 : l2;
      const std::vector<double>& on = stage == 0 ? o1 : o2;
      const double target = 0.5 * budget * budget * (stage == 0 ? t1 : t2);
      std::vector<int> prob;
      std::vector<double> size(nsec, 0.0);
      for (int q = 0; q < nsec; ++q) {
        if (stage == 0 ? h->bysrc[q].empty() : h->bydst[q].empty()) continue;
        prob.push_back(q);
        const bool sw = stage == 1 && h->swap2[q];
        const double M = stage == 0 ? h->rows1[q] : (sw ? h->n[q] : h->m[q]);
        const double Nn = sw ? h->m[q] : h->n[q];
        const double K = (stage == 0 ? h->nkb1[q] : h->nkb2[q]) * (double)oz::KB;
        size[q] = 2.0 * std::ceil(M / oz::TILE_M) * oz::TILE_M * std::ceil(Nn / oz::BN) * oz::BN * K;
      }
      auto err2 = [&](int q, int l) {
        if (on[q] <= 0.0 || l > LPRED) return 0.0;
        const double e = std::pow(10.0, pred[((size_t)stage * nsec + q) * nl + (l - LMIN)] + margin);
        return e * e * on[q];
      };
      double tot = 0.0;
      for (int q : prob) tot += err2(q, smax);
      while (tot <= target) {
        int best = -1;
        double bscore = -1.0, bdelta = 0.0;
        for (int q : prob) {
          const int l = lev[q];
          if (l <= LMIN) continue;
          const double d = err2(q, l - 1) - err2(q, l);
          if (tot + d > target) continue;
          const double saved = size[q] * (double)(l * (l + 1) / 2 - (l - 1) * l / 2);
          const double score = d <= 0.0 ? 1e300 : saved / d;
          if (score > bscore) {
            bscore = score;
            best = q;
            bdelta = d;
          }
        }
        if (best < 0) break;
        lev[best] -= 1;
        tot += bdelta;
      }
    }
  }
  if (int rc = h->set_levels(l1.data(), l2.data())) return rc;
  for (int q = 0; q < nsec; ++q) {
    if (s1) s1[q] = l1[q];
    if (s2) s2[q] = l2[q];
  }
  return OZ_OK;
}
