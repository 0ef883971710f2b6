// Davidson eigensolver around heff_apply (paper, section "Theory of TNS/DMRG regarding error
// analysis": the two-site update is the lowest eigenpair of H_eff found with a Krylov method;
// section "Numerical procedure": iterations stop at a residual threshold).
//
// Everything runs on the device in FP64 except the H_eff product itself (emulated or native, as
// the handle says): block dot products with a fixed-order two-stage reduction (bitwise
// reproducible), a one-CTA cyclic Jacobi eigensolver (oz_jacobi.cuh) for the small projected matrix, residual and
// diagonal preconditioner fused in one pass, classical Gram-Schmidt applied twice, restart to the
// two lowest Ritz vectors.  The host only sequences launches and reads two scalars per iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ozdmrg.h"
#include "oz_internal.cuh"
#include "oz_jacobi.cuh"

namespace {

constexpr int DMAX = 32;      // largest subspace (and largest matrix of oz_symeig_small)
constexpr int RT = 256;       // threads of the vector kernels
constexpr int MAX_SWEEPS = 60;

#define DV_CU(call)                                                                        \
  do {                                                                                     \
    cudaError_t _e = (call);                                                               \
    if (_e != cudaSuccess)                                                                 \
      return oz::api_fail(_e == cudaErrorMemoryAllocation ? OZ_ENOMEM : OZ_ECUDA,          \
                          std::string(#call) + ": " + cudaGetErrorString(_e));             \
  } while (0)

inline long long cdiv(long long a, long long b) { return (a + b - 1) / b; }

struct VecSet {
  const double* p[DMAX];
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-partial dot products of x with Y_0..Y_{m-1}: partial[j * gridDim.x + block].
__global__ void __launch_bounds__(RT) multidot_kernel(const double* __restrict__ x, VecSet Y, int m, long long n,
                                                      double* __restrict__ partial) {
  double acc[DMAX];
#pragma unroll
  for (int j = 0; j < DMAX; ++j) acc[j] = 0.0;
  const long long stride = (long long)gridDim.x * RT;
  for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < n; i += stride) {
    const double xi = x[i];
#pragma unroll
    for (int j = 0; j < DMAX; ++j)
      if (j < m) acc[j] = fma(xi, Y.p[j][i], acc[j]);
  }
  __shared__ double red[RT / 32][DMAX];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < DMAX; ++j) {
    if (j < m) {
      double v = warp_sum(acc[j]);
      if (lane == 0) red[warp][j] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < m) {
    double s = 0.0;
    for (int w = 0; w < RT / 32; ++w) s += red[w][threadIdx.x];
    partial[(long long)threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
}

// Sum of nb partials of one quantity, in a fixed order (one block).
__device__ double block_sum_fixed(const double* __restrict__ p, int nb, double* sh) {
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += RT) s += p[b];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < RT / 32; ++w) t += sh[w];
  __syncthreads();
  return t;  // valid in thread 0
}

// out[j] = sum of the partials of quantity j, j < m.
__global__ void __launch_bounds__(RT) reduce_kernel(const double* __restrict__ partial, int nb, int m,
                                                    double* __restrict__ out) {
  __shared__ double sh[RT / 32];
  for (int j = 0; j < m; ++j) {
    double t = block_sum_fixed(partial + (long long)j * nb, nb, sh);
    if (threadIdx.x == 0) out[j] = t;
  }
}

// Projected matrix update for the new vector k: G[j][k] = G[k][j] = (v_j.w_k + v_k.w_j)/2, j <= k
// (pA: w_k against v_0..v_k; pB: v_k against w_0..w_k).
__global__ void __launch_bounds__(RT) gram_kernel(const double* __restrict__ pA, const double* __restrict__ pB,
                                                  int nb, int k, double* __restrict__ G, int ldg) {
  __shared__ double sh[RT / 32];
  for (int j = 0; j <= k; ++j) {
    double a = block_sum_fixed(pA + (long long)j * nb, nb, sh);
    double b = block_sum_fixed(pB + (long long)j * nb, nb, sh);
    if (threadIdx.x == 0) {
      double g = 0.5 * (a + b);
      G[j * ldg + k] = g;
      G[k * ldg + j] = g;
    }
  }
}

// Eigenpairs of a symmetric m x m matrix (m <= 32) by the one-CTA cyclic Jacobi solver of
// oz_jacobi.cuh.  Eigenvalues ascending into w[0..m); the first nvec eigenvectors into V (row-major
// m x nvec, leading dimension ldv).  info[0] = number of sweeps (-1: not converged).
// Warm start (Qin, qin_m > 0): when the matrix is the previous one (qin_m x qin_m, diagonalised by
// the orthogonal Qin) bordered by new rows and columns, Jacobi starts from A = W^T G W with
// W = Qin (+) identity -- diagonal but for the border -- and accumulates its rotations onto W, so a
// subspace that grows by one vector per iteration needs one or two sweeps instead of a full solve.
// Qout (may alias Qin; leading dimension DMAX) receives all m eigenvectors, unsorted.
__global__ void __launch_bounds__(RT) symeig_kernel(const double* __restrict__ Gin, int m, int ldg,
                                                    double* __restrict__ w, double* __restrict__ V, int ldv,
                                                    int nvec, int* __restrict__ info, const double* Qin = nullptr,
                                                    int qin_m = 0, double* Qout = nullptr) {
  __shared__ double A[DMAX][DMAX + 1], Q[DMAX][DMAX + 1], Tm[DMAX][DMAX + 1];
  __shared__ double cs[DMAX / 2], sn[DMAX / 2];
  __shared__ int pp[DMAX / 2], qq[DMAX / 2];
  __shared__ double red[2 * (RT / 32)];
  __shared__ int stop;
  __shared__ int order[DMAX];
  const int tid = threadIdx.x;
  for (int idx = tid; idx < m * m; idx += RT) {
    int i = idx / m, j = idx % m;
    A[i][j] = 0.5 * (Gin[i * ldg + j] + Gin[j * ldg + i]);
  }
  const bool warm = Qin != nullptr && qin_m > 0 && qin_m <= m;
  if (warm) {
    for (int idx = tid; idx < m * m; idx += RT) {
      const int i = idx / m, j = idx % m;
      Q[i][j] = (i < qin_m && j < qin_m) ? Qin[i * DMAX + j] : (i == j ? 1.0 : 0.0);
    }
    __syncthreads();
    for (int idx = tid; idx < m * m; idx += RT) {  // Tm = G W
      const int i = idx / m, j = idx % m;
      double acc = 0.0;
      for (int k = 0; k < m; ++k) acc = fma(A[i][k], Q[k][j], acc);
      Tm[i][j] = acc;
    }
    __syncthreads();
    for (int idx = tid; idx < m * m; idx += RT) {  // A = W^T Tm
      const int i = idx / m, j = idx % m;
      double acc = 0.0;
      for (int k = 0; k < m; ++k) acc = fma(Q[k][i], Tm[k][j], acc);
      A[i][j] = acc;
    }
    __syncthreads();
    for (int idx = tid; idx < m * m; idx += RT) {  // symmetric to the last bit
      const int i = idx / m, j = idx % m;
      Tm[i][j] = 0.5 * (A[i][j] + A[j][i]);
    }
    __syncthreads();
    for (int idx = tid; idx < m * m; idx += RT) A[idx / m][idx % m] = Tm[idx / m][idx % m];
  }
  __syncthreads();
  const int sweeps =
      oz::jacobi_smem(&A[0][0], &Q[0][0], DMAX + 1, m, {cs, sn, pp, qq, red, &stop}, MAX_SWEEPS, !warm,
                      warm ? 1e-18 : 0.0);
  oz::jacobi_order(&A[0][0], DMAX + 1, m, false, order);
  if (tid == 0) info[0] = sweeps;
  for (int i = tid; i < m; i += RT) w[i] = A[order[i]][order[i]];
  const int nv = min(nvec, m);
  for (int idx = tid; idx < m * nv; idx += RT) {
    const int i = idx / nv, k = idx % nv;
    V[i * ldv + k] = Q[i][order[k]];
  }
  if (Qout)
    for (int idx = tid; idx < m * m; idx += RT) Qout[(idx / m) * DMAX + idx % m] = Q[idx / m][idx % m];
}

// Ritz vector, residual and preconditioned correction in one pass (y = first eigenvector of the
// projected matrix, theta = its eigenvalue):
//   x = V y, r = W y - theta x, d = r / (theta - diag) with |theta - diag| floored at 1e-12.
// Block partials of |r|^2 into partial[block].
__global__ void __launch_bounds__(RT) ritz_kernel(VecSet Vs, VecSet Ws, int m, const double* __restrict__ eig,
                                                  const double* __restrict__ diag, long long n,
                                                  double* __restrict__ x, double* __restrict__ d,
                                                  double* __restrict__ partial) {
  __shared__ double y[DMAX];
  __shared__ double sh[RT / 32];
  if (threadIdx.x < m) y[threadIdx.x] = eig[DMAX + threadIdx.x * 2];
  __syncthreads();
  const double theta = eig[0];
  double acc = 0.0;
  const long long stride = (long long)gridDim.x * RT;
  for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < n; i += stride) {
    double xv = 0.0, wv = 0.0;
    for (int j = 0; j < m; ++j) {
      xv = fma(y[j], Vs.p[j][i], xv);
      wv = fma(y[j], Ws.p[j][i], wv);
    }
    const double r = wv - theta * xv;
    double den = theta - diag[i];
    if (fabs(den) < 1e-12) den = den < 0.0 ? -1e-12 : 1e-12;
    x[i] = xv;
    d[i] = r / den;
    acc = fma(r, r, acc);
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < RT / 32; ++k) s += sh[k];
    partial[blockIdx.x] = s;
  }
}

// Restart: out0 = sum_j Y[j][0] S_j, out1 = sum_j Y[j][1] S_j for the V and the W sets.
__global__ void __launch_bounds__(RT) restart_kernel(VecSet Vs, VecSet Ws, int m, const double* __restrict__ eig,
                                                     long long n, double* __restrict__ v0, double* __restrict__ v1,
                                                     double* __restrict__ w0, double* __restrict__ w1) {
  __shared__ double y[DMAX][2];
  if (threadIdx.x < m) {
    y[threadIdx.x][0] = eig[DMAX + threadIdx.x * 2];
    y[threadIdx.x][1] = eig[DMAX + threadIdx.x * 2 + 1];
  }
  __syncthreads();
  const long long stride = (long long)gridDim.x * RT;
  for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < n; i += stride) {
    double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
    for (int j = 0; j < m; ++j) {
      const double v = Vs.p[j][i], wv = Ws.p[j][i];
      a0 = fma(y[j][0], v, a0);
      a1 = fma(y[j][1], v, a1);
      b0 = fma(y[j][0], wv, b0);
      b1 = fma(y[j][1], wv, b1);
    }
    v0[i] = a0;
    v1[i] = a1;
    w0[i] = b0;
    w1[i] = b1;
  }
}

// One Gram-Schmidt pass: d -= sum_j coef[j] V_j.
__global__ void __launch_bounds__(RT) project_out_kernel(double* __restrict__ d, VecSet Vs, int m,
                                                         const double* __restrict__ coef, long long n) {
  __shared__ double c[DMAX];
  if (threadIdx.x < m) c[threadIdx.x] = coef[threadIdx.x];
  __syncthreads();
  const long long stride = (long long)gridDim.x * RT;
  for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < n; i += stride) {
    double s = 0.0;
    for (int j = 0; j < m; ++j) s = fma(c[j], Vs.p[j][i], s);
    d[i] = d[i] - s;
  }
}

// dst = src / sqrt(*nrm2) unless the norm is below `floor` or not finite; then flag[0] = 1 and
// dst is left as it was.
__global__ void __launch_bounds__(RT) normalize_kernel(const double* __restrict__ src, double* __restrict__ dst,
                                                       long long n, const double* __restrict__ nrm2, double floor,
                                                       int* __restrict__ flag) {
  const double nd = sqrt(*nrm2);
  if (!(nd >= floor) || !isfinite(nd)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) flag[0] = 1;
    return;
  }
  const long long stride = (long long)gridDim.x * RT;
  for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < n; i += stride) dst[i] = src[i] / nd;
}

// x = sum_j y[j * ystride] S_j (Ritz vector of a Krylov basis).
__global__ void __launch_bounds__(RT) combine_kernel(VecSet Vs, int m, const double* __restrict__ y, int ystride,
                                                     long long n, double* __restrict__ x) {
  __shared__ double c[DMAX];
  if (threadIdx.x < m) c[threadIdx.x] = y[threadIdx.x * ystride];
  __syncthreads();
  const long long stride = (long long)gridDim.x * RT;
  for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < n; i += stride) {
    double s = 0.0;
    for (int j = 0; j < m; ++j) s = fma(c[j], Vs.p[j][i], s);
    x[i] = s;
  }
}

// Lanczos tridiagonal entries: T[j][j] = alpha, T[j][j+1] = T[j+1][j] = sqrt(beta2) (when j+1 < ld).
__global__ void set_tri_kernel(double* __restrict__ T, int ld, int j, const double* __restrict__ alpha,
                               const double* __restrict__ beta2, double* __restrict__ beta_out) {
  if (threadIdx.x == 0) {
    T[j * ld + j] = *alpha;
    const double b = sqrt(*beta2);
    *beta_out = b;
    if (j + 1 < ld) {
      T[j * ld + j + 1] = b;
      T[(j + 1) * ld + j] = b;
    }
  }
}

// ---- diagonal of H_eff
struct DiagTask {
  const double* L;
  const double* R;
  double coef;
  int m, n;
  long long offl, offr;
};

__global__ void diag_extract_kernel(const DiagTask* __restrict__ t, double* __restrict__ dl,
                                    double* __restrict__ dr) {
  const DiagTask d = t[blockIdx.x];
  for (int i = threadIdx.x; i < d.m; i += blockDim.x) dl[d.offl + i] = d.L[(long long)i * (d.m + 1)];
  for (int j = threadIdx.x; j < d.n; j += blockDim.x) dr[d.offr + j] = d.coef * d.R[(long long)j * (d.n + 1)];
}

// diag[(q,i,j)] = sum over the diagonal tasks t of sector q (in task order) of dl_t[i] dr_t[j].
__global__ void diag_sum_kernel(const long long* __restrict__ psioff, const int* __restrict__ ncols, int nsec,
                                const int* __restrict__ tfirst, const long long* __restrict__ offl,
                                const long long* __restrict__ offr, const double* __restrict__ dl,
                                const double* __restrict__ dr, double* __restrict__ out) {
  const long long dim = psioff[nsec];
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < dim; idx += stride) {
    int lo = 0, hi = nsec - 1;  // sector q with psioff[q] <= idx < psioff[q+1]
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (psioff[mid] <= idx) lo = mid;
      else hi = mid - 1;
    }
    const int q = lo;
    const long long e = idx - psioff[q];
    const int nq = ncols[q];
    const int i = (int)(e / nq), j = (int)(e % nq);
    double s = 0.0;
    for (int t = tfirst[q]; t < tfirst[q + 1]; ++t) s = fma(dl[offl[t] + i], dr[offr[t] + j], s);
    out[idx] = s;
  }
}

int grid_for(long long n, int nsm) { return (int)std::max(1ll, std::min<long long>(4ll * nsm, cdiv(n, RT))); }

}  // namespace

namespace oz {
int build_heff_diag(int nsec, const int* m, const int* n, const long long* psioff, int ntask, const oz_task* tasks,
                    double* d_diag) {
  std::vector<int> tfirst(nsec + 1, 0);
  std::vector<std::vector<int>> per(nsec);
  for (int t = 0; t < ntask; ++t)
    if (tasks[t].src == tasks[t].dst) per[tasks[t].src].push_back(t);
  std::vector<DiagTask> dt;
  std::vector<long long> offl, offr;
  long long nl = 0, nr = 0;
  for (int q = 0; q < nsec; ++q) {
    tfirst[q] = (int)dt.size();
    for (int t : per[q]) {
      dt.push_back({tasks[t].d_L, tasks[t].d_R, tasks[t].coef, m[q], n[q], nl, nr});
      offl.push_back(nl);
      offr.push_back(nr);
      nl += m[q];
      nr += n[q];
    }
  }
  tfirst[nsec] = (int)dt.size();
  std::vector<int> nc(n, n + nsec);
  const long long dim = psioff[nsec];
  // one allocation for every table
  size_t b_dt = dt.size() * sizeof(DiagTask), b_po = (nsec + 1) * 8, b_nc = nsec * 4, b_tf = (nsec + 1) * 4;
  size_t b_ol = offl.size() * 8, b_or = offr.size() * 8, b_dl = nl * 8, b_dr = nr * 8;
  auto a = [](size_t x) { return (x + 255) & ~(size_t)255; };
  size_t total = a(b_dt) + a(b_po) + a(b_nc) + a(b_tf) + a(b_ol) + a(b_or) + a(b_dl) + a(b_dr) + 256;
  char* buf = nullptr;
  DV_CU(cudaMalloc(&buf, total));
  char* p = buf;
  auto take = [&](size_t b) {
    char* r = p;
    p += a(b);
    return r;
  };
  DiagTask* d_dt = (DiagTask*)take(b_dt);
  long long* d_po = (long long*)take(b_po);
  int* d_nc = (int*)take(b_nc);
  int* d_tf = (int*)take(b_tf);
  long long* d_ol = (long long*)take(b_ol);
  long long* d_or = (long long*)take(b_or);
  double* d_dl = (double*)take(b_dl);
  double* d_dr = (double*)take(b_dr);
  cudaError_t e = cudaSuccess;
  if (!dt.empty()) {
    e = cudaMemcpy(d_dt, dt.data(), b_dt, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_ol, offl.data(), b_ol, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_or, offr.data(), b_or, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMemcpy(d_po, psioff, b_po, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_nc, nc.data(), b_nc, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_tf, tfirst.data(), b_tf, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !dt.empty()) {
    diag_extract_kernel<<<(unsigned)dt.size(), 128>>>(d_dt, d_dl, d_dr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    unsigned g = (unsigned)std::max(1ll, std::min(cdiv(dim, 256), 1ll << 16));
    diag_sum_kernel<<<g, 256>>>(d_po, d_nc, nsec, d_tf, d_ol, d_or, d_dl, d_dr, d_diag);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(buf);
  if (e != cudaSuccess) return api_fail(OZ_ECUDA, std::string("H_eff diagonal: ") + cudaGetErrorString(e));
  return OZ_OK;
}
}  // namespace oz

// ------------------------------------------------------------------------------------------------
// Davidson state
// ------------------------------------------------------------------------------------------------
struct oz_davidson_s {
  oz_heff* h = nullptr;
  int device = 0, nsm = 0, nb = 1, max_sub = 24;
  long long n = 0, ldn = 0;
  double tol = 1e-10;
  char* mem = nullptr;
  std::vector<double*> vphys, wphys;  // physical slots
  std::vector<int> vmap, wmap;        // logical subspace vector -> physical slot
  double *x = nullptr, *G = nullptr, *eig = nullptr, *pA = nullptr, *pB = nullptr, *scal = nullptr;
  double* Qw = nullptr;  // eigenvectors of the last projected matrix (warm start of the next one)
  int qw_m = 0;          // its order (0: none)
  int* flag = nullptr;  // [0] breakdown / bad norm, [1] Jacobi sweeps
  double* host = nullptr;  // page-locked: theta, theta1, |r|^2, flag
  int m = 0;
  bool started = false, converged = false;
  double theta = 0.0, resid = 0.0;
  int iters = 0;

  VecSet set(const std::vector<double*>& phys, const std::vector<int>& map, int count) const {
    VecSet s{};
    for (int j = 0; j < count; ++j) s.p[j] = phys[map[j]];
    return s;
  }
  int free_slot(const std::vector<int>& map, std::initializer_list<int> also) const {
    for (int p = 0; p < (int)vphys.size(); ++p) {
      bool used = std::find(map.begin(), map.end(), p) != map.end();
      for (int a : also) used = used || a == p;
      if (!used) return p;
    }
    return -1;
  }
  // partial dots of x against the first `count` vectors of a set, into `part`
  int dots(const double* xv, VecSet s, int count, double* part, cudaStream_t st) {
    multidot_kernel<<<nb, RT, 0, st>>>(xv, s, count, n, part);
    DV_CU(cudaGetLastError());
    return OZ_OK;
  }
  int norm_into(const double* src, double* dst, double floor, cudaStream_t st) {
    VecSet one{};
    one.p[0] = src;
    DV_CU(cudaMemsetAsync(flag, 0, 4, st));
    if (int rc = dots(src, one, 1, pA, st)) return rc;
    reduce_kernel<<<1, RT, 0, st>>>(pA, nb, 1, scal + 8);
    normalize_kernel<<<nb, RT, 0, st>>>(src, dst, n, scal + 8, floor, flag);
    DV_CU(cudaGetLastError());
    return OZ_OK;
  }
  // G entries of logical vector k against 0..k
  int gram(int k, cudaStream_t st) {
    VecSet vs = set(vphys, vmap, k + 1), ws = set(wphys, wmap, k + 1);
    if (int rc = dots(wphys[wmap[k]], vs, k + 1, pA, st)) return rc;
    if (int rc = dots(vphys[vmap[k]], ws, k + 1, pB, st)) return rc;
    gram_kernel<<<1, RT, 0, st>>>(pA, pB, nb, k, G, DMAX);
    DV_CU(cudaGetLastError());
    return OZ_OK;
  }
  int read_flag(cudaStream_t st, int* f) {
    DV_CU(cudaMemcpyAsync(host + 3, flag, 4, cudaMemcpyDeviceToHost, st));
    DV_CU(cudaStreamSynchronize(st));
    std::memcpy(f, host + 3, 4);
    return OZ_OK;
  }
};

extern "C" int oz_davidson_create(oz_heff* h, int max_sub, double tol, oz_davidson** out) {
  if (!out) return oz::api_fail(OZ_EINVAL, "out is null");
  *out = nullptr;
  if (!h) return oz::api_fail(OZ_EINVAL, "handle is null");
  if (max_sub < 3 || max_sub > DMAX) return oz::api_fail(OZ_EINVAL, "max_sub must be in 3..32");
  if (!(tol > 0.0)) return oz::api_fail(OZ_EINVAL, "tol must be positive");
  DV_CU(cudaSetDevice(oz::heff_device(h)));
  oz_davidson* d = new oz_davidson_s();
  d->h = h;
  d->device = oz::heff_device(h);
  d->nsm = oz::heff_nsm(h);
  d->n = oz::heff_dim(h);
  d->ldn = cdiv(d->n, 32) * 32;
  d->nb = grid_for(d->n, d->nsm);
  d->max_sub = max_sub;
  d->tol = tol;
  const int nslot = max_sub + 3;
  const size_t vec = (size_t)d->ldn * 8;
  const size_t small = 2 * (size_t)DMAX * DMAX * 8 + (size_t)DMAX * 3 * 8 + 2 * (size_t)DMAX * d->nb * 8 + 64 * 8 + 64;
  const size_t total = (2 * (size_t)nslot + 1) * vec + small + 1024;
  cudaError_t e = cudaMalloc(&d->mem, total);
  if (e != cudaSuccess) {
    delete d;
    return oz::api_fail(e == cudaErrorMemoryAllocation ? OZ_ENOMEM : OZ_ECUDA, "Davidson workspace cudaMalloc");
  }
  e = cudaMallocHost(&d->host, 64);
  if (e != cudaSuccess) {
    cudaFree(d->mem);
    delete d;
    return oz::api_fail(OZ_ECUDA, "Davidson cudaMallocHost");
  }
  char* p = d->mem;
  for (int s = 0; s < nslot; ++s, p += vec) d->vphys.push_back((double*)p);
  for (int s = 0; s < nslot; ++s, p += vec) d->wphys.push_back((double*)p);
  d->x = (double*)p;
  p += vec;
  d->G = (double*)p;
  p += (size_t)DMAX * DMAX * 8;
  d->Qw = (double*)p;
  p += (size_t)DMAX * DMAX * 8;
  d->eig = (double*)p;
  p += (size_t)DMAX * 3 * 8;
  d->pA = (double*)p;
  p += (size_t)DMAX * d->nb * 8;
  d->pB = (double*)p;
  p += (size_t)DMAX * d->nb * 8;
  d->scal = (double*)p;
  p += 64 * 8;
  d->flag = (int*)p;
  e = cudaMemset(d->G, 0, (size_t)DMAX * DMAX * 8);
  if (e != cudaSuccess) {
    cudaFreeHost(d->host);
    cudaFree(d->mem);
    delete d;
    return oz::api_fail(OZ_ECUDA, "cudaMemset");
  }
  *out = d;
  return OZ_OK;
}

extern "C" int oz_davidson_destroy(oz_davidson* d) {
  if (!d) return OZ_OK;
  cudaSetDevice(d->device);
  cudaDeviceSynchronize();
  if (d->host) cudaFreeHost(d->host);
  if (d->mem) cudaFree(d->mem);
  delete d;
  return OZ_OK;
}

extern "C" int davidson_start(oz_davidson* d, const double* d_x0, oz_stream_t stream) {
  if (!d || !d_x0) return oz::api_fail(OZ_EINVAL, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  d->vmap.assign(1, 0);
  d->wmap.assign(1, 0);
  d->m = 1;
  d->qw_m = 0;
  d->started = d->converged = false;
  d->iters = 0;
  DV_CU(cudaMemsetAsync(d->flag, 0, 8, st));
  if (int rc = d->norm_into(d_x0, d->vphys[0], DBL_MIN, st)) return rc;
  int f = 0;
  if (int rc = d->read_flag(st, &f)) return rc;
  if (f) return oz::api_fail(OZ_EINVAL, "the start vector has zero or non-finite norm");
  if (int rc = heff_apply(d->h, d->vphys[0], d->wphys[0], stream)) return rc;
  if (int rc = d->gram(0, st)) return rc;
  d->started = true;
  return OZ_OK;
}

extern "C" int davidson_step(oz_davidson* d, double* theta, double* resid, int* converged, oz_stream_t stream) {
  if (!d || !theta || !resid || !converged) return oz::api_fail(OZ_EINVAL, "null argument");
  if (!d->started) return oz::api_fail(OZ_EINVAL, "davidson_start has not been called");
  cudaStream_t st = (cudaStream_t)stream;
  if (d->converged) {
    *theta = d->theta;
    *resid = d->resid;
    *converged = 1;
    return OZ_OK;
  }
  const int m = d->m;
  d->iters += 1;
  // lowest eigenpairs of the projected matrix, Ritz vector, residual, correction
  // the subspace grew by one vector since the last solve unless it was restarted: warm start
  const bool warm = d->qw_m > 0 && d->qw_m == m - 1;
  symeig_kernel<<<1, RT, 0, st>>>(d->G, m, DMAX, d->eig, d->eig + DMAX, 2, 2, d->flag + 1, warm ? d->Qw : nullptr,
                                  warm ? d->qw_m : 0, d->Qw);
  DV_CU(cudaGetLastError());
  d->qw_m = m;
  const int fd = d->free_slot(d->vmap, {});
  VecSet vs = d->set(d->vphys, d->vmap, m), ws = d->set(d->wphys, d->wmap, m);
  ritz_kernel<<<d->nb, RT, 0, st>>>(vs, ws, m, d->eig, oz::heff_diag_ptr(d->h), d->n, d->x, d->vphys[fd], d->pA);
  DV_CU(cudaGetLastError());
  reduce_kernel<<<1, RT, 0, st>>>(d->pA, d->nb, 1, d->scal);
  DV_CU(cudaMemcpyAsync(d->host, d->eig, 16, cudaMemcpyDeviceToHost, st));
  DV_CU(cudaMemcpyAsync(d->host + 2, d->scal, 8, cudaMemcpyDeviceToHost, st));
  DV_CU(cudaStreamSynchronize(st));
  d->theta = d->host[0];
  d->resid = std::sqrt(d->host[2]);
  *theta = d->theta;
  *resid = d->resid;
  *converged = 0;
  if (!std::isfinite(d->theta) || !std::isfinite(d->resid))
    return oz::api_fail(OZ_ENONFINITE, "the Ritz value or residual is not finite");
  if (d->resid <= d->tol) {
    d->converged = true;
    *converged = 1;
    return OZ_OK;
  }
  if (m >= d->max_sub) {
    // restart from the two lowest Ritz vectors
    const int a = d->free_slot(d->vmap, {fd}), b = d->free_slot(d->vmap, {fd, a});
    const int wa = d->free_slot(d->wmap, {}), wb = d->free_slot(d->wmap, {wa});
    restart_kernel<<<d->nb, RT, 0, st>>>(vs, ws, m, d->eig, d->n, d->vphys[a], d->vphys[b], d->wphys[wa],
                                         d->wphys[wb]);
    DV_CU(cudaGetLastError());
    d->vmap = {a, b};
    d->wmap = {wa, wb};
    d->m = 2;
    d->qw_m = 0;  // a new basis: the next projected matrix is solved from scratch
    if (int rc = d->gram(0, st)) return rc;
    if (int rc = d->gram(1, st)) return rc;
  }
  // classical Gram-Schmidt, twice, then normalise
  const int mc = d->m;
  VecSet vc = d->set(d->vphys, d->vmap, mc);
  double* dv = d->vphys[fd];
  for (int pass = 0; pass < 2; ++pass) {
    if (int rc = d->dots(dv, vc, mc, d->pA, st)) return rc;
    reduce_kernel<<<1, RT, 0, st>>>(d->pA, d->nb, mc, d->scal + 16);
    project_out_kernel<<<d->nb, RT, 0, st>>>(dv, vc, mc, d->scal + 16, d->n);
    DV_CU(cudaGetLastError());
  }
  if (int rc = d->norm_into(dv, dv, 1e-14, st)) return rc;
  int f = 0;
  if (int rc = d->read_flag(st, &f)) return rc;
  if (f) return oz::api_fail(OZ_ENOCONV, "Davidson correction vanished after orthogonalisation");
  const int wf = d->free_slot(d->wmap, {});
  if (int rc = heff_apply(d->h, dv, d->wphys[wf], stream)) return rc;
  d->vmap.push_back(fd);
  d->wmap.push_back(wf);
  d->m = mc + 1;
  if (int rc = d->gram(d->m - 1, st)) return rc;
  return OZ_OK;
}

extern "C" int davidson_ritz(oz_davidson* d, double* d_x, oz_stream_t stream) {
  if (!d || !d_x) return oz::api_fail(OZ_EINVAL, "null argument");
  if (!d->started || d->iters == 0) return oz::api_fail(OZ_EINVAL, "no Ritz vector yet (call davidson_step)");
  cudaStream_t st = (cudaStream_t)stream;
  if (int rc = d->norm_into(d->x, d_x, DBL_MIN, st)) return rc;
  int f = 0;
  if (int rc = d->read_flag(st, &f)) return rc;
  if (f) return oz::api_fail(OZ_ENONFINITE, "the Ritz vector has zero or non-finite norm");
  return OZ_OK;
}

extern "C" int davidson_solve(oz_heff* h, double* d_psi, double tol, int max_iter, double* energy, int* iters,
                              oz_stream_t stream) {
  if (!h || !d_psi || !energy || !iters) return oz::api_fail(OZ_EINVAL, "null argument");
  if (max_iter < 1) return oz::api_fail(OZ_EINVAL, "max_iter must be positive");
  oz_davidson* d = nullptr;
  if (int rc = oz_davidson_create(h, 24, tol, &d)) return rc;
  int rc = davidson_start(d, d_psi, stream);
  int conv = 0;
  double th = 0.0, rs = 0.0;
  while (rc == OZ_OK && !conv && d->iters < max_iter) rc = davidson_step(d, &th, &rs, &conv, stream);
  if (d->iters > 0 && (rc == OZ_OK || rc == OZ_ENOCONV)) {
    int r2 = davidson_ritz(d, d_psi, stream);
    if (rc == OZ_OK) rc = r2;
  }
  *energy = th;
  *iters = d->iters;
  if (rc == OZ_OK && !conv) rc = oz::api_fail(OZ_ENOCONV, "Davidson reached max_iter without convergence");
  oz_davidson_destroy(d);
  return rc;
}

extern "C" int oz_symeig_small(const double* d_G, int m, int ldg, double* d_w, double* d_V, int ldv,
                               oz_stream_t stream) {
  if (!d_G || !d_w || !d_V) return oz::api_fail(OZ_EINVAL, "null argument");
  if (m < 1 || m > DMAX) return oz::api_fail(OZ_EINVAL, "m must be in 1..32");
  if (ldg < m || ldv < m) return oz::api_fail(OZ_EINVAL, "leading dimension too small");
  cudaStream_t st = (cudaStream_t)stream;
  int* info = nullptr;
  DV_CU(cudaMalloc(&info, 4));
  symeig_kernel<<<1, RT, 0, st>>>(d_G, m, ldg, d_w, d_V, ldv, m, info);
  cudaError_t e = cudaGetLastError();
  int sweeps = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&sweeps, info, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(info);
  if (e != cudaSuccess) return oz::api_fail(OZ_ECUDA, cudaGetErrorString(e));
  if (sweeps < 0) return oz::api_fail(OZ_ENOCONV, "Jacobi sweeps did not converge");
  return OZ_OK;
}

// Lanczos with full reorthogonalisation (classical Gram-Schmidt twice against the whole basis)
// and explicit restart from the Ritz vector every `krylov` vectors; convergence when the
// residual estimate beta_j |y_j| of the lowest Ritz pair is at most eps.
extern "C" int lanczos_solve(oz_heff* h, double* d_psi, double eps, int max_iter, int krylov, double* energy,
                             int* iters, oz_stream_t stream) {
  if (!h || !d_psi || !energy || !iters) return oz::api_fail(OZ_EINVAL, "null argument");
  if (max_iter < 1 || krylov < 2 || krylov > DMAX - 1 || !(eps > 0.0))
    return oz::api_fail(OZ_EINVAL, "max_iter >= 1, krylov in 2..31 and eps > 0 required");
  cudaStream_t st = (cudaStream_t)stream;
  oz_davidson* d = nullptr;
  if (int rc = oz_davidson_create(h, krylov + 1, eps, &d)) return rc;
  struct Guard {
    oz_davidson* d;
    ~Guard() { oz_davidson_destroy(d); }
  } guard{d};
  d->vmap.clear();
  for (int j = 0; j <= krylov; ++j) d->vmap.push_back(j);
  double* w = d->wphys[0];
  double* T = d->G;
  const long long n = d->n;
  if (int rc = d->norm_into(d_psi, d->vphys[0], DBL_MIN, st)) return rc;
  int f = 0;
  if (int rc = d->read_flag(st, &f)) return rc;
  if (f) return oz::api_fail(OZ_EINVAL, "the start vector has zero or non-finite norm");
  int total = 0, conv = 0;
  double theta = 0.0;
  while (true) {
    DV_CU(cudaMemsetAsync(T, 0, (size_t)DMAX * DMAX * 8, st));
    d->qw_m = 0;
    int j = 0;
    bool restart = false, stop = false;
    for (; j < krylov; ++j) {
      if (int rc = heff_apply(h, d->vphys[j], w, stream)) return rc;
      VecSet one{};
      one.p[0] = d->vphys[j];
      if (int rc = d->dots(w, one, 1, d->pA, st)) return rc;
      reduce_kernel<<<1, RT, 0, st>>>(d->pA, d->nb, 1, d->scal + 4);  // alpha_j
      VecSet vc = d->set(d->vphys, d->vmap, j + 1);
      for (int pass = 0; pass < 2; ++pass) {
        if (int rc = d->dots(w, vc, j + 1, d->pA, st)) return rc;
        reduce_kernel<<<1, RT, 0, st>>>(d->pA, d->nb, j + 1, d->scal + 16);
        project_out_kernel<<<d->nb, RT, 0, st>>>(w, vc, j + 1, d->scal + 16, n);
      }
      VecSet ww{};
      ww.p[0] = w;
      if (int rc = d->dots(w, ww, 1, d->pA, st)) return rc;
      reduce_kernel<<<1, RT, 0, st>>>(d->pA, d->nb, 1, d->scal + 5);  // beta_j^2
      set_tri_kernel<<<1, 32, 0, st>>>(T, DMAX, j, d->scal + 4, d->scal + 5, d->scal + 6);
      // T grows by one row and column per step: warm start from the last solve's eigenvectors
      const bool warm = d->qw_m > 0 && d->qw_m == j;
      symeig_kernel<<<1, RT, 0, st>>>(T, j + 1, DMAX, d->eig, d->eig + DMAX, 2, 1, d->flag + 1,
                                      warm ? d->Qw : nullptr, warm ? d->qw_m : 0, d->Qw);
      DV_CU(cudaGetLastError());
      d->qw_m = j + 1;
      DV_CU(cudaMemcpyAsync(d->host, d->eig, 8, cudaMemcpyDeviceToHost, st));
      DV_CU(cudaMemcpyAsync(d->host + 1, d->scal + 6, 8, cudaMemcpyDeviceToHost, st));
      DV_CU(cudaMemcpyAsync(d->host + 2, d->eig + DMAX + 2 * j, 8, cudaMemcpyDeviceToHost, st));
      DV_CU(cudaStreamSynchronize(st));
      theta = d->host[0];
      const double beta = d->host[1], est = beta * std::fabs(d->host[2]);
      ++total;
      if (!std::isfinite(theta) || !std::isfinite(beta))
        return oz::api_fail(OZ_ENONFINITE, "the Lanczos recurrence produced a non-finite value");
      if (est <= eps) {
        conv = 1;
        stop = true;
      } else if (total >= max_iter || beta < 1e-14) {
        stop = true;  // iteration limit, or an invariant subspace that still misses eps
      } else if (j + 1 == krylov) {
        restart = true;
      } else {
        // v_{j+1} = w / beta
        normalize_kernel<<<d->nb, RT, 0, st>>>(w, d->vphys[j + 1], n, d->scal + 5, 0.0, d->flag);
        DV_CU(cudaGetLastError());
        continue;
      }
      break;
    }
    // Ritz vector of the basis so far: x = V y, normalised into v_0 (and into psi at the end)
    VecSet vc = d->set(d->vphys, d->vmap, j + 1);
    combine_kernel<<<d->nb, RT, 0, st>>>(vc, j + 1, d->eig + DMAX, 2, n, d->x);
    DV_CU(cudaGetLastError());
    if (int rc = d->norm_into(d->x, stop ? d_psi : d->vphys[0], DBL_MIN, st)) return rc;
    if (stop || !restart) break;
  }
  *energy = theta;
  *iters = total;
  return conv ? OZ_OK : oz::api_fail(OZ_ENOCONV, "Lanczos stopped before its residual estimate reached eps");
}
