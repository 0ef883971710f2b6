// Two-site DMRG sweep around heff_apply (paper, section "Theory of TNS/DMRG regarding error
// analysis": sweep the chain; at every bond solve the lowest eigenpair of the effective
// Hamiltonian of the two-site tensor with a Krylov method, then truncate it by a singular value
// decomposition and renormalise the block operators; the energy approaches the exact ground
// state from above).
//
// Operators: the MPO of oz_mpo.cuh.  A block (sites 0..b on the left, b+1..L-1 on the right)
// holds, for every MPO state w on its boundary bond, the block-sparse matrix of the partial
// Hamiltonian string w in its basis (the environment).  At bond (i, i+1):
//   L_w = sum_w' E_left[w'] (x) W_i[w', w]      on LE = left block (x) site i,
//   R_w = sum_w'' W_{i+1}[w, w''] (x) E_right[w''] on RE = site i+1 (x) right block,
//   H_eff = sum_w L_w (x) R_w,  i.e.  Y = sum_w L_w psi R_w^T  over quantum-number sectors,
// which is exactly the task list of heff_apply (emulated or native, as the precision says).
// Truncation and renormalisation follow the same readings as the explicit-basis oracle: keep the
// whole enlarged block when it has at most D states, else the largest eigenvalues (> 1e-14, at
// most D, never cutting a group of equal ones) of the per-sector reduced density matrices; the new
// environment is U^T L_w U (U^T... on the right).  Everything on the device is FP64 except the
// emulated H_eff products: a block Kronecker-accumulate kernel builds L_w and R_w, a one-CTA
// Jacobi kernel per sector diagonalises the density matrices, a list-driven small-GEMM kernel does
// the density matrices and the projections, and the Davidson solver of oz_davidson.cu runs the
// eigenproblem.  The host builds index tables and picks the kept states.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "ozdmrg.h"
#include "oz_gemm.cuh"
#include "oz_internal.cuh"
#include "oz_jacobi.cuh"
#include "oz_mpo.cuh"

using oz::QN;

namespace {

constexpr int EIG_MAX = 112;          // largest density-matrix sector of the on-chip eigensolver
constexpr int EIG_MAX_GLOBAL = 1024;  // largest sector of the global-memory fallback
constexpr int EIG_THREADS = 256;
constexpr double LAMBDA_MIN = 1e-14;  // density-matrix eigenvalues kept must exceed this

#define DM_CU(call)                                                                 \
  do {                                                                              \
    cudaError_t _e = (call);                                                        \
    if (_e != cudaSuccess)                                                          \
      return oz::api_fail(_e == cudaErrorMemoryAllocation ? OZ_ENOMEM : OZ_ECUDA,   \
                          std::string(#call) + ": " + cudaGetErrorString(_e));      \
  } while (0)
#define DM_RC(call)                 \
  do {                              \
    int _rc = (call);               \
    if (_rc != OZ_OK) return _rc;   \
  } while (0)

inline bool same(QN a, QN b) { return a.n == b.n && a.s == b.s; }
inline QN add(QN a, QN b) { return {a.n + b.n, a.s + b.s}; }
inline QN sub(QN a, QN b) { return {a.n - b.n, a.s - b.s}; }

// ------------------------------------------------------------------------------------------------
// kernels
// ------------------------------------------------------------------------------------------------
struct KronJob {
  long long dst;    // element offset of the region's first element in the destination arena
  long long src;    // element offset of the source block in the source arena
  int ldd, lds, rows, cols;
  double scale;
};

// One CTA per destination region: region = sum of scale * source block over its jobs, in order.
__global__ void kron_accumulate_kernel(const KronJob* __restrict__ jobs, const int* __restrict__ gstart,
                                       const double* __restrict__ src, double* __restrict__ dst) {
  const int g0 = gstart[blockIdx.x], g1 = gstart[blockIdx.x + 1];
  const KronJob J0 = jobs[g0];
  for (int idx = threadIdx.x; idx < J0.rows * J0.cols; idx += blockDim.x) {
    const int r = idx / J0.cols, c = idx % J0.cols;
    double acc = 0.0;
    for (int g = g0; g < g1; ++g) {
      const KronJob& J = jobs[g];
      acc = fma(J.scale, src[J.src + (long long)r * J.lds + c], acc);
    }
    dst[J0.dst + (long long)r * J0.ldd + c] = acc;
  }
}

struct GemmJob {
  const double* A;
  const double* B;
  double* C;
  int M, N, K, lda, ldb, ldc, ta, tb;
};

// C = op(A) op(B), one CTA per job (small FP64 blocks).
__global__ void small_gemm_kernel(const GemmJob* __restrict__ jobs) {
  const GemmJob J = jobs[blockIdx.x];
  for (int idx = threadIdx.x; idx < J.M * J.N; idx += blockDim.x) {
    const int i = idx / J.N, j = idx % J.N;
    double s = 0.0;
    for (int k = 0; k < J.K; ++k) {
      const double a = J.ta ? J.A[(long long)k * J.lda + i] : J.A[(long long)i * J.lda + k];
      const double b = J.tb ? J.B[(long long)j * J.ldb + k] : J.B[(long long)k * J.ldb + j];
      s = fma(a, b, s);
    }
    J.C[(long long)i * J.ldc + j] = s;
  }
}

struct EigJob {
  const double* A;  // m x m symmetric
  double* w;        // m eigenvalues, descending
  double* V;        // m x m, column k = eigenvector of w[k]
  int m;
};

size_t eig_smem_bytes(int m) {
  const int h = (m + 1) / 2;
  return (size_t)(2 * m * (m + 1) + 2 * h + 2 * (EIG_THREADS / 32)) * 8 + (size_t)(2 * h + 1 + m) * 4 + 64;
}

__global__ void __launch_bounds__(EIG_THREADS) block_eig_kernel(const EigJob* __restrict__ jobs,
                                                                int* __restrict__ info) {
  extern __shared__ double sm[];
  const EigJob J = jobs[blockIdx.x];
  const int m = J.m, lda = m + 1, h = (m + 1) / 2;
  double* A = sm;
  double* Q = A + m * lda;
  double* cs = Q + m * lda;
  double* sn = cs + h;
  double* red = sn + h;
  int* pp = reinterpret_cast<int*>(red + 2 * (EIG_THREADS / 32));
  int* qq = pp + h;
  int* stop = qq + h;
  int* order = stop + 1;
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int i = idx / m, j = idx % m;
    A[i * lda + j] = 0.5 * (J.A[i * m + j] + J.A[j * m + i]);
  }
  __syncthreads();
  const int sweeps = oz::jacobi_smem(A, Q, lda, m, {cs, sn, pp, qq, red, stop}, 60);
  oz::jacobi_order(A, lda, m, true, order);
  if (threadIdx.x == 0) info[blockIdx.x] = sweeps;
  for (int i = threadIdx.x; i < m; i += blockDim.x) J.w[i] = A[order[i] * lda + order[i]];
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int i = idx / m, k = idx % m;
    J.V[i * m + k] = Q[i * lda + order[k]];
  }
}

// Larger sectors (EIG_MAX < m <= EIG_MAX_GLOBAL): the same Jacobi sweeps on the matrix in global
// memory, in place (J.A is the density matrix, overwritten; J.V receives the eigenvectors), with
// only the rotation scratch and the ordering in shared memory.
__global__ void __launch_bounds__(EIG_THREADS) block_eig_global_kernel(const EigJob* __restrict__ jobs,
                                                                       int* __restrict__ info) {
  extern __shared__ double gsm[];
  const EigJob J = jobs[blockIdx.x];
  const int m = J.m, h = (m + 1) / 2;
  double* A = const_cast<double*>(J.A);
  double* Q = J.V;
  double* cs = gsm;
  double* sn = cs + h;
  double* red = sn + h;
  int* pp = reinterpret_cast<int*>(red + 2 * (EIG_THREADS / 32));
  int* qq = pp + h;
  int* stop = qq + h;
  int* order = stop + 1;
  for (long long idx = threadIdx.x; idx < (long long)m * m; idx += blockDim.x) {
    const int i = (int)(idx / m), j = (int)(idx % m);
    if (i < j) {
      const double v = 0.5 * (A[(long long)i * m + j] + A[(long long)j * m + i]);
      A[(long long)i * m + j] = v;
      A[(long long)j * m + i] = v;
    }
  }
  __syncthreads();
  const int sweeps = oz::jacobi_smem(A, Q, m, m, {cs, sn, pp, qq, red, stop}, 60);
  // descending order, ties by index: the rank of every diagonal entry
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double a = A[(long long)i * m + i];
    int r = 0;
    for (int k = 0; k < m; ++k) {
      const double b = A[(long long)k * m + k];
      r += (b > a) || (b == a && k < i);
    }
    order[r] = i;
  }
  __syncthreads();
  if (threadIdx.x == 0) info[blockIdx.x] = sweeps;
  for (int k = threadIdx.x; k < m; k += blockDim.x) J.w[k] = A[(long long)order[k] * m + order[k]];
  __syncthreads();
  // columns of Q in that order: through A, which is no longer needed
  for (long long idx = threadIdx.x; idx < (long long)m * m; idx += blockDim.x) A[idx] = Q[idx];
  __syncthreads();
  for (long long idx = threadIdx.x; idx < (long long)m * m; idx += blockDim.x) {
    const int i = (int)(idx / m), k = (int)(idx % m);
    Q[idx] = A[(long long)i * m + order[k]];
  }
}

size_t eig_global_smem_bytes(int m) {
  const int h = (m + 1) / 2;
  return (size_t)(2 * h + 2 * (EIG_THREADS / 32)) * 8 + (size_t)(2 * h + 1 + m) * 4 + 64;
}

// Block partials of x . y (fixed order inside a block; the host adds the blocks in order).
__global__ void dot_kernel(const double* __restrict__ x, const double* __restrict__ y, long long n,
                           double* __restrict__ part) {
  __shared__ double sh[256];
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s = fma(x[i], y[i], s);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  // SplitMix64 (Steele, Lea and Flood, OOPSLA 2014), the published constants
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Davidson start vector: uniform in (-1, 1) from a counter-based generator.
__global__ void random_vector_kernel(double* __restrict__ x, long long n, unsigned long long key) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long r = splitmix64(key ^ splitmix64((unsigned long long)i));
    x[i] = ((double)(r >> 11) + 0.5) * 0x1.0p-52 - 1.0;
  }
}

// ------------------------------------------------------------------------------------------------
// host structures
// ------------------------------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  int reserve(size_t b) {
    if (b <= bytes) return OZ_OK;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    DM_CU(cudaMalloc(&p, std::max<size_t>(b, 256)));
    bytes = std::max<size_t>(b, 256);
    return OZ_OK;
  }
  template <class T>
  int upload(const std::vector<T>& v, cudaStream_t st) {
    DM_RC(reserve(v.size() * sizeof(T)));
    if (!v.empty()) DM_CU(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    return OZ_OK;
  }
};

struct Basis {
  std::vector<QN> q;
  std::vector<int> dim;
  std::vector<std::vector<long long>> pat;  // determinant pattern of every state (-1: rotated)
  int find(QN x) const {
    for (size_t i = 0; i < q.size(); ++i)
      if (same(q[i], x)) return (int)i;
    return -1;
  }
  long long total() const {
    long long t = 0;
    for (int d : dim) t += d;
    return t;
  }
};

// Product basis of a block and a site.  Left: block (x) site; right: site (x) block.  Sectors in
// order of first appearance, pieces ordered by site state then block sector.
struct Enlarged {
  Basis b;
  std::vector<std::array<int, 4>> sec, off;  // [block sector][site state] -> enlarged sector, offset
};

Enlarged enlarge(const Basis& blk, int site, bool left) {
  Enlarged E;
  E.sec.assign(blk.q.size(), {-1, -1, -1, -1});
  E.off.assign(blk.q.size(), {0, 0, 0, 0});
  for (int s = 0; s < 4; ++s)
    for (size_t a = 0; a < blk.q.size(); ++a) {
      const QN qn = add(blk.q[a], QN{oz::SITE_N[s], oz::SITE_S[s]});
      int k = E.b.find(qn);
      if (k < 0) {
        k = (int)E.b.q.size();
        E.b.q.push_back(qn);
        E.b.dim.push_back(0);
        E.b.pat.emplace_back();
      }
      E.sec[a][s] = k;
      E.off[a][s] = E.b.dim[k];
      E.b.dim[k] += blk.dim[a];
      for (long long p : blk.pat[a]) {
        const long long sp = (long long)s << (2 * site);
        E.b.pat[k].push_back(p < 0 ? -1 : (p | sp));
      }
      (void)left;
    }
  return E;
}

// Block-sparse operators on a basis, one per MPO state of a bond: the block of state w on input
// sector `in` maps to sector out[w][in] (= in + delta[w]) and sits at element offset off[w][in].
struct Ops {
  std::vector<QN> delta;
  std::vector<std::vector<int>> out;
  std::vector<std::vector<long long>> off;
  DevBuf mem;
  long long elems = 0;
  const double* ptr(int w, int in) const { return (const double*)mem.p + off[w][in]; }
};

// Environment = operators of a block on its own basis, and how that basis came out of the
// truncation of an enlarged basis `src` (absent for the start's reference blocks): every state kept
// (ident), or per src sector q the new sector newidx[q] (-1: dropped) spanned by k[q] kept vectors,
// row-major src.b.dim[q] x k[q] at U + uoff[q].  The kept vectors carry a two-site vector from one
// bond to the next (the start of the next eigensolver run).
struct Env {
  Basis basis;
  Ops ops;
  bool has_src = false, ident = false;
  Enlarged src;
  std::vector<int> k, newidx;
  std::vector<long long> uoff;
  DevBuf U;
};

}  // namespace

// ------------------------------------------------------------------------------------------------
// DMRG state
// ------------------------------------------------------------------------------------------------
struct oz_dmrg_s {
  oz_ctx* ctx = nullptr;
  int L = 0, N = 0, twosz = 0, D = 0;
  oz_prec prec{7, 0, OZ_MODE_EAGER};
  oz_prec renorm{7, 0, OZ_MODE_NATIVE};  // precision of the renormalisation products U^T O U
  oz_prec rdm{7, 0, OZ_MODE_NATIVE};     // precision of the density matrices psi psi^T
  int solver = OZ_SOLVER_DAVIDSON;        // eigensolver of the two-site update
  int check_fp64 = 0;                     // re-evaluate every Ritz vector with the FP64 H_eff
  double tol = 1e-10;
  unsigned long long seed = 0;
  oz::Mpo mpo;
  cudaStream_t st = nullptr;
  std::vector<std::unique_ptr<Env>> left;   // left[b + 1]: block 0..b, states of bond b
  std::vector<std::unique_ptr<Env>> right;  // right[b]: block b+1..L-1, states of bond b
  std::vector<oz_dmrg_step> steps;
  long long nsolve = 0;
  DevBuf jobs, groups, work, eigw, eigv, rho, info;
  // the last two-site solution and its layout (start-vector prediction of the next bond)
  int predict = 1;
  struct Prev {
    bool valid = false, truncated = false;
    int bond = -1, dir = 0;
    long long dim = 0;
    std::vector<int> le, re, m, n;
    std::vector<long long> psioff;
    Enlarged LE, RE;
  } prev;
  DevBuf prev_psi, pred_tmp, pred_jobs;
  // verification record of emulated renormalisation and density-matrix products (oz_dmrg_set_trace)
  struct TraceRec {
    int kind, step, M, N, K, S, level;
    std::vector<double> A, B, C;  // op(A) M x K, op(B) K x N, C M x N, row-major
  };
  int trace_stride = 0;
  std::vector<TraceRec> trace;
  QN target() const { return {N, twosz}; }
};

namespace {

// Host copy of rows x cols of a row-major device matrix (leading dimension ld), transposed into
// cols x rows when `trans` is set.
int fetch_matrix(const double* src, long long ld, int rows, int cols, bool trans, std::vector<double>* out,
                 cudaStream_t st) {
  std::vector<double> tmp((size_t)rows * cols);
  DM_CU(cudaMemcpy2DAsync(tmp.data(), (size_t)cols * 8, src, (size_t)ld * 8, (size_t)cols * 8, rows,
                          cudaMemcpyDeviceToHost, st));
  DM_CU(cudaStreamSynchronize(st));
  if (!trans) {
    out->swap(tmp);
    return OZ_OK;
  }
  out->assign((size_t)rows * cols, 0.0);
  for (int r = 0; r < rows; ++r)
    for (int c = 0; c < cols; ++c) (*out)[(size_t)c * rows + r] = tmp[(size_t)r * cols + c];
  return OZ_OK;
}

// Records products 0, stride, 2 stride, ... of an emulated batch that has completed on d->st (so
// every batch, i.e. every truncating bond, leaves at least one record): kind 0 = renormalisation
// T = O U, 1 = renormalisation U^T T, 2 = density matrix.
int trace_batch(oz_dmrg* d, int kind, const std::vector<oz::EmuJob>& jobs, int S, int lv) {
  if (d->trace_stride <= 0) return OZ_OK;
  for (size_t idx = 0; idx < jobs.size(); idx += (size_t)d->trace_stride) {
    const oz::EmuJob& j = jobs[idx];
    oz_dmrg_s::TraceRec r;
    r.kind = kind;
    r.step = (int)d->steps.size();
    r.M = j.M;
    r.N = j.N;
    r.K = j.K;
    r.S = S;
    r.level = lv;
    // op(A) = A (M x K) or the transpose of the stored K x M matrix
    DM_RC(j.transA ? fetch_matrix(j.A, j.lda, j.K, j.M, true, &r.A, d->st)
                   : fetch_matrix(j.A, j.lda, j.M, j.K, false, &r.A, d->st));
    // op(B) = B (K x N) or the transpose of the stored N x K matrix
    DM_RC(j.transB ? fetch_matrix(j.B, j.ldb, j.N, j.K, true, &r.B, d->st)
                   : fetch_matrix(j.B, j.ldb, j.K, j.N, false, &r.B, d->st));
    DM_RC(fetch_matrix(j.C, j.ldc, j.M, j.N, false, &r.C, d->st));
    d->trace.push_back(std::move(r));
  }
  return OZ_OK;
}

// Operators of the enlarged block: L_w (left) for the states of bond `site`, or R_w (right) for
// the states of bond `site` - 1.
int build_ops(oz_dmrg* d, const Env& E, const Enlarged& X, int site, bool left, Ops* out) {
  const oz::Mpo& M = d->mpo;
  const int bond = left ? site : site - 1;
  const int nst = M.chi(bond);
  const int nsec = (int)X.b.q.size();
  out->delta = M.delta[bond + 1];
  if (!left)
    for (auto& q : out->delta) q = QN{-q.n, -q.s};  // R_w changes the right side by -delta
  out->out.assign(nst, std::vector<int>(nsec, -1));
  out->off.assign(nst, std::vector<long long>(nsec, -1));
  // pass 1: which blocks receive contributions; jobs with block-relative destinations
  struct Pend {
    int w, in;
    long long roff;  // region offset inside the block
    KronJob j;
  };
  std::vector<Pend> pend;
  for (const oz::MpoEntry& e : M.W[site]) {
    const int wE = left ? e.row : e.col;   // state of the environment
    const int w = left ? e.col : e.row;    // state of the new operator
    for (int so = 0; so < 4; ++so)
      for (int si = 0; si < 4; ++si) {
        const double v = e.m[so * 4 + si];
        if (v == 0.0) continue;
        for (size_t a = 0; a < E.basis.q.size(); ++a) {
          const int ao = E.ops.out[wE][a];
          if (ao < 0 || E.ops.off[wE][a] < 0) continue;
          const int Qi = X.sec[a][si], Qo = X.sec[ao][so];
          if (out->out[w][Qi] < 0) out->out[w][Qi] = Qo;
          if (out->out[w][Qi] != Qo) return oz::api_fail(OZ_EINVAL, "MPO state mixes quantum-number changes");
          KronJob j{};
          j.src = E.ops.off[wE][a];
          j.lds = E.basis.dim[a];
          j.rows = E.basis.dim[ao];
          j.cols = E.basis.dim[a];
          j.scale = v;
          j.ldd = X.b.dim[Qi];
          pend.push_back({w, Qi, (long long)X.off[ao][so] * X.b.dim[Qi] + X.off[a][si], j});
        }
      }
  }
  long long tot = 0;
  for (int w = 0; w < nst; ++w)
    for (int q = 0; q < nsec; ++q)
      if (out->out[w][q] >= 0) {
        out->off[w][q] = tot;
        tot += (long long)X.b.dim[out->out[w][q]] * X.b.dim[q];
      }
  out->elems = tot;
  DM_RC(out->mem.reserve((size_t)std::max(tot, 1ll) * 8));
  DM_CU(cudaMemsetAsync(out->mem.p, 0, (size_t)std::max(tot, 1ll) * 8, d->st));
  if (pend.empty()) return OZ_OK;
  std::vector<KronJob> jobs;
  jobs.reserve(pend.size());
  for (auto& p : pend) {
    p.j.dst = out->off[p.w][p.in] + p.roff;
    jobs.push_back(p.j);
  }
  // host-side bounds check of every region against both arenas before the launch
  for (const KronJob& j : jobs) {
    const long long send = j.src + (long long)(j.rows - 1) * j.lds + j.cols;
    const long long dend = j.dst + (long long)(j.rows - 1) * j.ldd + j.cols;
    if (j.rows <= 0 || j.cols <= 0 || j.src < 0 || send > E.ops.elems || j.dst < 0 || dend > tot ||
        j.cols > j.lds || j.cols > j.ldd)
      return oz::api_fail(OZ_EINVAL, "internal: operator block outside its arena");
  }
  std::stable_sort(jobs.begin(), jobs.end(), [](const KronJob& a, const KronJob& b) { return a.dst < b.dst; });
  std::vector<int> gs;
  for (size_t i = 0; i < jobs.size(); ++i)
    if (i == 0 || jobs[i].dst != jobs[i - 1].dst) gs.push_back((int)i);
  gs.push_back((int)jobs.size());
  DM_RC(d->jobs.upload(jobs, d->st));
  DM_RC(d->groups.upload(gs, d->st));
  kron_accumulate_kernel<<<(unsigned)(gs.size() - 1), 128, 0, d->st>>>(
      (const KronJob*)d->jobs.p, (const int*)d->groups.p, (const double*)E.ops.mem.p, (double*)out->mem.p);
  DM_CU(cudaGetLastError());
  DM_CU(cudaStreamSynchronize(d->st));  // job tables are reused by the next call
  return OZ_OK;
}

// New environment from the operators of an enlarged block and the kept states: per enlarged sector
// Q, U[Q] (device, dim[Q] x k[Q] row-major) or keep_all (U = identity on every sector).
int project(oz_dmrg* d, const Enlarged& X, Ops& ops, bool keep_all, const std::vector<const double*>& U,
            const std::vector<int>& k, const std::vector<std::vector<long long>>& pats, Env* out) {
  const int nsec = (int)X.b.q.size();
  out->has_src = true;
  out->src = X;
  out->ident = keep_all;
  if (keep_all) {
    out->basis = X.b;
    out->ops.delta = ops.delta;
    out->ops.out = ops.out;
    out->ops.off = ops.off;
    out->ops.elems = ops.elems;
    std::swap(out->ops.mem.p, ops.mem.p);
    std::swap(out->ops.mem.bytes, ops.mem.bytes);
    return OZ_OK;
  }
  std::vector<int> newidx(nsec, -1);
  out->basis = Basis();
  for (int q = 0; q < nsec; ++q)
    if (k[q] > 0) {
      newidx[q] = (int)out->basis.q.size();
      out->basis.q.push_back(X.b.q[q]);
      out->basis.dim.push_back(k[q]);
      out->basis.pat.push_back(pats[q]);
    }
  // keep the kept vectors (the eigenvector arena is reused by the next truncation)
  out->k = k;
  out->newidx = newidx;
  out->uoff.assign(nsec, -1);
  long long ut = 0;
  for (int q = 0; q < nsec; ++q)
    if (k[q] > 0) {
      out->uoff[q] = ut;
      ut += (long long)X.b.dim[q] * k[q];
    }
  DM_RC(out->U.reserve((size_t)std::max(ut, 1ll) * 8));
  for (int q = 0; q < nsec; ++q)
    if (k[q] > 0)
      DM_CU(cudaMemcpyAsync((double*)out->U.p + out->uoff[q], U[q], (size_t)X.b.dim[q] * k[q] * 8,
                            cudaMemcpyDeviceToDevice, d->st));
  const int nst = (int)ops.delta.size(), nn = (int)out->basis.q.size();
  out->ops.delta = ops.delta;
  out->ops.out.assign(nst, std::vector<int>(nn, -1));
  out->ops.off.assign(nst, std::vector<long long>(nn, -1));
  long long tot = 0, ttot = 0;
  std::vector<GemmJob> g1, g2;
  std::vector<long long> toff;
  for (int w = 0; w < nst; ++w)
    for (int q = 0; q < nsec; ++q) {
      const int qo = ops.out[w][q];
      if (qo < 0 || newidx[q] < 0 || newidx[qo] < 0) continue;
      out->ops.out[w][newidx[q]] = newidx[qo];
      out->ops.off[w][newidx[q]] = tot;
      tot += (long long)k[qo] * k[q];
      toff.push_back(ttot);
      ttot += (long long)X.b.dim[qo] * k[q];
    }
  out->ops.elems = tot;
  DM_RC(out->ops.mem.reserve((size_t)std::max(tot, 1ll) * 8));
  DM_RC(d->work.reserve((size_t)std::max(ttot, 1ll) * 8));
  size_t t = 0;
  for (int w = 0; w < nst; ++w)
    for (int q = 0; q < nsec; ++q) {
      const int qo = ops.out[w][q];
      if (qo < 0 || newidx[q] < 0 || newidx[qo] < 0) continue;
      if (ops.off[w][q] < 0 || ops.off[w][q] + (long long)X.b.dim[qo] * X.b.dim[q] > ops.elems || !U[q] || !U[qo])
        return oz::api_fail(OZ_EINVAL, "internal: projection block outside its arena");
      double* T = (double*)d->work.p + toff[t++];
      // T = Op[qo <- q] U[q]  (dim[qo] x k[q]);  E = U[qo]^T T  (k[qo] x k[q])
      g1.push_back({ops.ptr(w, q), U[q], T, X.b.dim[qo], k[q], X.b.dim[q], X.b.dim[q], k[q], k[q], 0, 0});
      g2.push_back({U[qo], T, (double*)out->ops.mem.p + out->ops.off[w][newidx[q]], k[qo], k[q], X.b.dim[qo], k[qo],
                    k[q], k[q], 1, 0});
    }
  if (!g1.empty() && d->renorm.mode == OZ_MODE_EAGER) {
    // emulated renormalisation: both passes as grouped Ozaki products
    std::vector<oz::EmuJob> e1, e2;
    for (const GemmJob& g : g1) e1.push_back({g.A, g.lda, 0, g.B, g.ldb, 0, g.C, g.ldc, g.M, g.N, g.K});
    for (const GemmJob& g : g2) e2.push_back({g.A, g.lda, 1, g.B, g.ldb, 0, g.C, g.ldc, g.M, g.N, g.K});
    const int S = d->renorm.slices, lv = d->renorm.level ? d->renorm.level : d->renorm.slices;
    DM_RC(oz::emulated_batch(d->ctx, e1, S, lv, d->st));
    DM_RC(trace_batch(d, 0, e1, S, lv));
    DM_RC(oz::emulated_batch(d->ctx, e2, S, lv, d->st));
    DM_RC(trace_batch(d, 1, e2, S, lv));
  } else if (!g1.empty()) {
    DM_RC(d->jobs.upload(g1, d->st));
    small_gemm_kernel<<<(unsigned)g1.size(), 128, 0, d->st>>>((const GemmJob*)d->jobs.p);
    DM_CU(cudaGetLastError());
    DM_CU(cudaStreamSynchronize(d->st));
    DM_RC(d->jobs.upload(g2, d->st));
    small_gemm_kernel<<<(unsigned)g2.size(), 128, 0, d->st>>>((const GemmJob*)d->jobs.p);
    DM_CU(cudaGetLastError());
    DM_CU(cudaStreamSynchronize(d->st));
  }
  return OZ_OK;
}

// Two-site problem of bond i with the current environments.
struct Bond {
  Enlarged LE, RE;
  Ops Lw, Rw;
  std::vector<oz_task> tasks;
  std::vector<int> le, re;            // psi sector -> LE sector, RE sector
  std::vector<long long> psioff;
  std::vector<int> m, n;
  long long dim = 0;
  int ntask = 0;
  oz_heff* h = nullptr;
  ~Bond() {
    if (h) oz_heff_destroy(h);
  }
};

int make_bond(oz_dmrg* d, int i, Bond* B) {
  const Env* EL = d->left[i].get();       // block 0..i-1 (bond i-1)
  const Env* ER = d->right[i + 1].get();  // block i+2..L-1 (bond i+1)
  if (!EL || !ER) return oz::api_fail(OZ_EINVAL, "environments of this bond are not built");
  B->LE = enlarge(EL->basis, i, true);
  B->RE = enlarge(ER->basis, i + 1, false);
  DM_RC(build_ops(d, *EL, B->LE, i, true, &B->Lw));
  DM_RC(build_ops(d, *ER, B->RE, i + 1, false, &B->Rw));
  const QN T = d->target();
  std::vector<int> psi_of_le(B->LE.b.q.size(), -1);
  B->psioff.assign(1, 0);
  for (size_t q = 0; q < B->LE.b.q.size(); ++q) {
    const int r = B->RE.b.find(sub(T, B->LE.b.q[q]));
    if (r < 0) continue;
    psi_of_le[q] = (int)B->le.size();
    B->le.push_back((int)q);
    B->re.push_back(r);
    B->m.push_back(B->LE.b.dim[q]);
    B->n.push_back(B->RE.b.dim[r]);
    B->psioff.push_back(B->psioff.back() + (long long)B->LE.b.dim[q] * B->RE.b.dim[r]);
  }
  B->dim = B->psioff.back();
  if (B->le.empty()) return oz::api_fail(OZ_EINVAL, "the two-site space of this bond is empty");
  std::vector<oz_task> tasks;
  const int nst = (int)B->Lw.delta.size();
  for (int w = 0; w < nst; ++w)
    for (size_t p = 0; p < B->le.size(); ++p) {
      const int qo = B->Lw.out[w][B->le[p]], ro = B->Rw.out[w][B->re[p]];
      if (qo < 0 || ro < 0) continue;
      const int dst = psi_of_le[qo];
      if (dst < 0 || B->re[dst] != ro) continue;
      tasks.push_back({(int)p, dst, 1.0, B->Lw.ptr(w, B->le[p]), B->Rw.ptr(w, B->re[p])});
    }
  B->ntask = (int)tasks.size();
  B->tasks = tasks;
  DM_CU(cudaStreamSynchronize(d->st));
  return oz_heff_create(d->ctx, (int)B->le.size(), B->m.data(), B->n.data(), (int)tasks.size(), tasks.data(),
                        &d->prec, &B->h);
}

// Kept states of one side from the two-site vector psi (device, the layout of B).  Fills U (device
// pointers into d->eigv), k and patterns per enlarged sector, or sets keep_all.
int choose_states(oz_dmrg* d, Bond& B, const double* psi, bool left, bool* keep_all, std::vector<const double*>* U,
                  std::vector<int>* k, std::vector<std::vector<long long>>* pats, double* discarded) {
  const Enlarged& X = left ? B.LE : B.RE;
  const int nsec = (int)X.b.q.size();
  U->assign(nsec, nullptr);
  k->assign(nsec, 0);
  pats->assign(nsec, {});
  *discarded = 0.0;
  if (X.b.total() <= d->D) {
    *keep_all = true;
    return OZ_OK;
  }
  *keep_all = false;
  // density matrix per sector with a psi block: rho = psi psi^T (left) or psi^T psi (right)
  std::vector<int> sec_of(B.le.size());
  std::vector<long long> roff(B.le.size());
  long long rtot = 0;
  for (size_t p = 0; p < B.le.size(); ++p) {
    sec_of[p] = left ? B.le[p] : B.re[p];
    const int md = left ? B.m[p] : B.n[p];
    if (md > EIG_MAX_GLOBAL)
      return oz::api_fail(OZ_EINVAL, "a density-matrix sector exceeds " + std::to_string(EIG_MAX_GLOBAL) +
                                         " states (eigensolver limit)");
    roff[p] = rtot;
    rtot += (long long)md * md;
  }
  DM_RC(d->rho.reserve((size_t)rtot * 8));
  DM_RC(d->eigv.reserve((size_t)rtot * 8));
  long long wtot = 0;
  for (size_t p = 0; p < B.le.size(); ++p) wtot += left ? B.m[p] : B.n[p];
  DM_RC(d->eigw.reserve((size_t)wtot * 8));
  std::vector<GemmJob> gj;
  std::vector<EigJob> ej, ejg;  // on-chip sectors, global-memory sectors
  std::vector<long long> woff(B.le.size());
  long long wo = 0;
  int mmax = 1, mgmax = 1;
  for (size_t p = 0; p < B.le.size(); ++p) {
    const int mp = B.m[p], np = B.n[p];
    const double* P = psi + B.psioff[p];
    double* R = (double*)d->rho.p + roff[p];
    if (left)
      gj.push_back({P, P, R, mp, mp, np, np, np, mp, 0, 1});
    else
      gj.push_back({P, P, R, np, np, mp, np, np, np, 1, 0});
    const int md = left ? mp : np;
    woff[p] = wo;
    const EigJob job{R, (double*)d->eigw.p + wo, (double*)d->eigv.p + roff[p], md};
    if (md <= EIG_MAX) {
      ej.push_back(job);
      mmax = std::max(mmax, md);
    } else {
      ejg.push_back(job);
      mgmax = std::max(mgmax, md);
    }
    wo += md;
  }
  if (d->rdm.mode == OZ_MODE_EAGER) {
    // emulated density matrices: rho = psi psi^T (left) or psi^T psi (right)
    std::vector<oz::EmuJob> ejb;
    for (const GemmJob& g : gj)
      ejb.push_back({g.A, g.lda, g.ta, g.B, g.ldb, g.tb, g.C, g.ldc, g.M, g.N, g.K});
    const int lv = d->rdm.level ? d->rdm.level : d->rdm.slices;
    DM_RC(oz::emulated_batch(d->ctx, ejb, d->rdm.slices, lv, d->st));
    DM_RC(trace_batch(d, 2, ejb, d->rdm.slices, lv));
  } else {
    DM_RC(d->jobs.upload(gj, d->st));
    small_gemm_kernel<<<(unsigned)gj.size(), 128, 0, d->st>>>((const GemmJob*)d->jobs.p);
    DM_CU(cudaGetLastError());
    DM_CU(cudaStreamSynchronize(d->st));
  }
  // both job lists in one upload: on-chip jobs first, then the global-memory ones
  std::vector<EigJob> all_jobs(ej);
  all_jobs.insert(all_jobs.end(), ejg.begin(), ejg.end());
  DM_RC(d->jobs.upload(all_jobs, d->st));
  DM_RC(d->info.reserve(all_jobs.size() * 4));
  if (!ej.empty()) {
    const size_t smem = eig_smem_bytes(mmax);
    DM_CU(cudaFuncSetAttribute(block_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    block_eig_kernel<<<(unsigned)ej.size(), EIG_THREADS, smem, d->st>>>((const EigJob*)d->jobs.p, (int*)d->info.p);
    DM_CU(cudaGetLastError());
  }
  if (!ejg.empty()) {
    const size_t smem = eig_global_smem_bytes(mgmax);
    DM_CU(cudaFuncSetAttribute(block_eig_global_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    block_eig_global_kernel<<<(unsigned)ejg.size(), EIG_THREADS, smem, d->st>>>(
        (const EigJob*)d->jobs.p + ej.size(), (int*)d->info.p + ej.size());
    DM_CU(cudaGetLastError());
  }
  std::vector<double> w(wtot);
  std::vector<int> info(all_jobs.size());
  DM_CU(cudaMemcpyAsync(w.data(), d->eigw.p, (size_t)wtot * 8, cudaMemcpyDeviceToHost, d->st));
  DM_CU(cudaMemcpyAsync(info.data(), d->info.p, all_jobs.size() * 4, cudaMemcpyDeviceToHost, d->st));
  DM_CU(cudaStreamSynchronize(d->st));
  for (int x : info)
    if (x < 0) return oz::api_fail(OZ_ENOCONV, "density-matrix Jacobi sweeps did not converge");
  // global selection: at most D eigenvalues above LAMBDA_MIN, never cutting a group of equal ones
  std::vector<double> all(w.begin(), w.end());
  std::sort(all.begin(), all.end(), [](double a, double b) { return a > b; });
  std::vector<double> cand;
  for (double x : all)
    if (x > LAMBDA_MIN) cand.push_back(x);
  int kk = std::min<int>(d->D, (int)cand.size());
  const double lmax = cand.empty() ? 0.0 : cand[0];
  while (kk > 0 && kk < (int)cand.size() && cand[kk - 1] - cand[kk] <= 1e-12 * lmax + 1e-8 * cand[kk - 1]) --kk;
  if (kk == 0) return oz::api_fail(OZ_EINVAL, "truncation kept no state");
  const double cut = cand[kk - 1];
  double kept_w = 0.0, all_w = 0.0;
  for (double x : all) all_w += std::max(x, 0.0);
  int kept = 0;
  for (size_t p = 0; p < B.le.size(); ++p) {
    const int md = left ? B.m[p] : B.n[p];
    int kp = 0;
    while (kp < md && w[woff[p] + kp] >= cut) {
      kept_w += w[woff[p] + kp];
      ++kp;
    }
    const int q = sec_of[p];
    (*k)[q] = kp;
    kept += kp;
    if (kp == 0) continue;
    // U[q] = first kp columns of the eigenvector matrix (md x md): copy into a compact block
    double* dstU = (double*)d->eigv.p + roff[p];  // compacted in place, row by row (kp <= md)
    DM_CU(cudaMemcpy2DAsync(d->rho.p, (size_t)kp * 8, dstU, (size_t)md * 8, (size_t)kp * 8, md,
                            cudaMemcpyDeviceToDevice, d->st));
    DM_CU(cudaMemcpyAsync(dstU, d->rho.p, (size_t)kp * md * 8, cudaMemcpyDeviceToDevice, d->st));
    (*U)[q] = dstU;
    (*pats)[q].assign(kp, -1);
  }
  DM_CU(cudaStreamSynchronize(d->st));
  if (kept != kk) return oz::api_fail(OZ_EINVAL, "inconsistent truncation");
  *discarded = std::max(0.0, all_w - kept_w);
  return OZ_OK;
}

// Right blocks of the start: the reference determinant (orbitals filled from 0, up then down
// counts (N + 2Sz)/2 and (N - 2Sz)/2) restricted to sites b+1..L-1.
int reference_site_state(const oz_dmrg* d, int site) {
  const int nup = (d->N + d->twosz) / 2, ndn = (d->N - d->twosz) / 2;
  return (site < nup ? 1 : 0) | (site < ndn ? 2 : 0);
}

int init_environments(oz_dmrg* d) {
  const int L = d->L;
  d->left.clear();
  d->right.clear();
  d->left.resize(L + 1);
  d->right.resize(L + 1);
  // vacuum blocks: the single MPO state of the boundary bond acts as the 1 x 1 identity
  auto vacuum = [&](int bond, std::unique_ptr<Env>* slot) -> int {
    auto E = std::make_unique<Env>();
    E->basis.q = {QN{0, 0}};
    E->basis.dim = {1};
    E->basis.pat = {{0}};
    E->ops.delta = d->mpo.delta[bond + 1];
    E->ops.out = {{0}};
    E->ops.off = {{0}};
    E->ops.elems = 1;
    DM_RC(E->ops.mem.reserve(8));
    const double one = 1.0;
    DM_CU(cudaMemcpy(E->ops.mem.p, &one, 8, cudaMemcpyHostToDevice));
    *slot = std::move(E);
    return OZ_OK;
  };
  DM_RC(vacuum(-1, &d->left[0]));
  DM_RC(vacuum(L - 1, &d->right[L - 1]));
  for (int b = L - 2; b >= 0; --b) {
    const Env& ER = *d->right[b + 1];
    Enlarged X = enlarge(ER.basis, b + 1, false);
    Ops R;
    DM_RC(build_ops(d, ER, X, b + 1, false, &R));
    const int s = reference_site_state(d, b + 1);
    // the block of the start has one state in sector 0
    const int q = X.sec[0][s];
    const int row = X.off[0][s];
    std::vector<double> u(X.b.dim[q], 0.0);
    u[row] = 1.0;
    DevBuf ub;
    DM_RC(ub.upload(u, d->st));
    std::vector<const double*> U(X.b.q.size(), nullptr);
    std::vector<int> k(X.b.q.size(), 0);
    std::vector<std::vector<long long>> pats(X.b.q.size());
    U[q] = (const double*)ub.p;
    k[q] = 1;
    pats[q] = {X.b.pat[q][row]};
    auto E = std::make_unique<Env>();
    DM_RC(project(d, X, R, false, U, k, pats, E.get()));
    d->right[b] = std::move(E);
  }
  return OZ_OK;
}

// Start vector of bond i from the previous bond's solution (White's transformation of the two-site
// vector): at a turning point the same problem (the vector itself); after a left-to-right step
// psi' = U_L^T psi, with the right block's states expanded over (site i+1 block) by the vectors
// that made that block; after a right-to-left step the mirror image.  Returns *ok = false when no
// prediction applies (first pass, reference blocks); the caller then draws a random start.
int predict_start(oz_dmrg* d, int i, int dir, const Bond& B, double* psi, bool* ok) {
  *ok = false;
  const auto& P = d->prev;
  if (!d->predict || !P.valid) return OZ_OK;
  if (P.bond == i && !P.truncated && P.le == B.le && P.re == B.re && P.m == B.m && P.n == B.n) {
    DM_CU(cudaMemcpyAsync(psi, d->prev_psi.p, (size_t)B.dim * 8, cudaMemcpyDeviceToDevice, d->st));
    *ok = true;
    return OZ_OK;
  }
  if (!P.truncated || P.dir != dir || P.bond != (dir == 0 ? i - 1 : i + 1)) return OZ_OK;
  // T: the truncated side of the previous vector; X: the block whose states are expanded
  const Env* T = dir == 0 ? d->left[i].get() : d->right[i + 1].get();
  const Env* X = dir == 0 ? d->right[i].get() : d->left[i + 1].get();
  if (!T || !X || !T->has_src || !X->has_src) return OZ_OK;
  const Enlarged& Bx = dir == 0 ? B.RE : B.LE;  // the new enlarged basis X's states are expanded over
  if (X->src.b.q.size() != Bx.b.q.size() || X->src.b.dim != Bx.b.dim) return OZ_OK;
  if (T->src.b.dim != (dir == 0 ? P.LE : P.RE).b.dim) return OZ_OK;  // T was cut from the previous bond
  // new psi sector of (LE sector, RE sector)
  auto psi_sector = [&](int le, int re) {
    for (size_t p = 0; p < B.le.size(); ++p)
      if (B.le[p] == le && B.re[p] == re) return (int)p;
    return -1;
  };
  // inverse of X's sector map: X sector -> src (= Bx) sector
  std::vector<int> xsrc(X->basis.q.size(), -1);
  for (size_t q = 0; q < X->src.b.q.size(); ++q) {
    const int nq = X->ident ? (int)q : X->newidx[q];
    if (nq >= 0) xsrc[nq] = (int)q;
  }
  const double* Tsrc = (const double*)d->prev_psi.p;
  const int np = (int)P.le.size();
  // step 1: the truncated side, one product per previous block (or the block itself when all states
  // were kept): tmp_p = U^T psi_p (left) or psi_p U (right)
  std::vector<long long> toff(np, -1);
  std::vector<int> trows(np, 0), tcols(np, 0), tsec(np, -1);
  long long tt = 0;
  for (int p = 0; p < np; ++p) {
    const int q = dir == 0 ? P.le[p] : P.re[p];
    const int nq = T->ident ? q : T->newidx[q];
    if (nq < 0) continue;
    tsec[p] = nq;
    trows[p] = dir == 0 ? (T->ident ? P.m[p] : T->k[q]) : P.m[p];
    tcols[p] = dir == 0 ? P.n[p] : (T->ident ? P.n[p] : T->k[q]);
    toff[p] = tt;
    tt += (long long)trows[p] * tcols[p];
  }
  DM_RC(d->pred_tmp.reserve((size_t)std::max(tt, 1ll) * 8));
  double* tmp = (double*)d->pred_tmp.p;
  std::vector<GemmJob> g1, g2;
  for (int p = 0; p < np; ++p) {
    if (toff[p] < 0) continue;
    const int q = dir == 0 ? P.le[p] : P.re[p];
    const double* src = Tsrc + P.psioff[p];
    if (T->ident) {
      DM_CU(cudaMemcpyAsync(tmp + toff[p], src, (size_t)P.m[p] * P.n[p] * 8, cudaMemcpyDeviceToDevice, d->st));
    } else if (dir == 0) {
      // k x n = (m x k)^T (m x n)
      g1.push_back({(const double*)T->U.p + T->uoff[q], src, tmp + toff[p], trows[p], tcols[p], P.m[p], T->k[q],
                    P.n[p], tcols[p], 1, 0});
    } else {
      // m x k = (m x n) (n x k)
      g1.push_back({src, (const double*)T->U.p + T->uoff[q], tmp + toff[p], trows[p], tcols[p], P.n[p], P.n[p],
                    T->k[q], tcols[p], 0, 0});
    }
  }
  // step 2: the other side's block states expanded over (site x block) of the new bond
  DM_CU(cudaMemsetAsync(psi, 0, (size_t)B.dim * 8, d->st));
  const Enlarged& Pold = dir == 0 ? P.RE : P.LE;  // the previous enlarged basis holding X's states
  const Enlarged& Bt = dir == 0 ? B.LE : B.RE;    // the new enlarged basis holding the truncated side
  for (int p = 0; p < np; ++p) {
    if (toff[p] < 0) continue;
    const int r = dir == 0 ? P.re[p] : P.le[p];
    for (size_t a = 0; a < Pold.sec.size(); ++a)
      for (int sg = 0; sg < 4; ++sg) {
        if (Pold.sec[a][sg] != r) continue;
        const int xs = xsrc[a];                                  // Bx sector the states of a came from
        const int ts = Bt.sec[tsec[p]][sg];                      // sector of (truncated side, site) piece
        if (xs < 0 || ts < 0) continue;
        const int pn = dir == 0 ? psi_sector(ts, xs) : psi_sector(xs, ts);
        if (pn < 0) continue;
        const int da = X->basis.dim[a];
        const long long poff = Pold.off[a][sg];
        const long long boff = Bt.off[tsec[p]][sg];
        double* dst = psi + B.psioff[pn];
        if (dir == 0) {
          // rows boff.. of the new block (n columns = Bx dim of xs) = tmp[:, poff..poff+da] V^T
          double* C = dst + boff * B.n[pn];
          const double* A = tmp + toff[p] + poff;
          if (X->ident)
            DM_CU(cudaMemcpy2DAsync(C, (size_t)B.n[pn] * 8, A, (size_t)tcols[p] * 8, (size_t)da * 8, trows[p],
                                    cudaMemcpyDeviceToDevice, d->st));
          else
            g2.push_back({A, (const double*)X->U.p + X->uoff[xs], C, trows[p], B.n[pn], da, tcols[p], da, B.n[pn], 0,
                          1});
        } else {
          // columns boff.. of the new block (m rows = Bx dim of xs) = W tmp[poff..poff+da, :]
          double* C = dst + boff;
          const double* Bm = tmp + toff[p] + poff * tcols[p];
          if (X->ident)
            DM_CU(cudaMemcpy2DAsync(C, (size_t)B.n[pn] * 8, Bm, (size_t)tcols[p] * 8, (size_t)tcols[p] * 8, da,
                                    cudaMemcpyDeviceToDevice, d->st));
          else
            g2.push_back({(const double*)X->U.p + X->uoff[xs], Bm, C, B.m[pn], tcols[p], da, da, tcols[p], B.n[pn], 0,
                          0});
        }
      }
  }
  if (!g1.empty()) {
    DM_RC(d->pred_jobs.upload(g1, d->st));
    small_gemm_kernel<<<(unsigned)g1.size(), 128, 0, d->st>>>((const GemmJob*)d->pred_jobs.p);
    DM_CU(cudaGetLastError());
    DM_CU(cudaStreamSynchronize(d->st));  // the job table is reused below
  }
  if (!g2.empty()) {
    DM_RC(d->pred_jobs.upload(g2, d->st));
    small_gemm_kernel<<<(unsigned)g2.size(), 128, 0, d->st>>>((const GemmJob*)d->pred_jobs.p);
    DM_CU(cudaGetLastError());
  }
  // a usable start has a finite norm well away from zero (the discarded weight is small)
  DevBuf part;
  DM_RC(part.reserve(1024 * 8));
  const int nb = (int)std::min<long long>(1024, (B.dim + 255) / 256);
  dot_kernel<<<nb, 256, 0, d->st>>>(psi, psi, B.dim, (double*)part.p);
  DM_CU(cudaGetLastError());
  std::vector<double> ph(nb);
  DM_CU(cudaMemcpyAsync(ph.data(), part.p, (size_t)nb * 8, cudaMemcpyDeviceToHost, d->st));
  DM_CU(cudaStreamSynchronize(d->st));
  double nrm = 0.0;
  for (double v : ph) nrm += v;
  *ok = std::isfinite(nrm) && nrm > 1e-6;
  return OZ_OK;
}

// The solution of bond i (its Ritz vector in psi) as the source of the next prediction.
int remember(oz_dmrg* d, int i, int dir, bool truncated, const Bond& B, const double* psi) {
  auto& P = d->prev;
  P.valid = false;
  DM_RC(d->prev_psi.reserve((size_t)B.dim * 8));
  DM_CU(cudaMemcpyAsync(d->prev_psi.p, psi, (size_t)B.dim * 8, cudaMemcpyDeviceToDevice, d->st));
  P.bond = i;
  P.dir = dir;
  P.truncated = truncated;
  P.dim = B.dim;
  P.le = B.le;
  P.re = B.re;
  P.m = B.m;
  P.n = B.n;
  P.psioff = B.psioff;
  P.LE = B.LE;
  P.RE = B.RE;
  P.valid = true;
  return OZ_OK;
}

int solve_bond(oz_dmrg* d, int i, int dir, int sweep, bool truncate) {
  Bond B;
  DM_RC(make_bond(d, i, &B));
  DevBuf psi;
  DM_RC(psi.reserve((size_t)B.dim * 8));
  const unsigned long long key = d->seed * 0x2545F4914F6CDD1Dull + (unsigned long long)(++d->nsolve);
  bool predicted = false;
  DM_RC(predict_start(d, i, dir, B, (double*)psi.p, &predicted));
  if (!predicted) {
    random_vector_kernel<<<(unsigned)std::min<long long>(1024, (B.dim + 255) / 256), 256, 0, d->st>>>(
        (double*)psi.p, B.dim, key);
    DM_CU(cudaGetLastError());
  }
  double E = 0.0;
  int iters = 0;
  // a Davidson run that stops short of the tolerance (iteration limit, or a correction that
  // vanishes because the operator is no longer symmetric to that accuracy, e.g. after coarse
  // emulated renormalisation) still leaves its best Ritz pair: the sweep goes on with it and the
  // step records it as not converged
  int rc = d->solver == OZ_SOLVER_LANCZOS ? lanczos_solve(B.h, (double*)psi.p, d->tol, 1000, 30, &E, &iters, d->st)
                                           : davidson_solve(B.h, (double*)psi.p, d->tol, 1000, &E, &iters, d->st);
  if (rc != OZ_OK && rc != OZ_ENOCONV) return rc;
  const int conv = rc == OZ_OK;
  // energy of the same (normalised) vector under the FP64 H_eff of the bond: the variational
  // reference of an emulated Ritz value
  double E64 = E;
  if (d->check_fp64 && d->prec.mode == OZ_MODE_EAGER) {
    oz_prec nat{d->prec.slices, 0, OZ_MODE_NATIVE};
    oz_heff* hn = nullptr;
    DM_RC(oz_heff_create(d->ctx, (int)B.le.size(), B.m.data(), B.n.data(), (int)B.tasks.size(), B.tasks.data(), &nat,
                         &hn));
    DevBuf y, part;
    int rc2 = y.reserve((size_t)B.dim * 8);
    if (!rc2) rc2 = part.reserve(1024 * 8);
    if (!rc2) rc2 = heff_apply(hn, (const double*)psi.p, (double*)y.p, d->st);
    oz_heff_destroy(hn);
    if (rc2) return rc2;
    const int nb = (int)std::min<long long>(1024, (B.dim + 255) / 256);
    dot_kernel<<<nb, 256, 0, d->st>>>((const double*)psi.p, (const double*)y.p, B.dim, (double*)part.p);
    DM_CU(cudaGetLastError());
    std::vector<double> ph(nb);
    DM_CU(cudaMemcpyAsync(ph.data(), part.p, (size_t)nb * 8, cudaMemcpyDeviceToHost, d->st));
    DM_CU(cudaStreamSynchronize(d->st));
    E64 = 0.0;
    for (double v : ph) E64 += v;
  }
  DM_RC(oz_status(d->ctx, d->st));
  oz_dmrg_step s{};
  s.sweep = sweep;
  s.dir = dir;
  s.bond = i;
  s.dim = (int)B.dim;
  s.nterm = (int)B.Lw.delta.size();
  s.ntask = B.ntask;
  s.iters = iters;
  s.converged = conv;
  s.energy = E;
  s.energy_fp64 = E64;
  s.nonvariational = E < E64 - 1e-8 ? 1 : 0;
  s.predicted = predicted ? 1 : 0;
  if (truncate) {
    const bool left = dir == 0;
    bool keep_all = false;
    std::vector<const double*> U;
    std::vector<int> k;
    std::vector<std::vector<long long>> pats;
    double disc = 0.0;
    DM_RC(choose_states(d, B, (const double*)psi.p, left, &keep_all, &U, &k, &pats, &disc));
    auto Env_ = std::make_unique<Env>();
    DM_RC(project(d, left ? B.LE : B.RE, left ? B.Lw : B.Rw, keep_all, U, k, pats, Env_.get()));
    s.kept = (int)Env_->basis.total();
    s.rotated = keep_all ? 0 : 1;
    s.discarded = disc;
    if (left) d->left[i + 1] = std::move(Env_);
    else d->right[i] = std::move(Env_);
  }
  DM_RC(remember(d, i, dir, truncate, B, (const double*)psi.p));
  d->steps.push_back(s);
  return OZ_OK;
}

}  // namespace

extern "C" int oz_dmrg_create(oz_ctx* ctx, const double* h1, const double* eri, int L, int nelec, int twosz, int D,
                              const oz_prec* prec, double davidson_tol, unsigned long long seed, oz_dmrg** out) {
  if (!out) return oz::api_fail(OZ_EINVAL, "out is null");
  *out = nullptr;
  if (!ctx || !h1 || !eri || !prec) return oz::api_fail(OZ_EINVAL, "null argument");
  if (L < 2 || L > 64) return oz::api_fail(OZ_EINVAL, "L must be in 2..64");
  if (nelec < 0 || nelec > 2 * L || ((nelec + twosz) & 1) || std::abs(twosz) > nelec ||
      std::abs(twosz) > 2 * L - nelec)
    return oz::api_fail(OZ_EINVAL, "no state with this electron number and spin");
  if (D < 1) return oz::api_fail(OZ_EINVAL, "D must be positive");
  if (!(davidson_tol > 0.0)) return oz::api_fail(OZ_EINVAL, "davidson_tol must be positive");
  auto d = std::make_unique<oz_dmrg_s>();
  d->ctx = ctx;
  d->L = L;
  d->N = nelec;
  d->twosz = twosz;
  d->D = D;
  d->prec = *prec;
  d->tol = davidson_tol;
  d->seed = seed;
  std::string err;
  if (int rc = oz::build_mpo(h1, eri, L, &d->mpo, &err)) return oz::api_fail(rc, err);
  DM_CU(cudaSetDevice(oz::ctx_device(ctx)));
  DM_CU(cudaStreamCreateWithFlags(&d->st, cudaStreamNonBlocking));
  if (int rc = init_environments(d.get())) {
    cudaStreamDestroy(d->st);
    return rc;
  }
  *out = d.release();
  return OZ_OK;
}

extern "C" int oz_dmrg_set_prediction(oz_dmrg* d, int on) {
  if (!d) return oz::api_fail(OZ_EINVAL, "null handle");
  d->predict = on ? 1 : 0;
  return OZ_OK;
}

extern "C" int oz_dmrg_set_solver(oz_dmrg* d, int solver, double tol, int check_fp64) {
  if (!d) return oz::api_fail(OZ_EINVAL, "null handle");
  if (solver != OZ_SOLVER_DAVIDSON && solver != OZ_SOLVER_LANCZOS) return oz::api_fail(OZ_EINVAL, "unknown solver");
  if (!(tol > 0.0)) return oz::api_fail(OZ_EINVAL, "tol must be positive");
  d->solver = solver;
  d->tol = tol;
  d->check_fp64 = check_fp64 ? 1 : 0;
  return OZ_OK;
}

namespace {
int check_sub_prec(const oz_prec* prec) {
  if (!prec) return oz::api_fail(OZ_EINVAL, "null argument");
  if (prec->mode != OZ_MODE_EAGER && prec->mode != OZ_MODE_NATIVE) return oz::api_fail(OZ_EINVAL, "unknown mode");
  const int lv = prec->level ? prec->level : prec->slices;
  if (prec->slices < 1 || prec->slices > 9 || lv < 1 || lv > prec->slices || lv > oz::MAX_LEVEL)
    return oz::api_fail(OZ_EINVAL, "slices must be in 1..9 and the level in 1..min(S, 8)");
  return OZ_OK;
}
}  // namespace

extern "C" int oz_dmrg_set_renorm_prec(oz_dmrg* d, const oz_prec* prec) {
  if (!d) return oz::api_fail(OZ_EINVAL, "null handle");
  DM_RC(check_sub_prec(prec));
  d->renorm = *prec;
  return OZ_OK;
}

extern "C" int oz_dmrg_set_rdm_prec(oz_dmrg* d, const oz_prec* prec) {
  if (!d) return oz::api_fail(OZ_EINVAL, "null handle");
  DM_RC(check_sub_prec(prec));
  d->rdm = *prec;
  return OZ_OK;
}

extern "C" int oz_dmrg_destroy(oz_dmrg* d) {
  if (!d) return OZ_OK;
  cudaStreamSynchronize(d->st);
  d->left.clear();
  d->right.clear();
  cudaStreamDestroy(d->st);
  delete d;
  return OZ_OK;
}

extern "C" int oz_dmrg_run(oz_dmrg* d, int nsweeps, double* energies) {
  if (!d) return oz::api_fail(OZ_EINVAL, "null handle");
  if (nsweeps < 0) return oz::api_fail(OZ_EINVAL, "nsweeps must be >= 0");
  const int L = d->L;
  const int first = (int)d->steps.size();
  int sweep0 = 0;
  for (const auto& s : d->steps) sweep0 = std::max(sweep0, s.sweep + 1);
  for (int k = 0; k < nsweeps; ++k) {
    for (int i = 0; i <= L - 2; ++i) DM_RC(solve_bond(d, i, 0, sweep0 + k, i < L - 2));
    for (int i = L - 2; i >= 0; --i) DM_RC(solve_bond(d, i, 1, sweep0 + k, i > 0));
  }
  if (energies)
    for (size_t s = first; s < d->steps.size(); ++s) energies[s - first] = d->steps[s].energy;
  return OZ_OK;
}

extern "C" int oz_dmrg_steps(const oz_dmrg* d, oz_dmrg_step* out, int cap, int* n) {
  if (!d || !n) return oz::api_fail(OZ_EINVAL, "null argument");
  *n = (int)d->steps.size();
  if (out)
    for (int i = 0; i < std::min(cap, *n); ++i) out[i] = d->steps[i];
  return OZ_OK;
}

extern "C" int oz_dmrg_bond_heff(oz_dmrg* d, int bond, const double* d_psi, double* d_y, long long* patterns,
                                 long long* dim, oz_stream_t stream) {
  if (!d || !dim) return oz::api_fail(OZ_EINVAL, "null argument");
  if (bond < 0 || bond > d->L - 2) return oz::api_fail(OZ_EINVAL, "bond out of range");
  Bond B;
  DM_RC(make_bond(d, bond, &B));
  *dim = B.dim;
  if (patterns) {
    long long idx = 0;
    for (size_t p = 0; p < B.le.size(); ++p) {
      const auto& pl = B.LE.b.pat[B.le[p]];
      const auto& pr = B.RE.b.pat[B.re[p]];
      for (long long a : pl)
        for (long long b : pr) patterns[idx++] = (a < 0 || b < 0) ? -1 : (a | b);
    }
  }
  if (d_psi && d_y) {
    DM_RC(heff_apply(B.h, d_psi, d_y, stream));
    DM_CU(cudaStreamSynchronize((cudaStream_t)stream));
  }
  return OZ_OK;
}

extern "C" int dmrg_sweep(oz_ctx* ctx, const double* h1, const double* eri, int L, int nelec, int twosz, int D,
                          int nsweeps, const oz_prec* prec, double davidson_tol, unsigned long long seed,
                          double* energies) {
  oz_dmrg* d = nullptr;
  DM_RC(oz_dmrg_create(ctx, h1, eri, L, nelec, twosz, D, prec, davidson_tol, seed, &d));
  const int rc = oz_dmrg_run(d, nsweeps, energies);
  oz_dmrg_destroy(d);
  return rc;
}

extern "C" int oz_dmrg_set_trace(oz_dmrg* d, int stride) {
  if (!d) return oz::api_fail(OZ_EINVAL, "null handle");
  if (stride < 0) return oz::api_fail(OZ_EINVAL, "stride must be >= 0");
  d->trace_stride = stride;
  d->trace.clear();
  return OZ_OK;
}

extern "C" int oz_dmrg_trace(const oz_dmrg* d, long long i, int* info, double* A, double* B, double* C,
                             long long* n) {
  if (!d) return oz::api_fail(OZ_EINVAL, "null handle");
  if (n) *n = (long long)d->trace.size();
  if (i < 0) return OZ_OK;
  if (i >= (long long)d->trace.size()) return oz::api_fail(OZ_EINVAL, "trace record index out of range");
  const oz_dmrg_s::TraceRec& r = d->trace[(size_t)i];
  if (info) {
    const int v[7] = {r.kind, r.step, r.M, r.N, r.K, r.S, r.level};
    std::memcpy(info, v, sizeof(v));
  }
  if (A) std::memcpy(A, r.A.data(), r.A.size() * 8);
  if (B) std::memcpy(B, r.B.data(), r.B.size() * 8);
  if (C) std::memcpy(C, r.C.data(), r.C.size() * 8);
  return OZ_OK;
}
