// Term sharding of H_eff psi over several GPUs (host partition and the ordered reduction).
//
// H_eff psi = sum over tasks of coef L psi[src] R^T into Y[dst] splits over the tasks: every rank
// keeps the operator blocks of its own tasks (where the memory goes) and computes a partial Y
// with heff_apply on a handle built from those tasks; the partial vectors are then exchanged and
// summed.  The paper runs its sweeps on one multi-GPU node; it does not describe how the
// effective-Hamiltonian work is divided, so this follows the natural split of the sum.
//
//  * oz_heff_partition: a deterministic balanced assignment of tasks to ranks (host only, the
//    same on every rank): tasks in descending order of FP64 flop cost, each onto the rank with
//    the least work so far (ties to the lower rank, equal costs in task order).
//  * oz_reduce_ordered: out = ((p_0 + p_1) + p_2) + ... in FP64, element by element in rank
//    order, so the reduced vector does not depend on the order in which the parts arrived.
//  * oz_heff_apply_streamed: the same split on ONE GPU for structures whose operator digit planes
//    do not fit at once: the groups of the partition are built, applied and released one after
//    the other, their partial vectors summed in group order as they come.
#include <cuda_runtime.h>

#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "ozdmrg.h"
#include "oz_internal.cuh"

namespace {

constexpr int MAX_PARTS = 64;

struct Parts {
  const double* p[MAX_PARTS];
};

__global__ void reduce_ordered_kernel(const __grid_constant__ Parts parts, int nparts, long long len,
                                      double* __restrict__ out) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride) {
    double acc = parts.p[0][i];
    for (int r = 1; r < nparts; ++r) acc = __dadd_rn(acc, parts.p[r][i]);
    out[i] = acc;
  }
}

}  // namespace

extern "C" int oz_heff_partition(int nsec, const int* m, const int* n, int ntask, const int* src, const int* dst,
                                 int world, int* owner) {
  if (world < 1) return oz::api_fail(OZ_EINVAL, "world must be >= 1");
  if (nsec <= 0 || ntask < 0 || !m || !n || (ntask > 0 && (!src || !dst || !owner)))
    return oz::api_fail(OZ_EINVAL, "bad structure");
  std::vector<long long> cost(ntask);
  for (int t = 0; t < ntask; ++t) {
    const int s = src[t], d = dst[t];
    if (s < 0 || s >= nsec || d < 0 || d >= nsec) return oz::api_fail(OZ_EINVAL, "task sector out of range");
    // FP64 flops of the task: T = L psi[src] (m[d] x m[s] x n[s]), then T R^T (m[d] x n[s] x n[d])
    cost[t] = 2ll * m[d] * m[s] * n[s] + 2ll * m[d] * n[s] * n[d];
  }
  std::vector<int> ord(ntask);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<long long> load(world, 0);
  for (int t : ord) {
    int r = 0;
    for (int k = 1; k < world; ++k)
      if (load[k] < load[r]) r = k;
    owner[t] = r;
    load[r] += cost[t];
  }
  return OZ_OK;
}

extern "C" int oz_reduce_ordered(const double* const* d_parts, int nparts, long long len, double* d_out,
                                 oz_stream_t stream) {
  if (nparts < 1 || nparts > MAX_PARTS) return oz::api_fail(OZ_EINVAL, "nparts must be in 1..64");
  if (len < 0 || !d_parts || (len > 0 && !d_out)) return oz::api_fail(OZ_EINVAL, "bad arguments");
  if (len == 0) return OZ_OK;
  Parts P{};
  for (int r = 0; r < nparts; ++r) {
    if (!d_parts[r]) return oz::api_fail(OZ_EINVAL, "a part is null");
    P.p[r] = d_parts[r];
  }
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return oz::api_fail(OZ_ECUDA, std::string("device query: ") + cudaGetErrorString(e));
  const long long want = (len + 255) / 256;
  const int grid = (int)std::min<long long>(want, 8ll * nsm);
  reduce_ordered_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(P, nparts, len, d_out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return oz::api_fail(OZ_ECUDA, std::string("reduce_ordered: ") + cudaGetErrorString(e));
  return OZ_OK;
}

extern "C" int oz_heff_apply_streamed(oz_ctx* ctx, int nsec, const int* m, const int* n, int ntask,
                                      const oz_task* tasks, const oz_prec* prec, int chunks, const double* d_psi,
                                      double* d_y, oz_stream_t stream) {
  if (!ctx || !prec || !d_psi || !d_y) return oz::api_fail(OZ_EINVAL, "null argument");
  if (chunks < 1) return oz::api_fail(OZ_EINVAL, "chunks must be >= 1");
  if (nsec <= 0 || ntask < 0 || !m || !n || (ntask > 0 && !tasks)) return oz::api_fail(OZ_EINVAL, "bad structure");
  long long dim = 0;
  for (int q = 0; q < nsec; ++q) {
    if (m[q] <= 0 || n[q] <= 0) return oz::api_fail(OZ_EINVAL, "sector dims must be positive");
    dim += (long long)m[q] * n[q];
  }
  std::vector<int> src(ntask), dst(ntask), owner(ntask);
  for (int t = 0; t < ntask; ++t) {
    src[t] = tasks[t].src;
    dst[t] = tasks[t].dst;
  }
  if (int rc = oz_heff_partition(nsec, m, n, ntask, src.data(), dst.data(), chunks, owner.data())) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  double* part = nullptr;  // the partial product of one group
  if (chunks > 1) {
    cudaError_t e = cudaMalloc(&part, (size_t)std::max(dim, 1ll) * 8);
    if (e != cudaSuccess)
      return oz::api_fail(e == cudaErrorMemoryAllocation ? OZ_ENOMEM : OZ_ECUDA, "streamed partial vector");
  }
  int rc = OZ_OK;
  std::vector<oz_task> group;
  group.reserve(ntask);
  for (int r = 0; r < chunks && rc == OZ_OK; ++r) {
    group.clear();
    for (int t = 0; t < ntask; ++t)
      if (owner[t] == r) group.push_back(tasks[t]);
    // group 0 writes d_y; every later group writes its partial and is added in group order
    double* out = r == 0 ? d_y : part;
    oz_heff* h = nullptr;
    rc = oz_heff_create(ctx, nsec, m, n, (int)group.size(), group.data(), prec, &h);
    if (rc == OZ_OK) rc = heff_apply(h, d_psi, out, stream);
    if (rc == OZ_OK) rc = oz_status(ctx, stream);  // surfaces device-side conditions of the group
    if (h) {
      const int rd = oz_heff_destroy(h);
      if (rc == OZ_OK) rc = rd;
    }
    if (rc == OZ_OK && r > 0) {
      const double* pp[2] = {d_y, part};
      rc = oz_reduce_ordered(pp, 2, dim, d_y, stream);
    }
  }
  if (part) {
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(part);
    if (rc == OZ_OK && e != cudaSuccess) rc = oz::api_fail(OZ_ECUDA, std::string("streamed: ") + cudaGetErrorString(e));
  }
  return rc;
}
