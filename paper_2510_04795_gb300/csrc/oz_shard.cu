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
