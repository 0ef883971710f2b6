// Grouped persistent Ozaki GEMM on tcgen05 (declarations).
#pragma once
#include <vector>
#include "oz_common.cuh"

namespace oz {

constexpr int BN = 64;              // output tile columns (MMA N)
constexpr int NBUF = 512 / BN;      // TMEM accumulator buffers of BN columns

constexpr int MAX_LEVEL = 9;        // slice levels supported by the BN = 64 kernel
// Levels up to 8 keep one TMEM buffer per diagonal of the slice grid.  Level 9 (nine 64-column
// accumulators do not fit in TMEM's 512 columns) runs each tile in two passes over its k-blocks:
// diagonals 0..7, then diagonal 8 alone, both into the same exact sums.
constexpr int SPLIT_LEVEL = 9;
__host__ __device__ constexpr int passes_of(int s) { return s == SPLIT_LEVEL ? 2 : 1; }
// Longest reduction of one product.  The exact sum of an output element is bounded by
// K 2^14 sum_g (g+1) 2^(8(s-1-g)) (digit products are at most 2^14 in magnitude) and must stay below
// 2^95, the range of the epilogue's 96-bit sums: any K <= 2^20 at levels up to 8, K <= 130,048
// (= 8128 k-blocks of 16) at level 9.
constexpr long long MAX_K = 1ll << 20;
constexpr long long MAX_K_LEVEL9 = 130048;
inline long long max_k_of_level(int s) { return s >= SPLIT_LEVEL ? MAX_K_LEVEL9 : MAX_K; }

// output modes: dense C[row * ldc + col]; row table (C + rowdst[row] + col, with per-row |max|);
// dense transposed C[col * ldc + row]
enum : int { OUT_DENSE = 0, OUT_ROWTABLE = 1, OUT_DENSE_T = 2 };

// One emulated product C = alpha * (A B) + beta * C at slice level s.
// A: M x K as tiled digit planes (TILE_M-row tiles), B^T: N x K as tiled planes (BN-row tiles).
struct GemmProblem {
  const __half* A;
  const __half* B;
  const int* ea;               // per A row exponent
  const int* eb;               // per B^T row (output column) exponent
  int M, N, nkb;               // sizes, k-blocks of KB
  int SA, SB;                  // planes stored per k-block in A / B^T
  int s;                       // slice level (1..MAX_LEVEL)
  int mode;                    // OUT_DENSE, OUT_ROWTABLE or OUT_DENSE_T
  double* C;                   // dense: C + row * ldc + col;  rowtable: C + rowdst[row] + col
  long long ldc;
  const long long* rowdst;
  const int* rowslot;
  unsigned long long* rowmax;  // rowtable: max |C| per destination slot (atomicMax), may be null
  double alpha, beta;
};

struct GemmTile {
  int prob, mb, nb, pad;
};

size_t gemm_smem_bytes(int smax, bool pair, bool ho = false);
// tiles == nullptr: a single problem (*single) with implicit tiles i -> (i / nnb, i % nnb);
// otherwise smax is the largest slice level among the launch's problems (sizes the pipeline stages).
// d_first (grid + 1 entries, optional): unit b processes tiles [d_first[b], d_first[b+1]) in order;
// without it unit b takes tiles b, b + grid, ...  A unit is one CTA, or with pair = true a CTA pair
// (cluster of two CTAs on two SMs) computing 256 x 64 tiles: tile.mb then counts 256-row blocks, and
// every B^T operand must store the two 32-row halves of each k-block of a 64-row tile one after the
// other (SliceSeg::half_major).  ho selects the epilogue layout: false, 16 owner warps of 16 columns
// (short tiles: fast final conversion); true, 8 owners of 32 columns with lane quarter 1 handed over
// by a loader warp so that the MMA issuer's scheduler partition runs no exact arithmetic (long,
// drain-heavy tiles).  Results are identical.  CTA pairs use the first.
cudaError_t launch_gemm(const GemmProblem* d_probs, const GemmTile* d_tiles, int ntiles, int grid,
                        const GemmProblem* single, int smax, int* d_err, cudaStream_t st,
                        const int* d_first = nullptr, bool pair = false, bool ho = false);
// The epilogue layout for a launch whose tiles average `kb_per_tile` k-blocks.
inline bool gemm_handover_for(double kb_per_tile) { return kb_per_tile >= 48.0; }
// CTA pairs that can run concurrently on the current device for `nsm` SMs (0: none).
int gemm_pair_units(int nsm);
// Balanced assignment of a tile list to `grid` CTAs (longest processing time first, cost of a
// tile = k-blocks x slice pairs + a fixed epilogue share): reorders `tiles` so that CTA b owns
// the range [first[b], first[b+1]).
void balance_tiles(const std::vector<GemmProblem>& probs, std::vector<GemmTile>& tiles, int grid,
                   std::vector<int>& first);
// Schedules of a tile list over `grid` CTAs: balanced (longest first, each CTA's tiles in
// descending cost), balanced with each CTA's tiles in ascending cost, or strided (CTA b takes
// tiles b, b + grid, ... of the given order).
enum : int { SCHED_BALANCED = 0, SCHED_BALANCED_ASC = 1, SCHED_STRIDED = 2, SCHED_COUNT = 3 };
void schedule_tiles(const std::vector<GemmProblem>& probs, std::vector<GemmTile>& tiles, int grid, int mode,
                    std::vector<int>& first);

}  // namespace oz
