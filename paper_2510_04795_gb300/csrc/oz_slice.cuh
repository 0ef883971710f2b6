// Slicing: FP64 rectangles -> shared exponents + balanced INT8 digits stored as FP16 in
// pre-tiled tcgen05 operand layout.
#pragma once
#include <vector>

#include "oz_common.cuh"

namespace oz {

// One rectangle of source values copied into an operand (rows = MMA M or N side, K = reduction).
// Destination element (r0 + i, k0 + j), i < rows, j < cols, comes from
//   trans == 0: src[i * ld + j]      trans == 1: src[j * ld + i]
// multiplied by `scale` (one FP64 rounding) when scale != 1.  k0 must be a multiple of 8.
// The digit pass covers prows x pcols (>= rows x cols) and writes zero digits outside the source.
struct SliceSeg {
  const double* src;
  long long ld;
  int rows, cols;
  int prows, pcols;
  int r0, k0;
  int trans;
  int S;                       // digit planes stored by the operand
  double scale;
  __half* dst;                 // tiled planes: [row tile][k-block][plane][TR x 32 halves]
  int TR;                      // rows per tile of the operand: 128 for A, BN = 64 for B
  int nkb;                     // k-blocks of the operand
  unsigned long long* rowmax;  // per operand row: bit pattern of max |value|
  int* rowexp;                 // per operand row: shared exponent (written by the digit pass)
  long long unit0;             // first digit-pass work unit of this segment (prefix over segments)
  long long unit0m;            // first rowmax-pass work unit of this segment
  int half_major;              // TR = 64 only: the two 32-row halves of each k-block stored apart
                               // ([tile][k-block][half][plane][32 x 16]), for CTA-pair products
};

// Up to 4 segments passed by value (no host-to-device copy for single products).
constexpr int SEGPACK = 4;
struct SegPack {
  SliceSeg seg[SEGPACK];
};

constexpr int ROWMAX_SPAN = 512;  // K elements per rowmax thread of a trans = 1 segment
constexpr int RM_CHUNK = 2048;    // K elements per rowmax warp of a trans = 0 segment
constexpr int RM_ROWS = 8;        // rows per rowmax warp of a trans = 0 segment

// rowmax-pass thread slots of a segment (a multiple of 32; unit0m prefixes are sums of these)
long long rowmax_units(int rows, int cols, int trans);
long long digit_units(int prows, int pcols);
// segments from d_segs (device array) or, when d_segs == nullptr, from pack (nseg <= SEGPACK);
// d_ctaseg (optional, device) = the launch's CTA -> first segment table (rowmax_cta_table /
// digits_cta_table of the same segments and total), which bounds each thread's segment search
cudaError_t launch_rowmax(const SliceSeg* d_segs, const SegPack* pack, int nseg, long long total, int* flags,
                          cudaStream_t st, const int* d_ctaseg = nullptr);
cudaError_t launch_digits(const SliceSeg* d_segs, const SegPack* pack, int nseg, long long total, int S,
                          cudaStream_t st, const int* d_ctaseg = nullptr);
std::vector<int> rowmax_cta_table(const std::vector<SliceSeg>& segs, long long total);
std::vector<int> digits_cta_table(const std::vector<SliceSeg>& segs, long long total);
// untile digits of rows [0,rows) x [0,cols) of an A-role operand into int8 d_out[t][i][j]
cudaError_t launch_untile(const __half* dig, int TR, int nkb, int S, int rows, int cols, int8_t* out,
                          cudaStream_t st);

}  // namespace oz
