// Slicing kernels: the fixed-point conversion and 8-bit split of the Ozaki scheme
// (paper, section "Theory of emulated FP64 arithmetic", steps 1 and 2; S slices carry
// 8S-1 magnitude bits plus sign, section "Numerical procedure").
//
//  * rowmax pass: max |x| of every operand row (bit pattern, atomicMax), coalesced reads.
//  * digit pass:  e = smallest integer with max|x| <= (127/128) 2^e;  X = RN_even(x 2^(8S-1-e));
//                 balanced base-256 digits d_1..d_S in [-128,127]; each written as an FP16
//                 value into the tcgen05 operand tiles (16-byte stores, 8 K-elements each).
// Only integer operations touch the values after the (optional) scale multiply.
#include "oz_slice.cuh"

#include <vector>

namespace oz {

// Segment of a work unit: binary search over the unit prefixes, restricted to the CTA's range
// [ctaseg[b], ctaseg[b + 1]] when the launch carries that table (launches over many segments).
template <bool MAXPASS>
__device__ __forceinline__ const SliceSeg& find_seg(const SliceSeg* segs, const SegPack& pack, int nseg,
                                                    long long unit, const int* ctaseg) {
  const SliceSeg* base = segs ? segs : pack.seg;
  int lo = 0, hi = nseg - 1;
  if (ctaseg) {
    lo = __ldg(ctaseg + blockIdx.x);
    hi = __ldg(ctaseg + blockIdx.x + 1);
  }
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    long long u0 = MAXPASS ? base[mid].unit0m : base[mid].unit0;
    if (u0 <= unit) lo = mid; else hi = mid - 1;
  }
  return base[lo];
}

__device__ __forceinline__ unsigned long long absbits(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
}

// Row maxima, two access patterns chosen per segment so that every warp load is coalesced:
//  * trans == 0 (rows contiguous in memory): one warp per (RM_ROWS rows, RM_CHUNK columns); lane l
//    reads columns l, l + 32, ... of all its rows together (256 consecutive bytes per warp load,
//    2 RM_ROWS loads in flight per lane), then a warp-shuffle max and one atomicMax per row;
//  * trans == 1 (consecutive rows adjacent in memory): one thread per (row, ROWMAX_SPAN
//    columns), consecutive threads on consecutive rows (256 consecutive bytes per warp load).
// Segment slot counts are multiples of 32, so no warp straddles two segments.
// Bit pattern of max_j |RN(c x_j)| from that of max_j |x_j|: rounding is monotonic, so the maximum of
// the scaled magnitudes is the scaled maximum, RN(|c| max_j |x_j|) -- one multiply per row instead of
// one per element.  NaN and Inf patterns pass through (their products stay non-finite).
__device__ __forceinline__ unsigned long long scaled_max(unsigned long long mb, double c) {
  if (c == 1.0 || mb == 0ull) return mb;
  return absbits(__dmul_rn(__longlong_as_double((long long)mb), fabs(c)));
}

// |x| as 32-bit halves (x = lo, y = hi) of its bit pattern
__device__ __forceinline__ uint2 ldg_bits(const double* p) {
  const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
  return make_uint2(v.x, v.y & 0x7FFFFFFFu);
}
// (mh, ml) = max((mh, ml), v) in the order of the 64-bit patterns, with 32-bit comparisons
__device__ __forceinline__ void max_hl(uint32_t& mh, uint32_t& ml, uint2 v) {
  const bool gt = v.y > mh || (v.y == mh && v.x > ml);
  mh = gt ? v.y : mh;
  ml = gt ? v.x : ml;
}

__global__ void __launch_bounds__(256) rowmax_kernel(const SliceSeg* __restrict__ segs,
                                                     const __grid_constant__ SegPack pack, int nseg, long long total,
                                                     int* __restrict__ flags, const int* __restrict__ ctaseg) {
  const long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= total) return;  // total is a multiple of 32: whole warps leave together
  const SliceSeg& g = find_seg<true>(segs, pack, nseg, u, ctaseg);
  const long long lu = u - g.unit0m;
  unsigned long long mx = 0;
  int row = -1;
  if (!g.trans) {
    // warp w of the segment: column chunk w % nch of the rows RM_ROWS (w / nch) .. + RM_ROWS - 1
    const int lane = (int)(lu & 31);
    const long long w = lu >> 5;
    const int nch = (g.cols + RM_CHUNK - 1) / RM_CHUNK;
    const int r0 = (int)(w / nch) * RM_ROWS, nr = min(g.rows - r0, RM_ROWS);
    const int j0 = (int)(w % nch) * RM_CHUNK, j1 = min(g.cols, j0 + RM_CHUNK);
    const double* rp = g.src + (long long)r0 * g.ld;
    // all rows of the warp at once: 2 RM_ROWS loads in flight per lane whatever the row length.
    // (16-byte loads of aligned column pairs were measured slower: their registers halve the
    // resident warps.)  The maxima are kept as 32-bit halves and compared with 32-bit integer
    // operations only: the magnitudes are non-negative, so (hi, lo) order is the 64-bit order.
    uint32_t mh[RM_ROWS], ml[RM_ROWS];
#pragma unroll
    for (int r = 0; r < RM_ROWS; ++r) mh[r] = ml[r] = 0u;
    int j = j0 + lane;
    for (; j + 32 < j1; j += 64) {
      uint2 b0[RM_ROWS], b1[RM_ROWS];
#pragma unroll
      for (int r = 0; r < RM_ROWS; ++r) {
        b0[r] = r < nr ? ldg_bits(rp + r * g.ld + j) : make_uint2(0u, 0u);
        b1[r] = r < nr ? ldg_bits(rp + r * g.ld + j + 32) : make_uint2(0u, 0u);
      }
#pragma unroll
      for (int r = 0; r < RM_ROWS; ++r) {
        max_hl(mh[r], ml[r], b0[r]);
        max_hl(mh[r], ml[r], b1[r]);
      }
    }
    if (j < j1) {
#pragma unroll
      for (int r = 0; r < RM_ROWS; ++r)
        if (r < nr) max_hl(mh[r], ml[r], ldg_bits(rp + r * g.ld + j));
    }
    // 8 row maxima over 32 lanes in 3 halving exchanges and 2 plain ones: after the exchange over
    // lane bit 16 (8, 4) a lane keeps the half of its rows selected by that bit, so lane 4k ends
    // with the maximum of row k over all lanes
    static_assert(RM_ROWS == 8, "the exchange below reduces 8 rows");
#pragma unroll
    for (int o = 16, n = RM_ROWS; o >= 4; o >>= 1, n >>= 1) {
      const bool hi = (lane & o) != 0;
#pragma unroll
      for (int i = 0; i < RM_ROWS / 2; ++i) {
        if (i < n / 2) {
          const uint32_t sh = hi ? mh[i] : mh[i + n / 2], sl = hi ? ml[i] : ml[i + n / 2];
          const uint32_t kh = hi ? mh[i + n / 2] : mh[i], kl = hi ? ml[i + n / 2] : ml[i];
          const uint2 recv = make_uint2(__shfl_xor_sync(0xffffffffu, sl, o), __shfl_xor_sync(0xffffffffu, sh, o));
          mh[i] = kh;
          ml[i] = kl;
          max_hl(mh[i], ml[i], recv);
        }
      }
    }
#pragma unroll
    for (int o = 2; o > 0; o >>= 1) {
      const uint2 recv = make_uint2(__shfl_xor_sync(0xffffffffu, ml[0], o), __shfl_xor_sync(0xffffffffu, mh[0], o));
      max_hl(mh[0], ml[0], recv);
    }
    const unsigned long long m0 = ((unsigned long long)mh[0] << 32) | ml[0];
    const int r = lane >> 2;
    if ((lane & 3) == 0 && r < nr) {
      const unsigned long long mm = scaled_max(m0, g.scale);
      if (mm >= 0x7FF0000000000000ull) atomicOr(flags, 1);  // Inf or NaN in the input
      if (mm) atomicMax(g.rowmax + g.r0 + r0 + r, mm);
    }
    return;
  } else {
    const long long nsp = (g.cols + ROWMAX_SPAN - 1) / ROWMAX_SPAN;
    if (lu >= (long long)g.rows * nsp) return;
    row = (int)(lu % g.rows);
    const int sp = (int)(lu / g.rows);
    const int j0 = sp * ROWMAX_SPAN, j1 = min(g.cols, j0 + ROWMAX_SPAN);
    uint32_t mh = 0u, ml = 0u;
    for (int j = j0; j < j1; ++j) max_hl(mh, ml, ldg_bits(g.src + (long long)j * g.ld + row));
    mx = scaled_max(((unsigned long long)mh << 32) | ml, g.scale);
  }
  if (row < 0) return;
  if (mx >= 0x7FF0000000000000ull) atomicOr(flags, 1);  // Inf or NaN in the input
  if (mx) atomicMax(g.rowmax + g.r0 + row, mx);
}

// RN_even(|x| * 2^sh) for the 53-bit significand M of x and a shift sh; exact integer result.
// A right shift by r rounds to nearest even as floor((M + 2^(r-1) - 1 + q0) / 2^r), q0 the lowest
// bit of the truncated quotient: a remainder below the half stays below 2^r, above it reaches
// 2^r, and exactly the half rounds up only when q0 = 1.  (No 64-bit comparisons: on this GPU those
// issue to the FP64 pipe.)  M < 2^53, so M + 2^62 does not overflow.
__device__ __forceinline__ unsigned long long round_shift(unsigned long long M, int sh) {
  if (sh >= 0) return M << sh;  // caller guarantees no overflow
  const int r = -sh;
  if (r >= 64) return 0ull;     // M < 2^53 <= 2^(r-1): below the half
  const unsigned long long q0 = (M >> r) & 1ull;
  return (M + ((1ull << (r - 1)) - 1ull) + q0) >> r;
}

// fixed point of one value: X = RN_even(|x| 2^(8S-1-e)) with sign; S <= 8 (fits int64)
__device__ __forceinline__ long long fixed_point64(double x, int e, int S) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  int be = (int)((b >> 52) & 0x7FF);
  unsigned long long f = b & ((1ull << 52) - 1);
  // (a zero gives M = 0 and X = 0 through the same arithmetic)
  unsigned long long M = be ? (f | (1ull << 52)) : f;
  int bee = be ? be : 1;
  int sh = bee - 1075 + 8 * S - 1 - e;
  long long X = (long long)round_shift(M, sh);
  return (b >> 63) ? -X : X;
}

__device__ __forceinline__ __int128 fixed_point128(double x, int e, int S) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  int be = (int)((b >> 52) & 0x7FF);
  unsigned long long f = b & ((1ull << 52) - 1);
  if (be == 0 && f == 0) return 0;
  unsigned long long M = be ? (f | (1ull << 52)) : f;
  int bee = be ? be : 1;
  int sh = bee - 1075 + 8 * S - 1 - e;
  __int128 X = sh >= 0 ? ((__int128)M << sh) : (__int128)round_shift(M, sh);
  return (b >> 63) ? -X : X;
}

template <int S>
__global__ void __launch_bounds__(256) digits_kernel(const SliceSeg* __restrict__ segs,
                                                     const __grid_constant__ SegPack pack, int nseg, long long total,
                                                     const int* __restrict__ ctaseg) {
  long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long u = tid >> 3;
  if (u >= total) return;
  int r8 = (int)(tid & 7);
  const SliceSeg& g = find_seg<false>(segs, pack, nseg, u, ctaseg);
  // unit -> (8-row group, 8-column chunk) of the segment, by 32-bit division: a segment's source is
  // resident FP64 data (below 2^35 elements in 288 GB), so it has fewer than 2^30 units of 64 elements
  const uint32_t lu = (uint32_t)(u - g.unit0);
  const uint32_t nkc = (uint32_t)(g.pcols + 7) >> 3;
  const uint32_t rgi = lu / nkc;
  const int rg = (int)rgi, c = (int)(lu - rgi * nkc);
  int i = rg * 8 + r8;
  if (i >= g.prows) return;
  int R = g.r0 + i;
  const bool rowok = i < g.rows;
  const bool scaled = g.scale != 1.0;  // one FP64 compare per thread
  int e = rowok ? exponent_from_maxbits(g.rowmax[R]) : 0;
  if (c == 0) g.rowexp[R] = e;
  // the 8 values: one 64-byte run of the row, read as four 16-byte loads where it is aligned
  double vals[8];
  const int j0 = c * 8;
  if (!rowok) {
#pragma unroll
    for (int q = 0; q < 8; ++q) vals[q] = 0.0;
  } else if (!g.trans) {
    const double* rp = g.src + (long long)i * g.ld + j0;
    if (j0 + 8 <= g.cols && ((reinterpret_cast<uintptr_t>(rp) & 15) == 0)) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const double2 w = __ldg(reinterpret_cast<const double2*>(rp) + q);
        vals[2 * q] = w.x;
        vals[2 * q + 1] = w.y;
      }
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) vals[q] = j0 + q < g.cols ? __ldg(rp + q) : 0.0;
    }
  } else {
    const double* cp = g.src + (long long)j0 * g.ld + i;
#pragma unroll
    for (int q = 0; q < 8; ++q) vals[q] = j0 + q < g.cols ? __ldg(cp + (long long)q * g.ld) : 0.0;
  }
  if (scaled) {
#pragma unroll
    for (int q = 0; q < 8; ++q) vals[q] = __dmul_rn(vals[q], g.scale);
  }
  int K = g.k0 + c * 8;
  // TR is 64 or 128
  const int trs = g.TR == 128 ? 7 : 6;
  int rt = R >> trs, rr = R & (g.TR - 1), kb = K >> KB_SHIFT, kk = K & (KB - 1);
  // plane t of (row, k) at base + t * pstride; a half-major operand stores the 32-row halves of each
  // k-block of a tile one after the other (each half: S planes of 32 rows)
  long long base;
  int pstride;
  if (g.half_major) {
    base = ((((long long)rt * g.nkb + kb) * 2 + (rr >> 5)) * g.S) * (long long)(32 * KB) + tile_off(rr & 31, kk);
    pstride = 32 * KB;
  } else {
    base = (((long long)rt * g.nkb + kb) * g.S) * (long long)(g.TR * KB) + tile_off(rr, kk);
    pstride = g.TR * KB;
  }
  if constexpr (S <= 8) {
    // Balanced base-256 digits by one add: with Y = X + sum_t 128 * 256^t (0 <= Y < 256^S because
    // the exponent rule keeps |X| <= 127 * 256^(S-1)), byte t of Y is d + 128 for the digit of
    // weight 256^t.  Each byte b becomes the FP16 value 1024 + b by placing it under the exponent
    // bits 0x6400, and one half2 subtraction of 1152 leaves the digit itself, exactly.
    constexpr unsigned long long BIAS = 0x8080808080808080ull >> (8 * (8 - S));
    uint32_t ylo[8], yhi[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const unsigned long long Y = (unsigned long long)fixed_point64(vals[q], e, S) + BIAS;
      ylo[q] = (uint32_t)Y;
      yhi[q] = (uint32_t)(Y >> 32);
    }
    const __half2 off = __halves2half2(__float2half_rn(1152.0f), __float2half_rn(1152.0f));
#pragma unroll
    for (int t = 0; t < S; ++t) {
      const int bi = S - 1 - t;  // plane t holds the digit of weight 256^(S-1-t)
      // byte bi of element 2p into byte 0 and of element 2p+1 into byte 2 (selector nibbles 0, 2)
      const uint32_t sel = (uint32_t)((bi & 3) | (((bi & 3) + 4) << 8));
      uint4 o;
      uint32_t* op = reinterpret_cast<uint32_t*>(&o);
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const uint32_t a = bi < 4 ? ylo[2 * p] : yhi[2 * p], b = bi < 4 ? ylo[2 * p + 1] : yhi[2 * p + 1];
        const uint32_t bits = (__byte_perm(a, b, sel) & 0x00FF00FFu) | 0x64006400u;
        __half2 h = *reinterpret_cast<const __half2*>(&bits);
        h = __hsub2(h, off);
        op[p] = *reinterpret_cast<uint32_t*>(&h);
      }
      *reinterpret_cast<uint4*>(g.dst + base + (long long)t * pstride) = o;
    }
  } else {
    // S = 9: the fixed-point value needs more than 64 bits
    int d[S][8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const double v = vals[q];
      {
        __int128 X = fixed_point128(v, e, S);
#pragma unroll
        for (int t = S - 1; t >= 0; --t) {
          int dd = (int)((X + 128) & 255) - 128;
          d[t][q] = dd;
          X = (X - dd) >> 8;
        }
      }
    }
#pragma unroll
    for (int t = 0; t < S; ++t) {
      __half2 h0 = __halves2half2(__int2half_rn(d[t][0]), __int2half_rn(d[t][1]));
      __half2 h1 = __halves2half2(__int2half_rn(d[t][2]), __int2half_rn(d[t][3]));
      __half2 h2 = __halves2half2(__int2half_rn(d[t][4]), __int2half_rn(d[t][5]));
      __half2 h3 = __halves2half2(__int2half_rn(d[t][6]), __int2half_rn(d[t][7]));
      uint4 w;
      w.x = *reinterpret_cast<uint32_t*>(&h0);
      w.y = *reinterpret_cast<uint32_t*>(&h1);
      w.z = *reinterpret_cast<uint32_t*>(&h2);
      w.w = *reinterpret_cast<uint32_t*>(&h3);
      *reinterpret_cast<uint4*>(g.dst + base + (long long)t * pstride) = w;
    }
  }
}

long long rowmax_units(int rows, int cols, int trans) {
  if (rows <= 0 || cols <= 0) return 0;
  if (!trans) return 32ll * ((rows + RM_ROWS - 1) / RM_ROWS) * ((cols + RM_CHUNK - 1) / RM_CHUNK);
  const long long t = (long long)rows * ((cols + ROWMAX_SPAN - 1) / ROWMAX_SPAN);
  return (t + 31) / 32 * 32;
}
long long digit_units(int prows, int pcols) { return (long long)((prows + 7) / 8) * ((pcols + 7) / 8); }

cudaError_t launch_rowmax(const SliceSeg* d_segs, const SegPack* pack, int nseg, long long total, int* flags,
                          cudaStream_t st, const int* d_ctaseg) {
  if (total <= 0) return cudaSuccess;
  SegPack p{};
  if (!d_segs) p = *pack;
  long long blocks = (total + 255) / 256;
  rowmax_kernel<<<(unsigned)blocks, 256, 0, st>>>(d_segs, p, nseg, total, flags, d_ctaseg);
  return cudaGetLastError();
}

// CTA -> first segment tables of the two slicing launches: CTA b of the rowmax launch covers the
// thread slots [256 b, 256 b + 256), CTA b of the digit launch the units [32 b, 32 b + 32); entry
// b is the segment holding the CTA's first slot or unit, and the last entry is nseg - 1.
static std::vector<int> cta_table(const std::vector<SliceSeg>& segs, long long total, long long per_cta,
                                  bool maxpass) {
  const long long nb = (total + per_cta - 1) / per_cta;
  std::vector<int> t((size_t)nb + 1);
  int k = 0;
  const int n = (int)segs.size();
  for (long long b = 0; b < nb; ++b) {
    const long long u = b * per_cta;
    while (k + 1 < n && (maxpass ? segs[k + 1].unit0m : segs[k + 1].unit0) <= u) ++k;
    t[(size_t)b] = k;
  }
  t[(size_t)nb] = n - 1;
  return t;
}
std::vector<int> rowmax_cta_table(const std::vector<SliceSeg>& segs, long long total) {
  return cta_table(segs, total, 256, true);
}
std::vector<int> digits_cta_table(const std::vector<SliceSeg>& segs, long long total) {
  return cta_table(segs, total, 32, false);
}

__global__ void untile_kernel(const __half* __restrict__ dig, int TR, int nkb, int S, int rows, int cols,
                              int8_t* __restrict__ out) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long total = (long long)S * rows * cols;
  if (idx >= total) return;
  int j = (int)(idx % cols);
  int i = (int)((idx / cols) % rows);
  int t = (int)(idx / ((long long)rows * cols));
  int rt = i / TR, rr = i % TR, kb = j >> KB_SHIFT, kk = j & (KB - 1);
  long long off = (((long long)rt * nkb + kb) * S + t) * (long long)(TR * KB) + tile_off(rr, kk);
  out[idx] = (int8_t)__half2int_rn(dig[off]);
}

cudaError_t launch_untile(const __half* dig, int TR, int nkb, int S, int rows, int cols, int8_t* out,
                          cudaStream_t st) {
  long long total = (long long)S * rows * cols;
  if (total <= 0) return cudaSuccess;
  untile_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(dig, TR, nkb, S, rows, cols, out);
  return cudaGetLastError();
}

cudaError_t launch_digits(const SliceSeg* d_segs, const SegPack* pack, int nseg, long long total, int S,
                          cudaStream_t st, const int* d_ctaseg) {
  if (total <= 0) return cudaSuccess;
  SegPack p{};
  if (!d_segs) p = *pack;
  long long blocks = (total * 8 + 255) / 256;
  switch (S) {
#define OZ_CASE(s) case s: digits_kernel<s><<<(unsigned)blocks, 256, 0, st>>>(d_segs, p, nseg, total, d_ctaseg); break;
    OZ_CASE(1) OZ_CASE(2) OZ_CASE(3) OZ_CASE(4) OZ_CASE(5) OZ_CASE(6) OZ_CASE(7) OZ_CASE(8) OZ_CASE(9)
#undef OZ_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace oz
