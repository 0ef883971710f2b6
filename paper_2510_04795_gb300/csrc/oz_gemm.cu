// Grouped persistent Ozaki GEMM (paper, section "Theory of emulated FP64 arithmetic", steps 3-4:
// every kept slice pair A^t B^u multiplied in low precision, products accumulated at high
// precision and converted back to FP64; the pairs with t + u > s + 1 -- the "lower-triangular"
// part of the s x s grid -- are skipped).
//
// Carrier: the INT8 digits are exact FP16 values; tcgen05.mma.kind::f16 multiplies them into an
// FP32 accumulator in TMEM.  Every product is an integer of magnitude <= 2^14 and every
// accumulator group holds at most GROUP_TERMS = 1008 products, so each FP32 partial sum is an
// integer below 2^24 and the accumulation is exact (checked on the device against int64).
//
// One CTA per SM, persistent over a tile list:
//   warp 0       producer: cp.async.bulk of pre-tiled digit planes into a ring of shared-memory stages
//   warp 1       TMEM owner and single-thread MMA issuer; diagonal g = t+u (0-based) of the slice
//                grid accumulates into its own TMEM buffer (BN columns), A reused through the
//                collector across the u loop; a buffer whose group is full is handed to the
//                epilogue ("drain": one tcgen05.commit) and replaced by a free one
//   epilogue     replays the same deterministic drain/buffer schedule: owner warps of exact running
//                sums read each drained buffer, add q * 256^(s-1-g) into their sums, then round
//                once to FP64 scaled by 2^(ea+eb-8s-6), apply alpha/beta, store (and for the
//                row-table mode record a per-row |max| for the next slicing).  Two layouts, chosen
//                per launch (gemm_kernel<PAIR, HO>, see EpiCfg): 16 owners of 16 columns, or 8 owners
//                of 32 columns with the MMA issuer's scheduler partition kept free of the exact
//                arithmetic (a loader warp hands TMEM lane quarter 1 to owners elsewhere).
// CTA pairs (gemm_kernel<true, false>, clusters of two CTAs on two SMs): one tile is 256 x 64; each CTA
// loads its own 128 A rows and one 32-row half of the 64 B^T rows (the operand stores the halves of
// each k-block apart), the first CTA's thread issues cta_group::2 MMAs of M = 256 for both (each CTA
// accumulates its 128 rows in its own TMEM), commits signal the barriers of both CTAs, the second
// CTA's warp 1 forwards its operand arrivals to the first CTA's stage barriers, and both epilogues
// release drained buffers on the first CTA's barriers.  One issuing thread then drives two SMs.
// Measured on GB300 it is not faster: a pair instruction takes about as long in the running kernel
// as two single-CTA ones on two SMs, and each drain waits for the slower of two epilogues, so the
// single-CTA tiles stay the default.
// The drain schedule: diagonal g takes p = 16(g+1) products per k-block; its groups hold
// floor(GROUP_TERMS/p) k-blocks (the first group of long tiles is shortened per diagonal so that the
// drains of different diagonals do not coincide).  The first k-block of a tile is issued diagonal by
// diagonal, heaviest first, so that it starts while the previous tile's last buffers are drained.
// Every wait is bounded; a timeout sets *err and all roles leave their loops.
#include "oz_gemm.cuh"

#include <algorithm>
#include <atomic>
#include <utility>
#include <vector>

namespace oz {

constexpr int A_TILE_BYTES = TILE_M * KB * 2;             // 4 KB per plane
constexpr int B_TILE_BYTES = BN * KB * 2;                 // 2 KB per plane
constexpr int BH_BYTES = B_TILE_BYTES / 2;                // a CTA pair: each CTA's half (32 rows) of a B^T plane
__host__ __device__ constexpr int plane_bytes(bool pair) { return A_TILE_BYTES + (pair ? BH_BYTES : B_TILE_BYTES); }
constexpr int MAX_STAGES = 4;
constexpr int HO_SLOTS = 4;                               // hand-over slots of lane quarter 1
constexpr int HO_BYTES = HO_SLOTS * 32 * BN * 4;
// Final-stage staging: per owner warp, 32 rows x ZC columns of 16-byte exact sums (converted in
// place to doubles); row stride (ZC + 1) x 16 bytes against bank conflicts.
constexpr int ZC = 4;
constexpr int ZS_LD = ZC + 1;
// Two epilogue layouts, chosen per launch (a warp runs on scheduler partition warp % 4 and may read
// only TMEM lane quarter warp % 4):
//  * HO = false: 18 warps -- 0 producer, 1 MMA issuer, 2..17 owners of the exact sums, four per lane
//    quarter with 16 columns each.  Many owners keep the final conversion of short tiles fast.
//  * HO = true: 12 warps, 3 per partition -- 0 producer, 1 issuer; owners of 32 columns: quarter 0:
//    4, 8; quarter 2: 2, 6; quarter 3: 3, 7; quarter 1: 10, 11 (partitions 2 and 3), fed by warp 5,
//    the loader of lane quarter 1, which reads the drained buffer's lanes 32..63 and hands them over
//    through shared memory, so that the issuer's partition runs no exact arithmetic; warp 9 idles.
//    Drain-heavy long tiles run faster this way.
template <bool HO>
struct EpiCfg {
  static constexpr int NWARPS = HO ? 12 : 18;
  static constexpr int NTHREADS = 32 * NWARPS;
  static constexpr int OWNERS = HO ? 8 : 16;              // warps holding exact sums
  static constexpr int CW = BN / (HO ? 2 : 4);            // columns per owner
  static constexpr int READERS = HO ? 7 : 16;             // warps reading TMEM per drain
  static constexpr int ZS_BYTES = OWNERS * 32 * ZS_LD * 16 + (HO ? HO_BYTES : 0);
};
constexpr int SMEM_LIMIT = 232448;                        // opt-in shared memory per block

struct Shared {
  unsigned long long full[MAX_STAGES], empty[MAX_STAGES], accf[NBUF], acce[NBUF], fin;
  unsigned long long hfull[HO_SLOTS], hempty[HO_SLOTS];  // quarter-1 hand-over: loader -> owners 10, 11
  uint32_t tmem;
  int abort;
};

// pipeline stages that fit next to the staging area for slice level smax
static int zs_bytes(bool ho) { return ho ? EpiCfg<true>::ZS_BYTES : EpiCfg<false>::ZS_BYTES; }
int gemm_stages(int smax, bool pair, bool ho) {
  const int avail = SMEM_LIMIT - zs_bytes(ho) - (int)sizeof(Shared) - 1024;
  const int n = avail / (smax * plane_bytes(pair));
  return n < MAX_STAGES ? n : MAX_STAGES;
}
size_t gemm_smem_bytes(int smax, bool pair, bool ho) {
  return (size_t)gemm_stages(smax, pair, ho) * smax * plane_bytes(pair) + zs_bytes(ho) + sizeof(Shared) + 1024;
}

__device__ __forceinline__ uint32_t bar(const unsigned long long* p) { return smem_u32(p); }

// position in the stage ring: stage index and the parity of its current fill
struct Ring {
  int stg, ph, n;
  __device__ __forceinline__ void advance() {
    if (++stg == n) {
      stg = 0;
      ph ^= 1;
    }
  }
};

// Deterministic TMEM buffer assignment, replayed identically by the MMA issuer and the epilogue:
// the n-th acquisition returns buffer n while n < NBUF, afterwards the buffer of post n - NBUF.
struct BufRing {
  uint32_t ring;  // buffers of the last 8 posts, 4 bits each
  int nacq, npost;
  __device__ __forceinline__ uint32_t next() {
    const uint32_t b = nacq < NBUF ? (uint32_t)nacq : (ring >> (4 * ((nacq - NBUF) & 7))) & 0xFu;
    ++nacq;
    return b;
  }
  __device__ __forceinline__ void posted(uint32_t b) {
    const int j = npost & 7;
    ring = (ring & ~(0xFu << (4 * j))) | (b << (4 * j));
    ++npost;
  }
};

// k-block of the first drain of diagonal g and the drain period (both in k-blocks)
__device__ __forceinline__ void drain_plan(int g, int S, bool stagger, int& first, int& period) {
  const int p = 16 * (g + 1);
  period = GROUP_TERMS / p;
  const int room0 = stagger ? GROUP_TERMS - p * ((g * period) / S) : GROUP_TERMS;
  first = room0 / p;
}
__device__ __forceinline__ bool stagger_of(int nkb) { return nkb >= 64; }

struct MmaCtl {
  Ring rg;
  BufRing r;
  uint32_t acce_par;  // per buffer parity of the next "drained" wait
};

__device__ __forceinline__ uint32_t acquire(Shared& sh, MmaCtl& c, volatile int* abort) {
  const bool reused = c.r.nacq >= NBUF;
  const uint32_t b = c.r.next();
  if (reused) {
    mbar_wait(bar(&sh.acce[b]), (c.acce_par >> b) & 1u, abort);
    c.acce_par ^= 1u << b;
    tc_fence_after();
  }
  return b;
}
template <bool PAIR>
__device__ __forceinline__ void commit_to(uint32_t mbar) {
  if constexpr (PAIR) tc_commit_pair(mbar);
  else tc_commit(mbar);
}
template <bool PAIR, int COL>
__device__ __forceinline__ void mma_issue(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  if constexpr (PAIR) mma_f16_pair<COL>(d, a, b, id, acc);
  else mma_f16<COL>(d, a, b, id, acc);
}
template <bool PAIR>
__device__ __forceinline__ void post(Shared& sh, MmaCtl& c, uint32_t b) {
  commit_to<PAIR>(bar(&sh.accf[b]));
  c.r.posted(b);
}

// The MMAs of one tile: PAIR = one instruction of M = 256 over the CTA pair (issued by the first
// CTA; each CTA holds its own A rows and half of the B^T rows at the same shared-memory offsets).
template <int S, bool PAIR>
__device__ void mma_tile(Shared& sh, MmaCtl& c, uint32_t tmem, uint32_t stage0, uint32_t stage_bytes, uint32_t boff,
                         int nkb, volatile int* abort) {
  constexpr uint32_t IDESC = idesc_f16(PAIR ? 2 * TILE_M : TILE_M, BN);
  constexpr int BPL = PAIR ? BH_BYTES : B_TILE_BYTES;  // bytes between the B^T planes of a stage
  uint32_t buf[S];
  int nxt[S], per[S];
  const bool stag = stagger_of(nkb);
  int nmin = 1 << 30;
#pragma unroll
  for (int g = 0; g < S; ++g) {
    drain_plan(g, S, stag, nxt[g], per[g]);
    nmin = min(nmin, nxt[g]);
  }
  // ---- k-block 0: diagonal by diagonal (heaviest first), each as soon as its buffer is free
  {
    if (!mbar_wait(bar(&sh.full[c.rg.stg]), (uint32_t)c.rg.ph, abort)) return;
    const uint32_t aaddr = stage0 + c.rg.stg * stage_bytes;
    const uint64_t ad0 = smem_desc(aaddr, 128, 128 * KB_CM);
    const uint64_t bd0 = smem_desc(aaddr + boff, 128, 128 * KB_CM);
#pragma unroll
    for (int g = S - 1; g >= 0; --g) {
      buf[g] = acquire(sh, c, abort);
      const uint32_t d = tmem + buf[g] * BN;
#pragma unroll
      for (int t = 0; t <= g; ++t)
        mma_issue<PAIR, 0>(d, ad0 + (uint64_t)((t * A_TILE_BYTES) >> 4), bd0 + (uint64_t)(((g - t) * BPL) >> 4), IDESC,
                           t > 0 ? 1u : 0u);
    }
    commit_to<PAIR>(bar(&sh.empty[c.rg.stg]));
    c.rg.advance();
  }
  uint32_t fresh = 0u;  // diagonals whose current buffer has not been written yet
  for (int kb = 1; kb < nkb; ++kb) {
    if (kb == nmin) {
      nmin = 1 << 30;
#pragma unroll
      for (int g = 0; g < S; ++g) {
        if (nxt[g] == kb) {
          post<PAIR>(sh, c, buf[g]);
          buf[g] = acquire(sh, c, abort);
          fresh |= 1u << g;
          nxt[g] += per[g];
        }
        nmin = min(nmin, nxt[g]);
      }
    }
    if (!mbar_wait(bar(&sh.full[c.rg.stg]), (uint32_t)c.rg.ph, abort)) return;
    const uint32_t aaddr = stage0 + c.rg.stg * stage_bytes;
    const uint64_t ad0 = smem_desc(aaddr, 128, 128 * KB_CM);
    const uint64_t bd0 = smem_desc(aaddr + boff, 128, 128 * KB_CM);
#pragma unroll
    for (int t = 0; t < S; ++t) {
      const uint64_t ad = ad0 + (uint64_t)((t * A_TILE_BYTES) >> 4);
#pragma unroll
      for (int u = 0; u < S - t; ++u) {
        const int g = t + u;
        const uint64_t bd = bd0 + (uint64_t)((u * BPL) >> 4);
        const uint32_t d = tmem + buf[g] * BN;
        // the first product of a k-block into diagonal g is the one with t = 0
        const uint32_t acc = (t == 0) ? (((fresh >> g) & 1u) ^ 1u) : 1u;
        const int nu = S - t;
        if (nu == 1) mma_issue<PAIR, 0>(d, ad, bd, IDESC, acc);
        else if (u == 0) mma_issue<PAIR, 1>(d, ad, bd, IDESC, acc);
        else if (u == nu - 1) mma_issue<PAIR, 3>(d, ad, bd, IDESC, acc);
        else mma_issue<PAIR, 2>(d, ad, bd, IDESC, acc);
      }
    }
    fresh = 0u;
    commit_to<PAIR>(bar(&sh.empty[c.rg.stg]));
    c.rg.advance();
  }
#pragma unroll
  for (int g = 0; g < S; ++g) post<PAIR>(sh, c, buf[g]);
}

// Second pass of a level-9 tile: diagonal 8 alone (pairs t + u = 8, t = 0..8) into one buffer at a
// time; a group holds GROUP_TERMS / 144 = 7 k-blocks, so the buffer is handed to the epilogue at
// k-blocks 7, 14, ... and at the end of the tile.
constexpr int LAST_DIAG = SPLIT_LEVEL - 1;
constexpr int LAST_PERIOD = GROUP_TERMS / (16 * (LAST_DIAG + 1));
template <bool PAIR>
__device__ void mma_last_diagonal(Shared& sh, MmaCtl& c, uint32_t tmem, uint32_t stage0, uint32_t stage_bytes,
                                  uint32_t boff, int nkb, volatile int* abort) {
  constexpr uint32_t IDESC = idesc_f16(PAIR ? 2 * TILE_M : TILE_M, BN);
  constexpr int BPL = PAIR ? BH_BYTES : B_TILE_BYTES;
  uint32_t buf = acquire(sh, c, abort);
  uint32_t acc0 = 0u;  // accumulate flag of the first product into the current buffer
  int left = LAST_PERIOD;
  for (int kb = 0; kb < nkb; ++kb) {
    if (left == 0) {
      post<PAIR>(sh, c, buf);
      buf = acquire(sh, c, abort);
      acc0 = 0u;
      left = LAST_PERIOD;
    }
    --left;
    if (!mbar_wait(bar(&sh.full[c.rg.stg]), (uint32_t)c.rg.ph, abort)) return;
    const uint32_t aaddr = stage0 + c.rg.stg * stage_bytes;
    const uint64_t ad0 = smem_desc(aaddr, 128, 128 * KB_CM);
    const uint64_t bd0 = smem_desc(aaddr + boff, 128, 128 * KB_CM);
    const uint32_t d = tmem + buf * BN;
#pragma unroll
    for (int t = 0; t <= LAST_DIAG; ++t)
      mma_issue<PAIR, 0>(d, ad0 + (uint64_t)((t * A_TILE_BYTES) >> 4), bd0 + (uint64_t)(((LAST_DIAG - t) * BPL) >> 4),
                         IDESC, t > 0 ? 1u : acc0);
    acc0 = 1u;
    commit_to<PAIR>(bar(&sh.empty[c.rg.stg]));
    c.rg.advance();
  }
  post<PAIR>(sh, c, buf);
}

// a warp's 32 TMEM lanes x 16 or 32 columns
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, uint32_t (&r)[16]) { tmem_ld16(taddr, r); }
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, uint32_t (&r)[32]) { tmem_ld32(taddr, r); }

// Epilogue roles of the drains (see the epilogue layouts above)
enum : int { ROLE_TMEM_OWNER = 0, ROLE_LOADER = 1, ROLE_HO_OWNER = 2 };

// Epilogue side of one drain of buffer b:
//  * a TMEM owner waits until the MMAs into the buffer are complete, reads its 32 lanes x CW
//    columns, releases the buffer and adds q * 2^shl into its exact running sums (one 96-bit
//    two's-complement integer z2:z1:z0 per output element);
//  * a quarter-1 owner takes its 32 columns from the loader's hand-over slot instead, frees it, and
//    adds in the same way (drain_load below is the loader's side).
// Slots are used in drain order by the loader and both quarter-1 owners (hcount counts drains).
// (In a CTA pair the buffer is released on the first CTA's barrier, where the issuer waits for it.)
template <int CW>
__device__ __forceinline__ bool drain_into(Shared& sh, const float4* ho, int role, uint32_t tmem, int lq, int cg,
                                           int lane, uint32_t b, int shl, uint32_t& accf_par, uint32_t& hcount,
                                           volatile int* abort, uint32_t (&z0)[CW], uint32_t (&z1)[CW],
                                           uint32_t (&z2)[CW], bool remote_release) {
  uint32_t v[CW];
  if (role == ROLE_TMEM_OWNER) {
    if (!mbar_wait(bar(&sh.accf[b]), (accf_par >> b) & 1u, abort)) return false;
    accf_par ^= 1u << b;
    tc_fence_after();
    tmem_ld_cols(tmem + ((uint32_t)(lq * 32) << 16) + b * BN + cg * CW, v);
    tmem_wait_ld();
    tc_fence_before();
    __syncwarp();
    if (lane == 0) {
      if (remote_release) mbar_arrive_remote(mapa_shared(bar(&sh.acce[b]), 0));
      else mbar_arrive(bar(&sh.acce[b]));
    }
  } else {
    const uint32_t slot = hcount % HO_SLOTS, ph = (hcount / HO_SLOTS) & 1u;
    ++hcount;
    if (!mbar_wait(bar(&sh.hfull[slot]), ph, abort)) return false;
    const float4* hs = ho + slot * (BN / 4) * 32 + cg * (CW / 4) * 32;
#pragma unroll
    for (int c = 0; c < CW / 4; ++c) {
      const float4 f = hs[c * 32 + lane];
      v[4 * c] = __float_as_uint(f.x);
      v[4 * c + 1] = __float_as_uint(f.y);
      v[4 * c + 2] = __float_as_uint(f.z);
      v[4 * c + 3] = __float_as_uint(f.w);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(bar(&sh.hempty[slot]));
  }
  if (shl >= 64) {
    // level 9, diagonal 0: weight 2^64, the top word alone (the sums are kept modulo 2^96)
#pragma unroll
    for (int j = 0; j < CW; ++j) z2[j] += (uint32_t)__float2int_rn(__uint_as_float(v[j]));
    return true;
  }
#pragma unroll
  for (int j = 0; j < CW; ++j) w96_add_shifted(z0[j], z1[j], z2[j], __float2int_rn(__uint_as_float(v[j])), shl);
  return true;
}

// The loader's side of one drain: lanes 32..63 of buffer b, all 64 columns, read and released, then
// written to the next hand-over slot ([slot][column / 4][lane][4] floats) once both quarter-1 owners
// have taken its previous contents.
__device__ __forceinline__ bool drain_load(Shared& sh, float4* ho, uint32_t tmem, int lane, uint32_t b,
                                           uint32_t& accf_par, uint32_t& hcount, volatile int* abort,
                                           bool remote_release) {
  if (!mbar_wait(bar(&sh.accf[b]), (accf_par >> b) & 1u, abort)) return false;
  accf_par ^= 1u << b;
  tc_fence_after();
  constexpr int CW = BN / 2;  // the two halves of the 64 columns
  uint32_t v[CW], u[CW];
  tmem_ld32(tmem + (32u << 16) + b * BN, v);
  tmem_ld32(tmem + (32u << 16) + b * BN + CW, u);
  tmem_wait_ld();
  tc_fence_before();
  __syncwarp();
  if (lane == 0) {
    if (remote_release) mbar_arrive_remote(mapa_shared(bar(&sh.acce[b]), 0));
    else mbar_arrive(bar(&sh.acce[b]));
  }
  const uint32_t slot = hcount % HO_SLOTS, ph = (hcount / HO_SLOTS) & 1u;
  ++hcount;
  if (!mbar_wait(bar(&sh.hempty[slot]), ph ^ 1u, abort)) return false;
  float4* hs = ho + slot * (BN / 4) * 32;
#pragma unroll
  for (int c = 0; c < CW / 4; ++c) {
    hs[c * 32 + lane] = make_float4(__uint_as_float(v[4 * c]), __uint_as_float(v[4 * c + 1]),
                                    __uint_as_float(v[4 * c + 2]), __uint_as_float(v[4 * c + 3]));
    hs[(CW / 4 + c) * 32 + lane] = make_float4(__uint_as_float(u[4 * c]), __uint_as_float(u[4 * c + 1]),
                                               __uint_as_float(u[4 * c + 2]), __uint_as_float(u[4 * c + 3]));
  }
  __syncwarp();
  if (lane == 0) mbar_arrive(bar(&sh.hfull[slot]));
  return true;
}

// The drain schedule of one tile, replayed in the issuer's order: the buffers of k-block 0, then
// the mid-tile drains ordered by (k-block, diagonal), then the final buffers; drain(b, shl) handles
// buffer b whose diagonal carries the weight 2^shl.  Level 9: the first pass takes diagonals 0..7
// on the level-8 plan, the second diagonal 8 alone, drained every LAST_PERIOD k-blocks.
template <typename F>
__device__ __forceinline__ bool replay_drains(int S, int nkb, BufRing& er, F&& drain) {
  const bool stag = stagger_of(nkb);
  uint32_t bufs[SPLIT_LEVEL - 1];  // a pass has at most 8 diagonals
  int nxt[SPLIT_LEVEL - 1], per[SPLIT_LEVEL - 1];
  bool ok = true;
  for (int pass = 0; pass < passes_of(S) && ok; ++pass) {
    const int g0 = pass ? SPLIT_LEVEL - 1 : 0;                 // first diagonal of the pass
    const int nd = pass ? 1 : (S == SPLIT_LEVEL ? S - 1 : S);  // its diagonals
    for (int d = nd - 1; d >= 0; --d) bufs[d] = er.next();
    for (int d = 0; d < nd; ++d) {
      if (pass) nxt[d] = per[d] = LAST_PERIOD;
      else drain_plan(d, nd, stag, nxt[d], per[d]);
    }
    while (ok) {
      int kbmin = nkb, dsel = -1;
      for (int d = 0; d < nd; ++d)
        if (nxt[d] < kbmin) {
          kbmin = nxt[d];
          dsel = d;
        }
      if (dsel < 0) break;
      ok = drain(bufs[dsel], 8 * (S - 1 - g0 - dsel));
      er.posted(bufs[dsel]);
      bufs[dsel] = er.next();
      nxt[dsel] += per[dsel];
    }
    for (int d = 0; d < nd && ok; ++d) {
      ok = drain(bufs[d], 8 * (S - 1 - g0 - d));
      er.posted(bufs[d]);
    }
  }
  return ok;
}

__device__ __forceinline__ void tile_of(const GemmTile* tiles, const GemmProblem* probs, const GemmProblem& single,
                                        int idx, const GemmProblem*& P, int& mb, int& nb) {
  if (tiles) {
    GemmTile t = tiles[idx];
    P = probs + t.prob;
    mb = t.mb;
    nb = t.nb;
  } else {
    int nnb = (single.N + BN - 1) / BN;
    P = &single;
    mb = idx / nnb;
    nb = idx % nnb;
  }
}

template <bool PAIR, bool HO>
__global__ void __launch_bounds__(EpiCfg<HO>::NTHREADS, 1)
    gemm_kernel(const GemmProblem* __restrict__ probs, const GemmTile* __restrict__ tiles, int ntiles,
                const int* __restrict__ first,
                const __grid_constant__ GemmProblem single, int smax, int nstage, int* __restrict__ err) {
  using E = EpiCfg<HO>;
  constexpr int CW = E::CW;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int BPL = PAIR ? BH_BYTES : B_TILE_BYTES;  // bytes of one B^T plane in a stage
  const uint32_t stage_bytes = (uint32_t)(smax * plane_bytes(PAIR)), boff = (uint32_t)(smax * A_TILE_BYTES);
  longlong2* zstage = reinterpret_cast<longlong2*>(smem + nstage * stage_bytes);
  Shared& sh = *reinterpret_cast<Shared*>(smem + nstage * stage_bytes + E::ZS_BYTES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int* abort = &sh.abort;
  const uint32_t stage0 = smem_u32(smem);
  // CTA pair: rank 0 issues the MMAs of both; rank 1 forwards its operand arrivals to rank 0
  const uint32_t rank = PAIR ? cluster_rank() : 0u;
  const bool lead = rank == 0;

  if (threadIdx.x == 0) {
    for (int i = 0; i < nstage; ++i) {
      // the first CTA of a pair also waits for the second one's copies (one forwarded arrival)
      mbar_init(bar(&sh.full[i]), PAIR && lead ? 2 : 1);
      mbar_init(bar(&sh.empty[i]), 1);
    }
    for (int i = 0; i < NBUF; ++i) {
      mbar_init(bar(&sh.accf[i]), 1);
      mbar_init(bar(&sh.acce[i]), PAIR ? 2 * E::READERS : E::READERS);
    }
    mbar_init(bar(&sh.fin), 1);
    for (int i = 0; i < HO_SLOTS; ++i) {
      mbar_init(bar(&sh.hfull[i]), 1);
      mbar_init(bar(&sh.hempty[i]), 2);
    }
    sh.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    if constexpr (PAIR) tmem_alloc_pair(smem_u32(&sh.tmem), 512);
    else tmem_alloc(smem_u32(&sh.tmem), 512);
  }
  tc_fence_before();
  if constexpr (PAIR) cluster_sync();
  else __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh.tmem;
  // this CTA's (pair's) tiles: the range [first[b], first[b+1]) of a host-balanced list, or every
  // grid-th tile; all roles (of both CTAs of a pair) walk the same sequence
  const int unit = PAIR ? (int)cluster_id() : (int)blockIdx.x;
  const int units = PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;
  const int it0 = first ? first[unit] : unit;
  const int it1 = first ? first[unit + 1] : ntiles;
  const int istep = first ? 1 : units;

  if (warp == 0) {
    // ------------------------------------------------------------------ producer
    if (lane == 0) {
      Ring rg{0, 0, nstage};
      long long fills = 0;
      for (int idx = it0; idx < it1 && !*abort; idx += istep) {
        const GemmProblem* P;
        int mb, nb;
        tile_of(tiles, probs, single, idx, P, mb, nb);
        const int nkb = P->nkb, s = P->s, SA = P->SA, SB = P->SB;
        // a pair's tile is 256 rows: this CTA's A tile is 2 mb + rank; its B^T half is the rank-th
        // 32-row half of the 64-row tile nb (the operand stores the two halves of each k-block apart).
        // An operand with an odd number of 128-row tiles has no A tile for the second CTA of its last
        // pair: that CTA loads only its B^T half, and the rows it computes lie beyond M (never stored).
        const int ma = PAIR ? 2 * mb + (int)rank : mb;
        const bool a_in = !PAIR || ma * TILE_M < P->M;
        const char* Ab = reinterpret_cast<const char*>(P->A) + (long long)ma * nkb * SA * A_TILE_BYTES;
        const char* Bb = reinterpret_cast<const char*>(P->B) + (long long)nb * nkb * SB * B_TILE_BYTES +
                         (PAIR ? (long long)rank * SB * BH_BYTES : 0ll);
        bool stop = false;
        // one fill per k-block and pass (level 9: the k-blocks twice)
        const int nfill = passes_of(s) * nkb;
        for (int f = 0; f < nfill; ++f) {
          const int kb = f < nkb ? f : f - nkb;
          // a stage is refilled once the MMAs of its previous fill have completed
          if (fills >= nstage && !mbar_wait(bar(&sh.empty[rg.stg]), (uint32_t)(rg.ph ^ 1), abort)) {
            stop = true;
            break;
          }
          mbar_expect_tx(bar(&sh.full[rg.stg]), (uint32_t)(s * ((a_in ? A_TILE_BYTES : 0) + BPL)));
          const uint32_t dA = stage0 + rg.stg * stage_bytes;
          if (a_in)
            bulk_g2s(dA, Ab + (long long)kb * SA * A_TILE_BYTES, (uint32_t)(s * A_TILE_BYTES), bar(&sh.full[rg.stg]));
          bulk_g2s(dA + boff, Bb + (long long)kb * SB * B_TILE_BYTES, (uint32_t)(s * BPL), bar(&sh.full[rg.stg]));
          ++fills;
          rg.advance();
        }
        if (stop) break;
      }
      // let the copies still in flight land before the CTA can exit: wait for the last fill of
      // every stage that was filled
      volatile int never = 0;
      for (int i = 0; i < nstage && i < fills; ++i) {
        rg.stg = rg.stg == 0 ? nstage - 1 : rg.stg - 1;
        if (rg.stg == nstage - 1) rg.ph ^= 1;
        mbar_wait(bar(&sh.full[rg.stg]), (uint32_t)rg.ph, &never);
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && lead) {
      // ------------------------------------------------------------------ MMA issuer
      MmaCtl c{Ring{0, 0, nstage}, BufRing{0u, 0, 0}, 0u};
      for (int idx = it0; idx < it1 && !*abort; idx += istep) {
        const GemmProblem* P;
        int mb, nb;
        tile_of(tiles, probs, single, idx, P, mb, nb);
        const int nkb = P->nkb;
        switch (P->s) {
          case 1: mma_tile<1, PAIR>(sh, c, tmem, stage0, stage_bytes, boff, nkb, abort); break;
          case 2: mma_tile<2, PAIR>(sh, c, tmem, stage0, stage_bytes, boff, nkb, abort); break;
          case 3: mma_tile<3, PAIR>(sh, c, tmem, stage0, stage_bytes, boff, nkb, abort); break;
          case 4: mma_tile<4, PAIR>(sh, c, tmem, stage0, stage_bytes, boff, nkb, abort); break;
          case 5: mma_tile<5, PAIR>(sh, c, tmem, stage0, stage_bytes, boff, nkb, abort); break;
          case 6: mma_tile<6, PAIR>(sh, c, tmem, stage0, stage_bytes, boff, nkb, abort); break;
          case 7: mma_tile<7, PAIR>(sh, c, tmem, stage0, stage_bytes, boff, nkb, abort); break;
          case 8:
          case 9:  // level 9: the level-8 pass, then diagonal 8 alone
            mma_tile<8, PAIR>(sh, c, tmem, stage0, stage_bytes, boff, nkb, abort);
            if (P->s == SPLIT_LEVEL) mma_last_diagonal<PAIR>(sh, c, tmem, stage0, stage_bytes, boff, nkb, abort);
            break;
          default: *abort = 1; break;
        }
      }
      // all issued MMAs complete before TMEM is released
      commit_to<PAIR>(bar(&sh.fin));
      volatile int never = 0;
      mbar_wait(bar(&sh.fin), 0, &never);
    } else if (PAIR && lane == 0) {
      // ------------------------------------------------------------------ forwarder (second CTA)
      // every fill of this CTA's stage ring, once its copies have landed, counts as one arrival on
      // the first CTA's barrier of the same stage, which its issuer waits on
      Ring rg{0, 0, nstage};
      for (int idx = it0; idx < it1 && !*abort; idx += istep) {
        const GemmProblem* P;
        int mb, nb;
        tile_of(tiles, probs, single, idx, P, mb, nb);
        bool stop = false;
        const int nfill = passes_of(P->s) * P->nkb;
        for (int f = 0; f < nfill; ++f) {
          if (!mbar_wait(bar(&sh.full[rg.stg]), (uint32_t)rg.ph, abort)) {
            stop = true;
            break;
          }
          mbar_arrive_remote(mapa_shared(bar(&sh.full[rg.stg]), 0));
          rg.advance();
        }
        if (stop) break;
      }
    }
  } else if (HO && warp == 5) {
    // ------------------------------------------------------------------ loader of lane quarter 1
    uint32_t accf_par = 0, hcount = 0;
    BufRing er{0u, 0, 0};
    float4* ho = reinterpret_cast<float4*>(zstage + E::OWNERS * 32 * ZS_LD);
    for (int idx = it0; idx < it1 && !*abort; idx += istep) {
      const GemmProblem* P;
      int mb, nb;
      tile_of(tiles, probs, single, idx, P, mb, nb);
      if (!replay_drains(P->s, P->nkb, er, [&](uint32_t b, int) {
            return drain_load(sh, ho, tmem, lane, b, accf_par, hcount, abort, PAIR && !lead);
          }))
        break;
    }
  } else if (!HO || warp != 9) {
    // ------------------------------------------------------------------ owners of the exact sums
    const int role = HO && warp >= 10 ? ROLE_HO_OWNER : ROLE_TMEM_OWNER;
    const int lq = warp & 3;                               // TMEM lane quarter this warp may read
    const int rq = role == ROLE_HO_OWNER ? 1 : lq;         // lane quarter (rows) of its exact sums
    const int cg = role == ROLE_HO_OWNER ? warp - 10 : (warp - 2) >> 2;  // column group of the tile
    // owner index (staging area): HO: 2, 3, 4, 6, 7, 8, 10, 11 -> 0..7; else warp - 2
    const int oi = !HO ? warp - 2 : (role == ROLE_HO_OWNER ? warp - 4 : (warp < 5 ? warp - 2 : warp - 3));
    uint32_t accf_par = 0, hcount = 0;
    BufRing er{0u, 0, 0};
    longlong2* zs = zstage + oi * 32 * ZS_LD;
    const float4* ho = reinterpret_cast<const float4*>(zstage + E::OWNERS * 32 * ZS_LD);
    for (int idx = it0; idx < it1 && !*abort; idx += istep) {
      const GemmProblem* P;
      int mb, nb;
      tile_of(tiles, probs, single, idx, P, mb, nb);
      // per-tile operands of the final stage, loaded now so that their latency hides behind the drains
      const int M = P->M, N = P->N, mode = P->mode;
      const int row = (PAIR ? 2 * mb + (int)rank : mb) * TILE_M + rq * 32 + lane;
      const bool rowok = row < M;
      const int col0 = nb * BN + cg * CW;
      const int ebl = (lane < CW && col0 + lane < N) ? __ldg(P->eb + col0 + lane) : 0;
      const int ea_raw = rowok ? __ldg(P->ea + row) : 0;
      double* crow = nullptr;
      const bool tmode = mode == OUT_DENSE_T;
      if (rowok) {
        if (mode == OUT_DENSE) crow = P->C + (long long)row * P->ldc + col0;
        else if (tmode) crow = P->C + (long long)col0 * P->ldc + row;  // element jj at crow[jj * ldc]
        else crow = P->C + __ldg(P->rowdst + row) + col0;
      }
      const long long cstr = tmode ? P->ldc : 1;
      // exact running sum per element, a 96-bit two's-complement integer z2:z1:z0 (|Z| < 2^95 within
      // the reduction lengths max_k_of_level admits)
      uint32_t z0[CW], z1[CW], z2[CW];
#pragma unroll
      for (int j = 0; j < CW; ++j) {
        z0[j] = 0u;
        z1[j] = 0u;
        z2[j] = 0u;
      }
      const int S = P->s;
      const bool ok = replay_drains(S, P->nkb, er, [&](uint32_t b, int shl) {
        return drain_into(sh, ho, role, tmem, lq, cg, lane, b, shl, accf_par, hcount, abort, z0, z1, z2,
                          PAIR && !lead);
      });
      if (!ok) break;
      // ---- one rounding to FP64, scaling; the exact sums pass through shared memory ZC columns at a
      //      time so that the conversion code exists once (compact loop), and the stores are coalesced
      const int ncol = min(CW, N - col0);
      const int ea = ea_raw - 8 * S - 6;
      const double alpha = P->alpha, beta = P->beta;
      const bool plain = (mode == OUT_ROWTABLE) || ((alpha == 1.0) && (beta == 0.0));
      // row-table mode: max |value| of the row's outputs, as 32-bit halves of the bit pattern
      // (compared with 32-bit integer operations; 64-bit comparisons would issue to the FP64 pipe)
      const bool tabmax = mode == OUT_ROWTABLE && P->rowmax;
      uint32_t mxh = 0u, mxl = 0u;
#pragma unroll
      for (int c4 = 0; c4 < CW / ZC; ++c4) {
        if (c4 * ZC < ncol) {
#pragma unroll
          for (int j = 0; j < ZC; ++j)
            zs[lane * ZS_LD + j] = make_longlong2((long long)(((unsigned long long)z1[c4 * ZC + j] << 32) | z0[c4 * ZC + j]),
                                                  (long long)(int)z2[c4 * ZC + j]);
          __syncwarp();
#pragma unroll 1
          for (int j = 0; j < ZC; ++j) {
            const int jj = c4 * ZC + j;
            const int ebj = __shfl_sync(0xffffffffu, ebl, jj);
            double v = 0.0;
            if (rowok && jj < ncol) {
              const longlong2 z = zs[lane * ZS_LD + j];
              v = w96_to_double((uint32_t)z.x, (uint32_t)((unsigned long long)z.x >> 32), (uint32_t)z.y, ea + ebj);
              if (!plain) {
                v = __dmul_rn(alpha, v);
                if (beta != 0.0) v = __dadd_rn(v, __dmul_rn(beta, crow[jj * cstr]));
              }
              if (tabmax) {
                const uint32_t bh = (uint32_t)__double2hiint(v) & 0x7FFFFFFFu, bl = (uint32_t)__double2loint(v);
                const bool gt = bh > mxh || (bh == mxh && bl > mxl);
                mxh = gt ? bh : mxh;
                mxl = gt ? bl : mxl;
              }
              // transposed output: the warp's lanes are consecutive rows, i.e. consecutive addresses
              if (tmode) crow[jj * cstr] = v;
            }
            reinterpret_cast<double*>(zs + lane * ZS_LD + j)[0] = v;
          }
          __syncwarp();
          // coalesced stores: each pass writes (32 / ZC) rows x ZC consecutive doubles
#pragma unroll 1
          for (int p = 0; p < ZC && !tmode; ++p) {
            const int r = p * (32 / ZC) + lane / ZC, cc = lane % ZC;
            double* base =
                reinterpret_cast<double*>(__shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(crow), r));
            if (base && c4 * ZC + cc < ncol) base[c4 * ZC + cc] = reinterpret_cast<const double*>(zs + r * ZS_LD + cc)[0];
          }
          __syncwarp();
        }
      }
      if (tabmax && rowok && (mxh | mxl))
        atomicMax(P->rowmax + __ldg(P->rowslot + row), ((unsigned long long)mxh << 32) | mxl);
    }
  }

  tc_fence_before();
  if constexpr (PAIR) cluster_sync();  // both CTAs' epilogues are done with TMEM, remote arrivals are in
  else __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    if constexpr (PAIR) tmem_dealloc_pair(tmem, 512);
    else tmem_dealloc(tmem, 512);
  }
  if (threadIdx.x == 0 && sh.abort) atomicOr(err, 2);
}

void schedule_tiles(const std::vector<GemmProblem>& probs, std::vector<GemmTile>& tiles, int grid, int mode,
                    std::vector<int>& first) {
  if (mode == SCHED_STRIDED) {
    // CTA b takes tiles b, b + grid, ... of the given order
    std::vector<GemmTile> out;
    out.reserve(tiles.size());
    first.assign(grid + 1, 0);
    for (int b = 0; b < grid; ++b) {
      first[b] = (int)out.size();
      for (size_t i = b; i < tiles.size(); i += grid) out.push_back(tiles[i]);
    }
    first[grid] = (int)out.size();
    tiles.swap(out);
    return;
  }
  balance_tiles(probs, tiles, grid, first);
  if (mode == SCHED_BALANCED_ASC)
    for (int b = 0; b < grid; ++b) std::reverse(tiles.begin() + first[b], tiles.begin() + first[b + 1]);
}

void balance_tiles(const std::vector<GemmProblem>& probs, std::vector<GemmTile>& tiles, int grid,
                   std::vector<int>& first) {
  // cost in MMA units: k-blocks x slice pairs, plus about 130 MMAs' worth of epilogue per tile
  auto cost = [&](const GemmTile& t) {
    const GemmProblem& P = probs[t.prob];
    return (long long)P.nkb * (P.s * (P.s + 1) / 2) + 130;
  };
  std::vector<int> ord(tiles.size());
  for (size_t i = 0; i < tiles.size(); ++i) ord[i] = (int)i;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return cost(tiles[a]) > cost(tiles[b]); });
  // longest first onto the least loaded CTA (ties: lowest index)
  std::vector<long long> load(grid, 0);
  std::vector<std::vector<int>> own(grid);
  std::vector<std::pair<long long, int>> heap;
  for (int b = 0; b < grid; ++b) heap.push_back({0, b});
  auto cmp = [](const std::pair<long long, int>& x, const std::pair<long long, int>& y) {
    return x.first != y.first ? x.first > y.first : x.second > y.second;
  };
  std::make_heap(heap.begin(), heap.end(), cmp);
  for (int i : ord) {
    std::pop_heap(heap.begin(), heap.end(), cmp);
    auto& top = heap.back();
    own[top.second].push_back(i);
    top.first += cost(tiles[i]);
    std::push_heap(heap.begin(), heap.end(), cmp);
  }
  std::vector<GemmTile> out;
  out.reserve(tiles.size());
  first.assign(grid + 1, 0);
  for (int b = 0; b < grid; ++b) {
    first[b] = (int)out.size();
    for (int i : own[b]) out.push_back(tiles[i]);
  }
  first[grid] = (int)out.size();
  tiles.swap(out);
}

namespace {
// The shared-memory opt-in of a kernel belongs to the current device's context: record it per
// device ordinal (bit d of a process-wide mask).  Setting it twice is harmless, so two host threads
// racing on the same device need no lock.
template <bool PAIR, bool HO>
cudaError_t opt_in_smem() {
  static std::atomic<unsigned long long> attr_set{0ull};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
  if (!bit || !(attr_set.load(std::memory_order_acquire) & bit)) {
    e = cudaFuncSetAttribute(gemm_kernel<PAIR, HO>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT);
    if (e != cudaSuccess) return e;
    attr_set.fetch_or(bit, std::memory_order_release);
  }
  return cudaSuccess;
}
}  // namespace

int gemm_pair_units(int nsm) {
  // CTA pairs that run at the same time on the current device (clusters of 2, one CTA per SM)
  if (opt_in_smem<true, false>() != cudaSuccess) return 0;
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)(nsm / 2 * 2), 1, 1);
  cfg.blockDim = dim3(EpiCfg<false>::NTHREADS, 1, 1);
  cfg.dynamicSmemBytes = gemm_smem_bytes(MAX_LEVEL, true, false);
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, gemm_kernel<true, false>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n < nsm / 2 ? n : nsm / 2;
}

cudaError_t launch_gemm(const GemmProblem* d_probs, const GemmTile* d_tiles, int ntiles, int grid,
                        const GemmProblem* single, int smax, int* d_err, cudaStream_t st, const int* d_first,
                        bool pair, bool ho) {
  if (ntiles <= 0) return cudaSuccess;
  if (pair) ho = false;  // CTA pairs keep the 18-warp layout
  cudaError_t e = pair ? opt_in_smem<true, false>() : (ho ? opt_in_smem<false, true>() : opt_in_smem<false, false>());
  if (e != cudaSuccess) return e;
  GemmProblem one{};
  if (single) {
    one = *single;
    smax = one.s;
  }
  if (smax < 1 || smax > MAX_LEVEL) return cudaErrorInvalidValue;
  const int nstage = gemm_stages(smax, pair, ho);
  const int g = d_first ? grid : (grid < ntiles ? grid : ntiles);
  if (!pair) {
    if (ho)
      gemm_kernel<false, true><<<g, EpiCfg<true>::NTHREADS, gemm_smem_bytes(smax, false, true), st>>>(
          d_probs, d_tiles, ntiles, d_first, one, smax, nstage, d_err);
    else
      gemm_kernel<false, false><<<g, EpiCfg<false>::NTHREADS, gemm_smem_bytes(smax, false, false), st>>>(
          d_probs, d_tiles, ntiles, d_first, one, smax, nstage, d_err);
    return cudaGetLastError();
  }
  // g CTA pairs: clusters of two CTAs on two SMs
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)(2 * g), 1, 1);
  cfg.blockDim = dim3(EpiCfg<false>::NTHREADS, 1, 1);
  cfg.dynamicSmemBytes = gemm_smem_bytes(smax, true, false);
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, gemm_kernel<true, false>, d_probs, d_tiles, ntiles, d_first, one, smax, nstage,
                            d_err);
}

}  // namespace oz
