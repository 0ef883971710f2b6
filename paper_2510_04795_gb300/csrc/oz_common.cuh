// Shared device helpers: mbarriers, bulk async copies, tcgen05 (TMEM, MMA), descriptors.
// Everything here is sm_103a inline PTX; nothing falls back to another architecture.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_fp16.h>

#ifndef OZ_DEVICE_INLINE
#define OZ_DEVICE_INLINE __device__ __forceinline__
#endif

namespace oz {

// Digit tiles: K-blocks of KB FP16 digits; "core matrices" of 8 rows x 8 K-elements
// (128 contiguous bytes) in the no-swizzle K-major canonical layout of tcgen05.mma.
constexpr int KB_SHIFT = 4;
constexpr int KB = 1 << KB_SHIFT;      // K elements per k-block (one MMA K-step of 16)
constexpr int KB_CM = KB / 8;          // core matrices along K in one k-block
constexpr int TILE_M = 128;            // A-operand tile rows (MMA M)
constexpr int GROUP_TERMS = 1008;      // products per FP32 accumulator group: 1008 * 2^14 < 2^24

// element offset (in halves) of (r, k) inside one R x KB tile
OZ_DEVICE_INLINE int tile_off(int r, int k) {
  return (((r >> 3) * KB_CM + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7);
}

OZ_DEVICE_INLINE uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// ----------------------------------------------------------------------------------------------
// mbarrier
// ----------------------------------------------------------------------------------------------
OZ_DEVICE_INLINE void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
OZ_DEVICE_INLINE void mbar_arrive(uint32_t a) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(a) : "memory");
}
OZ_DEVICE_INLINE void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(a), "r"(bytes)
               : "memory");
}
OZ_DEVICE_INLINE bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.b32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}

// Spin budget for every wait in the library's kernels (clock64 cycles, about 2 s at 2 GHz).
constexpr long long WAIT_BUDGET = 1ll << 32;

// Bounded wait.  Returns false (and never blocks again) once `abort` is set or the budget runs out.
OZ_DEVICE_INLINE bool mbar_wait(uint32_t a, uint32_t parity, volatile int* abort) {
  if (mbar_try(a, parity)) return true;
  long long t0 = clock64();
  while (true) {
    if (mbar_try(a, parity)) return true;
    if (*abort) return false;
    if (clock64() - t0 > WAIT_BUDGET) {
      *abort = 1;
      return false;
    }
  }
}

// ----------------------------------------------------------------------------------------------
// bulk async copy global -> shared (16-byte aligned, size multiple of 16)
// ----------------------------------------------------------------------------------------------
OZ_DEVICE_INLINE void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

// ----------------------------------------------------------------------------------------------
// tcgen05
// ----------------------------------------------------------------------------------------------
OZ_DEVICE_INLINE void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
OZ_DEVICE_INLINE void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
OZ_DEVICE_INLINE void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
OZ_DEVICE_INLINE void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
OZ_DEVICE_INLINE void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

// Shared-memory matrix descriptor, no swizzle, K-major: LBO = stride between core matrices
// along K, SBO = stride between 8-row groups; bit 46 = descriptor version for tcgen05.
OZ_DEVICE_INLINE uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// Instruction descriptor of kind::f16: D = F32, A = B = F16, both K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// collector usage for A: 0 none, 1 fill, 2 use, 3 lastuse
template <int COL>
OZ_DEVICE_INLINE void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  if constexpr (COL == 0)
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc));
  else if constexpr (COL == 1)
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], %1, %2, "
        "%3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc));
  else if constexpr (COL == 2)
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16.collector::a::use [%0], %1, %2, "
        "%3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc));
  else
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%0], %1, "
        "%2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc));
}

// ---- CTA pairs (cta_group::2): one MMA of M = 256 over two CTAs of a cluster of 2.  CTA rank r
// supplies rows 128 r .. 128 r + 127 of A and rows N/2 r .. N/2 r + N/2 - 1 of B^T from the same
// shared-memory offsets, and receives its 128 rows of D in its own TMEM at the same address; the
// allocation is collective (both CTAs allocate and obtain the same address).
OZ_DEVICE_INLINE uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
OZ_DEVICE_INLINE uint32_t cluster_id() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
OZ_DEVICE_INLINE void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// shared::cluster address of the same shared-memory offset in CTA `rank` of the cluster
OZ_DEVICE_INLINE uint32_t mapa_shared(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
// arrive on an mbarrier of another CTA of the cluster (shared::cluster address)
OZ_DEVICE_INLINE void mbar_arrive_remote(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
OZ_DEVICE_INLINE void tmem_alloc_pair(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
OZ_DEVICE_INLINE void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// completion of the issuing thread's earlier pair MMAs, signalled on the mbarrier at this offset in
// both CTAs of the pair
OZ_DEVICE_INLINE void tc_commit_pair(uint32_t mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(mbar),
      "h"((uint16_t)3)
      : "memory");
}
template <int COL>
OZ_DEVICE_INLINE void mma_f16_pair(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  if constexpr (COL == 0)
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc));
  else if constexpr (COL == 1)
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::2.kind::f16.collector::a::fill [%0], %1, %2, "
        "%3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc));
  else if constexpr (COL == 2)
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::2.kind::f16.collector::a::use [%0], %1, %2, "
        "%3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc));
  else
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::2.kind::f16.collector::a::lastuse [%0], %1, "
        "%2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc));
}

// 32 lanes x 32 columns of 32-bit TMEM words: thread i of the warp gets lane (base+i), 32 columns.
OZ_DEVICE_INLINE void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%"
      "20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
OZ_DEVICE_INLINE void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
OZ_DEVICE_INLINE void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ----------------------------------------------------------------------------------------------
// exact integer <-> FP64 helpers (integer arithmetic only: FP64 units are scarce on this GPU)
// ----------------------------------------------------------------------------------------------

// Shared exponent of a row/column from the bit pattern of max|x|: the smallest e with
// max|x| <= (127/128) 2^e; 0 for an all-zero row.
OZ_DEVICE_INLINE int exponent_from_maxbits(unsigned long long mb) {
  if (mb == 0ull) return 0;
  int be = (int)(mb >> 52);
  unsigned long long f = mb & ((1ull << 52) - 1);
  if (be == 0) {  // subnormal: normalise so that the value is (1.f') 2^(-1022 - shift)
    int lz = __clzll((long long)f) - 11;  // leading zeros within the 53-bit field (bit 52 empty)
    f = (f << lz) & ((1ull << 52) - 1);
    be = 1 - lz;
  }
  int ex = be - 1022;                      // value = m 2^ex with m in [0.5, 1)
  return (f > (63ull << 46)) ? ex + 1 : ex;  // m <= 127/128  <=>  f <= 63 * 2^46
}

// RN_even(Z * 2^E) as IEEE binary64, Z a signed 128-bit integer.
static __device__ __noinline__ double int128_to_double(__int128 Z, int E) {
  if (Z == 0) return 0.0;
  unsigned long long sign = 0;
  unsigned __int128 a;
  if (Z < 0) {
    sign = 1ull << 63;
    a = (unsigned __int128)(-Z);
  } else {
    a = (unsigned __int128)Z;
  }
  unsigned long long hi = (unsigned long long)(a >> 64), lo = (unsigned long long)a;
  int nb = hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo);  // bit length
  int e2 = nb - 1 + E;                                                        // binary exponent of leading bit
  int drop;                                                                   // bits to drop from a
  if (e2 >= -1022) {
    drop = nb - 53;
  } else {
    drop = -1074 - E;  // keep bits at weight >= 2^-1074
  }
  unsigned long long mant;
  if (drop <= 0) {
    mant = (unsigned long long)(a << (-drop));
  } else if (drop >= 128) {
    return __longlong_as_double((long long)sign);  // far below half the smallest subnormal
  } else {
    unsigned __int128 q = a >> drop;
    unsigned __int128 rem = a - (q << drop);
    unsigned __int128 half = (unsigned __int128)1 << (drop - 1);
    if (rem > half || (rem == half && (q & 1))) q += 1;
    mant = (unsigned long long)q;
  }
  unsigned long long bits;
  if (e2 >= -1022) {
    if (mant >> 53) {  // rounding carried into a new bit
      mant >>= 1;
      e2 += 1;
    }
    if (e2 > 1023) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull));
    bits = sign | ((unsigned long long)(e2 + 1023) << 52) | (mant & ((1ull << 52) - 1));
  } else {
    bits = sign | mant;  // subnormal (mant may reach 2^52: that is the smallest normal, encoded alike)
  }
  return __longlong_as_double((long long)bits);
}

// RN_even((zhi * 2^32 + zlo) * 2^E): fast path for results in the normal range (64-bit integer
// operations only), general path otherwise.
OZ_DEVICE_INLINE double split_to_double(long long zhi, long long zlo, int E) {
  const unsigned long long L1 = (unsigned long long)zhi << 32;
  unsigned long long l = L1 + (unsigned long long)zlo;
  unsigned long long h = (unsigned long long)((zhi >> 32) + (zlo >> 63) + (l < L1 ? 1ll : 0ll));
  const unsigned long long sign = h & 0x8000000000000000ull;
  if (sign) {
    l = ~l + 1ull;
    h = ~h + (l == 0ull ? 1ull : 0ull);
  }
  if ((h | l) == 0ull) return 0.0;
  int nb;
  unsigned long long top;
  bool sticky;
  if (h) {
    const int lz = __clzll((long long)h);
    nb = 128 - lz;
    top = lz ? ((h << lz) | (l >> (64 - lz))) : h;
    sticky = (lz ? (l << lz) : l) != 0ull;
  } else {
    const int lz = __clzll((long long)l);
    nb = 64 - lz;
    top = l << lz;
    sticky = false;
  }
  int e2 = nb - 1 + E;
  if (e2 < -1022 || e2 > 1022) return int128_to_double(((__int128)zhi << 32) + (__int128)zlo, E);
  unsigned long long m = top >> 11;
  const unsigned long long g = top & 0x7FFull;
  if (g > 0x400ull || (g == 0x400ull && (sticky || (m & 1ull)))) {
    m += 1ull;
    if (m >> 53) {
      m >>= 1;
      e2 += 1;
    }
  }
  return __longlong_as_double((long long)(sign | ((unsigned long long)(e2 + 1023) << 52) | (m & ((1ull << 52) - 1))));
}

// RN_even(Z * 2^E) for the 96-bit two's-complement integer Z = w2:w1:w0 (|Z| < 2^95), with the
// rounding of split_to_double in 32-bit word arithmetic only: normalised by whole words and one
// funnel shift, rounded to 53 bits (ties to even) with a sticky bit, and assembled directly;
// results outside the normal range take the general path.
OZ_DEVICE_INLINE double w96_to_double(uint32_t w0, uint32_t w1, uint32_t w2, int E) {
  const uint32_t v0 = w0, v1 = w1, v2 = w2;
  const uint32_t sign = w2 & 0x80000000u;
  if (sign) asm("sub.cc.u32 %0, 0, %0;\n\tsubc.cc.u32 %1, 0, %1;\n\tsubc.u32 %2, 0, %2;" : "+r"(w0), "+r"(w1), "+r"(w2));
  if ((w0 | w1 | w2) == 0u) return 0.0;
  int lz = 0;
  if (w2 == 0u) {
    w2 = w1;
    w1 = w0;
    w0 = 0u;
    lz = 32;
    if (w2 == 0u) {
      w2 = w1;
      w1 = 0u;
      lz = 64;
    }
  }
  const int sft = __clz((int)w2);
  if (sft) {
    w2 = __funnelshift_l(w1, w2, sft);
    w1 = __funnelshift_l(w0, w1, sft);
    w0 <<= sft;
  }
  lz += sft;
  int e2 = 95 - lz + E;
  uint32_t mh = w2 >> 11, ml = (w2 << 21) | (w1 >> 11);
  const uint32_t g = w1 & 0x7FFu;
  if (g > 0x400u || (g == 0x400u && (w0 != 0u || (ml & 1u)))) {
    asm("add.cc.u32 %0, %0, 1;\n\taddc.u32 %1, %1, 0;" : "+r"(ml), "+r"(mh));
    if (mh >> 21) {
      mh = 1u << 20;
      ml = 0u;
      e2 += 1;
    }
  }
  if (e2 < -1022 || e2 > 1023) {
    const __int128 Z = (__int128)(((unsigned __int128)(int32_t)v2 << 64) | ((unsigned __int128)v1 << 32) | v0);
    return int128_to_double(Z, E);
  }
  return __hiloint2double((int)(sign | ((uint32_t)(e2 + 1023) << 20) | (mh & 0xFFFFFu)), (int)ml);
}

// The same for Z = zhi * 2^32 + zlo (|zhi|, |zlo| < 2^62, so |Z| < 2^95).
OZ_DEVICE_INLINE double z96_to_double(long long zhi, long long zlo, int E) {
  const uint32_t l0 = (uint32_t)zlo, l1 = (uint32_t)((unsigned long long)zlo >> 32);
  const uint32_t h0 = (uint32_t)zhi, h1 = (uint32_t)((unsigned long long)zhi >> 32);
  const uint32_t sx = (uint32_t)((int32_t)l1 >> 31);
  uint32_t w1, w2;
  asm("add.cc.u32 %0, %2, %3;\n\taddc.u32 %1, %4, %5;" : "=r"(w1), "=r"(w2) : "r"(l1), "r"(h0), "r"(h1), "r"(sx));
  return w96_to_double(l0, w1, w2, E);
}

// Z += x * 2^sh for an int32 x and 0 <= sh < 64, on the 96-bit two's-complement Z = w2:w1:w0.
OZ_DEVICE_INLINE void w96_add_shifted(uint32_t& w0, uint32_t& w1, uint32_t& w2, int x, int sh) {
  const int b = sh & 31;
  const uint32_t lo = (uint32_t)x << b;
  const uint32_t hi = b ? (uint32_t)(x >> (32 - b)) : (uint32_t)(x >> 31);
  const uint32_t sg = (uint32_t)(x >> 31);
  if (sh < 32) {
    asm("add.cc.u32 %0, %0, %3;\n\taddc.cc.u32 %1, %1, %4;\n\taddc.u32 %2, %2, %5;"
        : "+r"(w0), "+r"(w1), "+r"(w2)
        : "r"(lo), "r"(hi), "r"(sg));
  } else {
    asm("add.cc.u32 %0, %0, %2;\n\taddc.u32 %1, %1, %3;" : "+r"(w1), "+r"(w2) : "r"(lo), "r"(hi));
  }
}

}  // namespace oz
