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
// One CTA per SM, persistent over a tile list; 10 warps:
//   warp 0       producer: cp.async.bulk of pre-tiled digit planes into an NSTAGE ring
//   warp 1       TMEM owner and single-thread MMA issuer; diagonal g = t+u-2 of the slice grid
//                accumulates into its own TMEM buffer (BN columns), A reused through the
//                collector across the u loop; a full buffer is handed to the epilogue ("drain")
//                and replaced by a free one, so the MMA never waits on the epilogue while a
//                spare buffer exists
//   warps 2..9   epilogue: exact 128-bit running sums Z += q * 256^(s-1-g) per output element,
//                then one round-to-nearest-even to FP64 scaled by 2^(ea+eb-8s-6), alpha/beta,
//                store (and for the row-table mode a per-row |max| for the next slicing).
// Every wait is bounded; a timeout sets *err and all roles leave their loops.
#include "oz_gemm.cuh"

namespace oz {

constexpr int A_TILE_BYTES = TILE_M * KB * 2;   // 8 KB per plane
constexpr int B_TILE_BYTES = BN * KB * 2;       // 4 KB per plane
constexpr int STAGE_BYTES = MAX_LEVEL * (A_TILE_BYTES + B_TILE_BYTES);
constexpr int NTHREADS = 320;

struct Shared {
  unsigned long long full[NSTAGE], empty[NSTAGE], accf[NBUF], acce[NBUF], qfull[QN], fin;
  int4 rec[QN];
  uint32_t tmem;
  int abort;
};

size_t gemm_smem_bytes() { return (size_t)NSTAGE * STAGE_BYTES + sizeof(Shared) + 1024; }

struct MmaCtl {
  long long it;      // k-block iterations issued (ring position)
  int fresh;         // buffers never used yet
  int qseq;          // drain records posted
  int reclaim;       // next record whose buffer is reused
  uint32_t acce_par; // per buffer parity of the next "drained" wait
};

__device__ __forceinline__ uint32_t bar(const unsigned long long* p) { return smem_u32(p); }

__device__ __noinline__ void post(Shared& sh, MmaCtl& c, uint32_t b, int shift, int flags) {
  tc_commit(bar(&sh.accf[b]));
  int slot = c.qseq % QN;
  sh.rec[slot] = make_int4((int)b, shift, flags, 0);
  mbar_arrive(bar(&sh.qfull[slot]));
  c.qseq++;
}

__device__ __noinline__ uint32_t acquire(Shared& sh, MmaCtl& c, volatile int* abort) {
  if (c.fresh < NBUF) return (uint32_t)c.fresh++;
  int slot = c.reclaim % QN;
  uint32_t b = (uint32_t)sh.rec[slot].x;
  c.reclaim++;
  mbar_wait(bar(&sh.acce[b]), (c.acce_par >> b) & 1u, abort);
  c.acce_par ^= 1u << b;
  tc_fence_after();
  return b;
}

// MMAs of one output tile at slice level S.  Per k-block (one K-step of 16) diagonal g = t + u
// (0-based) receives g + 1 slice-pair products of 16 terms each; before the k-block, every diagonal
// whose group could not absorb them is drained (its buffer handed to the epilogue and replaced), so
// the MMA sequence itself is branch-free.  First groups are shortened by a per-diagonal offset so
// that the drains of different diagonals fall into different k-blocks.
template <int S>
__device__ void mma_tile(Shared& sh, MmaCtl& c, uint32_t tmem, uint32_t stage0, int nkb, volatile int* abort) {
  constexpr uint32_t IDESC = idesc_f16(TILE_M, BN);
  uint32_t buf[S];
  int room[S];
#pragma unroll
  for (int g = 0; g < S; ++g) {
    buf[g] = acquire(sh, c, abort);
    const int per = 16 * (g + 1);
    const int period = GROUP_TERMS / per;              // k-blocks per full group
    room[g] = GROUP_TERMS - per * ((g * period) / S);   // staggered first group
  }
  uint32_t fresh = (1u << S) - 1u;  // diagonals whose current buffer has not been written yet
  for (int kb = 0; kb < nkb; ++kb) {
    const int stg = (int)(c.it % NSTAGE);
    const uint32_t par = (uint32_t)((c.it / NSTAGE) & 1);
#pragma unroll
    for (int g = 0; g < S; ++g) {
      if (room[g] < 16 * (g + 1)) {
        post(sh, c, buf[g], 8 * (S - 1 - g), 0);
        buf[g] = acquire(sh, c, abort);
        room[g] = GROUP_TERMS;
        fresh |= 1u << g;
      }
      room[g] -= 16 * (g + 1);
    }
    if (!mbar_wait(bar(&sh.full[stg]), par, abort)) return;
    const uint32_t aaddr = stage0 + stg * STAGE_BYTES;
    const uint64_t ad0 = smem_desc(aaddr, 128, 128 * KB_CM);
    const uint64_t bd0 = smem_desc(aaddr + MAX_LEVEL * A_TILE_BYTES, 128, 128 * KB_CM);
#pragma unroll
    for (int t = 0; t < S; ++t) {
      const uint64_t ad = ad0 + (uint64_t)((t * A_TILE_BYTES) >> 4);
#pragma unroll
      for (int u = 0; u < S - t; ++u) {
        const int g = t + u;
        const uint64_t bd = bd0 + (uint64_t)((u * B_TILE_BYTES) >> 4);
        const uint32_t d = tmem + buf[g] * BN;
        // the first product of a k-block into diagonal g is the one with t = 0
        const uint32_t acc = (t == 0) ? (((fresh >> g) & 1u) ^ 1u) : 1u;
        const int nu = S - t;
        if (nu == 1) mma_f16<0>(d, ad, bd, IDESC, acc);
        else if (u == 0) mma_f16<1>(d, ad, bd, IDESC, acc);
        else if (u == nu - 1) mma_f16<3>(d, ad, bd, IDESC, acc);
        else mma_f16<2>(d, ad, bd, IDESC, acc);
      }
    }
    fresh = 0u;
    tc_commit(bar(&sh.empty[stg]));
    c.it++;
  }
#pragma unroll
  for (int g = 0; g < S; ++g) post(sh, c, buf[g], 8 * (S - 1 - g), g == S - 1 ? 1 : 0);
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

__global__ void __launch_bounds__(NTHREADS, 1)
    gemm_kernel(const GemmProblem* __restrict__ probs, const GemmTile* __restrict__ tiles, int ntiles,
                const __grid_constant__ GemmProblem single, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  Shared& sh = *reinterpret_cast<Shared*>(smem + NSTAGE * STAGE_BYTES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int* abort = &sh.abort;
  const uint32_t stage0 = smem_u32(smem);

  if (threadIdx.x == 0) {
    for (int i = 0; i < NSTAGE; ++i) {
      mbar_init(bar(&sh.full[i]), 1);
      mbar_init(bar(&sh.empty[i]), 1);
    }
    for (int i = 0; i < NBUF; ++i) {
      mbar_init(bar(&sh.accf[i]), 1);
      mbar_init(bar(&sh.acce[i]), 8);
    }
    for (int i = 0; i < QN; ++i) mbar_init(bar(&sh.qfull[i]), 1);
    mbar_init(bar(&sh.fin), 1);
    sh.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(&sh.tmem), 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh.tmem;

  if (warp == 0) {
    // ------------------------------------------------------------------ producer
    if (lane == 0) {
      long long it = 0;
      for (int idx = blockIdx.x; idx < ntiles && !*abort; idx += gridDim.x) {
        const GemmProblem* P;
        int mb, nb;
        tile_of(tiles, probs, single, idx, P, mb, nb);
        const int nkb = P->nkb, s = P->s, SA = P->SA, SB = P->SB;
        const char* Ab = reinterpret_cast<const char*>(P->A) + (long long)mb * nkb * SA * A_TILE_BYTES;
        const char* Bb = reinterpret_cast<const char*>(P->B) + (long long)nb * nkb * SB * B_TILE_BYTES;
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int stg = (int)(it % NSTAGE);
          if (it >= NSTAGE && !mbar_wait(bar(&sh.empty[stg]), (uint32_t)(((it / NSTAGE) - 1) & 1), abort)) break;
          mbar_expect_tx(bar(&sh.full[stg]), (uint32_t)(s * (A_TILE_BYTES + B_TILE_BYTES)));
          const uint32_t dA = stage0 + stg * STAGE_BYTES;
          bulk_g2s(dA, Ab + (long long)kb * SA * A_TILE_BYTES, (uint32_t)(s * A_TILE_BYTES), bar(&sh.full[stg]));
          bulk_g2s(dA + MAX_LEVEL * A_TILE_BYTES, Bb + (long long)kb * SB * B_TILE_BYTES,
                   (uint32_t)(s * B_TILE_BYTES), bar(&sh.full[stg]));
        }
      }
      // let the copies still in flight land before the CTA can exit
      for (long long j = it - NSTAGE; j < it; ++j) {
        if (j < 0) continue;
        volatile int never = 0;
        mbar_wait(bar(&sh.full[j % NSTAGE]), (uint32_t)((j / NSTAGE) & 1), &never);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      MmaCtl c{0, 0, 0, 0, 0u};
      for (int idx = blockIdx.x; idx < ntiles && !*abort; idx += gridDim.x) {
        const GemmProblem* P;
        int mb, nb;
        tile_of(tiles, probs, single, idx, P, mb, nb);
        const int nkb = P->nkb;
        switch (P->s) {
          case 1: mma_tile<1>(sh, c, tmem, stage0, nkb, abort); break;
          case 2: mma_tile<2>(sh, c, tmem, stage0, nkb, abort); break;
          case 3: mma_tile<3>(sh, c, tmem, stage0, nkb, abort); break;
          case 4: mma_tile<4>(sh, c, tmem, stage0, nkb, abort); break;
          case 5: mma_tile<5>(sh, c, tmem, stage0, nkb, abort); break;
          case 6: mma_tile<6>(sh, c, tmem, stage0, nkb, abort); break;
          case 7: mma_tile<7>(sh, c, tmem, stage0, nkb, abort); break;
          case 8: mma_tile<8>(sh, c, tmem, stage0, nkb, abort); break;
          default: *abort = 1; break;
        }
      }
      // all issued MMAs complete before TMEM is released
      tc_commit(bar(&sh.fin));
      volatile int never = 0;
      mbar_wait(bar(&sh.fin), 0, &never);
    }
  } else {
    // ------------------------------------------------------------------ epilogue
    const int lq = warp & 3;            // TMEM lane quarter this warp may access
    const int ch = (warp - 2) >> 2;     // column half of the BN-wide tile
    long long eseq = 0;
    uint32_t accf_par = 0;
    for (int idx = blockIdx.x; idx < ntiles && !*abort; idx += gridDim.x) {
      const GemmProblem* P;
      int mb, nb;
      tile_of(tiles, probs, single, idx, P, mb, nb);
      // exact running sum Z = zhi * 2^32 + zlo; drains with shift < 32 go to zlo, the others to zhi
      // (each part stays below 2^62 in magnitude for levels <= 8 and fewer than 2^14 groups per diagonal)
      long long zlo[32], zhi[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        zlo[j] = 0ll;
        zhi[j] = 0ll;
      }
      bool ok = true;
      while (true) {
        const int slot = (int)(eseq % QN);
        if (!mbar_wait(bar(&sh.qfull[slot]), (uint32_t)((eseq / QN) & 1), abort)) { ok = false; break; }
        volatile int* rp = reinterpret_cast<volatile int*>(&sh.rec[slot]);
        const int4 r = make_int4(rp[0], rp[1], rp[2], rp[3]);
        const uint32_t b = (uint32_t)r.x;
        if (!mbar_wait(bar(&sh.accf[b]), (accf_par >> b) & 1u, abort)) { ok = false; break; }
        accf_par ^= 1u << b;
        tc_fence_after();
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(lq * 32) << 16) + b * BN + ch * 32, v);
        tmem_wait_ld();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(&sh.acce[b]));
        const int shl = r.y;
        if (shl < 32) {
#pragma unroll
          for (int j = 0; j < 32; ++j) zlo[j] += (long long)__float2int_rn(__uint_as_float(v[j])) << shl;
        } else {
          const int sh2 = shl - 32;
#pragma unroll
          for (int j = 0; j < 32; ++j) zhi[j] += (long long)__float2int_rn(__uint_as_float(v[j])) << sh2;
        }
        ++eseq;
        if (r.z & 1) break;
      }
      if (!ok) break;
      // ---- one rounding to FP64, scaling, store
      const int M = P->M, N = P->N, s = P->s, mode = P->mode;
      const int row = mb * TILE_M + lq * 32 + lane;
      if (row < M) {
        const int* __restrict__ eb = P->eb;
        const int ea = __ldg(P->ea + row) - 8 * s - 6;
        const int col0 = nb * BN + ch * 32;
        const int ncol = min(32, N - col0);
        if (mode == OUT_DENSE) {
          double* crow = P->C + (long long)row * P->ldc + col0;
          const double alpha = P->alpha, beta = P->beta;
          const bool plain = (alpha == 1.0) && (beta == 0.0);
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            if (j < ncol) {
              const __int128 Z = ((__int128)zhi[j] << 32) + (__int128)zlo[j];
              double c = int128_to_double(Z, ea + __ldg(eb + col0 + j));
              if (!plain) {
                c = __dmul_rn(alpha, c);
                if (beta != 0.0) c = __dadd_rn(c, __dmul_rn(beta, crow[j]));
              }
              crow[j] = c;
            }
          }
        } else {
          double* crow = P->C + __ldg(P->rowdst + row) + col0;
          unsigned long long mx = 0;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            if (j < ncol) {
              const __int128 Z = ((__int128)zhi[j] << 32) + (__int128)zlo[j];
              const double c = int128_to_double(Z, ea + __ldg(eb + col0 + j));
              crow[j] = c;
              const unsigned long long bb = (unsigned long long)__double_as_longlong(c) & 0x7FFFFFFFFFFFFFFFull;
              mx = bb > mx ? bb : mx;
            }
          }
          unsigned long long* rmax = P->rowmax;
          if (rmax && mx) atomicMax(rmax + __ldg(P->rowslot + row), mx);
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
  if (threadIdx.x == 0 && sh.abort) atomicOr(err, 2);
}

cudaError_t launch_gemm(const GemmProblem* d_probs, const GemmTile* d_tiles, int ntiles, int grid,
                        const GemmProblem* single, int* d_err, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  static bool attr = false;
  const size_t smem = gemm_smem_bytes();
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  GemmProblem one{};
  if (single) one = *single;
  gemm_kernel<<<grid < ntiles ? grid : ntiles, NTHREADS, smem, st>>>(d_probs, d_tiles, ntiles, one, d_err);
  return cudaGetLastError();
}

}  // namespace oz
