// Split-precision tensor-core contraction on tcgen05 (sm_103a), kind::tf32.
//
//   D[m][n] = sum_k A[m][k] B[n][k]
//
// The tensor core sums its FP32 accumulator with truncation, a bias of about
// one FP32 ulp per accumulation step toward zero: a coherent shrink of every
// dot product that would not average out over the thousands of pairs of an
// MBE(3) energy.  The operands are therefore cut into fixed-point slices
// (tf32_split.cuh): within each 32-wide k-chunk, row m of A is
//   A[m][k] = 2^e_m * sum_{s=1..4} a_s[m][k] 2^(-9 s),  a_s integer, |a_s| <= 2^9,
// with e_m common to the chunk (same for B; tf32_split.cuh).  A slice product of level
// l = s + t is then an integer multiple of 2^(e_m + e_n - 9 l) of magnitude
// <= 2^18, and a chunk sum of the level-2 product (32 terms) or of the two
// level-3 products (64 terms) stays below 2^24 units: it is computed EXACTLY
// whatever the accumulator's rounding.  The seven products of levels 4-5 are
// 2^-18 smaller and share a third (rounded) accumulator; levels >= 6 (below
// 2^-45 of the chunk scale) are dropped.  After every chunk the drain warps
// fold the three level sums into a TMEM-resident (hi, lo) FP32 pair with
// error-free two-sums.
//
// Persistent CTAs (one per SM) over output tiles of 128 rows (TMEM lanes) x up
// to 64 columns:
//   warp 0     TMA producer: the eight 128B-swizzled K-major slice tiles of a
//              k-chunk per stage, two stages
//   warp 1     TMEM allocation and the single MMA-issuing thread (10 MMAs per
//              8-wide k-step)
//   warps 2-5  drain and the transposed epilogue store
// TMEM columns: two buffers of three level accumulators (6 x 64), hi and lo.
// Every mbarrier wait is bounded; a timeout sets ERR_TC_TIMEOUT in *err, the
// roles leave their loops, the producer waits (bounded) for its copies in flight
// and the MMA thread for its last commit, and the CTA frees its tensor memory
// and returns without hanging.
#pragma once
#include <cuda.h>
#include <stdint.h>

#include "tc_job.h"
#include "tf32_split.cuh"

namespace osv {
namespace tc {

constexpr int BK = 32;                       // k per stage (one 128-byte swizzle row of TF32)
constexpr int BROWS = 32;                    // rows of one TMA box of the B operand
constexpr int A_TILE = BM * BK * 4;          // 16 KB per A slice tile
constexpr int B_TILE = BN * BK * 4;          // 8 KB per B slice tile (filled up to n rows)
constexpr int STAGE = NSL * (A_TILE + B_TILE);
constexpr int NSTAGE = 2;
constexpr int SMEM = NSTAGE * STAGE + 1024;  // + slack for 1024-byte alignment
constexpr int NTHREADS = 192;
constexpr int TMEM_COLS = 512;
constexpr int COL_HI = 6 * BN, COL_LO = 7 * BN;
constexpr long long WAIT_LIMIT = 1ll << 26;  // try_wait polls before a wait is declared stuck
constexpr int ERR_TC_TIMEOUT = 16;           // same bit as ERR_TIMEOUT of the library

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < WAIT_LIMIT; it++) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred P1;\n mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n selp.b32 %0, 1, 0, P1;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms 1024 B apart
__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

#define OSV_TMEM_LD16(taddr, r)                                                                                   \
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, " \
               "[%16];"                                                                                           \
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),  \
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),         \
                 "=r"(r[15])                                                                                      \
               : "r"(taddr))
#define OSV_TMEM_ST16(taddr, r)                                                                                    \
  asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15," \
               "%16};" ::"r"(taddr),                                                                               \
               "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),  \
               "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]))

// Epi: functor epi(job, row, col, hi, lo) storing the tile element (row < m_valid,
// col < n_valid) whose value is hi + lo; or, when Epi::kWarp, epi.warp(job, row,
// col0, hi[16], lo[16]) called by every lane of a drain warp (row = its TMEM lane,
// rows past m_valid included) for the columns col0 .. col0 + 15, for epilogues
// that combine the 32 rows of a warp (fixed-point slicing along the rows).
template <class Epi>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_tf32x3(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
             const Job* __restrict__ jobs, int n_jobs, int K, int* err, Epi epi) {
  extern __shared__ uint8_t dsm[];
  __shared__ __align__(8) uint64_t bar_full[NSTAGE], bar_empty[NSTAGE], bar_accf[2], bar_acce[2];
  __shared__ uint32_t s_tmem;
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dsm) + 1023) & ~(uintptr_t)1023);
  const uint32_t sbase = su32(sm);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nch = (K + BK - 1) / BK;

  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&s_tmem)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTAGE; s++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar_full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar_empty[s])));
    }
    for (int b = 0; b < 2; b++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar_accf[b])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(su32(&bar_acce[b])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = s_tmem;
  bool ok = true;
  // Persistent: the CTA takes tiles blockIdx.x, + gridDim.x, ...; g counts the
  // k-chunks this CTA has passed through the pipeline, so the stage and
  // accumulator-buffer phases carry over from one tile to the next and the MMAs
  // of a tile overlap the epilogue of the one before.  A role leaves its loops at
  // its first timed-out wait.

  if (warp == 0) {
    if (lane == 0) {                                             // ---- TMA producer
      long long g = 0;
      for (int tile = blockIdx.x; ok && tile < n_jobs; tile += gridDim.x) {
        const Job jb = jobs[tile];
        const int nbox = (jb.n_valid + BROWS - 1) / BROWS;
        const uint32_t bytes = NSL * (A_TILE + nbox * BROWS * BK * 4);
        for (int c = 0; c < nch; c++, g++) {
          const int s = (int)(g & 1);
          if (g >= NSTAGE) ok &= mbar_wait(su32(&bar_empty[s]), (uint32_t)(((g - NSTAGE) >> 1) & 1));
          if (!ok) break;
          const uint32_t fb = su32(&bar_full[s]);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(bytes) : "memory");
          const uint32_t st = sbase + s * STAGE;
          for (int sl = 0; sl < NSL; sl++)
            tma_load_2d(st + sl * A_TILE, &tmA, fb, c * BK, jb.a_row + sl * jb.a_sstride);
          for (int sl = 0; sl < NSL; sl++)
            for (int bx = 0; bx < nbox; bx++)
              tma_load_2d(st + NSL * A_TILE + sl * B_TILE + bx * BROWS * BK * 4, &tmB, fb, c * BK,
                          jb.b_row + sl * jb.b_sstride + bx * BROWS);
        }
      }
      if (!ok) {
        // leaving early: let the copies already issued land first (bounded waits).  Only
        // the last armed chunk of each stage can be outstanding: a stage is re-armed only
        // after its previous chunk was consumed.
        for (long long gg = g - 1; gg >= 0 && gg >= g - NSTAGE; gg--)
          mbar_wait(su32(&bar_full[gg & 1]), (uint32_t)((gg >> 1) & 1));
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {                                             // ---- MMA issuer
      // slice products (A slice, B slice, level accumulator 0/1/2 for levels 2 / 3 / 4-5)
      const int pa[10] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3};
      const int pb[10] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0};
      const int pl[10] = {0, 1, 1, 2, 2, 2, 2, 2, 2, 2};
      // chunks this CTA runs; a stage is released only to a later chunk (no arrive may
      // be left in flight when the CTA exits)
      const long long g_total = (long long)nch * ((n_jobs - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x);
      long long g = 0;
      for (int tile = blockIdx.x; ok && tile < n_jobs; tile += gridDim.x) {
        const int npad = (jobs[tile].n_valid + 15) & ~15;
        const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(npad >> 3) << 17) |
                               ((uint32_t)(BM >> 4) << 24);
        for (int c = 0; c < nch; c++, g++) {
          const int s = (int)(g & 1), b = (int)(g & 1);
          ok &= mbar_wait(su32(&bar_full[s]), (uint32_t)((g >> 1) & 1));
          if (g >= 2) ok &= mbar_wait(su32(&bar_acce[b]), (uint32_t)(((g - 2) >> 1) & 1));
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t st = sbase + s * STAGE;
          bool first[3] = {true, true, true};
          for (int q = 0; q < 10; q++) {
            const uint32_t dacc = tmem + (uint32_t)((3 * b + pl[q]) * BN);
            for (int ks = 0; ks < BK / 8; ks++) {
              const uint64_t da = desc_sw128(st + pa[q] * A_TILE + ks * 32);
              const uint64_t db = desc_sw128(st + NSL * A_TILE + pb[q] * B_TILE + ks * 32);
              mma_tf32(dacc, da, db, idesc, first[pl[q]] ? 0u : 1u);
              first[pl[q]] = false;
            }
          }
          if (g + NSTAGE < g_total)
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                su32(&bar_empty[s])));
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              su32(&bar_accf[b])));
        }
      }
      // leaving early: the last commit completes when every MMA issued so far has, so
      // wait for it (bounded) before the tensor memory is released
      if (!ok && g > 0) mbar_wait(su32(&bar_accf[(g - 1) & 1]), (uint32_t)(((g - 1) >> 1) & 1));
    }
  } else {                                                       // ---- drain + epilogue (warps 2..5)
    const int q = warp & 3;                                      // TMEM lane quarter of this warp
    const uint32_t lrow = tmem + ((uint32_t)(32 * q) << 16);
    const int row = 32 * q + lane;
    long long g = 0;
    for (int tile = blockIdx.x; ok && tile < n_jobs; tile += gridDim.x) {
      const Job jb = jobs[tile];
      const int npad = (jb.n_valid + 15) & ~15;
      for (int c = 0; c < nch; c++, g++) {
        const int b = (int)(g & 1);
        ok &= mbar_wait(su32(&bar_accf[b]), (uint32_t)((g >> 1) & 1));
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        for (int n0 = 0; n0 < npad; n0 += 16) {
          uint32_t x2[16], x3[16], x4[16], h[16], l[16];
          OSV_TMEM_LD16(lrow + (3 * b + 0) * BN + n0, x2);
          OSV_TMEM_LD16(lrow + (3 * b + 1) * BN + n0, x3);
          OSV_TMEM_LD16(lrow + (3 * b + 2) * BN + n0, x4);
          if (c > 0) {
            OSV_TMEM_LD16(lrow + COL_HI + n0, h);
            OSV_TMEM_LD16(lrow + COL_LO + n0, l);
          } else {
#pragma unroll
            for (int u = 0; u < 16; u++) h[u] = l[u] = 0u;
          }
          asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
          for (int u = 0; u < 16; u++) {
            float sh = __uint_as_float(h[u]), sl = __uint_as_float(l[u]), e;
            two_sum(sh, __uint_as_float(x2[u]), sh, e);
            sl += e;
            two_sum(sh, __uint_as_float(x3[u]), sh, e);
            sl += e;
            two_sum(sh, __uint_as_float(x4[u]), sh, e);
            sl += e;
            h[u] = __float_as_uint(sh);
            l[u] = __float_as_uint(sl);
          }
          OSV_TMEM_ST16(lrow + COL_HI + n0, h);
          OSV_TMEM_ST16(lrow + COL_LO + n0, l);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&bar_acce[b])) : "memory");
      }
      if (!ok) break;
      for (int n0 = 0; n0 < npad; n0 += 16) {
        uint32_t h[16], l[16];
        OSV_TMEM_LD16(lrow + COL_HI + n0, h);
        OSV_TMEM_LD16(lrow + COL_LO + n0, l);
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if constexpr (Epi::kWarp) {
          epi.warp(jb, row, n0, h, l);
        } else if (row < jb.m_valid) {
#pragma unroll
          for (int u = 0; u < 16; u++)
            if (n0 + u < jb.n_valid) epi(jb, row, n0 + u, __uint_as_float(h[u]), __uint_as_float(l[u]));
        }
      }
    }
  }
  if (!ok) atomicOr(err, ERR_TC_TIMEOUT);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

// Grid of the persistent kernel: one CTA per SM, at most one per tile.
inline int persistent_grid(int n_jobs) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
  }
  return n_jobs < sms ? n_jobs : sms;
}

}  // namespace tc
}  // namespace osv
