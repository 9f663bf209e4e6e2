// FP32 GEMM on the tcgen05 tensor cores (kind::tf32) with 3xTF32 splitting,
// the engine of the FP32 bulk of the mixed path: Cholesky trailing updates,
// the rank-2k updates of the skew tridiagonalization, the back-transform and
// the refinement's corrections.
//
//   C = alpha * op(A) * op(B) + beta * C      (column-major FP32, optional
//                                               restriction to C's lower triangle)
//
// Splitting. Every FP32 operand value x is written as hi + lo with
// hi = x rounded to TF32 (10 explicit mantissa bits) and lo = x - hi (exact in
// FP32); the product is accumulated as hi*hi + hi*lo + lo*hi in FP32 in TMEM,
// which drops only lo*lo (about 2^-22 relative) and leaves FP32-level accuracy.
// With split = 0 a single TF32 pass runs (10-bit operands).
//
// Layout. Column-major operands are staged by TMA in their natural layout:
// op(A) = A (M contiguous) and op(B) = B^T (N contiguous) arrive "MN-major",
// op(A) = A^T and op(B) = B arrive "K-major" (K contiguous). The splitter warps
// write hi and lo of every tile in the K-major 128-byte-swizzled layout the MMA
// reads (transposing MN-major tiles on the way, bank-conflict free), so no
// operand is transposed or copied in global memory. Tiles are 128 x 128 with
// 32-deep K stages.
//
// Structure (448 threads, one persistent CTA per SM over the output tiles):
//   warp 0     TMA producer: raw FP32 tiles of op(A) and op(B) into a 3-slot
//              ring (32 KiB per slot)
//   warps 10-13 splitters: raw slot -> hi and lo tiles in a 2-slot MMA ring
//              (64 KiB per slot), then a proxy fence so that the tensor cores
//              see the generic-proxy stores
//   warp 1     TMEM owner and MMA issuer (one thread): 3 (or 1) tcgen05.mma
//              per 8-deep K step; each 32-deep K block accumulates afresh in
//              one of two 128 x 128 FP32 TMEM buffers
//   warps 2-9  epilogue: adds each K block's TMEM buffer into registers with
//              round-to-nearest FP32 while the MMA fills the other buffer,
//              then writes alpha acc + beta C (one row and 64 columns per thread)
//
// Accumulation. The tensor cores truncate their FP32 sums at every MMA step,
// so a K-long run through one accumulator collects a bias of order
// (K/8) 2^-24 relative to the sum; restarting every 32 and summing the blocks
// in registers bounds it by 4 steps and keeps the result at FP32 level.
// Every wait is bounded; on timeout the CTA records BSE_ERR_TIMEOUT in the
// caller's status word, lets its copies and MMAs drain, frees TMEM and returns.
#include <cuda.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "common.cuh"
#include "gemm_simt.cuh"
#include "ptx_sm100.cuh"
#include "tc32.cuh"

namespace bse {
namespace tc32 {

using namespace ptx;

constexpr int BM = 128, BN = 128, BK = 32;
constexpr int RSTAGES = 3, MSTAGES = 2;
constexpr int TILE_BYTES = BM * BK * 4;        // 16 KiB: one 128 x 32 FP32 operand tile
constexpr int RAW_BYTES = 2 * TILE_BYTES;      // raw slot: A, B
constexpr int MMA_BYTES = 4 * TILE_BYTES;      // MMA slot: A.hi, B.hi, A.lo, B.lo
constexpr int SMEM_BYTES = RSTAGES * RAW_BYTES + MSTAGES * MMA_BYTES + 1024 + 256;
constexpr int THREADS = 448;
constexpr uint32_t TMEM_COLS = 2 * BN;         // two FP32 accumulators
constexpr int kGroupM = 8;                     // row tiles per L2 band

struct Params {
  int M, N, K;
  int a_mn, b_mn;  // operand is MN-major (1) or K-major (0)
  int split;       // 1: 3xTF32, 0: 1xTF32
  int uplo;        // 0 all of C, 1 lower triangle i >= j, 2 strict lower i > j (M == N)
  int tiles_m, tiles_n, tiles;
  float alpha, beta;
  float* C;
  long ldc;
  int* status;
};

// Tile t -> (row tile, column tile). Full C: bands of kGroupM row tiles walked
// column by column so co-resident CTAs share operand tiles in L2. Lower
// triangle: the tiles with tm >= tn, row by row.
__device__ __forceinline__ void tile_coords(const Params& P, int t, int& tm, int& tn) {
  if (P.uplo) {
    int r = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((long)r * (r + 1) / 2 > t) --r;
    while ((long)(r + 1) * (r + 2) / 2 <= t) ++r;
    tm = r;
    tn = t - r * (r + 1) / 2;
    return;
  }
  const int group = t / (kGroupM * P.tiles_n);
  const int first_m = group * kGroupM;
  const int gm = min(kGroupM, P.tiles_m - first_m);
  const int in_group = t - group * kGroupM * P.tiles_n;
  tm = first_m + in_group % gm;
  tn = in_group / gm;
}

// kind::tf32, D = F32, A = B = TF32, both K-major, N = BN, M = BM.
__host__ __device__ constexpr uint32_t make_idesc() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}

// Descriptor of the 8-deep K slice ks (0..3) of a K-major 128 x 32 tile: rows of
// 32 FP32 (128 B, swizzled), 8-row groups 1 KiB apart; the slice is a 32-byte
// step inside the rows.
__device__ __forceinline__ uint64_t tile_desc(uint32_t saddr, int ks) {
  return make_desc_sw128(saddr + (uint32_t)ks * 32u, 16, 1024);
}

// Byte offset of element (row r, k) in a K-major 128-byte-swizzled tile.
__device__ __forceinline__ uint32_t kmaj_off(int r, int k) {
  return (uint32_t)r * 128u + ((uint32_t)((k >> 2) ^ (r & 7)) << 4) + (uint32_t)(k & 3) * 4u;
}

__device__ __forceinline__ uint32_t rna_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__global__ void __launch_bounds__(THREADS, 1)
    tc32_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const Params P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* raw_ring = smem;
  uint8_t* mma_ring = smem + RSTAGES * RAW_BYTES;
  uint64_t* raw_full = reinterpret_cast<uint64_t*>(mma_ring + MSTAGES * MMA_BYTES);
  uint64_t* raw_empty = raw_full + RSTAGES;
  uint64_t* mma_full = raw_empty + RSTAGES;
  uint64_t* mma_empty = mma_full + MSTAGES;
  uint64_t* tfull = mma_empty + MSTAGES;  // [2]
  uint64_t* tempty = tfull + 2;           // [2]
  uint64_t* drain = tempty + 2;           // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* err = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int KB = (P.K + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < RSTAGES; ++s) {
      mbar_init(&raw_full[s], 1);
      mbar_init(&raw_empty[s], 128);
    }
    for (int s = 0; s < MSTAGES; ++s) {
      mbar_init(&mma_full[s], 128);
      mbar_init(&mma_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 256);
    }
    mbar_init(drain, 1);
    *err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // TMA producer: one raw slot (A and B tiles of one K stage) per iteration
      int it = 0;
      uint32_t issued = 0, last_par = 0;
      for (int t = blockIdx.x; t < P.tiles && !*err; t += gridDim.x) {
        int tm, tn;
        tile_coords(P, t, tm, tn);
        const int m0 = tm * BM, n0 = tn * BN;
        for (int kb = 0; kb < KB; ++kb, ++it) {
          const int rs = it % RSTAGES;
          const uint32_t ph = (it / RSTAGES) & 1;
          if (!mbar_wait(&raw_empty[rs], ph ^ 1, err)) break;
          uint8_t* sa = raw_ring + rs * RAW_BYTES;
          uint8_t* sb = sa + TILE_BYTES;
          mbar_expect_tx(&raw_full[rs], RAW_BYTES);
          const int k0 = kb * BK;
          if (P.a_mn) {
#pragma unroll
            for (int j = 0; j < BM / 32; ++j) tma_load_2d(sa + j * (BK * 128), &tmA, m0 + 32 * j, k0, &raw_full[rs]);
          } else {
            tma_load_2d(sa, &tmA, k0, m0, &raw_full[rs]);
          }
          if (P.b_mn) {
#pragma unroll
            for (int j = 0; j < BN / 32; ++j) tma_load_2d(sb + j * (BK * 128), &tmB, n0 + 32 * j, k0, &raw_full[rs]);
          } else {
            tma_load_2d(sb, &tmB, k0, n0, &raw_full[rs]);
          }
          issued |= 1u << rs;
          last_par = (last_par & ~(1u << rs)) | (ph << rs);
        }
      }
      // the CTA may leave early after an error: first let every issued copy land
      for (int rs = 0; rs < RSTAGES; ++rs)
        if (issued & (1u << rs)) mbar_drain(&raw_full[rs], (last_par >> rs) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = make_idesc();
      // Every 32-deep K block is a separate accumulation (TMEM buffer c & 1):
      // the tensor cores truncate their FP32 sums at each MMA, so long K runs
      // would collect a bias; the epilogue adds the blocks with rounded FP32.
      int it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < P.tiles && ok; t += gridDim.x) {
        for (int kb = 0; kb < KB; ++kb, ++it) {
          const int buf = it & 1;
          ok = mbar_wait(&tempty[buf], ((it >> 1) & 1) ^ 1, err);
          if (!ok) break;
          const int ms = it % MSTAGES;
          const uint32_t ph = (it / MSTAGES) & 1;
          ok = mbar_wait(&mma_full[ms], ph, err);
          if (!ok) break;
          tc_fence_after();
          const uint32_t d = tmem_base + (uint32_t)(buf * BN);
          const uint32_t sah = smem_u32(mma_ring + ms * MMA_BYTES);
          const uint32_t sbh = sah + TILE_BYTES, sal = sah + 2 * TILE_BYTES, sbl = sah + 3 * TILE_BYTES;
#pragma unroll
          for (int ks = 0; ks < BK / 8; ++ks) {
            const uint64_t ah = tile_desc(sah, ks), bh = tile_desc(sbh, ks);
            if (P.split) {
              // small terms first, the dominant hi*hi last
              umma_tf32(d, ah, tile_desc(sbl, ks), idesc, ks != 0);
              umma_tf32(d, tile_desc(sal, ks), bh, idesc, 1);
              umma_tf32(d, ah, bh, idesc, 1);
            } else {
              umma_tf32(d, ah, bh, idesc, ks != 0);
            }
          }
          umma_commit(&mma_empty[ms]);
          umma_commit(&tfull[buf]);
        }
      }
      // all issued MMAs complete before TMEM can be released
      umma_commit(drain);
      mbar_drain(drain, 0);
    }
  } else if (warp < 10) {
    // epilogue: TMEM lane quadrant q4 = warp % 4 holds output rows q4*32 .. q4*32+31;
    // two warps per quadrant, each thread = one output row and 64 of its columns,
    // the sums in registers across the K blocks
    const int q4 = warp & 3;
    const int half = (warp - 2) >> 2;
    constexpr int CW = BN / 2;
    int it = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < P.tiles && ok; t += gridDim.x) {
      int tm, tn;
      tile_coords(P, t, tm, tn);
      float acc[CW];
#pragma unroll
      for (int i = 0; i < CW; ++i) acc[i] = 0.0f;
      for (int kb = 0; kb < KB; ++kb, ++it) {
        const int buf = it & 1;
        ok = __all_sync(0xffffffffu, mbar_wait(&tfull[buf], (it >> 1) & 1, err));
        if (!ok) break;
        tc_fence_after();
        const uint32_t tb = tmem_base + (uint32_t)(buf * BN + half * CW) + ((uint32_t)(q4 * 32) << 16);
#pragma unroll
        for (int c0 = 0; c0 < CW; c0 += 16) {
          float v[16];
          tmem_ld16(tb + (uint32_t)c0, v);
#pragma unroll
          for (int i = 0; i < 16; ++i) acc[c0 + i] += v[i];
        }
        tc_fence_before();
        mbar_arrive(&tempty[buf]);
      }
      if (!ok) break;
      const int row = tm * BM + q4 * 32 + lane;
      const int n0 = tn * BN + half * CW;
      // last column this row may write (lower triangle) and the column limit
      int cmax = P.N - 1;
      if (P.uplo == 1) cmax = min(cmax, row);
      if (P.uplo == 2) cmax = min(cmax, row - 1);
      if (row >= P.M) cmax = -1;
      float* crow = P.C + row;
      if (P.beta != 0.0f) {
#pragma unroll
        for (int c0 = 0; c0 < CW; c0 += 16) {
          float old[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int col = n0 + c0 + i;
            old[i] = (col <= cmax) ? crow[(long)col * P.ldc] : 0.0f;
          }
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int col = n0 + c0 + i;
            if (col <= cmax) crow[(long)col * P.ldc] = fmaf(P.alpha, acc[c0 + i], P.beta * old[i]);
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < CW; ++i) {
          const int col = n0 + i;
          if (col <= cmax) crow[(long)col * P.ldc] = P.alpha * acc[i];
        }
      }
    }
  } else {
    // splitters (128 threads): raw slot -> K-major hi / lo tiles of an MMA slot
    const int tid = threadIdx.x - 320;
    const int sw = tid >> 5;  // splitter warp 0..3
    int it = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < P.tiles && ok; t += gridDim.x) {
      for (int kb = 0; kb < KB; ++kb, ++it) {
        const int rs = it % RSTAGES, ms = it % MSTAGES;
        ok = mbar_wait(&raw_full[rs], (it / RSTAGES) & 1, err) &&
             mbar_wait(&mma_empty[ms], ((it / MSTAGES) & 1) ^ 1, err);
        if (!ok) break;
        const uint8_t* raw = raw_ring + rs * RAW_BYTES;
        uint8_t* dst = mma_ring + ms * MMA_BYTES;
#pragma unroll
        for (int op = 0; op < 2; ++op) {
          const uint8_t* src = raw + op * TILE_BYTES;
          uint8_t* hi = dst + op * TILE_BYTES;
          uint8_t* lo = dst + (2 + op) * TILE_BYTES;
          const int mn = op == 0 ? P.a_mn : P.b_mn;
          if (mn) {
            // MN-major raw: four 32-column blocks of 32 K-rows (128 B, swizzled).
            // Lane = k; a warp reads the 4 consecutive rows mn0..mn0+3 at every k
            // (one float4 per lane) and scatters them to 4 K-major rows.
            const int k = lane;
#pragma unroll 2
            for (int q = sw; q < BM / 4; q += 4) {
              const int mn0 = 4 * q;
              const int chunk = (mn0 & 31) >> 2;
              const float4 x = *reinterpret_cast<const float4*>(src + (mn0 >> 5) * (BK * 128) + k * 128 +
                                                                (((chunk ^ (k & 7)) & 7) << 4));
              const float xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const uint32_t o = kmaj_off(mn0 + e, k);
                const float h = __uint_as_float(rna_tf32(xv[e]));
                *reinterpret_cast<float*>(hi + o) = h;
                if (P.split) *reinterpret_cast<float*>(lo + o) = xv[e] - h;
              }
            }
          } else {
            // K-major raw already has the MMA layout: elementwise hi / lo
#pragma unroll 4
            for (int i = tid; i < TILE_BYTES / 16; i += 128) {
              const float4 x = reinterpret_cast<const float4*>(src)[i];
              float4 h, l;
              h.x = __uint_as_float(rna_tf32(x.x));
              h.y = __uint_as_float(rna_tf32(x.y));
              h.z = __uint_as_float(rna_tf32(x.z));
              h.w = __uint_as_float(rna_tf32(x.w));
              reinterpret_cast<float4*>(hi)[i] = h;
              if (P.split) {
                l.x = x.x - h.x;
                l.y = x.y - h.y;
                l.z = x.z - h.z;
                l.w = x.w - h.w;
                reinterpret_cast<float4*>(lo)[i] = l;
              }
            }
          }
        }
        // make the generic-proxy stores visible to the tensor cores (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&mma_full[ms]);
        mbar_arrive(&raw_empty[rs]);
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, TMEM_COLS);
  }
  if (threadIdx.x == 0 && *err && P.status) atomicCAS(P.status, 0, *err);
}

// ---- pre-split operands -------------------------------------------------------
// The same product from operands split once in global memory into K-major TF32
// planes hi = rna_tf32(x), lo = x - hi (rows of op(A) / op(B)^T, K contiguous,
// row pitch ldk). TMA then lands every tile already in the MMA's K-major
// 128-byte-swizzled layout, so no warp rewrites operands in shared memory: per
// 32-deep K block the tensor cores' operand reads (96 KiB) and the TMA writes
// (64 KiB) are the only shared-memory traffic, against 192 KiB with in-kernel
// splitting.
constexpr int PSTAGES = 3;                         // 64 KiB per stage: A.hi, B.hi, A.lo, B.lo
constexpr int P_SMEM_BYTES = PSTAGES * MMA_BYTES + 1024 + 256;
constexpr int P_THREADS = 320;                     // TMA warp, MMA warp, 8 epilogue warps

__global__ void __launch_bounds__(P_THREADS, 1)
    tc32p_kernel(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                 const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl, const Params P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* ring = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + PSTAGES * MMA_BYTES);
  uint64_t* empty = full + PSTAGES;
  uint64_t* tfull = empty + PSTAGES;  // [2]
  uint64_t* tempty = tfull + 2;       // [2]
  uint64_t* drain = tempty + 2;       // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* err = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int KB = (P.K + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int st = 0; st < PSTAGES; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 256);
    }
    mbar_init(drain, 1);
    *err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      uint32_t issued = 0, last_par = 0;
      for (int t = blockIdx.x; t < P.tiles && !*err; t += gridDim.x) {
        int tm, tn;
        tile_coords(P, t, tm, tn);
        const int m0 = tm * BM, n0 = tn * BN;
        for (int kb = 0; kb < KB; ++kb, ++it) {
          const int st = it % PSTAGES;
          const uint32_t ph = (it / PSTAGES) & 1;
          if (!mbar_wait(&empty[st], ph ^ 1, err)) break;
          uint8_t* sah = ring + st * MMA_BYTES;
          const int k0 = kb * BK;
          mbar_expect_tx(&full[st], MMA_BYTES);
          tma_load_2d(sah, &tmAh, k0, m0, &full[st]);
          tma_load_2d(sah + TILE_BYTES, &tmBh, k0, n0, &full[st]);
          tma_load_2d(sah + 2 * TILE_BYTES, &tmAl, k0, m0, &full[st]);
          tma_load_2d(sah + 3 * TILE_BYTES, &tmBl, k0, n0, &full[st]);
          issued |= 1u << st;
          last_par = (last_par & ~(1u << st)) | (ph << st);
        }
      }
      for (int st = 0; st < PSTAGES; ++st)
        if (issued & (1u << st)) mbar_drain(&full[st], (last_par >> st) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = make_idesc();
      int it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < P.tiles && ok; t += gridDim.x) {
        for (int kb = 0; kb < KB; ++kb, ++it) {
          const int buf = it & 1;
          ok = mbar_wait(&tempty[buf], ((it >> 1) & 1) ^ 1, err);
          if (!ok) break;
          const int st = it % PSTAGES;
          ok = mbar_wait(&full[st], (it / PSTAGES) & 1, err);
          if (!ok) break;
          tc_fence_after();
          const uint32_t d = tmem_base + (uint32_t)(buf * BN);
          const uint32_t sah = smem_u32(ring + st * MMA_BYTES);
          const uint32_t sbh = sah + TILE_BYTES, sal = sah + 2 * TILE_BYTES, sbl = sah + 3 * TILE_BYTES;
#pragma unroll
          for (int ks = 0; ks < BK / 8; ++ks) {
            const uint64_t ah = tile_desc(sah, ks), bh = tile_desc(sbh, ks);
            umma_tf32(d, ah, tile_desc(sbl, ks), idesc, ks != 0);
            umma_tf32(d, tile_desc(sal, ks), bh, idesc, 1);
            umma_tf32(d, ah, bh, idesc, 1);
          }
          umma_commit(&empty[st]);
          umma_commit(&tfull[buf]);
        }
      }
      umma_commit(drain);
      mbar_drain(drain, 0);
    }
  } else {
    // epilogue, as in tc32_kernel: warps 2..9, lane quadrant warp % 4, column half
    const int q4 = warp & 3;
    const int half = (warp - 2) >> 2;
    constexpr int CW = BN / 2;
    int it = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < P.tiles && ok; t += gridDim.x) {
      int tm, tn;
      tile_coords(P, t, tm, tn);
      float acc[CW];
#pragma unroll
      for (int i = 0; i < CW; ++i) acc[i] = 0.0f;
      for (int kb = 0; kb < KB; ++kb, ++it) {
        const int buf = it & 1;
        ok = __all_sync(0xffffffffu, mbar_wait(&tfull[buf], (it >> 1) & 1, err));
        if (!ok) break;
        tc_fence_after();
        const uint32_t tb = tmem_base + (uint32_t)(buf * BN + half * CW) + ((uint32_t)(q4 * 32) << 16);
#pragma unroll
        for (int c0 = 0; c0 < CW; c0 += 16) {
          float v[16];
          tmem_ld16(tb + (uint32_t)c0, v);
#pragma unroll
          for (int i = 0; i < 16; ++i) acc[c0 + i] += v[i];
        }
        tc_fence_before();
        mbar_arrive(&tempty[buf]);
      }
      if (!ok) break;
      const int row = tm * BM + q4 * 32 + lane;
      const int n0 = tn * BN + half * CW;
      int cmax = P.N - 1;
      if (P.uplo == 1) cmax = min(cmax, row);
      if (P.uplo == 2) cmax = min(cmax, row - 1);
      if (row >= P.M) cmax = -1;
      float* crow = P.C + row;
      if (P.beta != 0.0f) {
#pragma unroll
        for (int c0 = 0; c0 < CW; c0 += 16) {
          float old[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int col = n0 + c0 + i;
            old[i] = (col <= cmax) ? crow[(long)col * P.ldc] : 0.0f;
          }
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int col = n0 + c0 + i;
            if (col <= cmax) crow[(long)col * P.ldc] = fmaf(P.alpha, acc[c0 + i], P.beta * old[i]);
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < CW; ++i) {
          const int col = n0 + i;
          if (col <= cmax) crow[(long)col * P.ldc] = P.alpha * acc[i];
        }
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, TMEM_COLS);
  }
  if (threadIdx.x == 0 && *err && P.status) atomicCAS(P.status, 0, *err);
}

// hi / lo planes of op(X) (rows x K, K contiguous, pitch ldk) from a column-major
// X whose rows of op(X) are contiguous along K (kmaj: element (r, k) at
// X[k + r ld]) or along the rows (element (r, k) at X[r + k ld], transposed
// through shared memory). Columns k >= K of the planes are zero.
__global__ void tc32_split(int rows, int K, int ldk, const float* __restrict__ X, long ld, int kmaj,
                           float* __restrict__ hi, float* __restrict__ lo) {
  __shared__ float t[32][33];
  const int k0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  if (kmaj) {
    for (int y = ty; y < 32; y += 8) {
      const int r = r0 + y, k = k0 + tx;
      if (r < rows && k < ldk) {
        const float x = k < K ? X[k + (long)r * ld] : 0.f;
        const float h = __uint_as_float(rna_tf32(x));
        hi[k + (long)r * ldk] = h;
        lo[k + (long)r * ldk] = x - h;
      }
    }
    return;
  }
  for (int y = ty; y < 32; y += 8) {
    const int r = r0 + tx, k = k0 + y;  // read along the rows (contiguous in X)
    t[y][tx] = (r < rows && k < K) ? X[r + (long)k * ld] : 0.f;
  }
  __syncthreads();
  for (int y = ty; y < 32; y += 8) {
    const int r = r0 + y, k = k0 + tx;  // write along K
    if (r < rows && k < ldk) {
      const float x = t[tx][y];
      const float h = __uint_as_float(rna_tf32(x));
      hi[k + (long)r * ldk] = h;
      lo[k + (long)r * ldk] = x - h;
    }
  }
}

// ---- host side -------------------------------------------------------------

// 0: FP32 GEMMs on the SIMT kernel, 1: 3xTF32 tensor cores splitting in shared
// memory, 2: 3xTF32 on operands pre-split in global memory where that pays,
// 3: pre-split for every product
static std::atomic<int> g_mode{2};

static int sm_count() {
  static int count[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  if (!count[dev]) {
    int c = 0;
    if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c <= 0) c = 148;
    count[dev] = c;
  }
  return count[dev];
}

bool eligible(const GemmArgs& g) {
  if (g.M < 1 || g.N < 1 || g.K < 1 || g.batch > 1 || g.a_tri || g.b_tri) return false;
  if (g.c_uplo && g.M != g.N) return false;
  auto aligned = [](const void* p, long ld) {
    return (reinterpret_cast<uintptr_t>(p) & 15) == 0 && (ld & 3) == 0 && ld > 0 && ld < (1L << 37);
  };
  return aligned(g.A, g.lda) && aligned(g.B, g.ldb) && g.ldc >= g.M;
}

// Pre-split planes, one buffer per (device, stream), grown on demand. Growing
// waits for the stream (earlier products may still read the old buffer); the
// buffers live for the process.
struct SplitBuf {
  int dev;
  cudaStream_t stream;
  float* ptr;
  size_t bytes;
};
static std::mutex g_split_mu;
static SplitBuf g_split[64];
static int g_nsplit = 0;

static int split_buffer(size_t bytes, cudaStream_t s, float** out) {
  int dev = 0;
  BSE_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_split_mu);
  SplitBuf* b = nullptr;
  for (int i = 0; i < g_nsplit; ++i)
    if (g_split[i].dev == dev && g_split[i].stream == s) b = &g_split[i];
  if (!b) {
    if (g_nsplit == 64) {
      record_message("tc32 gemm: more than 64 (device, stream) pairs hold pre-split buffers");
      return BSE_ERR_ARG;
    }
    b = &g_split[g_nsplit++];
    *b = SplitBuf{dev, s, nullptr, 0};
  }
  if (b->bytes < bytes) {
    if (b->ptr) {
      BSE_CUDA(cudaStreamSynchronize(s));
      BSE_CUDA(cudaFree(b->ptr));
      b->ptr = nullptr;
      b->bytes = 0;
    }
    const size_t want = bytes + bytes / 4;
    void* p = nullptr;
    BSE_CUDA(cudaMalloc(&p, want));
    b->ptr = static_cast<float*>(p);
    b->bytes = want;
  }
  *out = b->ptr;
  return BSE_OK;
}

static int gemm_presplit(const GemmArgs& g, Params& P, cudaStream_t s) {
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [] {
    attr_err = cudaFuncSetAttribute(tc32p_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, P_SMEM_BYTES);
  });
  if (attr_err != cudaSuccess) {
    record_error("cudaFuncSetAttribute(tc32p_kernel)", attr_err, __FILE__, __LINE__);
    return BSE_ERR_CUDA;
  }
  const long ldk = (long)ceil_div(g.K, BK) * BK;
  const long ra = (long)P.tiles_m * BM, rb = (long)P.tiles_n * BN;  // rows padded to whole tiles
  const size_t plane_a = (size_t)ra * ldk, plane_b = (size_t)rb * ldk;
  float* buf = nullptr;
  BSE_TRY(split_buffer(2 * (plane_a + plane_b) * sizeof(float), s, &buf));
  float *ah = buf, *al = ah + plane_a, *bh = al + plane_a, *bl = bh + plane_b;
  const dim3 blk(32, 8);
  {
    KprofScope ks(K_TF32_SPLIT, s, 12.0 * ((double)g.M + g.N) * g.K, 0.0);
    kcount(1);  // two launches in this scope
    tc32_split<<<dim3((unsigned)(ldk / BK), (unsigned)ceil_div(g.M, 32)), blk, 0, s>>>(
        g.M, g.K, (int)ldk, reinterpret_cast<const float*>(g.A), g.lda, g.transA ? 1 : 0, ah, al);
    BSE_LAUNCH_CHECK();
    tc32_split<<<dim3((unsigned)(ldk / BK), (unsigned)ceil_div(g.N, 32)), blk, 0, s>>>(
        g.N, g.K, (int)ldk, reinterpret_cast<const float*>(g.B), g.ldb, g.transB ? 0 : 1, bh, bl);
    BSE_LAUNCH_CHECK();
  }
  CUtensorMap mah, mal, mbh, mbl;
  BSE_TRY(make_tensor_map_2d(&mah, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, ah, ldk, g.M, ldk * 4, BK, BM));
  BSE_TRY(make_tensor_map_2d(&mal, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, al, ldk, g.M, ldk * 4, BK, BM));
  BSE_TRY(make_tensor_map_2d(&mbh, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, bh, ldk, g.N, ldk * 4, BK, BN));
  BSE_TRY(make_tensor_map_2d(&mbl, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, bl, ldk, g.N, ldk * 4, BK, BN));
  P.K = (int)ldk;  // the padded columns are zero
  const int grid = P.tiles < sm_count() ? P.tiles : sm_count();
  double fl = 2.0 * g.M * (double)g.N * g.K;
  if (g.c_uplo) fl *= 0.5;
  KprofScope ks(K_GEMM_TF32, s, 0.0, fl);
  tc32p_kernel<<<grid, P_THREADS, P_SMEM_BYTES, s>>>(mah, mal, mbh, mbl, P);
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

// Pre-splitting costs one pass over both operands (read 4 B, write 8 B per
// entry of op(A) and op(B)) and saves the shared-memory splitting of every tile
// (measured at 8192^3: 9.9 ms in-kernel against 5.5 ms on split planes, about
// 8e-15 s per multiply-add). At about 6 TB/s the pass costs 2e-12 s per operand
// entry, so it pays once M N (halved for a triangular C) exceeds about
// 250 (M + N); the bound below is twice that, for split passes that run under
// copy bandwidth. Square products beyond about 1000 qualify, the skinny panel
// products (N <= 128), whose operands are read once anyway, do not.
static bool presplit_pays(const GemmArgs& g) {
  const double mn = (double)g.M * (double)g.N * (g.c_uplo ? 0.5 : 1.0);
  return mn >= 500.0 * ((double)g.M + (double)g.N);
}

int gemm(const GemmArgs& g, int split, int* status, cudaStream_t s) {
  if (!eligible(g)) {
    record_message("tc32 gemm: operand layout not supported (16-byte aligned bases, leading dimensions % 4)");
    return BSE_ERR_ARG;
  }
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [] {
    attr_err = cudaFuncSetAttribute(tc32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  });
  if (attr_err != cudaSuccess) {
    record_error("cudaFuncSetAttribute(tc32_kernel)", attr_err, __FILE__, __LINE__);
    return BSE_ERR_CUDA;
  }
  Params P{};
  P.M = g.M; P.N = g.N; P.K = g.K;
  // op(A) = A (column-major M x K): M contiguous -> MN-major; op(A) = A^T: K contiguous
  P.a_mn = g.transA ? 0 : 1;
  // op(B) = B (column-major K x N): K contiguous -> K-major; op(B) = B^T: N contiguous
  P.b_mn = g.transB ? 1 : 0;
  P.split = split ? 1 : 0;
  P.uplo = g.c_uplo;
  P.tiles_m = ceil_div(g.M, BM);
  P.tiles_n = ceil_div(g.N, BN);
  P.tiles = P.uplo ? P.tiles_m * (P.tiles_m + 1) / 2 : P.tiles_m * P.tiles_n;
  P.alpha = (float)g.alpha;
  P.beta = (float)g.beta;
  P.C = reinterpret_cast<float*>(g.C);
  P.ldc = g.ldc;
  P.status = status ? status : reinterpret_cast<int*>(current_status());
  const int md = g_mode.load(std::memory_order_relaxed);
  if (split && (md == 3 || (md == 2 && presplit_pays(g)))) return gemm_presplit(g, P, s);
  CUtensorMap ma, mb;
  if (P.a_mn)
    BSE_TRY(make_tensor_map_2d(&ma, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, g.A, g.M, g.K, g.lda * 4, 32, BK));
  else
    BSE_TRY(make_tensor_map_2d(&ma, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, g.A, g.K, g.M, g.lda * 4, BK, BM));
  if (P.b_mn)
    BSE_TRY(make_tensor_map_2d(&mb, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, g.B, g.N, g.K, g.ldb * 4, 32, BK));
  else
    BSE_TRY(make_tensor_map_2d(&mb, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, g.B, g.K, g.N, g.ldb * 4, BK, BN));
  const int grid = P.tiles < sm_count() ? P.tiles : sm_count();
  double fl = 2.0 * g.M * (double)g.N * g.K;
  if (g.c_uplo) fl *= 0.5;
  KprofScope ks(K_GEMM_TF32, s, 0.0, fl);
  tc32_kernel<<<grid, THREADS, SMEM_BYTES, s>>>(ma, mb, P);
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

int mode() { return g_mode.load(std::memory_order_relaxed); }

}  // namespace tc32
}  // namespace bse

extern "C" int bse_set_fp32_gemm(int mode) {
  if (mode < 0 || mode > 3) return BSE_ERR_ARG;
  bse::tc32::g_mode.store(mode);
  return BSE_OK;
}

extern "C" int bse_tc32_gemm(int M, int N, int K, float alpha, const float* A, int lda, int transA, const float* B,
                             int ldb, int transB, float beta, float* C, int ldc, int uplo, int split,
                             int* dev_status, void* stream) {
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C || !dev_status || uplo < 0 || uplo > 2) return BSE_ERR_ARG;
  if ((transA ? lda < K : lda < M) || (transB ? ldb < N : ldb < K) || ldc < M) return BSE_ERR_ARG;
  bse::GemmArgs g{};
  g.M = M; g.N = N; g.K = K;
  g.A = A; g.lda = lda; g.B = B; g.ldb = ldb; g.C = C; g.ldc = ldc;
  g.alpha = alpha; g.beta = beta; g.transA = transA != 0; g.transB = transB != 0;
  g.c_uplo = uplo; g.batch = 1;
  if (!bse::tc32::eligible(g)) {
    bse::record_message("bse_tc32_gemm: A and B need 16-byte aligned bases and leading dimensions divisible by 4");
    return BSE_ERR_ARG;
  }
  return bse::tc32::gemm(g, split, dev_status, (cudaStream_t)stream);
}
