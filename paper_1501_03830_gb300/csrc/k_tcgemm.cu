// Tensor-core GEMM for sm_103a: tcgen05.mma (bf16 x bf16 -> FP32 in TMEM) fed
// by TMA, used for the FP64-accurate products of the refinement (error-free
// digit splitting, see k_ozaki.cu) and testable on its own.
//
// One CTA owns a 128 x 256 output tile and runs a list of "units": unit u
// multiplies digit matrix a_digit[u] of A by digit matrix b_digit[u] of B over
// the whole K. The K range is cut into chunks of chunk_kb 64-deep blocks; each
// chunk accumulates afresh in one of two TMEM accumulators (256 FP32 columns
// each) while the threads drain the other into per-thread 32-bit registers.
// For digit products every chunk sum is an integer of magnitude <= 2^22, so the
// drain converts it exactly (adding 1.5 * 2^23 puts the integer in the low
// mantissa bits) and sums in int32: the exact sum over K is not limited by the
// FP32 accumulator's 24 bits, which lets the digits be wider (fewer of them).
// Consecutive units flagged as one group (digit pairs on one anti-diagonal
// p + q = d, which share a scale) share the integer sum, written once per group
// as an int32 plane; the FP64 scaling and summation of the planes is a separate
// elementwise pass (k_ozaki.cu). Both operands are K-major bf16 (A: rows x K,
// B: cols x K, K contiguous), staged by TMA with 128-byte swizzle into a
// 4-stage shared-memory ring guarded by mbarriers.
//
// Every probe and wait is bounded: a CTA that sees no progress for kIdleMax
// probes records BSE_ERR_TIMEOUT, stops issuing work, drains what it issued
// (bounded again), frees its TMEM and returns.
#include <cuda.h>
#include <stdint.h>

#include <mutex>

#include "common.cuh"
#include "ptx_sm100.cuh"
#include "tcgemm.cuh"

namespace bse {
namespace tc {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;  // 16 KiB
constexpr int B_BYTES = BN * BK * 2;  // 32 KiB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
// 8 warps, all of which drain TMEM (lane quadrant = warp % 4, column half =
// warp / 4); lane 0 of warp 0 also issues the TMA loads and lane 0 of warp 1
// the MMAs, both by non-blocking mbarrier probes between drains. Eight warps
// leave each thread up to 255 registers, which the 128 integer sums need.
constexpr int THREADS = 256;
constexpr int HALF_N = BN / 2;  // columns per thread
constexpr long kIdleMax = 1L << 26;  // probes without progress before a CTA gives up
constexpr uint32_t TMEM_COLS = 512;  // two 128 x 256 FP32 accumulators

using namespace ptx;

// K-major operand, rows of 64 bf16 = 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) { return make_desc_sw128(saddr, 16, 1024); }

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, N = 256, M = 128.
__host__ __device__ constexpr uint32_t make_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
// One CTA per 128 x 256 output tile, tiles walked in a grouped order (a band
// of kGroupM tile rows column by column) so the operand tiles that co-resident
// CTAs read stay in L2.
__global__ void __launch_bounds__(THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ TcParams P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;  // [2]
  uint64_t* tempty = tfull + 2;      // [2]
  uint64_t* drain = tempty + 2;      // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* err = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int kGroupM = 16;
  const int tiles_m = (P.M + BM - 1) / BM;
  const int tiles_n = (P.N + BN - 1) / BN;
  const int group = blockIdx.x / (kGroupM * tiles_n);
  const int first_m = group * kGroupM;
  const int gm = min(kGroupM, tiles_m - first_m);
  const int in_group = blockIdx.x - group * kGroupM * tiles_n;
  const int m0 = (first_m + in_group % gm) * BM;
  const int n0 = (in_group / gm) * BN;
  const int KB = (P.K + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], THREADS);
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

  const bool producer = warp == 0 && lane == 0;
  const bool issuer = warp == 1 && lane == 0;
  // producer state: next K block to load
  int p_it = 0, p_u = 0, p_kb = 0;
  uint32_t issued = 0, last_par = 0;  // per stage: a load was issued / its phase parity
  // MMA state: next K block to multiply, chunk, whether its TMEM buffer is held
  int m_it = 0, m_u = 0, m_kb = 0, m_ch = 0;
  bool m_have = false;
  const uint32_t idesc = make_idesc();
  // drain state
  const int q4 = warp & 3;
  const int cb = (warp >> 2) * HALF_N;
  const int row = m0 + q4 * 32 + lane;
  int d_u = 0, d_ch = 0, d_kb0 = 0, nfold = 0;
  int acc[HALF_N];  // integer sums (mode 1) or FP32 bit patterns (mode 0)
#pragma unroll
  for (int j = 0; j < HALF_N; ++j) acc[j] = 0;
  long idle = 0;

  while (d_u < P.units) {
    bool progress = false;
    if (producer) {
      while (p_u < P.units) {
        const int st = p_it % STAGES;
        const uint32_t ph = (p_it / STAGES) & 1;
        if (!mbar_test(&empty[st], ph ^ 1)) break;
        const int ya = P.a_digit[p_u] * P.a_rows + m0;
        const int yb = P.b_digit[p_u] * P.b_rows + n0;
        uint8_t* sa = smem + st * STAGE_BYTES;
        mbar_expect_tx(&full[st], STAGE_BYTES);
        tma_load_2d(sa, &tmA, p_kb * BK, ya, &full[st]);
        tma_load_2d(sa + A_BYTES, &tmB, p_kb * BK, yb, &full[st]);
        issued |= 1u << st;
        last_par = (last_par & ~(1u << st)) | (ph << st);
        ++p_it;
        if (++p_kb == KB) {
          p_kb = 0;
          ++p_u;
        }
        progress = true;
      }
    }
    if (issuer) {
      // one TMEM accumulator per chunk of chunk_kb K blocks
      while (m_u < P.units) {
        const int buf = m_ch & 1;
        if (!m_have) {
          if (!mbar_test(&tempty[buf], ((m_ch >> 1) & 1) ^ 1)) break;
          tc_fence_after();
          m_have = true;
        }
        const int st = m_it % STAGES;
        if (!mbar_test(&full[st], (m_it / STAGES) & 1)) break;
        tc_fence_after();
        const uint32_t sa = smem_u32(smem + st * STAGE_BYTES);
        const uint64_t da = make_desc(sa), db = make_desc(sa + A_BYTES);
        const uint32_t d = tmem_base + (uint32_t)(buf * BN);
        const int kc = m_kb % P.chunk_kb;
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk)
          umma_bf16(d, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc, (kc | kk) != 0);
        umma_commit(&empty[st]);
        ++m_it;
        ++m_kb;
        if (kc == P.chunk_kb - 1 || m_kb == KB) {
          umma_commit(&tfull[buf]);
          ++m_ch;
          m_have = false;
        }
        if (m_kb == KB) {
          m_kb = 0;
          ++m_u;
        }
        progress = true;
      }
    }
    __syncwarp();
    // drain the next chunk into the per-thread sums (warp-collective TMEM loads)
    const int buf = d_ch & 1;
    // every lane probes (each must observe the phase); the phase cannot move on
    // before this warp has drained it, so a late probe sees the same answer
    const bool ready = __all_sync(0xffffffffu, mbar_test(&tfull[buf], (d_ch >> 1) & 1));
    if (ready) {
      tc_fence_after();
      const uint32_t tb = tmem_base + (uint32_t)(buf * BN + cb) + ((uint32_t)(q4 * 32) << 16);
      if (P.mode == 1) {
#pragma unroll
        for (int c0 = 0; c0 < HALF_N; c0 += 32) {
          uint32_t r[32];
          tmem_ld32(tb + (uint32_t)c0, r);
          // exact: |chunk sum| <= 2^22, so adding 1.5 * 2^23 leaves it in the low mantissa bits
#pragma unroll
          for (int i = 0; i < 32; ++i)
            acc[c0 + i] += (int)(__float_as_uint(__uint_as_float(r[i]) + 12582912.0f) - 0x4B400000u);
        }
      } else {
#pragma unroll
        for (int c0 = 0; c0 < HALF_N; c0 += 32) {
          uint32_t r[32];
          tmem_ld32(tb + (uint32_t)c0, r);
#pragma unroll
          for (int i = 0; i < 32; ++i) acc[c0 + i] = __float_as_int(__int_as_float(acc[c0 + i]) + __uint_as_float(r[i]));
        }
      }
      tc_fence_before();
      mbar_arrive(&tempty[buf]);
      ++d_ch;
      d_kb0 += P.chunk_kb;
      if (d_kb0 >= KB) {
        d_kb0 = 0;
        if (P.fold[d_u]) {
          // end of a group of units: write the sums (FP32 C, or int32 plane nfold)
          const int ncols = min(HALF_N, P.N - (n0 + cb));
          if (row < P.M) {
            if (P.mode == 0) {
              float* cp = P.Cf + row + (long)(n0 + cb) * P.ldc;
#pragma unroll
              for (int j = 0; j < HALF_N; ++j)
                if (j < ncols) cp[(long)j * P.ldc] = __int_as_float(acc[j]);
            } else {
              int* cp = P.Si + (long)nfold * P.plane + row + (long)(n0 + cb) * P.ldc;
#pragma unroll
              for (int j = 0; j < HALF_N; ++j)
                if (j < ncols) cp[(long)j * P.ldc] = acc[j];
            }
          }
#pragma unroll
          for (int j = 0; j < HALF_N; ++j) acc[j] = 0;
          ++nfold;
        }
        ++d_u;
      }
      progress = true;
    }
    // bounded: a CTA that sees no progress for kIdleMax probes (or an error
    // recorded by another warp) stops
    if (__any_sync(0xffffffffu, progress)) {
      idle = 0;
    } else if (++idle > kIdleMax) {
      *err = BSE_ERR_TIMEOUT;
    }
    if (*err) break;
  }
  if (producer) {
    // the CTA may leave early after an error: first let every issued copy land
    for (int st = 0; st < STAGES; ++st)
      if (issued & (1u << st)) mbar_drain(&full[st], (last_par >> st) & 1);
  }
  if (issuer) {
    // all issued MMAs complete before TMEM can be released
    umma_commit(drain);
    mbar_drain(drain, 0);
  }
  __syncwarp();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, TMEM_COLS);
  }
  if (threadIdx.x == 0 && *err && P.status) atomicCAS(P.status, 0, *err);
}

// ---- host side -------------------------------------------------------------

}  // namespace tc

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

int make_tensor_map_2d(CUtensorMap* map, CUtensorMapDataType dt, const void* base, long inner, long outer,
                       long pitch_bytes, int box_inner, int box_outer) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    record_message("cuTensorMapEncodeTiled is not available");
    return BSE_ERR_CUDA;
  }
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  cuuint64_t strides[1] = {(cuuint64_t)pitch_bytes};
  cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    record_message("cuTensorMapEncodeTiled failed");
    return BSE_ERR_CUDA;
  }
  return BSE_OK;
}

namespace tc {

// rows x K bf16, K contiguous with row pitch ldk (elements); box BK x box_rows.
static int make_map(CUtensorMap* map, const void* base, long rows, long K, long ldk, int box_rows) {
  return make_tensor_map_2d(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, base, K, rows, ldk * 2, BK, box_rows);
}

int tc_gemm(const TcProblem& pb, cudaStream_t s) {
  if (pb.M <= 0 || pb.N <= 0 || pb.K <= 0 || pb.units <= 0) return BSE_OK;
  if (pb.units > kMaxUnits || pb.chunk_kb < 1 || !pb.fold[pb.units - 1] || (pb.ldk % 8) != 0 ||
      (reinterpret_cast<uintptr_t>(pb.A) % 16) != 0 ||
      (reinterpret_cast<uintptr_t>(pb.B) % 16) != 0) {
    record_message("tc_gemm: bad layout (K pitch a multiple of 8, bases 16-byte aligned, chunk >= 1, last unit folds)");
    return BSE_ERR_ARG;
  }
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [] {
    attr_err = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  });
  if (attr_err != cudaSuccess) {
    record_error("cudaFuncSetAttribute(tc_gemm_kernel)", attr_err, __FILE__, __LINE__);
    return BSE_ERR_CUDA;
  }
  CUtensorMap ma, mb;
  BSE_TRY(make_map(&ma, pb.A, (long)pb.a_rows * pb.a_digits, pb.K, pb.ldk, BM));
  BSE_TRY(make_map(&mb, pb.B, (long)pb.b_rows * pb.b_digits, pb.K, pb.ldk, BN));
  TcParams P{};
  P.M = pb.M; P.N = pb.N; P.K = pb.K;
  P.a_rows = pb.a_rows; P.b_rows = pb.b_rows;
  P.units = pb.units;
  P.chunk_kb = pb.chunk_kb;
  for (int u = 0; u < pb.units; ++u) {
    P.a_digit[u] = pb.a_digit[u];
    P.b_digit[u] = pb.b_digit[u];
    P.fold[u] = pb.fold[u];
  }
  P.mode = pb.mode; P.Cf = pb.Cf; P.Si = pb.Si; P.plane = pb.plane; P.ldc = pb.ldc;
  P.status = pb.status;
  const long tiles = (long)((pb.M + BM - 1) / BM) * ((pb.N + BN - 1) / BN);
  KprofScope ks(K_GEMM_TC, s, 0.0, 2.0 * pb.M * (double)pb.N * pb.K * pb.units);
  tc_gemm_kernel<<<(unsigned)tiles, THREADS, SMEM_BYTES, s>>>(ma, mb, P);
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

}  // namespace tc
}  // namespace bse

// C (M x N, FP32, column-major, ldc) = A (M x K bf16, K-major with pitch ldk) *
// B (N x K bf16, K-major with pitch ldk)^T on the tensor cores.
extern "C" int bse_tc_gemm_bf16(int M, int N, int K, const void* A, const void* B, int ldk, float* C, int ldc,
                                int* dev_status, void* stream) {
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C || ldk < K || ldc < M || !dev_status) return BSE_ERR_ARG;
  bse::tc::TcProblem pb{};
  pb.M = M; pb.N = N; pb.K = K; pb.ldk = ldk;
  pb.A = A; pb.B = B; pb.a_rows = M; pb.b_rows = N; pb.a_digits = 1; pb.b_digits = 1;
  pb.units = 1; pb.a_digit[0] = 0; pb.b_digit[0] = 0; pb.fold[0] = 1;
  pb.chunk_kb = 4;  // FP32 sums of 256-deep chunks: no long in-TMEM accumulation
  pb.mode = 0; pb.Cf = C; pb.ldc = ldc; pb.status = dev_status;
  return bse::tc::tc_gemm(pb, (cudaStream_t)stream);
}

