// BF16 tensor-core GEMMs for the MLP of the learned reaction step (Sec. 2.2: hidden layers of
// 1600, 800 and 400 GELU units; the paper runs it in half precision through libTorch,
// Sec. 2.1).  Here every layer is a hand-written tcgen05 GEMM fed by TMA with the layer's
// elementwise work fused into the TMEM epilogue.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "gemm_tc.cuh"
#include "internal.h"

namespace chem {

using bf16 = __nv_bfloat16;

// ------------------------------------------------------------------------------------------
// GELU (erf form, Hendrycks & Gimpel 2016) and its derivative.  erf by the rational
// approximation of Abramowitz & Stegun, Handbook of Mathematical Functions, eq. 7.1.26
// (Hastings): erf z = 1 - t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) e^{-z^2}, t = 1 / (1 + p z),
// z >= 0, |error| <= 1.5e-7 (6e-7 in FP32 arithmetic); GELU within 2.1e-7 max(1, |x|), far below
// the BF16 rounding of the outputs.  Arranged for few instructions: with a = |x| and z = a/sqrt2,
// w = (1 - erf z)/2 = t q(t) e^{-x^2/2} with the a_i halved and p/sqrt2 folded into t, and then
// Phi(x) = x >= 0 ? 1 - w : w, GELU x = x Phi(x), GELU' x = Phi(x) + x e^{-x^2/2} / sqrt(2 pi).
// One reciprocal and one base-2 exponential on the special-function unit.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// w = (1 - erf(|x| / sqrt2)) / 2 and e = e^{-x^2/2}
__device__ __forceinline__ float half_erfc_as(float x, float& e) {
  const float t = rcp_approx(fmaf(0.3275911f * 0.70710678118654752f, fabsf(x), 1.0f));
  float q = fmaf(t, 0.5f * 1.061405429f, 0.5f * -1.453152027f);
  q = fmaf(q, t, 0.5f * 1.421413741f);
  q = fmaf(q, t, 0.5f * -0.284496736f);
  q = fmaf(q, t, 0.5f * 0.254829592f);
  e = ex2_approx((x * -0.72134752044448170f) * x);   // -log2(e) / 2
  return (q * t) * e;
}
__device__ __forceinline__ float gelu_f(float x) {
  float e;
  const float w = half_erfc_as(x, e);
  const float r = x * w;
  return x >= 0.0f ? x - r : r;
}
__device__ __forceinline__ float dgelu_f(float x) {
  float e;
  const float w = half_erfc_as(x, e);
  return fmaf(x * 0.39894228040143268f, e, x >= 0.0f ? 1.0f - w : w);
}

// ------------------------------------------------------------------------------------------
// GEMM kernel
// ------------------------------------------------------------------------------------------
#ifndef CHEM_GEMM_STAGES_256
#define CHEM_GEMM_STAGES_256 2   // 2 stages of 48 KB: two CTAs per SM, one's epilogue overlaps the other's MMAs
#endif
#ifndef CHEM_GEMM_STAGES
#define CHEM_GEMM_STAGES 3
#endif

// staging buffer of one epilogue warp (32 rows x 32 BF16 columns), see store_rows_bf16
constexpr int kEpiWarpBytes = 32 * 64;

template <int BN>
struct TileCfg {
  static constexpr int STAGES = BN >= 224 ? CHEM_GEMM_STAGES_256 : CHEM_GEMM_STAGES;
  static constexpr uint32_t TMEM_COLS = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
  static constexpr size_t A_BYTES = (size_t)tc::BM * tc::BK * 2;
  static constexpr size_t B_BYTES = (size_t)BN * tc::BK * 2;
  static constexpr size_t SMEM = 1024 + STAGES * (A_BYTES + B_BYTES) + (2 * STAGES + 2) * 8 + 16 + 128 +
                                 8 * kEpiWarpBytes;
};

// Per-warp staging of a 32 x 32 BF16 block between the row-per-lane layout of the TMEM
// epilogue and row segments: a warp's store (load) then moves 8 whole 64-byte row segments
// (full 32-byte sectors) instead of 32 scattered 16-byte pieces.  Slot of (row r, 16-byte chunk
// c) in the 2 KB buffer: r * 64 + 16 ((c + (r >> 1)) & 3), free of bank conflicts both for one
// row per lane and for four lanes per row.
__device__ __forceinline__ uint32_t stage_slot(int r, int c) { return (uint32_t)(r * 64 + 16 * ((c + (r >> 1)) & 3)); }

// rows 0 .. nrows - 1 of `dst` (row stride ld elements, 32 columns) from the staging buffer,
// which holds this lane's row (lane = row) at stage_slot(lane, 0..3)
__device__ __forceinline__ void flush_rows_bf16(const uint8_t* wbuf, bf16* dst, int64_t ld, int nrows, int lane) {
  __syncwarp();
  const int c = lane & 3;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = (lane >> 2) + 8 * i;
    if (r < nrows) *(uint4*)(dst + (size_t)r * ld + 8 * c) = *(const uint4*)(wbuf + stage_slot(r, c));
  }
  __syncwarp();
}

// the reverse: this lane's row (lane = row - row0) of src into pk; rows past nrows read zero
__device__ __forceinline__ void load_rows_bf16(uint4 (&pk)[4], uint8_t* wbuf, const bf16* src, int64_t ld,
                                               int nrows, int lane) {
  const int c = lane & 3;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = (lane >> 2) + 8 * i;
    const uint4 v = r < nrows ? __ldg((const uint4*)(src + (size_t)r * ld + 8 * c)) : make_uint4(0u, 0u, 0u, 0u);
    *(uint4*)(wbuf + stage_slot(r, c)) = v;
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < 4; ++q) pk[q] = *(const uint4*)(wbuf + stage_slot(lane, q));
  __syncwarp();
}

// epilogue of one 32-column chunk of the accumulator rows of a warp: this lane's row is
// row = row0 + lane, columns col0 .. col0 + nv - 1; rows row0 .. row0 + nrows - 1 exist.
// Called by the whole warp (the staged BF16 paths synchronise it).
template <int EPI>
__device__ __forceinline__ void epi_chunk(float (&v)[32], int row, int col0, int nv, const GemmEpi& e,
                                          uint8_t* wbuf, int row0, int nrows, int lane) {
  if ((EPI == 0 || EPI == 2) && nv == 32) {
    if (EPI == 0) {
      // hidden layer forward: out = bf16(GELU(acc + b)); optional pre-activation copy.  Each
      // group of 8 columns goes to the staging buffer as soon as it is made (few live registers)
      if (e.bias) {
        // the chunk's 32 biases as eight 16-byte broadcast loads (col0 is a multiple of 32)
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 b4 = __ldg((const float4*)(e.bias + col0) + q);
          v[4 * q] += b4.x;
          v[4 * q + 1] += b4.y;
          v[4 * q + 2] += b4.z;
          v[4 * q + 3] += b4.w;
        }
      }
      if (e.zout) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          __align__(16) bf16 u[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) u[i] = __float2bfloat16_rn(v[8 * q + i]);
          *(uint4*)(wbuf + stage_slot(lane, q)) = *(const uint4*)u;
        }
        flush_rows_bf16(wbuf, e.zout + (size_t)row0 * e.ldo + col0, e.ldo, nrows, lane);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        __align__(16) bf16 t[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) t[i] = __float2bfloat16_rn(gelu_f(v[8 * q + i]));
        *(uint4*)(wbuf + stage_slot(lane, q)) = *(const uint4*)t;
      }
      flush_rows_bf16(wbuf, (bf16*)e.out + (size_t)row0 * e.ldo + col0, e.ldo, nrows, lane);
    } else {
      // hidden-layer backward: dZ = acc * GELU'(z)
      uint4 zk[4];
      load_rows_bf16(zk, wbuf, e.z + (size_t)row0 * e.ldz + col0, e.ldz, nrows, lane);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const bf16* zin = (const bf16*)&zk[q];
        __align__(16) bf16 t[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) t[i] = __float2bfloat16_rn(v[8 * q + i] * dgelu_f(__bfloat162float(zin[i])));
        *(uint4*)(wbuf + stage_slot(lane, q)) = *(const uint4*)t;
      }
      flush_rows_bf16(wbuf, (bf16*)e.out + (size_t)row0 * e.ldo + col0, e.ldo, nrows, lane);
    }
    return;
  }
  if (row - row0 >= nrows) return;
  // every loop below is unrolled over the 32 columns with the ragged bound as a predicate: an
  // index that depends on nv would put the accumulator chunk into local memory
  if (EPI == 0 || EPI == 1) {   // + bias
    if (e.bias) {
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] += (i < nv) ? __ldg(e.bias + col0 + i) : 0.0f;
    }
  }
  if (EPI == 0) {
    // hidden layer forward: out = bf16(GELU(acc + b)); optional pre-activation copy
    bf16* o = (bf16*)e.out + (size_t)row * e.ldo + col0;
    bf16* zo = e.zout ? e.zout + (size_t)row * e.ldo + col0 : nullptr;
    if (nv == 32) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        __align__(16) bf16 t[8], u[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          t[i] = __float2bfloat16_rn(gelu_f(v[8 * q + i]));
          u[i] = __float2bfloat16_rn(v[8 * q + i]);
        }
        *(uint4*)(o + 8 * q) = *(const uint4*)t;
        if (zo) *(uint4*)(zo + 8 * q) = *(const uint4*)u;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        if (i < nv) {
          o[i] = __float2bfloat16_rn(gelu_f(v[i]));
          if (zo) zo[i] = __float2bfloat16_rn(v[i]);
        }
      }
    }
  } else if (EPI == 1 || EPI == 3) {
    // output layer (acc + b) or weight gradient (acc), FP32
    float* o = (float*)e.out + (size_t)row * e.ldo + col0;
    if (nv == 32) {
#pragma unroll
      for (int q = 0; q < 8; ++q) *(float4*)(o + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i)
        if (i < nv) o[i] = v[i];
    }
  } else if (EPI == 2) {
    // hidden-layer backward: dZ = acc * GELU'(z)
    const bf16* zz = e.z + (size_t)row * e.ldz + col0;
    bf16* o = (bf16*)e.out + (size_t)row * e.ldo + col0;
#pragma unroll
    for (int i = 0; i < 32; ++i)
      if (i < nv) o[i] = __float2bfloat16_rn(v[i] * dgelu_f(__bfloat162float(zz[i])));
  }
}

// Epilogue 4 (short-K kernel only): the hidden-layer forward of epilogue 0 without the
// pre-activation copy, N a multiple of 32.  Each 32-column chunk is read from TMEM in four
// 8-column pieces: with a whole 32-float chunk plus the GELU temporaries live, the short-K
// kernel's 64 registers per thread spill.
__device__ __forceinline__ void epi_gelu_x8(uint32_t taddr, int col0, const GemmEpi& e, uint8_t* wbuf,
                                            int row0, int nrows, int lane) {
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    float v[8];
    tc::tmem_ld8(taddr + 8 * h, v);
    if (e.bias) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const float4 b4 = __ldg((const float4*)(e.bias + col0 + 8 * h) + q);
        v[4 * q] += b4.x;
        v[4 * q + 1] += b4.y;
        v[4 * q + 2] += b4.z;
        v[4 * q + 3] += b4.w;
      }
    }
    __align__(16) bf16 t[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) t[i] = __float2bfloat16_rn(gelu_f(v[i]));
    *(uint4*)(wbuf + stage_slot(lane, h)) = *(const uint4*)t;
  }
  flush_rows_bf16(wbuf, (bf16*)e.out + (size_t)row0 * e.ldo + col0, e.ldo, nrows, lane);
}

// S (1..STAGES, a launch argument) stages in the ring: min(STAGES, K slabs), so that a
// short K takes less shared memory and more CTAs share an SM
template <int BN, int EPI>
__global__ void __launch_bounds__(256, 4) gemm_bf16_kernel(const __grid_constant__ CUtensorMap ta,
                                                           const __grid_constant__ CUtensorMap tb,
                                                           GemmEpi e, int M, int N, int K, int S, int* err) {
  using C = TileCfg<BN>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = sA + S * C::A_BYTES;
  uint64_t* full = (uint64_t*)(sB + S * C::B_BYTES);
  uint64_t* empty = full + S;
  uint64_t* done = empty + S;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  uint8_t* stage = (uint8_t*)(((uintptr_t)(tmem_slot + 4) + 127) & ~(uintptr_t)127);   // 8 warps x 2 KB

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // N tiles fastest: the CTAs of one row block run together and share its A rows in L2
  const int m0 = blockIdx.y * tc::BM, n0 = blockIdx.x * BN;
  const int nkb = (K + tc::BK - 1) / tc::BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(done, 1);
    tc::fence_barrier_init();
  }
  if (warp == 2) tc::tmem_alloc(tmem_slot, C::TMEM_COLS);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (threadIdx.x == 0) {
    // TMA producer
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % S;
      if (kb >= S && !tc::mbar_wait(&empty[s], ((kb / S) & 1) ^ 1, err, 1)) break;
      tc::mbar_expect_tx(&full[s], (uint32_t)(C::A_BYTES + C::B_BYTES));
      tc::tma_load_2d(sA + s * C::A_BYTES, &ta, &full[s], kb * tc::BK, m0);
      tc::tma_load_2d(sB + s * C::B_BYTES, &tb, &full[s], kb * tc::BK, n0);
    }
  } else if (threadIdx.x == 32) {
    // single-thread MMA issue
    constexpr uint32_t idesc = tc::idesc_bf16_f32<tc::BM, BN>();
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % S;
      if (!tc::mbar_wait(&full[s], (kb / S) & 1, err, 2)) break;
      tc::tc_fence_after();
      const uint64_t da = tc::sw128_desc(sA + s * C::A_BYTES);
      const uint64_t db = tc::sw128_desc(sB + s * C::B_BYTES);
#pragma unroll
      for (int k = 0; k < tc::BK / tc::UMMA_K; ++k)
        tc::mma_bf16(tmem, da + (uint64_t)((k * tc::UMMA_K * 2) >> 4), db + (uint64_t)((k * tc::UMMA_K * 2) >> 4),
                     idesc, (kb > 0 || k > 0) ? 1u : 0u);
      tc::mma_commit(&empty[s]);
    }
    tc::mma_commit(done);
  }
  __syncwarp();
  const bool ok = tc::mbar_wait(done, 0, err, 3);
  tc::tc_fence_after();
  if (ok) {
    // 8 epilogue warps: warp w reads TMEM lanes 32 (w % 4) .. +31 (the rows it may access) and
    // every second 32-column chunk starting at chunk w / 4
    const int quarter = warp & 3;
    const int row0 = m0 + quarter * 32, row = row0 + lane;
    const int nrows = max(0, min(32, M - row0));
    uint8_t* wbuf = stage + warp * kEpiWarpBytes;
#pragma unroll 1
    for (int c0 = (warp >> 2) * 32; c0 < BN; c0 += 64) {
      if (n0 + c0 >= N) break;
      const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0;
      // the whole warp takes part (no early exit): the next tcgen05.ld and the staged stores
      // need every lane
      if constexpr (EPI == 4) {
        epi_gelu_x8(taddr, n0 + c0, e, wbuf, row0, nrows, lane);
      } else {
        float v[32];
        tc::tmem_ld32(taddr, v);
        epi_chunk<EPI>(v, row, n0 + c0, min(32, N - (n0 + c0)), e, wbuf, row0, nrows, lane);
      }
      __syncwarp();
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 2) tc::tmem_dealloc(tmem, C::TMEM_COLS);
}

// ------------------------------------------------------------------------------------------
// Persistent variant for long K: one CTA per SM walks a static tile schedule (N tiles fastest,
// so the CTAs working at one time share the A row block in L2).  Warp 0 (one thread) streams
// A/B slabs through an S-stage ring, warp 1 (one thread) issues the MMAs into one of two TMEM
// accumulators, warps 2-9 run the epilogue of the previous tile from the other accumulator, so
// the tensor core does not wait for the epilogue.  Barriers: full/empty per stage (TMA ->
// MMA -> TMA), acc_full/acc_empty per accumulator (MMA -> epilogue -> MMA).  All waits are
// bounded; after a timeout every role stops at its next wait.
// ------------------------------------------------------------------------------------------
template <int BN>
struct PersistCfg {
  static constexpr size_t A_BYTES = (size_t)tc::BM * tc::BK * 2;
  static constexpr size_t B_BYTES = (size_t)BN * tc::BK * 2;
  // as many stages as fit in 204 KB (at most 8; the ring must cover the L2 latency), leaving
  // 16 KB for the epilogue warps' staging buffers
  static constexpr int STAGES = (int)((204 * 1024) / (A_BYTES + B_BYTES)) < 8
                                    ? (int)((204 * 1024) / (A_BYTES + B_BYTES)) : 8;
  static constexpr uint32_t ACC_COLS = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
  static constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;
  static constexpr size_t SMEM = 1024 + STAGES * (A_BYTES + B_BYTES) + (2 * STAGES + 4) * 8 + 16 + 128 +
                                 8 * kEpiWarpBytes;
};

__device__ __forceinline__ bool gemm_failed(const int* err) { return *(const volatile int*)err != 0; }

template <int BN, int EPI>
__global__ void __launch_bounds__(320, 1) gemm_bf16_persistent(const __grid_constant__ CUtensorMap ta,
                                                                 const __grid_constant__ CUtensorMap tb,
                                                                 GemmEpi e, int M, int N, int K, int S, int* err) {
  using C = PersistCfg<BN>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = sA + S * C::A_BYTES;
  uint64_t* full = (uint64_t*)(sB + S * C::B_BYTES);
  uint64_t* empty = full + S;
  uint64_t* accf = empty + S;    // [2]
  uint64_t* acce = accf + 2;     // [2]
  uint32_t* tmem_slot = (uint32_t*)(acce + 2);
  uint8_t* stage = (uint8_t*)(((uintptr_t)(tmem_slot + 4) + 127) & ~(uintptr_t)127);   // 8 warps x 2 KB

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkb = (K + tc::BK - 1) / tc::BK;
  const int n_tiles = (N + BN - 1) / BN;
  // tile t: group t / per_group, then row block, then N tile (fastest)
  const int per_group = n_tiles * ((M + tc::BM - 1) / tc::BM);
  const int total = per_group * (e.groups > 1 ? e.groups : 1);

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&accf[b], 1);
      tc::mbar_init(&acce[b], 8);    // one arrival per epilogue warp
    }
    tc::fence_barrier_init();
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, C::TMEM_COLS);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // TMA producer over every K slab of every tile of this CTA
      int g = 0;
      for (int t = blockIdx.x; t < total && !gemm_failed(err); t += gridDim.x) {
        const int gr = t / per_group, r = t - gr * per_group;
        const int m0 = (r / n_tiles) * tc::BM, n0 = (r % n_tiles) * BN;
        const int ax = gr * e.a_col, ay = gr * e.a_row + m0, bx = gr * e.b_col, by = gr * e.b_row + n0;
        bool stop = false;
        for (int kb = 0; kb < nkb; ++kb, ++g) {
          const int s = g % S;
          if (g >= S && !tc::mbar_wait(&empty[s], ((g / S) & 1) ^ 1, err, 11)) { stop = true; break; }
          tc::mbar_expect_tx(&full[s], (uint32_t)(C::A_BYTES + C::B_BYTES));
          tc::tma_load_2d(sA + s * C::A_BYTES, &ta, &full[s], ax + kb * tc::BK, ay);
          tc::tma_load_2d(sB + s * C::B_BYTES, &tb, &full[s], bx + kb * tc::BK, by);
        }
        if (stop) break;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // single-thread MMA issue into the two accumulators in turn
      constexpr uint32_t idesc = tc::idesc_bf16_f32<tc::BM, BN>();
      int g = 0, it = 0;
      for (int t = blockIdx.x; t < total && !gemm_failed(err); t += gridDim.x, ++it) {
        const int b = it & 1, u = it >> 1;
        // accumulator b was last used by tile it - 2: wait for its epilogue
        if (u > 0 && !tc::mbar_wait(&acce[b], (u & 1) ^ 1, err, 12)) break;
        tc::tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)b * C::ACC_COLS;
        bool stop = false;
        for (int kb = 0; kb < nkb; ++kb, ++g) {
          const int s = g % S;
          if (!tc::mbar_wait(&full[s], (g / S) & 1, err, 13)) { stop = true; break; }
          tc::tc_fence_after();
          const uint64_t da = tc::sw128_desc(sA + s * C::A_BYTES);
          const uint64_t db = tc::sw128_desc(sB + s * C::B_BYTES);
#pragma unroll
          for (int k = 0; k < tc::BK / tc::UMMA_K; ++k)
            tc::mma_bf16(acc, da + (uint64_t)((k * tc::UMMA_K * 2) >> 4), db + (uint64_t)((k * tc::UMMA_K * 2) >> 4),
                         idesc, (kb > 0 || k > 0) ? 1u : 0u);
          tc::mma_commit(&empty[s]);
        }
        if (stop) break;
        tc::mma_commit(&accf[b]);
      }
    }
  } else {
    // epilogue warps 2..9: warp w reads TMEM lanes 32 (w % 4) .. +31 and every second
    // 32-column chunk starting at chunk (w - 2) / 4
    const int quarter = warp & 3, half = (warp - 2) >> 2;
    int it = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x, ++it) {
      const int b = it & 1, u = it >> 1;
      if (gemm_failed(err) || !tc::mbar_wait(&accf[b], u & 1, err, 14)) break;
      tc::tc_fence_after();
      const int gr = t / per_group, r = t - gr * per_group;
      const int m0 = (r / n_tiles) * tc::BM, n0 = (r % n_tiles) * BN;
      const int row0 = m0 + quarter * 32, row = row0 + lane;
      const int nrows = max(0, min(32, M - row0));
      uint8_t* wbuf = stage + (warp - 2) * kEpiWarpBytes;
      GemmEpi eg = e;
      if (gr) {
        constexpr size_t osz = (EPI == 0 || EPI == 2) ? 2 : 4;
        eg.out = (char*)e.out + (size_t)gr * (size_t)e.out_goff * osz;
        if (e.zout) eg.zout = e.zout + (size_t)gr * (size_t)e.out_goff;
        if (e.z) eg.z = e.z + (size_t)gr * (size_t)e.z_goff;
        if (e.bias) eg.bias = e.bias + (size_t)gr * (size_t)e.bias_goff;
      }
      const uint32_t acc = tmem + (uint32_t)b * C::ACC_COLS + ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
      for (int c0 = half * 32; c0 < BN; c0 += 64) {
        if (n0 + c0 >= N) break;
        float v[32];
        tc::tmem_ld32(acc + (uint32_t)c0, v);
        // the whole warp takes part (no early exit): the next tcgen05.ld and the staged
        // stores need every lane
        epi_chunk<EPI>(v, row, n0 + c0, min(32, N - (n0 + c0)), eg, wbuf, row0, nrows, lane);
        __syncwarp();
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&acce[b])) : "memory");
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tmem, C::TMEM_COLS);
}

// ------------------------------------------------------------------------------------------
// CTA-pair persistent GEMM: tiles of 256 x BN on two SMs (tcgen05.mma.cta_group::2).  Each CTA
// of the pair stages its own 128 rows of A and its own BN/2 rows of B per K slab, so one
// M = 256 MMA moves 28 % fewer operand bytes through each SM's shared memory per FLOP than the
// single-CTA 128 x BN tile.  Roles as in gemm_bf16_persistent, with:
//   * both producers count their TMA bytes on the even CTA's "full" barrier (two arrivals);
//   * the even CTA's thread 32 issues every MMA and commits to the "empty" and "accumulator
//     full" barriers of both CTAs at once (multicast commit);
//   * both CTAs' epilogue warps arrive on the even CTA's "accumulator empty" barrier
//     (16 arrivals) and each reads its own TMEM (accumulator rows 0-127 or 128-255).
// Every wait is bounded; both CTAs meet at a cluster barrier before TMEM is freed, so neither
// leaves while the other's MMAs may still read its shared memory.
// ------------------------------------------------------------------------------------------
template <int BN>
struct PairCfg {
  // KSUB 64-wide K boxes per stage: one barrier round trip and one commit per 128 of K
  static constexpr int KSUB = 2;
  static constexpr size_t A_BOX = (size_t)tc::BM * tc::BK * 2;
  static constexpr size_t B_BOX = (size_t)(BN / 2) * tc::BK * 2;
  static constexpr size_t A_BYTES = KSUB * A_BOX;
  static constexpr size_t B_BYTES = KSUB * B_BOX;
  static constexpr int STAGES = (int)((204 * 1024) / (A_BYTES + B_BYTES)) < 8
                                    ? (int)((204 * 1024) / (A_BYTES + B_BYTES)) : 8;
  static constexpr uint32_t ACC_COLS = BN <= 128 ? 128 : 256;
  static constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;
  static constexpr size_t SMEM = 1024 + STAGES * (A_BYTES + B_BYTES) + (2 * STAGES + 4) * 8 + 16 + 128 +
                                 8 * kEpiWarpBytes;
};

template <int BN, int EPI>
__global__ void __launch_bounds__(320, 1) gemm_bf16_pair(const __grid_constant__ CUtensorMap ta,
                                                           const __grid_constant__ CUtensorMap tb,
                                                           GemmEpi e, int M, int N, int K, int S, int* err) {
  static_assert(BN % 16 == 0 && BN >= 32 && BN <= 256, "pair tile width");
  using C = PairCfg<BN>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = sA + S * C::A_BYTES;
  uint64_t* full = (uint64_t*)(sB + S * C::B_BYTES);
  uint64_t* empty = full + S;
  uint64_t* accf = empty + S;    // [2]
  uint64_t* acce = accf + 2;     // [2]
  uint32_t* tmem_slot = (uint32_t*)(acce + 2);
  uint8_t* stage = (uint8_t*)(((uintptr_t)(tmem_slot + 4) + 127) & ~(uintptr_t)127);   // 8 warps x 2 KB

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = tc::cluster_rank();
  const int cid = blockIdx.x >> 1, ncl = gridDim.x >> 1;
  const int nkb = (K + C::KSUB * tc::BK - 1) / (C::KSUB * tc::BK);
  const int n_tiles = (N + BN - 1) / BN;
  // tile t: group t / per_group, then 256-row block, then N tile (fastest)
  const int per_group = n_tiles * ((M + 2 * tc::BM - 1) / (2 * tc::BM));
  const int total = per_group * (e.groups > 1 ? e.groups : 1);

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&full[s], 1);    // the even CTA's producer expects the bytes of both CTAs
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&accf[b], 1);
      tc::mbar_init(&acce[b], 16);   // one arrival per epilogue warp of both CTAs
    }
    tc::fence_barrier_init();
  }
  if (warp == 1) tc::tmem_alloc_pair(tmem_slot, C::TMEM_COLS);
  tc::tc_fence_before();
  __syncthreads();
  tc::cluster_sync();                // barriers of both CTAs initialised before any remote arrival
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // TMA producer of this CTA's halves; bytes counted on the even CTA's "full" barrier
      const uint32_t full0 = tc::mapa_shared(tc::smem_u32(full), 0);
      int g = 0;
      for (int t = cid; t < total && !gemm_failed(err); t += ncl) {
        const int gr = t / per_group, r = t - gr * per_group;
        const int m0 = (r / n_tiles) * 2 * tc::BM, n0 = (r % n_tiles) * BN;
        const int ax = gr * e.a_col, bx = gr * e.b_col;
        const int ay = gr * e.a_row + m0 + (int)rank * tc::BM, by = gr * e.b_row + n0 + (int)rank * (BN / 2);
        bool stop = false;
        for (int kb = 0; kb < nkb; ++kb, ++g) {
          const int s = g % S;
          if (g >= S && !tc::mbar_wait(&empty[s], ((g / S) & 1) ^ 1, err, 21)) { stop = true; break; }
          const uint32_t fb = full0 + (uint32_t)s * 8u;
          // the even CTA's stage fills once both CTAs' halves have landed; the odd CTA's bytes
          // may land before this arrival (the transaction count goes transiently negative)
          if (rank == 0) tc::mbar_expect_tx(&full[s], (uint32_t)(2 * (C::A_BYTES + C::B_BYTES)));
#pragma unroll
          for (int q = 0; q < C::KSUB; ++q) {
            const int kx = (kb * C::KSUB + q) * tc::BK;
            tc::tma_load_2d_pair(sA + s * C::A_BYTES + q * C::A_BOX, &ta, fb, ax + kx, ay);
            tc::tma_load_2d_pair(sB + s * C::B_BYTES + q * C::B_BOX, &tb, fb, bx + kx, by);
          }
        }
        if (stop) break;
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 0) {
      // the pair's MMAs, issued by the even CTA into the two accumulators in turn
      constexpr uint32_t idesc = tc::idesc_bf16_f32<2 * tc::BM, BN>();
      int g = 0, it = 0;
      for (int t = cid; t < total && !gemm_failed(err); t += ncl, ++it) {
        const int b = it & 1, u = it >> 1;
        if (u > 0 && !tc::mbar_wait(&acce[b], (u & 1) ^ 1, err, 22)) break;
        tc::tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)b * C::ACC_COLS;
        bool stop = false;
        for (int kb = 0; kb < nkb; ++kb, ++g) {
          const int s = g % S;
          if (!tc::mbar_wait(&full[s], (g / S) & 1, err, 23)) { stop = true; break; }
          tc::tc_fence_after();
#pragma unroll
          for (int q = 0; q < C::KSUB; ++q) {
            const uint64_t da = tc::sw128_desc(sA + s * C::A_BYTES + q * C::A_BOX);
            const uint64_t db = tc::sw128_desc(sB + s * C::B_BYTES + q * C::B_BOX);
#pragma unroll
            for (int k = 0; k < tc::BK / tc::UMMA_K; ++k)
              tc::mma_bf16_pair(acc, da + (uint64_t)((k * tc::UMMA_K * 2) >> 4),
                                db + (uint64_t)((k * tc::UMMA_K * 2) >> 4), idesc,
                                (kb > 0 || q > 0 || k > 0) ? 1u : 0u);
          }
          tc::mma_commit_pair(&empty[s]);
        }
        if (stop) break;
        tc::mma_commit_pair(&accf[b]);
      }
    }
  } else {
    // epilogue warps 2..9 of each CTA: this CTA's 128 accumulator rows
    const int quarter = warp & 3, half = (warp - 2) >> 2;
    const uint32_t acce0 = tc::mapa_shared(tc::smem_u32(acce), 0);
    int it = 0;
    for (int t = cid; t < total; t += ncl, ++it) {
      const int b = it & 1, u = it >> 1;
      if (gemm_failed(err) || !tc::mbar_wait(&accf[b], u & 1, err, 24)) break;
      tc::tc_fence_after();
      const int gr = t / per_group, r = t - gr * per_group;
      const int m0 = (r / n_tiles) * 2 * tc::BM + (int)rank * tc::BM, n0 = (r % n_tiles) * BN;
      const int row0 = m0 + quarter * 32, row = row0 + lane;
      const int nrows = max(0, min(32, M - row0));
      uint8_t* wbuf = stage + (warp - 2) * kEpiWarpBytes;
      GemmEpi eg = e;
      if (gr) {
        constexpr size_t osz = (EPI == 0 || EPI == 2) ? 2 : 4;
        eg.out = (char*)e.out + (size_t)gr * (size_t)e.out_goff * osz;
        if (e.zout) eg.zout = e.zout + (size_t)gr * (size_t)e.out_goff;
        if (e.z) eg.z = e.z + (size_t)gr * (size_t)e.z_goff;
        if (e.bias) eg.bias = e.bias + (size_t)gr * (size_t)e.bias_goff;
      }
      const uint32_t acc = tmem + (uint32_t)b * C::ACC_COLS + ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
      for (int c0 = half * 32; c0 < BN; c0 += 64) {
        if (n0 + c0 >= N) break;
        float v[32];
        tc::tmem_ld32(acc + (uint32_t)c0, v);
        epi_chunk<EPI>(v, row, n0 + c0, min(32, N - (n0 + c0)), eg, wbuf, row0, nrows, lane);
        __syncwarp();
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive_cluster(acce0 + (uint32_t)b * 8u);
    }
  }
  tc::tc_fence_before();
  __syncwarp();
  __syncthreads();
  tc::cluster_sync();                // no CTA leaves while the pair's MMAs may read its stages
  tc::tc_fence_after();
  if (warp == 1) tc::tmem_dealloc_pair(tmem, C::TMEM_COLS);
}

// ------------------------------------------------------------------------------------------
// host: tensor maps and launch
// ------------------------------------------------------------------------------------------
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
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

// 2-D BF16 row-major [rows, cols] with row stride ld (elements); box = 64 columns x box_rows
static int make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return set_error(CHEM_E_CUDA, "cuTensorMapEncodeTiled is unavailable");
  if (((uintptr_t)base & 15) || ((ld * 2) & 15))
    return set_error(CHEM_E_ARG, "GEMM operand must be 16-byte aligned with a row stride that is a multiple of 8 elements");
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)tc::BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(CHEM_E_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return CHEM_OK;
}

template <int BN, int EPI>
static int launch_pair_t(const bf16* A, int64_t lda, const bf16* B, int64_t ldb, int M, int N, int K,
                         const GemmEpi& e, int* err, cudaStream_t s) {
  using P = PairCfg<BN>;
  CUtensorMap ta, tb;
  int rc;
  const int G = e.groups > 1 ? e.groups : 1;
  // the maps span every group's operand, as for the single-CTA kernels
  if ((rc = make_map(&ta, A, M + (int64_t)(G - 1) * e.a_row, K + (int64_t)(G - 1) * e.a_col, lda, tc::BM))) return rc;
  if ((rc = make_map(&tb, B, N + (int64_t)(G - 1) * e.b_row, K + (int64_t)(G - 1) * e.b_col, ldb, BN / 2))) return rc;
  static int max_clusters = 0;
  static bool configured = false;
  const int nkb = (K + P::KSUB * tc::BK - 1) / (P::KSUB * tc::BK);
  const int S = nkb < P::STAGES ? nkb : P::STAGES;
  const size_t smem = 1024 + (size_t)S * (P::A_BYTES + P::B_BYTES) + (2 * (size_t)S + 4) * 8 + 16 + 128 +
                      8 * (size_t)kEpiWarpBytes;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(320, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (!configured) {
    if ((rc = cuda_check(cudaFuncSetAttribute(gemm_bf16_pair<BN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)P::SMEM), "gemm pair smem attribute")))
      return rc;
    cudaLaunchConfig_t q = cfg;
    q.dynamicSmemBytes = P::SMEM;
    q.gridDim = dim3(2, 1, 1);
    int nc = 0;
    if ((rc = cuda_check(cudaOccupancyMaxActiveClusters(&nc, gemm_bf16_pair<BN, EPI>, &q), "gemm pair occupancy")))
      return rc;
    if (nc <= 0) return set_error(CHEM_E_UNSUPPORTED, "gemm: no CTA pair fits on the device");
    max_clusters = nc;
    configured = true;
  }
  const int64_t total = (int64_t)((N + BN - 1) / BN) * ((M + 2 * tc::BM - 1) / (2 * tc::BM)) * G;
  if (total > 0x7fffffff) return set_error(CHEM_E_ARG, "gemm: too many tiles in one call");
  const int ncl = (int)std::min<int64_t>(total, (int64_t)max_clusters);
  cfg.gridDim = dim3(2 * (unsigned)ncl, 1, 1);
  return cuda_check(cudaLaunchKernelEx(&cfg, gemm_bf16_pair<BN, EPI>, ta, tb, e, M, N, K, S, err),
                    "gemm_bf16_pair launch");
}

template <int BN, int EPI>
static int launch_gemm_t(const bf16* A, int64_t lda, const bf16* B, int64_t ldb, int M, int N, int K,
                         const GemmEpi& e, int* err, cudaStream_t s) {
  CUtensorMap ta, tb;
  int rc;
  const int G = e.groups > 1 ? e.groups : 1;
  // the maps span every group's operand; a K slab that runs past a group's K reads the next
  // group's A columns, multiplied by the zeros that B's map supplies past its K extent
  if ((rc = make_map(&ta, A, M + (int64_t)(G - 1) * e.a_row, K + (int64_t)(G - 1) * e.a_col, lda, tc::BM))) return rc;
  if ((rc = make_map(&tb, B, N + (int64_t)(G - 1) * e.b_row, K + (int64_t)(G - 1) * e.b_col, ldb, BN))) return rc;
  const int nkb_all = (K + tc::BK - 1) / tc::BK;
  if constexpr (EPI == 4) {
    if (nkb_all > 2 || G > 1 || N % 32) return set_error(CHEM_E_ARG, "gemm: epilogue 4 needs K <= 128, N % 32 == 0");
  } else if (nkb_all > 2 || G > 1) {
    if constexpr (BN >= 128) {
      // long K, wide tiles, at least one 256-row block: CTA pairs (cta_group::2)
      if (M >= 2 * tc::BM) return launch_pair_t<BN, EPI>(A, lda, B, ldb, M, N, K, e, err, s);
    }
    // long K: persistent warp-specialised kernel, one CTA per SM
    using P = PersistCfg<BN>;
    static bool pconfigured = false;
    if (!pconfigured) {
      if ((rc = cuda_check(cudaFuncSetAttribute(gemm_bf16_persistent<BN, EPI>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P::SMEM),
                           "gemm smem attribute")))
        return rc;
      pconfigured = true;
    }
    const int S = nkb_all < P::STAGES ? nkb_all : P::STAGES;
    const size_t smem = 1024 + (size_t)S * (P::A_BYTES + P::B_BYTES) + (2 * (size_t)S + 4) * 8 + 16 + 128 +
                        8 * (size_t)kEpiWarpBytes;
    const int64_t total = (int64_t)((N + BN - 1) / BN) * ((M + tc::BM - 1) / tc::BM) * G;
    if (total > 0x7fffffff) return set_error(CHEM_E_ARG, "gemm: too many tiles in one call");
    static int sms = 0;
    if (!sms) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (sms <= 0) sms = 1;
    }
    const int grid = (int)std::min<int64_t>(total, (int64_t)sms);
    gemm_bf16_persistent<BN, EPI><<<grid, 320, smem, s>>>(ta, tb, e, M, N, K, S, err);
    return cuda_check(cudaGetLastError(), "gemm_bf16_persistent launch");
  }
  using Cfg = TileCfg<BN>;
  static bool configured = false;
  if (!configured) {
    if ((rc = cuda_check(cudaFuncSetAttribute(gemm_bf16_kernel<BN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)Cfg::SMEM), "gemm smem attribute")))
      return rc;
    configured = true;
  }
  const int nkb = (K + tc::BK - 1) / tc::BK;
  const int S = nkb < Cfg::STAGES ? nkb : Cfg::STAGES;
  const size_t smem = 1024 + (size_t)S * (Cfg::A_BYTES + Cfg::B_BYTES) + (2 * (size_t)S + 2) * 8 + 16 + 128 +
                      8 * (size_t)kEpiWarpBytes;
  if ((M + tc::BM - 1) / tc::BM > 65535) return set_error(CHEM_E_ARG, "gemm: more than 65535 row blocks in one call");
  dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + tc::BM - 1) / tc::BM));
  gemm_bf16_kernel<BN, EPI><<<grid, 256, smem, s>>>(ta, tb, e, M, N, K, S, err);
  return cuda_check(cudaGetLastError(), "gemm_bf16_kernel launch");
}

// C = A B^T with the epilogue `epi` (0: bias+GELU -> BF16 [+ pre-activation copy],
// 1: bias -> FP32, 2: * GELU'(z) -> BF16, 3: FP32).  BN (a multiple of 32, at most 256) is
// chosen from N.
int gemm_bf16(int epi, const bf16* A, int64_t lda, const bf16* B, int64_t ldb, int M, int N, int K,
              const GemmEpi& e, int* err, cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) return CHEM_OK;
  if (e.groups > 1) {
    // TMA column coordinates on 16-byte boundaries; 16-byte vector stores and z loads of
    // full 32-column chunks at every group's offset
    const int64_t ov = (epi == 0 || epi == 2) ? 8 : 4;
    if (e.a_row < 0 || e.b_row < 0 || e.a_col < 0 || e.b_col < 0 || (e.a_col & 7) || (e.b_col & 7) ||
        e.out_goff < 0 || e.z_goff < 0 || e.bias_goff < 0 || (N >= 32 && (e.out_goff % ov || e.z_goff % 8)))
      return set_error(CHEM_E_ARG, "gemm: group offsets must be non-negative, column offsets multiples of 8");
  }
  // tile width: N <= 128 takes the narrowest of 32/64/128 that covers it; wider layers take the
  // tile of at least 128 columns with the least padded width ceil(N / BN) BN, ties to the wider
  // (single CTAs: N = 1600 and 800 take 160, N = 400 and 2000 take 224, N = 1000 and 500 take
  // 256), or on CTA pairs the least padded width weighted by 1 + 128/BN (N = 800 and 400 take
  // 224, 1600, 2000, 1000 and 500 take 256) -- narrow tiles on wide layers would reload the A
  // tile once per 32 columns.  A short K (<= 128, the first layer) takes 128: its time is the
  // epilogue, and 128 TMEM columns per CTA let four CTAs share an SM instead of two.
  int bn = N <= 32 ? 32 : N <= 64 ? 64 : 128;
  if (N > 128 && K > 128) {
    static const int kBN[] = {256, 224, 160, 128};
    const bool pair = M >= 2 * tc::BM && K > 2 * tc::BK;
    int64_t best = INT64_MAX;
    for (int c : kBN) {
      const int64_t padded = (int64_t)((N + c - 1) / c) * c;
      // CTA pairs: time ~ padded width x (1 + 128 / BN) -- a wider MMA carries its fixed cost
      // over more columns (measured: the 800-wide layer runs 7 % faster at 224, padded to 896,
      // than at 160)
      const int64_t cost = pair ? padded * (c + 128) / c : padded;
      if (cost < best) { best = cost; bn = c; }
    }
  }
  // the first layer's forward without a pre-activation copy: the short-K kernel's lean GELU epilogue
  const bool gelu_x8 = epi == 0 && !e.zout && e.groups <= 1 && K <= 2 * tc::BK && N % 32 == 0;
#define CHEM_GEMM_CASE(BNV)                                                                    \
  if (bn == BNV) {                                                                             \
    switch (epi) {                                                                             \
      case 0:                                                                                  \
        if (gelu_x8) return launch_gemm_t<BNV, 4>(A, lda, B, ldb, M, N, K, e, err, s);         \
        return launch_gemm_t<BNV, 0>(A, lda, B, ldb, M, N, K, e, err, s);                      \
      case 1: return launch_gemm_t<BNV, 1>(A, lda, B, ldb, M, N, K, e, err, s);                \
      case 2: return launch_gemm_t<BNV, 2>(A, lda, B, ldb, M, N, K, e, err, s);                \
      default: return launch_gemm_t<BNV, 3>(A, lda, B, ldb, M, N, K, e, err, s);               \
    }                                                                                          \
  }
  CHEM_GEMM_CASE(32)
  CHEM_GEMM_CASE(64)
  CHEM_GEMM_CASE(128)
  CHEM_GEMM_CASE(160)
  CHEM_GEMM_CASE(224)
  CHEM_GEMM_CASE(256)
#undef CHEM_GEMM_CASE
  return set_error(CHEM_E_ARG, "gemm: unsupported tile");
}

// output layer of per-species networks, backward: one thread per element of dZ [B, G h]
__global__ void group_out_dgrad_kernel(const bf16* dU, int ldu, const bf16* W, const bf16* Z, int64_t B, int G, int h,
                                       bf16* dZ) {
  const int64_t w = (int64_t)G * h, n = B * w;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = i / w;
    const int c = (int)(i - b * w), g = c / h;
    const float acc = __bfloat162float(dU[b * ldu + g]) * __bfloat162float(W[c]);
    dZ[i] = __float2bfloat16_rn(acc * dgelu_f(__bfloat162float(Z[i])));
  }
}

int launch_group_out_dgrad(const bf16* dU, int ldu, const bf16* W, const bf16* Z, int64_t B, int G, int h, bf16* dZ,
                           cudaStream_t s) {
  const int64_t n = B * (int64_t)G * h;
  if (n <= 0) return CHEM_OK;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sms * 32));
  group_out_dgrad_kernel<<<grid, 256, 0, s>>>(dU, ldu, W, Z, B, G, h, dZ);
  return cuda_check(cudaGetLastError(), "group_out_dgrad_kernel launch");
}

}  // namespace chem

using namespace chem;

extern "C" int chem_selftest_gemm(int epi, int M, int N, int K, const void* A, const void* B, const float* bias,
                                  const void* z, void* out, int* err, chem_stream stream) {
  if (M < 0 || N < 0 || K < 0 || !A || !B || !out || !err) return set_error(CHEM_E_ARG, "chem_selftest_gemm: bad arguments");
  if (epi < 0 || epi > 3 || (epi == 2 && !z)) return set_error(CHEM_E_ARG, "chem_selftest_gemm: bad epilogue");
  GemmEpi e{};
  e.bias = bias;
  e.out = out;
  e.ldo = N;
  e.z = (const bf16*)z;
  e.ldz = N;
  e.zout = nullptr;
  return gemm_bf16(epi, (const bf16*)A, K, (const bf16*)B, K, M, N, K, e, err, (cudaStream_t)stream);
}

// G GEMMs in one launch with the group offsets of GemmEpi (row strides lda, ldb, ldo, ldz)
extern "C" int chem_selftest_gemm_grouped(int epi, int G, int M, int N, int K, const void* A, int64_t lda, int a_row,
                                          int a_col, const void* B, int64_t ldb, int b_row, int b_col,
                                          const float* bias, int bias_goff, const void* z, int64_t ldz, int64_t z_goff,
                                          void* out, int64_t ldo, int64_t out_goff, int* err, chem_stream stream) {
  if (G < 1 || M < 0 || N < 0 || K < 0 || !A || !B || !out || !err || ldo > INT_MAX || ldz > INT_MAX)
    return set_error(CHEM_E_ARG, "chem_selftest_gemm_grouped: bad arguments");
  if (epi < 0 || epi > 3 || (epi == 2 && !z)) return set_error(CHEM_E_ARG, "chem_selftest_gemm_grouped: bad epilogue");
  GemmEpi e{};
  e.bias = bias;
  e.out = out;
  e.ldo = (int)ldo;
  e.z = (const bf16*)z;
  e.ldz = (int)ldz;
  e.groups = G;
  e.a_row = a_row;
  e.a_col = a_col;
  e.b_row = b_row;
  e.b_col = b_col;
  e.out_goff = out_goff;
  e.z_goff = z_goff;
  e.bias_goff = bias_goff;
  return gemm_bf16(epi, (const bf16*)A, lda, (const bf16*)B, ldb, M, N, K, e, err, (cudaStream_t)stream);
}
