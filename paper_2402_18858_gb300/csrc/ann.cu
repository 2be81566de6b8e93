// The learned reaction step (Sec. 2.2): an MLP maps the cell state phi(t) = {T, p, F(Y)}
// (F = Box-Cox transform, Eq. 7, lambda = 0.1) to the change of the transformed mass
// fractions over dt, standing in for the direct integration of Eq. 2.  The paper runs it in
// half precision (Sec. 2.1); here it is BF16 on the tcgen05 tensor cores with FP32
// accumulation, trained by this file's own forward/backward kernels with the loss of
// Eqs. 8-9 and Adam.  Cells whose inputs fall outside the training range, whose prediction
// breaks element conservation or gives a non-physical temperature fall back to direct
// integration, so the step never returns an unchecked learned state.
//
// Reading of the output (the paper writes u* = Y(t+dt) - Y(t); its Eq. 7 transform is applied
// to the species): the network predicts u_k = (F(Y_k(t+dt)) - F(Y_k(t)) - mu_k) / sigma_k,
// z-scored over the training set; T(t+dt) follows from enthalpy conservation of the adiabatic
// constant-pressure cell, h(T(t+dt), Y(t+dt)) = h(T(t), Y(t)), solved by Newton's method.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

using bf16 = __nv_bfloat16;

namespace chem {

constexpr float kLambda = 0.1f;     // Box-Cox parameter (Sec. 2.2)
constexpr int kMaxLayers = 8;
constexpr int kInPad = 64;          // input features padded to one 64-wide K slab
constexpr int kStatBlock = 256;

// Box-Cox transform of a mass fraction (Eq. 7 read as (x^lambda - 1)/lambda, x clipped >= 0)
__device__ __forceinline__ float bct_x(float x) {
  return x > 0.0f ? (exp2f(kLambda * log2f(x)) - 1.0f) * (1.0f / kLambda) : -1.0f / kLambda;
}
__device__ __forceinline__ float bct_f(double y) { return bct_x((float)fmax(y, 0.0)); }
// inverse: x = (lambda z + 1)^(1/lambda) = t^10, 0 where t <= 0
__device__ __forceinline__ float ibct_f(float z) {
  const float t = fmaxf(kLambda * z + 1.0f, 0.0f);
  const float t2 = t * t, t4 = t2 * t2, t8 = t4 * t4;
  return t8 * t2;
}

}  // namespace chem

using namespace chem;

struct chem_ann_s {
  int device = 0;
  chem_mech_s* mech = nullptr;
  DevMech dm{};
  int K = 0, n_in = 0, n_out = 0, n_out_pad = 0, L = 0;
  // groups = 1: one network with K outputs.  groups = K: one network per species (Sec. 2.2),
  // all sharing the input; dims[] are then the widths of one species' network (output 1) and
  // every layer stores the K networks' weights stacked by species, W_l [K dims[l+1], dims[l]]
  int groups = 1;
  int dims[kMaxLayers + 1] = {0};
  int64_t n_params = 0;        // including padding
  void* dmem = nullptr;        // all parameter-sized device memory
  float *Wm[kMaxLayers], *bm[kMaxLayers], *gW[kMaxLayers], *gb[kMaxLayers];
  float *mW[kMaxLayers], *vW[kMaxLayers], *mb[kMaxLayers], *vb[kMaxLayers];
  bf16 *W[kMaxLayers], *WT[kMaxLayers];
  float* norm = nullptr;       // device: in_mean, in_std, in_min, in_max [n_in]; out_mean, out_std [n_out]
  std::vector<float> hnorm;    // host copy
  int step = 0;
  int* err = nullptr;          // device GEMM error flag
  // training scratch
  void* tmem_ = nullptr;
  int64_t tcap = 0;
  float* loss_part = nullptr;
};

// ------------------------------------------------------------------------------------------
// kernels
// ------------------------------------------------------------------------------------------
namespace {

// raw feature j of cell i: 0 -> T, 1 -> p, 2 + k -> F(Y_k)
__device__ __forceinline__ float raw_feature(int j, int64_t i, int64_t ld, const double* T, const double* p,
                                             const double* Y) {
  if (j == 0) return (float)T[i];
  if (j == 1) return (float)p[i];
  return bct_f(Y[(size_t)(j - 2) * ld + i]);
}

// heat-release coefficients of the L_HRR term (Eq. 10) per sample: c_bk = -rho (h_k(T0) - hbar)
// / (dt s) (h_k the mass enthalpy from NASA-7 at the initial temperature, hbar = sum Y0_k h_k,
// rho = p / (R T0 sum Y/W)) and the DI target r_b = sum_k c_bk (Y1_bk - Y0_bk); FP64
// arithmetic, FP32 results [n, K], [n].  The shift by hbar leaves the heat release of any
// mass-conserving change unchanged and keeps mass-sum errors (L_mass) out of L_HRR.
__global__ void hrr_coeff_kernel(DevMech m, int64_t n, int64_t ld, const double* T0, const double* p,
                                 const double* Y0, const double* Y1, double dt, double scale, float* c, float* r) {
  const int K = m.K;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double T = T0[i], invT = 1.0 / T;
    double sYW = 0.0;
    for (int k = 0; k < K; ++k) sYW += Y0[(size_t)k * ld + i] * m.invW[k];
    const double rho = p[i] / (kR * T * sYW);
    const double f = -rho * kR * T / (dt * scale);
    const int hi = T >= m.Tmid ? 1 : 0;
    // mass enthalpies over RT (the common factor R T goes into f) and their mean over Y0
    double hbar = 0.0;
    for (int k = 0; k < K; ++k) {
      const double* a = m.th + ((size_t)k * 2 + hi) * kThermoStride;
      const double hRT = a[5] + T * (a[6] + T * (a[7] + T * (a[8] + T * a[9]))) + a[10] * invT;
      hbar += Y0[(size_t)k * ld + i] * hRT * m.invW[k];
    }
    double acc = 0.0;
    for (int k = 0; k < K; ++k) {
      const double* a = m.th + ((size_t)k * 2 + hi) * kThermoStride;
      const double hRT = a[5] + T * (a[6] + T * (a[7] + T * (a[8] + T * a[9]))) + a[10] * invT;
      const double ck = f * (hRT * m.invW[k] - hbar);
      c[(size_t)i * K + k] = (float)ck;
      acc += ck * (Y1[(size_t)k * ld + i] - Y0[(size_t)k * ld + i]);
    }
    r[i] = (float)acc;
  }
}


// normalised BF16 features X[i][0..63]; range flag (bit 1) against the training min/max
__global__ void features_kernel(int64_t n, int64_t ld, const double* T, const double* p, const double* Y, int n_in,
                                const float* norm, float margin, bf16* X, int32_t* flags, float* bcty, int K,
                                const int32_t* idx) {
  const float* mean = norm;
  const float* sd = norm + n_in;
  const float* mn = norm + 2 * n_in;
  const float* mx = norm + 3 * n_in;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int flag = 0;
    const int64_t col = idx ? (int64_t)idx[i] : i;
    __align__(16) bf16 row[kInPad];
    for (int j = 0; j < kInPad; ++j) {
      float v = 0.0f;
      if (j < n_in) {
        const float r = raw_feature(j, col, ld, T, p, Y);
        const float span = mx[j] - mn[j];
        if (!(r >= mn[j] - margin * span && r <= mx[j] + margin * span)) flag = 1;
        v = (r - mean[j]) / sd[j];
        if (bcty && j >= 2) bcty[(size_t)i * K + (j - 2)] = r;
      }
      row[j] = __float2bfloat16_rn(v);
    }
    uint4* dst = (uint4*)(X + (size_t)i * kInPad);
#pragma unroll
    for (int q = 0; q < kInPad / 8; ++q) dst[q] = ((const uint4*)row)[q];
    if (flags) flags[i] = flag;
  }
}

// z-scored targets u_k = (F(Y1_k) - F(Y0_k) - mu_k)/sigma_k, padded to n_out_pad columns
__global__ void targets_kernel(int64_t n, int64_t ld, const double* Y0, const double* Y1, int K, int n_out_pad,
                               const float* out_mean, const float* out_sd, float* U) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    for (int k = 0; k < n_out_pad; ++k) {
      float v = 0.0f;
      if (k < K) v = (bct_f(Y1[(size_t)k * ld + i]) - bct_f(Y0[(size_t)k * ld + i]) - out_mean[k]) / out_sd[k];
      U[(size_t)i * n_out_pad + k] = v;
    }
}

// per-block partial statistics of the raw features (n_in) and raw targets (K):
// sum, sum of squares, min, max -> part[b][c][4] (deterministic: fixed-order tree per block)
__global__ void stats_partial_kernel(int64_t n, int64_t ld, const double* T, const double* p, const double* Y0,
                                     const double* Y1, int n_in, int K, double* part) {
  const int C = n_in + K;
  __shared__ double sh[4][kStatBlock];
  for (int c = 0; c < C; ++c) {
    double s = 0, q = 0, lo = 1e300, hi = -1e300;
    for (int64_t i = (int64_t)blockIdx.x * kStatBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kStatBlock) {
      double v;
      if (c < n_in) v = raw_feature(c, i, ld, T, p, Y0);
      else v = (double)(bct_f(Y1[(size_t)(c - n_in) * ld + i]) - bct_f(Y0[(size_t)(c - n_in) * ld + i]));
      s += v;
      q += v * v;
      lo = fmin(lo, v);
      hi = fmax(hi, v);
    }
    sh[0][threadIdx.x] = s;
    sh[1][threadIdx.x] = q;
    sh[2][threadIdx.x] = lo;
    sh[3][threadIdx.x] = hi;
    __syncthreads();
    for (int o = kStatBlock / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) {
        sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
        sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
        sh[2][threadIdx.x] = fmin(sh[2][threadIdx.x], sh[2][threadIdx.x + o]);
        sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + o]);
      }
      __syncthreads();
    }
    if (threadIdx.x == 0)
      for (int t = 0; t < 4; ++t) part[((size_t)blockIdx.x * C + c) * 4 + t] = sh[t][0];
    __syncthreads();
  }
}

// network output -> new state; flags: 1 range, 2 non-finite, 4 element residual, 8 T range, 16 |dT|
// FP32 work of the update (the enthalpy and element sums of the old and predicted states, T
// from h by Newton) reads FP32 copies of the NASA-7 and composition tables, so that no
// FP64 -> FP32 conversion runs per table entry; the element projection stays FP64 and skips
// the zero entries of the composition (a warp-uniform test: every thread is at the same
// species).  EC: compile-time bound on the element count (registers for the E x E system).
template <int EC>
__global__ void update_kernel(DevMech m, int64_t n, int64_t ld, double* T, const double* p, double* Y,
                              const float* U, int n_out_pad, const float* out_mean, const float* out_sd,
                              int32_t* flags, int32_t* status, float elem_tol, float Tmin, float Tmax, float dTmax,
                              const int32_t* idx) {
  const int K = m.K, E = m.E;
  const float Tmidf = (float)m.Tmid;
  for (int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; slot < n;
       slot += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx ? (int64_t)idx[slot] : slot;   // cell column; U, flags, status by slot
    int flag = flags[slot];
    if (flag == 0) {
      float yn[CHEM_MAX_SPECIES];    // prediction (inverse Box-Cox, renormalised)
      float yp[CHEM_MAX_SPECIES];    // the state T' is solved for: projected, or yn when flagged
      float eo[EC], en[EC];
      double eod[EC], lam[EC];
#pragma unroll
      for (int e = 0; e < EC; ++e) {
        eo[e] = en[e] = 0.0f;
        eod[e] = lam[e] = 0.0;
      }
      const float T0 = (float)T[i];
      // enthalpy of the old state (FP32 NASA-7 sums) and old element moles
      float h0 = 0.0f, ysum = 0.0f;
      bool finite = true;
      const int hi0 = T0 >= Tmidf ? 1 : 0;
      for (int k = 0; k < K; ++k) {
        const double y = Y[(size_t)k * ld + i];
        const float yf = narrow_f32(y);
        const float* a = m.th32 + ((size_t)k * 2 + hi0) * 16;
        const float hRT = a[5] + T0 * (a[6] + T0 * (a[7] + T0 * (a[8] + T0 * a[9]))) + a[10] / T0;
        h0 += yf * m.invW32[k] * hRT;
#pragma unroll
        for (int e = 0; e < EC; ++e) {
          if (e < E) {
            const float cf = m.compW32[(size_t)k * E + e];
            if (cf != 0.0f) {
              eod[e] = fma(y, m.compW[(size_t)k * E + e], eod[e]);
              eo[e] = fmaf(yf, cf, eo[e]);
            }
          }
        }
        const float z = bct_x((float)fmax(y, 0.0)) + U[(size_t)slot * n_out_pad + k] * out_sd[k] + out_mean[k];
        finite = finite && isfinite(z);   // ibct_f would map a NaN to 0 (fmaxf)
        const float v = ibct_f(z);
        yn[k] = v;
        ysum += v;
      }
      h0 *= T0;   // h/R per kg
      if (!finite || !(ysum > 0.0f) || !isfinite(ysum)) flag |= 2;
      if (!flag) {
        const float is = 1.0f / ysum;
        for (int k = 0; k < K; ++k) {
          yn[k] *= is;
#pragma unroll
          for (int e = 0; e < EC; ++e)
            if (e < E) en[e] = fmaf(yn[k], m.compW32[(size_t)k * E + e], en[e]);
        }
        float res = 0.0f;
#pragma unroll
        for (int e = 0; e < EC; ++e)
          if (e < E && eo[e] > 0.0f) res = fmaxf(res, fabsf(en[e] - eo[e]) / eo[e]);
        if (!(res <= elem_tol)) flag |= 4;
        if (!flag) {
          // accepted: project onto exact element conservation, min sum_k dY_k^2 / w_k with
          // w_k = Y_k subject to sum_k c_ke (Y_k + dY_k) = E_old_e (c = composition / W):
          // dY = diag(w) C^T lam, (C diag(w) C^T) lam = E_old - C Y.  In FP64: the E x E system
          // can be ill-conditioned (an element carried mostly by one abundant species), and
          // the projected state conserves the elements to FP64 rounding.  The matrix is
          // accumulated on its upper triangle and mirrored.
          double Mx[EC][EC + 1];
#pragma unroll
          for (int a1 = 0; a1 < EC; ++a1) {
#pragma unroll
            for (int a2 = 0; a2 < EC; ++a2) Mx[a1][a2] = 0.0;
            Mx[a1][EC] = eod[a1];
          }
          for (int k = 0; k < K; ++k) {
            const double wk = (double)yn[k];
#pragma unroll
            for (int a1 = 0; a1 < EC; ++a1) {
              if (a1 < E && m.compW32[(size_t)k * E + a1] != 0.0f) {
                const double c1 = m.compW[(size_t)k * E + a1] * wk;
                Mx[a1][EC] -= c1;
#pragma unroll
                for (int a2 = a1; a2 < EC; ++a2)
                  if (a2 < E && m.compW32[(size_t)k * E + a2] != 0.0f)
                    Mx[a1][a2] = fma(c1, m.compW[(size_t)k * E + a2], Mx[a1][a2]);
              }
            }
          }
#pragma unroll
          for (int a1 = 0; a1 < EC; ++a1)
#pragma unroll
            for (int a2 = 0; a2 < a1; ++a2) Mx[a1][a2] = Mx[a2][a1];
          // Gauss-Jordan with partial pivoting; elements absent from both states have a zero
          // row and column and keep lam = 0
          bool live[EC];
#pragma unroll
          for (int c = 0; c < EC; ++c) live[c] = c < E && Mx[c][c] > 0.0;
#pragma unroll
          for (int c = 0; c < EC; ++c) {
            if (!live[c]) continue;
            int piv = c;
#pragma unroll
            for (int r = c + 1; r < EC; ++r)
              if (live[r] && fabs(Mx[r][c]) > fabs(Mx[piv][c])) piv = r;
            // rows swapped through a select chain (indices stay compile-time constants)
#pragma unroll
            for (int r = c + 1; r < EC; ++r) {
              if (r == piv) {
#pragma unroll
                for (int j = 0; j <= EC; ++j) { const double t = Mx[c][j]; Mx[c][j] = Mx[r][j]; Mx[r][j] = t; }
              }
            }
            if (!(fabs(Mx[c][c]) > 0.0)) continue;
            const double d = 1.0 / Mx[c][c];
#pragma unroll
            for (int j = 0; j <= EC; ++j) Mx[c][j] *= d;
#pragma unroll
            for (int r = 0; r < EC; ++r) {
              if (r == c) continue;
              const double f = Mx[r][c];
#pragma unroll
              for (int j = 0; j <= EC; ++j) Mx[r][j] = fma(-f, Mx[c][j], Mx[r][j]);
            }
          }
#pragma unroll
          for (int c = 0; c < EC; ++c) lam[c] = (live[c] && fabs(Mx[c][c] - 1.0) < 1e-9) ? Mx[c][EC] : 0.0;
          for (int k = 0; k < K; ++k) {
            double cl = 0.0;
#pragma unroll
            for (int e = 0; e < EC; ++e)
              if (e < E && m.compW32[(size_t)k * E + e] != 0.0f) cl = fma(m.compW[(size_t)k * E + e], lam[e], cl);
            const double yd = (double)yn[k];
            yp[k] = (float)fmax(fma(yd, cl, yd), 0.0);
          }
        } else {
          for (int k = 0; k < K; ++k) yp[k] = yn[k];
        }
        // T from h(T, Y_new) = h0 by Newton's method
        float Tn = T0;
        for (int it = 0; it < 8; ++it) {
          const int hi = Tn >= Tmidf ? 1 : 0;
          float h = 0.0f, cp = 0.0f;
          for (int k = 0; k < K; ++k) {
            const float* a = m.th32 + ((size_t)k * 2 + hi) * 16;
            const float yw = yp[k] * m.invW32[k];
            const float cpR = a[0] + Tn * (a[1] + Tn * (a[2] + Tn * (a[3] + Tn * a[4])));
            const float hRT = a[5] + Tn * (a[6] + Tn * (a[7] + Tn * (a[8] + Tn * a[9]))) + a[10] / Tn;
            h += yw * hRT * Tn;
            cp += yw * cpR;
          }
          const float dT = (h - h0) / cp;
          Tn = fminf(fmaxf(Tn - dT, 200.0f), 6000.0f);
          if (fabsf(dT) < 1e-4f * Tn) break;
        }
        if (!isfinite(Tn)) flag |= 2;
        else if (Tn < Tmin || Tn > Tmax) flag |= 8;
        else if (dTmax > 0.0f && fabsf(Tn - T0) > dTmax) flag |= 16;
        if (!flag) {
          // the projected state in FP64 (accepted cells were projected)
          for (int k = 0; k < K; ++k) {
            double cl = 0.0;
#pragma unroll
            for (int e = 0; e < EC; ++e)
              if (e < E && m.compW32[(size_t)k * E + e] != 0.0f) cl = fma(m.compW[(size_t)k * E + e], lam[e], cl);
            const double yd = (double)yn[k];
            Y[(size_t)k * ld + i] = fmax(fma(yd, cl, yd), 0.0);
          }
          T[i] = (double)Tn;
        }
      }
    }
    flags[slot] = flag;
    status[slot] = flag ? CHEM_CELL_ANN_FALLBACK : CHEM_CELL_OK;
  }
}

int grid_for(int64_t n, int threads);

// update_kernel with its element bound chosen from the mechanism (C/H/O/N: 4)
static int launch_update(const DevMech& m, int64_t n, int64_t ld, double* T, const double* p, double* Y,
                         const float* U, int n_out_pad, const float* out_mean, const float* out_sd,
                         int32_t* flags, int32_t* status, float elem_tol, float Tmin, float Tmax, float dTmax,
                         const int32_t* idx, cudaStream_t s) {
  const unsigned grid = grid_for(n, 128);
#define CHEM_UPDATE_CASE(EC)                                                                                  \
  update_kernel<EC><<<grid, 128, 0, s>>>(m, n, ld, T, p, Y, U, n_out_pad, out_mean, out_sd, flags, status,  \
                                         elem_tol, Tmin, Tmax, dTmax, idx)
  if (m.E <= 3) CHEM_UPDATE_CASE(3);
  else if (m.E <= 4) CHEM_UPDATE_CASE(4);
  else CHEM_UPDATE_CASE(kMaxElem);
#undef CHEM_UPDATE_CASE
  return cuda_check(cudaGetLastError(), "update_kernel launch");
}

// deterministic compaction of cells with status != 0: per-block counts, scan, write
constexpr int kCompactBlock = 1024;

__global__ void compact_count_kernel(int64_t n, const int32_t* status, int32_t* blk_count) {
  __shared__ int ws[32];
  const int64_t i = (int64_t)blockIdx.x * kCompactBlock + threadIdx.x;
  const int f = (i < n && status[i] != 0) ? 1 : 0;
  const unsigned b = __ballot_sync(0xffffffffu, f);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = __popc(b);
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < kCompactBlock / 32; ++w) s += ws[w];
    blk_count[blockIdx.x] = s;
  }
}

__global__ void compact_scan_kernel(int nb, int32_t* blk_count, int32_t* total) {
  // single thread: exclusive scan in block order (nb <= a few thousand)
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int s = 0;
    for (int b = 0; b < nb; ++b) {
      const int c = blk_count[b];
      blk_count[b] = s;
      s += c;
    }
    *total = s;
  }
}

__global__ void compact_write_kernel(int64_t n, const int32_t* status, const int32_t* blk_off, int32_t* slots,
                                     int32_t* cols, const int32_t* idx) {
  __shared__ int ws[32];
  const int64_t i = (int64_t)blockIdx.x * kCompactBlock + threadIdx.x;
  const int f = (i < n && status[i] != 0) ? 1 : 0;
  const unsigned b = __ballot_sync(0xffffffffu, f);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) ws[w] = __popc(b);
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int q = 0; q < kCompactBlock / 32; ++q) {
      const int c = ws[q];
      ws[q] = s;
      s += c;
    }
  }
  __syncthreads();
  if (f) {
    const int q = blk_off[blockIdx.x] + ws[w] + __popc(b & ((1u << lane) - 1u));
    slots[q] = (int32_t)i;
    cols[q] = idx ? idx[i] : (int32_t)i;
  }
}

// DI statuses of the fallback cells back to the cells: 5 when DI succeeded, else DI's code
__global__ void scatter_status_kernel(int64_t nmax, const int32_t* n_dev, const int32_t* slots, const int32_t* st_slot,
                                      int32_t* status) {
  const int64_t nf = min(nmax, (int64_t)*n_dev);
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nf; s += (int64_t)gridDim.x * blockDim.x)
    status[slots[s]] = st_slot[s] == CHEM_CELL_OK ? CHEM_CELL_ANN_FALLBACK : st_slot[s];
}

// training loss (Eqs. 8-10) and its gradient w.r.t. the network output
//   L = w_data * mean_{b,k}(u - u_t)^2 + w_mass * mean_b |sum_k Y*_k - 1| + w_hrr * mean_b e_b^2,
//   Y*_k = F^-1(F(Y_k) + u_k sigma_k + mu_k),
//   e_b = sum_k c_bk (Y*_k - Y_k) - r_b   (the step-mean heat-release error, scaled)
// dU (BF16 [B, n_out_pad]) and its transpose dUT ([n_out_pad, B]); per-block loss partials.
__global__ void loss_grad_kernel(int64_t B, int K, int n_out_pad, const float* Up, const float* Ut, const float* bcty,
                                 const float* out_mean, const float* out_sd, float w_data, float w_mass,
                                 const float* hrr_c, const float* hrr_r, float w_hrr, bf16* dU, bf16* dUT,
                                 float* part) {
  __shared__ float sh[3][256];
  float ld = 0.0f, lm = 0.0f, lh = 0.0f;
  const float cdata = 2.0f * w_data / (float)(B * K);
  const bool mass = bcty && w_mass != 0.0f;
  const bool hrr = bcty && hrr_c && hrr_r && w_hrr != 0.0f;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < B; b += (int64_t)gridDim.x * blockDim.x) {
    float ysum = 0.0f, eb = 0.0f;
    if (mass || hrr) {
      for (int k = 0; k < K; ++k) {
        const float ys = ibct_f(bcty[b * K + k] + Up[b * n_out_pad + k] * out_sd[k] + out_mean[k]);
        ysum += ys;
        if (hrr) eb += hrr_c[b * K + k] * (ys - ibct_f(bcty[b * K + k]));
      }
    }
    if (hrr) {
      eb -= hrr_r[b];
      lh += eb * eb;
    }
    const float sgn = ysum > 1.0f ? 1.0f : (ysum < 1.0f ? -1.0f : 0.0f);
    if (mass) lm += fabsf(ysum - 1.0f);
    for (int k = 0; k < n_out_pad; ++k) {
      float g = 0.0f;
      if (k < K) {
        const float d = Up[b * n_out_pad + k] - Ut[b * n_out_pad + k];
        ld += d * d;
        g = cdata * d;
        if (mass || hrr) {
          const float ys = ibct_f(bcty[b * K + k] + Up[b * n_out_pad + k] * out_sd[k] + out_mean[k]);
          // dY*/du = Y*^(1 - lambda) sigma_k
          const float dys = (ys > 0.0f ? exp2f(0.9f * log2f(ys)) : 0.0f) * out_sd[k];
          float f = 0.0f;
          if (mass) f += w_mass / (float)B * sgn;
          if (hrr) f += w_hrr * 2.0f / (float)B * eb * hrr_c[b * K + k];
          g += f * dys;
        }
      }
      const bf16 gb = __float2bfloat16_rn(g);
      dU[b * n_out_pad + k] = gb;
      dUT[(int64_t)k * B + b] = gb;
    }
  }
  sh[0][threadIdx.x] = ld;
  sh[1][threadIdx.x] = lm;
  sh[2][threadIdx.x] = lh;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
      sh[2][threadIdx.x] += sh[2][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = sh[0][0] / (float)(B * K);
    part[3 * blockIdx.x + 1] = sh[1][0] / (float)B;
    part[3 * blockIdx.x + 2] = sh[2][0] / (float)B;
  }
}

__global__ void loss_final_kernel(int nb, const float* part, float w_data, float w_mass, float w_hrr, float* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float a = 0.0f, b = 0.0f, c = 0.0f;
    for (int i = 0; i < nb; ++i) {
      a += part[3 * i];
      b += part[3 * i + 1];
      c += part[3 * i + 2];
    }
    out[0] = w_data * a + w_mass * b + w_hrr * c;
    out[1] = a;
    out[2] = b;
    out[3] = c;
  }
}

// BF16 transpose [R, C] -> [C, R] through 32 x 33 shared tiles
__global__ void transpose_kernel(const bf16* in, int64_t R, int64_t C, bf16* out) {
  __shared__ bf16 t[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int64_t r = r0 + dy, c = c0 + threadIdx.x;
    t[dy][threadIdx.x] = (r < R && c < C) ? in[r * C + c] : __float2bfloat16_rn(0.0f);
  }
  __syncthreads();
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int64_t c = c0 + dy, r = r0 + threadIdx.x;
    if (c < C && r < R) out[c * R + r] = t[threadIdx.x][dy];
  }
}

// column sums of the first N columns of a BF16 [B, ld] matrix (bias gradients), one thread per
// column, fixed order
__global__ void colsum_kernel(const bf16* dZ, int64_t B, int N, int ld, float* out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  float s = 0.0f;
  for (int64_t b = 0; b < B; ++b) s += __bfloat162float(dZ[b * ld + c]);
  out[c] = s;
}

// position in the per-group transposes W^T [groups cols, ldt] of element i of W [groups gh, cols]
// (one group: the plain transpose [cols, rows])
__device__ __forceinline__ int64_t wt_index(int64_t i, int gh, int ldt, int cols) {
  const int64_t r = i / cols;
  const int c = (int)(i - r * cols);
  const int64_t g = r / gh;
  return (g * cols + c) * ldt + (r - g * gh);
}

// Adam (Kingma & Ba 2015) on FP32 masters; refreshes the BF16 copy and its transpose
__global__ void adam_kernel(int64_t n, int gh, int ldt, int cols, float* w, const float* g, float* mom, float* vel,
                            float lr, float b1, float b2, float eps, float bc1, float bc2, bf16* wb, bf16* wt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * mom[i] + (1.0f - b1) * gi;
    const float vi = b2 * vel[i] + (1.0f - b2) * gi * gi;
    mom[i] = mi;
    vel[i] = vi;
    const float wi = w[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    w[i] = wi;
    if (wb) {
      const bf16 q = __float2bfloat16_rn(wi);
      wb[i] = q;
      wt[wt_index(i, gh, ldt, cols)] = q;
    }
  }
}

__global__ void to_bf16_kernel(int64_t n, int gh, int ldt, int cols, const float* w, bf16* wb, bf16* wt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const bf16 q = __float2bfloat16_rn(w[i]);
    wb[i] = q;
    wt[wt_index(i, gh, ldt, cols)] = q;
  }
}

// Seeded permutation of 0..n-1 for the epoch's minibatch order, without a table: a 4-round
// Feistel network (a bijection) on the smallest domain 2^(2 hb) >= n, with cycle walking (apply
// it again until the value falls below n; the walk stays on the cycle through the start, so it
// ends, on average after fewer than 4 rounds since the domain is below 4 n; the bound only keeps
// the loop finite).  Round function: a 64-bit finaliser (splitmix64's) of (half, key, round).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ int64_t epoch_perm(int64_t i, int64_t n, int hb, uint64_t key) {
  const uint64_t mask = (1ull << hb) - 1ull;
  uint64_t x = (uint64_t)i;
  for (int walk = 0; walk < 4096; ++walk) {
    uint64_t L = x >> hb, R = x & mask;
    for (int r = 0; r < 4; ++r) {
      const uint64_t F = mix64(R ^ (key + 0x9E3779B97F4A7C15ull * (uint64_t)(r + 1))) & mask;
      const uint64_t t = R;
      R = L ^ F;
      L = t;
    }
    x = (L << hb) | R;
    if (x < (uint64_t)n) return (int64_t)x;
  }
  return i;   // not reached for a domain below 4 n (probability < (3/4)^4096)
}

__global__ void epoch_order_kernel(int64_t n, int hb, uint64_t key, int32_t* order) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    order[i] = (int32_t)epoch_perm(i, n, hb, key);
}

// rows r0 .. r0 + B - 1 of the epoch's order gathered into contiguous minibatch buffers
__global__ void gather_batch_kernel(int64_t n, int hb, uint64_t key, int64_t r0, int64_t B, const bf16* X,
                                    const float* Ut, int n_out_pad, const float* bcty, const float* hc, const float* hr,
                                    int K, bf16* Xb, float* Utb, float* bctyb, float* hcb, float* hrb) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < B; b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t src = epoch_perm(r0 + b, n, hb, key);
    const uint4* xs = (const uint4*)(X + (size_t)src * kInPad);
    uint4* xd = (uint4*)(Xb + (size_t)b * kInPad);
#pragma unroll
    for (int q = 0; q < kInPad / 8; ++q) xd[q] = xs[q];
    for (int k = 0; k < n_out_pad; ++k) Utb[(size_t)b * n_out_pad + k] = Ut[(size_t)src * n_out_pad + k];
    if (bcty)
      for (int k = 0; k < K; ++k) bctyb[(size_t)b * K + k] = bcty[(size_t)src * K + k];
    if (hc) {
      for (int k = 0; k < K; ++k) hcb[(size_t)b * K + k] = hc[(size_t)src * K + k];
      hrb[b] = hr[src];
    }
  }
}

// epoch mean of the per-step losses: acc[0..3] += step[0..3] (acc zeroed first); scale at the end
__global__ void loss_accumulate_kernel(const float* step, float* acc, float scale, int finish, float* out) {
  if (threadIdx.x < 4 && blockIdx.x == 0) {
    const float v = acc[threadIdx.x] + step[threadIdx.x];
    acc[threadIdx.x] = v;
    if (finish && out) out[threadIdx.x] = v * scale;
  }
}

int grid_for(int64_t n, int threads) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, (int64_t)sms * 32));
}

// ------------------------------------------------------------------------------------------
// host helpers
// ------------------------------------------------------------------------------------------
uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

double normal01(uint64_t& s) {
  // Box-Muller on two uniforms in (0, 1]
  const double u1 = ((splitmix64(s) >> 11) + 1.0) * (1.0 / 9007199254740992.0);
  const double u2 = ((splitmix64(s) >> 11) + 1.0) * (1.0 / 9007199254740992.0);
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

// defaults of the learned step's options (chem_ann_opts fields <= 0 or NaN select them)
void ann_fill_defaults(chem_ann_opts& o) {
  if (!(o.range_margin >= 0)) o.range_margin = 0.05;
  if (!(o.elem_tol > 0)) o.elem_tol = 1e-2;
  if (!(o.T_min > 0)) o.T_min = 250.0;
  if (!(o.T_max > 0)) o.T_max = 3500.0;
  di_fill_defaults(o.di);
}

int check_ann(chem_ann a) {
  if (!a || !a->dmem) return set_error(CHEM_E_ARG, "null or freed ANN handle");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != a->device) return set_error(CHEM_E_ARG, "ANN was created on another device");
  return CHEM_OK;
}


// parameter rows of layer l (all groups) and the width of its output activations
int rows_of(const chem_ann_s* a, int l) { return a->groups * a->dims[l + 1]; }
int width_of(const chem_ann_s* a, int l) { return l == a->L - 1 ? a->n_out_pad : rows_of(a, l); }
// row length of the per-group transposed weights W_l^T [groups dims[l], ldt]
int ldt_of(const chem_ann_s* a, int l) { return (a->dims[l + 1] + 7) & ~7; }

// training scratch for a batch of B rows
struct TrainBufs {
  bf16 *Z[kMaxLayers], *A[kMaxLayers], *AT[kMaxLayers], *dZ[kMaxLayers], *dZT[kMaxLayers];
  float* Up;
};

size_t train_bytes(const chem_ann_s* a, int64_t B) {
  size_t s = 0;
  for (int l = 0; l < a->L; ++l) {
    const size_t w = (size_t)width_of(a, l);
    s += 5 * B * w * 2 + 5 * 256;       // Z, A, AT, dZ, dZT
  }
  s += (size_t)B * kInPad * 2 + 256;   // XT
  s += (size_t)B * a->n_out_pad * 4 + 256;
  // minibatch staging of chem_ann_train_epoch: X, Ut, bcty, hrr_c, hrr_r, loss sums
  s += (size_t)B * kInPad * 2 + (size_t)B * a->n_out_pad * 4 + 2 * (size_t)B * a->K * 4 + (size_t)B * 4 + 6 * 256;
  return s;
}

// the staging block of chem_ann_train_epoch at the end of the training buffers
struct EpochBufs {
  bf16* X;
  float *Ut, *bcty, *hc, *hr, *acc;
};

EpochBufs epoch_bufs(const chem_ann_s* a, int64_t B) {
  const size_t stage = (size_t)B * kInPad * 2 + (size_t)B * a->n_out_pad * 4 + 2 * (size_t)B * a->K * 4 +
                       (size_t)B * 4 + 6 * 256;
  char* w = (char*)a->tmem_ + train_bytes(a, a->tcap) - stage;
  size_t off = 0;
  auto take = [&](size_t bytes) { void* p = w + off; off = (off + bytes + 255) & ~size_t(255); return p; };
  EpochBufs e;
  e.X = (bf16*)take((size_t)B * kInPad * 2);
  e.Ut = (float*)take((size_t)B * a->n_out_pad * 4);
  e.bcty = (float*)take((size_t)B * a->K * 4);
  e.hc = (float*)take((size_t)B * a->K * 4);
  e.hr = (float*)take((size_t)B * 4);
  e.acc = (float*)take(8 * sizeof(float));   // epoch sums [4], last step [4]
  return e;
}

}  // namespace

// ------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------
static int ann_create(chem_mech mech, const int* hidden, int n_hidden, uint64_t seed, bool per_species,
                      chem_ann* out) {
  if (!mech || !hidden || n_hidden < 1 || n_hidden > kMaxLayers - 1 || !out)
    return set_error(CHEM_E_ARG, "chem_ann_create: bad arguments");
  *out = nullptr;
  chem_ann_s* a = new chem_ann_s();
  a->mech = mech;
  a->dm = mech_dev(mech);
  a->K = a->dm.K;
  a->n_in = a->K + 2;
  if (a->n_in > kInPad) { delete a; return set_error(CHEM_E_UNSUPPORTED, "chem_ann_create: more than 62 species"); }
  a->n_out = a->K;
  a->n_out_pad = a->K <= 32 ? 32 : 64;
  a->groups = per_species ? a->K : 1;
  a->L = n_hidden + 1;
  a->dims[0] = kInPad;
  // hidden widths are stored rounded up to a multiple of 8 (16-byte rows for the TMA loads);
  // the extra units start with zero weights and biases, so their activations, gradients and
  // Adam updates stay exactly zero and the network is the one with the requested widths
  int real[kMaxLayers + 1] = {0};
  real[0] = a->n_in;
  for (int l = 0; l < n_hidden; ++l) {
    if (hidden[l] < 1 || hidden[l] > 8192) {
      delete a;
      return set_error(CHEM_E_ARG, "chem_ann_create: hidden widths must be in [1, 8192]");
    }
    a->dims[l + 1] = (hidden[l] + 7) & ~7;
    real[l + 1] = hidden[l];
  }
  real[a->L] = per_species ? 1 : a->n_out;
  a->dims[a->L] = per_species ? 1 : a->n_out_pad;

  int rc = cuda_check(cudaGetDevice(&a->device), "cudaGetDevice");
  if (rc) { delete a; return rc; }
  // parameter-sized memory: masters, grads, Adam m/v (FP32) and BF16 W, W^T per layer
  size_t total = 0;
  std::vector<size_t> off;
  auto take = [&](size_t bytes) { off.push_back(total); total += (bytes + 255) & ~size_t(255); };
  for (int l = 0; l < a->L; ++l) {
    const size_t nw = (size_t)rows_of(a, l) * a->dims[l], nb = rows_of(a, l);
    for (int t = 0; t < 4; ++t) { take(nw * 4); take(nb * 4); }   // master, grad, m, v
    take(nw * 2);
    take((size_t)a->groups * a->dims[l] * ldt_of(a, l) * 2);
    a->n_params += (int64_t)(nw + nb);
  }
  take((size_t)(4 * a->n_in + 2 * a->n_out) * 4);   // normalisation
  take(64);                                           // error flag
  take(4096 * 8);                                     // loss partials
  if (cudaMalloc(&a->dmem, total) != cudaSuccess) {
    cudaGetLastError();
    delete a;
    return set_error(CHEM_E_NOMEM, "chem_ann_create: cudaMalloc failed");
  }
  cudaMemset(a->dmem, 0, total);
  char* b = (char*)a->dmem;
  size_t q = 0;
  for (int l = 0; l < a->L; ++l) {
    a->Wm[l] = (float*)(b + off[q++]); a->bm[l] = (float*)(b + off[q++]);
    a->gW[l] = (float*)(b + off[q++]); a->gb[l] = (float*)(b + off[q++]);
    a->mW[l] = (float*)(b + off[q++]); a->mb[l] = (float*)(b + off[q++]);
    a->vW[l] = (float*)(b + off[q++]); a->vb[l] = (float*)(b + off[q++]);
    a->W[l] = (bf16*)(b + off[q++]); a->WT[l] = (bf16*)(b + off[q++]);
  }
  a->norm = (float*)(b + off[q++]);
  a->err = (int*)(b + off[q++]);
  a->loss_part = (float*)(b + off[q++]);
  // initial weights: N(0, 2/fan_in) on the real (unpadded) inputs, units and outputs of every
  // group, zero biases and zero padding
  uint64_t st = seed * 0x9E3779B97F4A7C15ull + 12345;
  for (int l = 0; l < a->L; ++l) {
    const int gh = a->dims[l + 1], rows = rows_of(a, l), cols = a->dims[l];
    const int real_cols = real[l], real_rows = real[l + 1];
    std::vector<float> w((size_t)rows * cols, 0.0f);
    const double sd = std::sqrt(2.0 / real_cols) * (l == a->L - 1 ? 0.5 : 1.0);
    for (int g = 0; g < a->groups; ++g)
      for (int r = 0; r < real_rows; ++r)
        for (int c = 0; c < real_cols; ++c) w[((size_t)g * gh + r) * cols + c] = (float)(sd * normal01(st));
    cudaMemcpy(a->Wm[l], w.data(), w.size() * 4, cudaMemcpyHostToDevice);
    to_bf16_kernel<<<grid_for((int64_t)w.size(), 256), 256>>>((int64_t)w.size(), gh, ldt_of(a, l), cols, a->Wm[l],
                                                             a->W[l], a->WT[l]);
  }
  // identity normalisation until chem_ann_set_norm / chem_ann_fit_norm
  a->hnorm.assign((size_t)4 * a->n_in + 2 * a->n_out, 0.0f);
  for (int j = 0; j < a->n_in; ++j) {
    a->hnorm[a->n_in + j] = 1.0f;
    a->hnorm[2 * a->n_in + j] = -3e38f;
    a->hnorm[3 * a->n_in + j] = 3e38f;
  }
  for (int k = 0; k < a->n_out; ++k) a->hnorm[4 * a->n_in + a->n_out + k] = 1.0f;
  cudaMemcpy(a->norm, a->hnorm.data(), a->hnorm.size() * 4, cudaMemcpyHostToDevice);
  if ((rc = cuda_check(cudaDeviceSynchronize(), "chem_ann_create"))) {
    cudaFree(a->dmem);
    delete a;
    return rc;
  }
  *out = a;
  return CHEM_OK;
}

extern "C" {

int chem_ann_create(chem_mech mech, const int* hidden, int n_hidden, uint64_t seed, chem_ann* out) {
  return ann_create(mech, hidden, n_hidden, seed, false, out);
}

int chem_ann_create_per_species(chem_mech mech, const int* hidden, int n_hidden, uint64_t seed, chem_ann* out) {
  return ann_create(mech, hidden, n_hidden, seed, true, out);
}

int chem_ann_layout(chem_ann a, int* groups, int* n_out_pad) {
  if (!a) return set_error(CHEM_E_ARG, "null ANN handle");
  if (groups) *groups = a->groups;
  if (n_out_pad) *n_out_pad = a->n_out_pad;
  return CHEM_OK;
}

void chem_ann_free(chem_ann a) {
  if (!a) return;
  if (a->tmem_) cudaFree(a->tmem_);
  if (a->dmem) cudaFree(a->dmem);
  a->dmem = nullptr;
  delete a;
}

int chem_ann_info(chem_ann a, int* n_in, int* n_out, int* n_layers, int* dims, int64_t* n_params) {
  if (!a) return set_error(CHEM_E_ARG, "null ANN handle");
  if (n_in) *n_in = a->n_in;
  if (n_out) *n_out = a->n_out;
  if (n_layers) *n_layers = a->L;
  if (dims)
    for (int l = 0; l <= a->L; ++l) dims[l] = a->dims[l];
  if (n_params) *n_params = a->n_params;
  return CHEM_OK;
}

int chem_ann_set_norm(chem_ann a, const float* host_norm) {
  int rc = check_ann(a);
  if (rc) return rc;
  if (!host_norm) return set_error(CHEM_E_ARG, "chem_ann_set_norm: null");
  std::vector<float> v(host_norm, host_norm + a->hnorm.size());
  for (int j = 0; j < a->n_in; ++j)
    if (!(v[a->n_in + j] > 0)) v[a->n_in + j] = 1.0f;
  for (int k = 0; k < a->n_out; ++k)
    if (!(v[4 * a->n_in + a->n_out + k] > 0)) v[4 * a->n_in + a->n_out + k] = 1.0f;
  a->hnorm = v;
  return cuda_check(cudaMemcpy(a->norm, v.data(), v.size() * 4, cudaMemcpyHostToDevice), "chem_ann_set_norm");
}

int chem_ann_get_norm(chem_ann a, float* host_norm) {
  if (!a || !host_norm) return set_error(CHEM_E_ARG, "chem_ann_get_norm: null");
  std::memcpy(host_norm, a->hnorm.data(), a->hnorm.size() * 4);
  return CHEM_OK;
}

int chem_ann_fit_norm(chem_ann a, int64_t n, int64_t ld, const double* T, const double* p, const double* Y0,
                      const double* Y1, chem_stream stream) {
  int rc = check_ann(a);
  if (rc) return rc;
  if (n < 2 || ld < n || !T || !p || !Y0 || !Y1) return set_error(CHEM_E_ARG, "chem_ann_fit_norm: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  const int C = a->n_in + a->K;
  const int nb = (int)std::min<int64_t>((n + kStatBlock - 1) / kStatBlock, 1024);
  double* part = nullptr;
  if ((rc = cuda_check(cudaMallocAsync((void**)&part, (size_t)nb * C * 4 * 8, s), "fit_norm alloc"))) return rc;
  stats_partial_kernel<<<nb, kStatBlock, 0, s>>>(n, ld, T, p, Y0, Y1, a->n_in, a->K, part);
  std::vector<double> hp((size_t)nb * C * 4);
  rc = cuda_check(cudaMemcpyAsync(hp.data(), part, hp.size() * 8, cudaMemcpyDeviceToHost, s), "fit_norm copy");
  if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "fit_norm sync");
  cudaFreeAsync(part, s);
  if (rc) return rc;
  std::vector<float> v(a->hnorm.size());
  for (int c = 0; c < C; ++c) {
    double sm = 0, sq = 0, lo = 1e300, hi = -1e300;
    for (int b = 0; b < nb; ++b) {
      const double* q = &hp[((size_t)b * C + c) * 4];
      sm += q[0];
      sq += q[1];
      lo = std::min(lo, q[2]);
      hi = std::max(hi, q[3]);
    }
    const double mean = sm / n, var = std::max(sq / n - mean * mean, 0.0);
    const double sd = std::sqrt(var) > 1e-12 * std::max(1.0, std::fabs(mean)) ? std::sqrt(var) : 1.0;
    if (c < a->n_in) {
      v[c] = (float)mean;
      v[a->n_in + c] = (float)sd;
      v[2 * a->n_in + c] = (float)lo;
      v[3 * a->n_in + c] = (float)hi;
    } else {
      const int k = c - a->n_in;
      v[4 * a->n_in + k] = (float)mean;
      v[4 * a->n_in + a->n_out + k] = (float)sd;
    }
  }
  return chem_ann_set_norm(a, v.data());
}

int chem_ann_features(chem_ann a, int64_t n, int64_t ld, const double* T, const double* p, const double* Y, void* X,
                      float* bcty, double range_margin, int32_t* flags, chem_stream stream) {
  int rc = check_ann(a);
  if (rc) return rc;
  if (n < 0 || ld < n || (n > 0 && (!T || !p || !Y || !X))) return set_error(CHEM_E_ARG, "chem_ann_features: bad arguments");
  if (flags && !(range_margin >= 0.0)) return set_error(CHEM_E_ARG, "chem_ann_features: range_margin must be >= 0");
  if (n == 0) return CHEM_OK;
  features_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(n, ld, T, p, Y, a->n_in, a->norm,
                                                                     (float)range_margin, (bf16*)X, flags, bcty,
                                                                     a->K, nullptr);
  return cuda_check(cudaGetLastError(), "features_kernel launch");
}

int chem_ann_update(chem_ann a, int64_t n, int64_t ld, double* T, const double* p, double* Y, const float* U,
                    const int32_t* idx, const chem_ann_opts* opts, int32_t* flags, int32_t* status,
                    chem_stream stream) {
  int rc = check_ann(a);
  if (rc) return rc;
  if (n < 0 || ld < n) return set_error(CHEM_E_ARG, "chem_ann_update: need 0 <= n <= ld");
  if (n == 0) return CHEM_OK;
  if (!T || !p || !Y || !U || !flags || !status) return set_error(CHEM_E_ARG, "chem_ann_update: null array");
  chem_ann_opts o{};
  if (opts) o = *opts;
  ann_fill_defaults(o);
  const float* om = a->norm + 4 * a->n_in;
  return launch_update(a->dm, n, ld, T, p, Y, U, a->n_out_pad, om, om + a->n_out, flags, status, (float)o.elem_tol,
                       (float)o.T_min, (float)o.T_max, (float)o.dT_max, idx, (cudaStream_t)stream);
}

int chem_ann_targets(chem_ann a, int64_t n, int64_t ld, const double* Y0, const double* Y1, float* U,
                     chem_stream stream) {
  int rc = check_ann(a);
  if (rc) return rc;
  if (n < 0 || ld < n || (n > 0 && (!Y0 || !Y1 || !U))) return set_error(CHEM_E_ARG, "chem_ann_targets: bad arguments");
  if (n == 0) return CHEM_OK;
  const float* om = a->norm + 4 * a->n_in;
  targets_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(n, ld, Y0, Y1, a->K, a->n_out_pad, om,
                                                                    om + a->n_out, U);
  return cuda_check(cudaGetLastError(), "targets_kernel launch");
}

int chem_ann_hrr_coeffs(chem_ann a, int64_t n, int64_t ld, const double* T0, const double* p, const double* Y0,
                        const double* Y1, double dt, double scale, float* hrr_c, float* hrr_r, chem_stream stream) {
  int rc = check_ann(a);
  if (rc) return rc;
  if (n < 0 || ld < n) return set_error(CHEM_E_ARG, "chem_ann_hrr_coeffs: need 0 <= n <= ld");
  if (!(dt > 0.0) || !(scale > 0.0)) return set_error(CHEM_E_ARG, "chem_ann_hrr_coeffs: dt and scale must be positive");
  if (n == 0) return CHEM_OK;
  if (!T0 || !p || !Y0 || !Y1 || !hrr_c || !hrr_r) return set_error(CHEM_E_ARG, "chem_ann_hrr_coeffs: null array");
  hrr_coeff_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(a->dm, n, ld, T0, p, Y0, Y1, dt, scale,
                                                                      hrr_c, hrr_r);
  return cuda_check(cudaGetLastError(), "hrr_coeff_kernel launch");
}

// forward pass over rows [0, M) of X (BF16 [M, 64]) into U (FP32 [M, n_out_pad]), through
// BF16 activation buffers act[l] ([M, width_of(l)]); optionally keeping pre-activations zs[l].
// Per-species networks: the first layer is one GEMM over all species' units (shared input),
// every later layer one launch of `groups` GEMMs, species g reading its own slice of the
// previous activations and writing its own slice (the output layer: column g of U).
static int forward_rows(chem_ann a, const bf16* X, int64_t M, bf16* const* act, bf16* const* zs, float* U,
                        cudaStream_t s) {
  int rc;
  const bf16* in = X;
  int64_t ld_in = kInPad;
  for (int l = 0; l < a->L; ++l) {
    const int Kd = a->dims[l];
    const bool grouped = a->groups > 1 && l > 0;
    const int N = grouped ? a->dims[l + 1] : rows_of(a, l);
    GemmEpi e{};
    e.bias = a->bm[l];
    if (grouped) {
      e.groups = a->groups;
      e.a_col = Kd;
      e.b_row = N;
      e.out_goff = N;
      e.bias_goff = N;
    }
    const bool last = l == a->L - 1;
    // the per-species output layer writes columns 0..K-1 of U; the padding columns read zero,
    // as the one-network output layer's zero padding rows give
    if (last && grouped &&
        (rc = cuda_check(cudaMemsetAsync(U, 0, (size_t)M * a->n_out_pad * sizeof(float), s), "U padding")))
      return rc;
    e.out = last ? (void*)U : (void*)act[l];
    e.ldo = width_of(a, l);
    e.zout = (!last && zs) ? zs[l] : nullptr;
    if ((rc = gemm_bf16(last ? 1 : 0, in, ld_in, a->W[l], Kd, (int)M, N, Kd, e, a->err, s))) return rc;
    in = act[l];
    ld_in = width_of(a, l);
  }
  return CHEM_OK;
}

// rows of the activation chunk used by inference. One network: 262144 rows (1.5 GB of BF16
// activations for the 1600-800-400 hidden layers); fewer, longer GEMM launches drain their
// last wave of tiles less often, which outweighs keeping the chunk in L2. Per-species
// networks: as many rows as keep the widest activation chunk near 400 MB, at most 32768.
static int64_t infer_chunk(const chem_ann_s* a) {
  if (a->groups == 1) return 262144;
  int wmax = 1;
  for (int l = 0; l < a->L - 1; ++l) wmax = std::max(wmax, width_of(a, l));
  const int64_t rows = ((int64_t)400 * 1024 * 1024 / (2 * (int64_t)wmax)) & ~(int64_t)127;
  return std::min<int64_t>(32768, std::max<int64_t>(128, rows));
}

size_t chem_ann_workspace_bytes(chem_ann a, int64_t n) {
  if (!a || n < 0) return 0;
  const int64_t mc = std::min<int64_t>(std::max<int64_t>(n, 1), infer_chunk(a));
  size_t s = 0;
  s += (size_t)n * kInPad * 2 + 256;                 // X
  s += (size_t)n * a->n_out_pad * 4 + 256;           // U
  for (int l = 0; l < a->L - 1; ++l) s += (size_t)mc * width_of(a, l) * 2 + 256;
  s += 4 * ((size_t)n * 4 + 256);                     // flags, slots, cell columns, DI slot status
  s += ((size_t)(n / kCompactBlock + 2) * 4 + 256) + 256 + 256;   // block counts, total, queue
  return s;
}

int chem_ann_forward(chem_ann a, const void* X, int64_t n, float* U, void* workspace, size_t ws_bytes,
                     chem_stream stream) {
  int rc = check_ann(a);
  if (rc) return rc;
  if (n < 0 || (n > 0 && (!X || !U))) return set_error(CHEM_E_ARG, "chem_ann_forward: bad arguments");
  if (n == 0) return CHEM_OK;
  if (!workspace || ws_bytes < chem_ann_workspace_bytes(a, n))
    return set_error(CHEM_E_WORKSPACE, "chem_ann_forward: workspace smaller than chem_ann_workspace_bytes()");
  const int64_t mc = std::min<int64_t>(n, infer_chunk(a));
  char* w = (char*)workspace;
  bf16* act[kMaxLayers];
  size_t o = (size_t)n * kInPad * 2 + 256 + (size_t)n * a->n_out_pad * 4 + 256;
  for (int l = 0; l < a->L - 1; ++l) {
    act[l] = (bf16*)(w + ((o + 255) & ~size_t(255)));
    o = ((o + 255) & ~size_t(255)) + (size_t)mc * width_of(a, l) * 2;
  }
  for (int64_t r0 = 0; r0 < n; r0 += mc) {
    const int64_t m = std::min(mc, n - r0);
    if ((rc = forward_rows(a, (const bf16*)X + r0 * kInPad, m, act, nullptr, U + r0 * a->n_out_pad,
                           (cudaStream_t)stream)))
      return rc;
  }
  return CHEM_OK;
}

int chem_ann_error(chem_ann a, int* host_err) {
  if (!a || !host_err) return set_error(CHEM_E_ARG, "chem_ann_error: null");
  int rc = cuda_check(cudaMemcpy(host_err, a->err, sizeof(int), cudaMemcpyDeviceToHost), "chem_ann_error");
  if (!rc) cudaMemset(a->err, 0, sizeof(int));
  return rc;
}

int chem_step_ann(chem_mech mech, chem_ann a, int64_t n, int64_t ld, double dt, double* T, const double* p,
                  double* Y, const int32_t* idx_in, const chem_ann_opts* opts, int32_t* status, void* workspace,
                  size_t ws_bytes, chem_stream stream) {
  int rc = check_ann(a);
  if (rc) return rc;
  if (!mech || mech != a->mech) return set_error(CHEM_E_ARG, "chem_step_ann: the ANN belongs to another mechanism");
  if (n < 0 || ld < n) return set_error(CHEM_E_ARG, "chem_step_ann: need 0 <= n <= ld");
  if (n == 0) return CHEM_OK;
  if (!T || !p || !Y || !status) return set_error(CHEM_E_ARG, "chem_step_ann: null array");
  if (n > (int64_t)0x7fffffff) return set_error(CHEM_E_ARG, "chem_step_ann: too many cells");
  if (!workspace || ws_bytes < chem_ann_workspace_bytes(a, n))
    return set_error(CHEM_E_WORKSPACE, "chem_step_ann: workspace smaller than chem_ann_workspace_bytes()");
  chem_ann_opts o{};
  if (opts) o = *opts;
  ann_fill_defaults(o);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t mc = std::min<int64_t>(n, infer_chunk(a));
  char* w = (char*)workspace;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  size_t off = 0;
  bf16* X = (bf16*)(w + off);
  off = al(off + (size_t)n * kInPad * 2);
  float* U = (float*)(w + off);
  off = al(off + (size_t)n * a->n_out_pad * 4);
  bf16* act[kMaxLayers];
  for (int l = 0; l < a->L - 1; ++l) {
    act[l] = (bf16*)(w + off);
    off = al(off + (size_t)mc * width_of(a, l) * 2);
  }
  int32_t* flags = (int32_t*)(w + off);
  off = al(off + (size_t)n * 4);
  int32_t* slots = (int32_t*)(w + off);
  off = al(off + (size_t)n * 4);
  int32_t* cols = (int32_t*)(w + off);
  off = al(off + (size_t)n * 4);
  int32_t* st_slot = (int32_t*)(w + off);
  off = al(off + (size_t)n * 4);
  const int nb = (int)((n + kCompactBlock - 1) / kCompactBlock);
  int32_t* blk = (int32_t*)(w + off);
  off = al(off + (size_t)(nb + 1) * 4);
  int32_t* nflag = (int32_t*)(w + off);
  off = al(off + 4);
  unsigned int* queue = (unsigned int*)(w + off);

  // 1. features and range flags
  features_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, ld, T, p, Y, a->n_in, a->norm, (float)o.range_margin, X, flags,
                                                  nullptr, a->K, idx_in);
  if ((rc = cuda_check(cudaGetLastError(), "features_kernel launch"))) return rc;
  // 2. MLP on the tensor cores, chunk by chunk
  for (int64_t r0 = 0; r0 < n; r0 += mc) {
    const int64_t m = std::min(mc, n - r0);
    if ((rc = forward_rows(a, X + r0 * kInPad, m, act, nullptr, U + r0 * a->n_out_pad, s))) return rc;
  }
  // 3. new state, checks
  const float* om = a->norm + 4 * a->n_in;
  if ((rc = launch_update(a->dm, n, ld, T, p, Y, U, a->n_out_pad, om, om + a->n_out, flags, status,
                          (float)o.elem_tol, (float)o.T_min, (float)o.T_max, (float)o.dT_max, idx_in, s)))
    return rc;
  if (!o.no_fallback) {
    // 4. compaction of flagged cells (deterministic order) and direct integration of those
    compact_count_kernel<<<nb, kCompactBlock, 0, s>>>(n, status, blk);
    compact_scan_kernel<<<1, 32, 0, s>>>(nb, blk, nflag);
    compact_write_kernel<<<nb, kCompactBlock, 0, s>>>(n, status, blk, slots, cols, idx_in);
    if ((rc = cuda_check(cudaMemsetAsync(queue, 0, 4, s), "queue reset"))) return rc;
    if ((rc = launch_di(a->dm, n, ld, dt, T, p, Y, cols, o.di, st_slot, nullptr, queue, s, nflag))) return rc;
    scatter_status_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, nflag, slots, st_slot, status);
    if ((rc = cuda_check(cudaGetLastError(), "fallback launch"))) return rc;
  }
  return CHEM_OK;
}

// training buffers for minibatches of up to B rows (library-owned, grown on demand)
static int ensure_train_bufs(chem_ann a, int64_t B, cudaStream_t s) {
  if (B <= a->tcap) return CHEM_OK;
  if (a->tmem_) { cudaStreamSynchronize(s); cudaFree(a->tmem_); a->tmem_ = nullptr; a->tcap = 0; }
  if (cudaMalloc(&a->tmem_, train_bytes(a, B)) != cudaSuccess) {
    cudaGetLastError();
    return set_error(CHEM_E_NOMEM, "chem_ann_train: cudaMalloc of training buffers failed");
  }
  a->tcap = B;
  return CHEM_OK;
}

// one optimisation step on a contiguous minibatch (buffers already sized for B)
static int train_step_impl(chem_ann a, const bf16* X, const float* Ut, const float* bcty, const float* hrr_c,
                           const float* hrr_r, int64_t B, const chem_train_opts* opts, float* loss_out,
                           cudaStream_t s) {
  int rc;
  // carve training buffers
  TrainBufs t{};
  char* w = (char*)a->tmem_;
  size_t off = 0;
  auto take = [&](size_t bytes) { void* p = w + off; off = (off + bytes + 255) & ~size_t(255); return p; };
  for (int l = 0; l < a->L; ++l) {
    const size_t n = (size_t)B * width_of(a, l);
    t.Z[l] = (bf16*)take(n * 2);
    t.A[l] = (bf16*)take(n * 2);
    t.AT[l] = (bf16*)take(n * 2);
    t.dZ[l] = (bf16*)take(n * 2);
    t.dZT[l] = (bf16*)take(n * 2);
  }
  bf16* XT = (bf16*)take((size_t)B * kInPad * 2);
  t.Up = (float*)take((size_t)B * a->n_out_pad * 4);
  // forward (pre-activations kept for GELU')
  bf16* act[kMaxLayers];
  bf16* zs[kMaxLayers];
  for (int l = 0; l < a->L; ++l) { act[l] = t.A[l]; zs[l] = t.Z[l]; }
  if ((rc = forward_rows(a, X, B, act, zs, t.Up, s))) return rc;
  // loss and dU
  const float* om = a->norm + 4 * a->n_in;
  const int nbl = (int)std::min<int64_t>((B + 255) / 256, 2048);
  const int Lo = a->L - 1;
  loss_grad_kernel<<<nbl, 256, 0, s>>>(B, a->K, a->n_out_pad, t.Up, Ut, bcty, om, om + a->n_out, opts->w_data,
                                      opts->w_mass, hrr_c, hrr_r, opts->w_hrr, t.dZ[Lo], t.dZT[Lo], a->loss_part);
  if (loss_out)
    loss_final_kernel<<<1, 32, 0, s>>>(nbl, a->loss_part, opts->w_data, opts->w_mass, opts->w_hrr, loss_out);
  // backward
  dim3 tb(32, 8);
  const int G = a->groups;
  for (int l = Lo; l >= 0; --l) {
    const int Kd = a->dims[l], wl = width_of(a, l);
    const bool grouped = G > 1 && l > 0;
    const int Ng = a->dims[l + 1];
    // input activations of layer l, transposed: [width, B]
    const bf16* inT;
    if (l == 0) {
      transpose_kernel<<<dim3((kInPad + 31) / 32, (unsigned)((B + 31) / 32)), tb, 0, s>>>(X, B, kInPad, XT);
      inT = XT;
    } else {
      const int win = width_of(a, l - 1);
      transpose_kernel<<<dim3((unsigned)((win + 31) / 32), (unsigned)((B + 31) / 32)), tb, 0, s>>>(t.A[l - 1], B, win,
                                                                                                   t.AT[l - 1]);
      inT = t.AT[l - 1];
    }
    if (l != Lo)
      transpose_kernel<<<dim3((unsigned)((wl + 31) / 32), (unsigned)((B + 31) / 32)), tb, 0, s>>>(t.dZ[l], B, wl, t.dZT[l]);
    // dW_l [rows, Kd] = dZ_l^T [rows, B] (A_{l-1}^T [Kd, B])^T, per species for grouped layers
    GemmEpi e{};
    e.out = a->gW[l];
    e.ldo = Kd;
    if (grouped) {
      e.groups = G;
      e.a_row = Ng;
      e.b_row = Kd;
      e.out_goff = (int64_t)Ng * Kd;
      if ((rc = gemm_bf16(3, t.dZT[l], B, inT, B, Ng, Kd, (int)B, e, a->err, s))) return rc;
    } else if ((rc = gemm_bf16(3, t.dZT[l], B, inT, B, rows_of(a, l), Kd, (int)B, e, a->err, s))) {
      return rc;
    }
    colsum_kernel<<<(rows_of(a, l) + 127) / 128, 128, 0, s>>>(t.dZ[l], B, rows_of(a, l), wl, a->gb[l]);
    if (l == 0) continue;
    // dZ_{l-1} = (dZ_l W_l) * GELU'(Z_{l-1}); B operand = W_l^T
    const int win = width_of(a, l - 1);
    if (!grouped) {
      GemmEpi e2{};
      e2.out = t.dZ[l - 1];
      e2.ldo = Kd;
      e2.z = t.Z[l - 1];
      e2.ldz = Kd;
      if ((rc = gemm_bf16(2, t.dZ[l], wl, a->WT[l], ldt_of(a, l), (int)B, Kd, rows_of(a, l), e2, a->err, s))) return rc;
    } else if (l == Lo) {
      // one output per species: dZ_{l-1}[b, g Kd + j] = dU[b, g] W[g, j] GELU'(Z)
      if ((rc = launch_group_out_dgrad(t.dZ[l], wl, a->W[l], t.Z[l - 1], B, G, Kd, t.dZ[l - 1], s))) return rc;
    } else {
      GemmEpi e2{};
      e2.out = t.dZ[l - 1];
      e2.ldo = win;
      e2.z = t.Z[l - 1];
      e2.ldz = win;
      e2.groups = G;
      e2.a_col = Ng;
      e2.b_row = Kd;
      e2.out_goff = Kd;
      e2.z_goff = Kd;
      if ((rc = gemm_bf16(2, t.dZ[l], wl, a->WT[l], ldt_of(a, l), (int)B, Kd, Ng, e2, a->err, s))) return rc;
    }
  }
  if ((rc = cuda_check(cudaGetLastError(), "training launches"))) return rc;
  if (!opts->apply) return CHEM_OK;
  // Adam
  a->step++;
  // bias corrections 1 - beta^t in FP64: in FP32, 1 - 0.999^t loses most of its digits to
  // cancellation for small t
  const float bc1 = (float)(1.0 - std::pow((double)opts->beta1, (double)a->step));
  const float bc2 = (float)(1.0 - std::pow((double)opts->beta2, (double)a->step));
  for (int l = 0; l < a->L; ++l) {
    const int rows = rows_of(a, l), cols = a->dims[l];
    const int64_t nw = (int64_t)rows * cols;
    adam_kernel<<<grid_for(nw, 256), 256, 0, s>>>(nw, a->dims[l + 1], ldt_of(a, l), cols, a->Wm[l], a->gW[l], a->mW[l],
                                                   a->vW[l], opts->lr, opts->beta1, opts->beta2, opts->eps, bc1, bc2,
                                                   a->W[l], a->WT[l]);
    adam_kernel<<<grid_for(rows, 256), 256, 0, s>>>(rows, 1, 1, 1, a->bm[l], a->gb[l], a->mb[l], a->vb[l], opts->lr,
                                                    opts->beta1, opts->beta2, opts->eps, bc1, bc2, nullptr, nullptr);
  }
  return cuda_check(cudaGetLastError(), "adam launch");
}

int chem_ann_train_step(chem_ann a, const void* Xv, const float* Ut, const float* bcty, const float* hrr_c,
                        const float* hrr_r, int64_t B, const chem_train_opts* opts, float* loss_out,
                        chem_stream stream) {
  int rc = check_ann(a);
  if (rc) return rc;
  if (B < 8 || B > (1 << 20) || B % 8 != 0 || !Xv || !Ut || !opts)
    return set_error(CHEM_E_ARG, "chem_ann_train_step: bad arguments (B must be a multiple of 8)");
  if (opts->w_hrr != 0.0f && (!bcty || !hrr_c || !hrr_r))
    return set_error(CHEM_E_ARG, "chem_ann_train_step: w_hrr != 0 needs bcty, hrr_c and hrr_r");
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = ensure_train_bufs(a, B, s))) return rc;
  return train_step_impl(a, (const bf16*)Xv, Ut, bcty, hrr_c, hrr_r, B, opts, loss_out, s);
}

// key of the minibatch order of (seed, epoch)
static uint64_t epoch_key(uint64_t seed, int epoch) {
  uint64_t st = seed * 0x9E3779B97F4A7C15ull ^ ((uint64_t)(uint32_t)epoch << 32);
  return splitmix64(st);
}

// half-width of the permutation domain: the smallest hb with 2^(2 hb) >= n
static int epoch_half_bits(int64_t n) {
  int hb = 1;
  while ((1ll << (2 * hb)) < n) ++hb;
  return hb;
}

int chem_ann_train_epoch(chem_ann a, const void* Xv, const float* Ut, const float* bcty, const float* hrr_c,
                         const float* hrr_r, int64_t n, const chem_train_epoch_opts* opts, float* loss_out,
                         chem_stream stream) {
  int rc = check_ann(a);
  if (rc) return rc;
  if (!opts || !Xv || !Ut) return set_error(CHEM_E_ARG, "chem_ann_train_epoch: null argument");
  const int64_t B = opts->batch;
  if (B < 8 || B > (1 << 20) || B % 8 != 0 || n < B || n > (int64_t)0x7fffffff)
    return set_error(CHEM_E_ARG, "chem_ann_train_epoch: need a batch that is a multiple of 8 in [8, 2^20] and "
                                 "batch <= n_samples <= 2^31 - 1");
  if (opts->step.w_hrr != 0.0f && (!bcty || !hrr_c || !hrr_r))
    return set_error(CHEM_E_ARG, "chem_ann_train_epoch: w_hrr != 0 needs bcty, hrr_c and hrr_r");
  if (opts->step.w_mass != 0.0f && !bcty)
    return set_error(CHEM_E_ARG, "chem_ann_train_epoch: w_mass != 0 needs bcty");
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = ensure_train_bufs(a, B, s))) return rc;
  const EpochBufs eb = epoch_bufs(a, B);
  const int64_t steps = n / B;
  const int64_t total = opts->total_steps > 0 ? opts->total_steps : steps;
  const int hb = epoch_half_bits(n);
  const uint64_t key = epoch_key(opts->seed, opts->epoch);
  const bool with_hrr = opts->step.w_hrr != 0.0f;
  if ((rc = cuda_check(cudaMemsetAsync(eb.acc, 0, 4 * sizeof(float), s), "chem_ann_train_epoch: loss sums"))) return rc;
  float* step_loss = eb.acc + 4;
  for (int64_t q = 0; q < steps; ++q) {
    gather_batch_kernel<<<grid_for(B, 128), 128, 0, s>>>(n, hb, key, q * B, B, (const bf16*)Xv, Ut, a->n_out_pad, bcty,
                                                        with_hrr ? hrr_c : nullptr, with_hrr ? hrr_r : nullptr, a->K,
                                                        eb.X, eb.Ut, eb.bcty, eb.hc, eb.hr);
    // cosine learning rate over the whole schedule
    chem_train_opts o = opts->step;
    const double t = std::min(1.0, (double)(opts->step0 + q) / (double)std::max<int64_t>(total - 1, 1));
    o.lr = (float)(opts->lr_min + 0.5 * ((double)opts->step.lr - opts->lr_min) * (1.0 + std::cos(M_PI * t)));
    if ((rc = train_step_impl(a, eb.X, eb.Ut, bcty ? eb.bcty : nullptr, with_hrr ? eb.hc : nullptr,
                              with_hrr ? eb.hr : nullptr, B, &o, step_loss, s)))
      return rc;
    loss_accumulate_kernel<<<1, 32, 0, s>>>(step_loss, eb.acc, 1.0f / (float)steps, q == steps - 1 ? 1 : 0, loss_out);
  }
  return cuda_check(cudaGetLastError(), "chem_ann_train_epoch launches");
}

int chem_selftest_epoch_order(int64_t n, uint64_t seed, int epoch, int32_t* order, chem_stream stream) {
  if (n < 1 || n > (int64_t)0x7fffffff || !order) return set_error(CHEM_E_ARG, "chem_selftest_epoch_order: bad arguments");
  epoch_order_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(n, epoch_half_bits(n), epoch_key(seed, epoch),
                                                                        order);
  return cuda_check(cudaGetLastError(), "epoch_order_kernel launch");
}

// parameters/gradients as one flat FP32 host array: per layer W [rows, dims[l]] then b [rows]
// (rows = groups dims[l+1], per-species networks stacked by species)
int chem_ann_get_params(chem_ann a, int which, float* host, int64_t count) {
  int rc = check_ann(a);
  if (rc) return rc;
  if (!host || count != a->n_params || which < 0 || which > 1) return set_error(CHEM_E_ARG, "chem_ann_get_params: bad arguments");
  cudaDeviceSynchronize();
  float* p = host;
  for (int l = 0; l < a->L; ++l) {
    const size_t nw = (size_t)rows_of(a, l) * a->dims[l], nb = rows_of(a, l);
    if ((rc = cuda_check(cudaMemcpy(p, which ? a->gW[l] : a->Wm[l], nw * 4, cudaMemcpyDeviceToHost), "get params"))) return rc;
    p += nw;
    if ((rc = cuda_check(cudaMemcpy(p, which ? a->gb[l] : a->bm[l], nb * 4, cudaMemcpyDeviceToHost), "get params"))) return rc;
    p += nb;
  }
  return CHEM_OK;
}

int chem_ann_set_params(chem_ann a, const float* host, int64_t count) {
  int rc = check_ann(a);
  if (rc) return rc;
  if (!host || count != a->n_params) return set_error(CHEM_E_ARG, "chem_ann_set_params: bad arguments");
  const float* p = host;
  for (int l = 0; l < a->L; ++l) {
    const int rows = rows_of(a, l), cols = a->dims[l];
    const size_t nw = (size_t)rows * cols;
    if ((rc = cuda_check(cudaMemcpy(a->Wm[l], p, nw * 4, cudaMemcpyHostToDevice), "set params"))) return rc;
    p += nw;
    if ((rc = cuda_check(cudaMemcpy(a->bm[l], p, rows * 4, cudaMemcpyHostToDevice), "set params"))) return rc;
    p += rows;
    to_bf16_kernel<<<grid_for((int64_t)nw, 256), 256>>>((int64_t)nw, a->dims[l + 1], ldt_of(a, l), cols, a->Wm[l],
                                                       a->W[l], a->WT[l]);
  }
  return cuda_check(cudaDeviceSynchronize(), "set params");
}

// checkpoint: header (species, layers, Adam step, normalisation size, flags: bit 0 Adam moments
// stored, bit 1 per-species networks), dims, normalisation, then masters and Adam moments
int chem_ann_save(chem_ann a, const char* path, int with_moments) {
  int rc = check_ann(a);
  if (rc) return rc;
  FILE* f = path ? std::fopen(path, "wb") : nullptr;
  if (!f) return set_error(CHEM_E_ARG, "chem_ann_save: cannot open file");
  cudaDeviceSynchronize();
  const char magic[8] = {'C', 'H', 'E', 'M', 'A', 'N', 'N', '2'};
  int hdr[5] = {a->K, a->L, a->step, (int)a->hnorm.size(), (with_moments ? 1 : 0) | (a->groups > 1 ? 2 : 0)};
  std::fwrite(magic, 1, 8, f);
  std::fwrite(hdr, 4, 5, f);
  std::fwrite(a->dims, 4, a->L + 1, f);
  std::fwrite(a->hnorm.data(), 4, a->hnorm.size(), f);
  for (int l = 0; l < a->L; ++l) {
    const size_t nw = (size_t)rows_of(a, l) * a->dims[l], nb = rows_of(a, l);
    const float* parts[6] = {a->Wm[l], a->bm[l], a->mW[l], a->mb[l], a->vW[l], a->vb[l]};
    const size_t sizes[6] = {nw, nb, nw, nb, nw, nb};
    for (int q = 0; q < (with_moments ? 6 : 2); ++q) {
      std::vector<float> h(sizes[q]);
      cudaMemcpy(h.data(), parts[q], sizes[q] * 4, cudaMemcpyDeviceToHost);
      std::fwrite(h.data(), 4, h.size(), f);
    }
  }
  const bool ok = std::ferror(f) == 0;
  std::fclose(f);
  return ok ? CHEM_OK : set_error(CHEM_E_ARG, "chem_ann_save: write failed");
}

int chem_ann_load(chem_mech mech, const char* path, chem_ann* out) {
  if (!mech || !path || !out) return set_error(CHEM_E_ARG, "chem_ann_load: bad arguments");
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return set_error(CHEM_E_ARG, std::string("chem_ann_load: cannot open ") + path);
  char magic[8];
  int hdr[5];
  if (std::fread(magic, 1, 8, f) != 8 || std::memcmp(magic, "CHEMANN2", 8) != 0 || std::fread(hdr, 4, 5, f) != 5 ||
      hdr[1] < 2 || hdr[1] > kMaxLayers) {
    std::fclose(f);
    return set_error(CHEM_E_PARSE, "chem_ann_load: not an ANN checkpoint");
  }
  int dims[kMaxLayers + 1];
  if (std::fread(dims, 4, hdr[1] + 1, f) != (size_t)hdr[1] + 1 || hdr[0] != mech_dev(mech).K) {
    std::fclose(f);
    return set_error(CHEM_E_PARSE, "chem_ann_load: checkpoint does not match the mechanism");
  }
  chem_ann a = nullptr;
  int rc = ann_create(mech, dims + 1, hdr[1] - 1, 0, (hdr[4] & 2) != 0, &a);
  if (rc) { std::fclose(f); return rc; }
  std::vector<float> norm(hdr[3]);
  bool ok = hdr[3] == (int)a->hnorm.size() && std::fread(norm.data(), 4, norm.size(), f) == norm.size();
  for (int l = 0; ok && l < a->L; ++l) {
    const size_t nw = (size_t)rows_of(a, l) * a->dims[l], nb = rows_of(a, l);
    float* parts[6] = {a->Wm[l], a->bm[l], a->mW[l], a->mb[l], a->vW[l], a->vb[l]};
    const size_t sizes[6] = {nw, nb, nw, nb, nw, nb};
    for (int q = 0; ok && q < ((hdr[4] & 1) ? 6 : 2); ++q) {   // without moments: Adam restarts from zero
      std::vector<float> h(sizes[q]);
      ok = std::fread(h.data(), 4, h.size(), f) == h.size();
      if (ok) cudaMemcpy(parts[q], h.data(), h.size() * 4, cudaMemcpyHostToDevice);
    }
    to_bf16_kernel<<<grid_for((int64_t)nw, 256), 256>>>((int64_t)nw, a->dims[l + 1], ldt_of(a, l), a->dims[l], a->Wm[l],
                                                       a->W[l], a->WT[l]);
  }
  std::fclose(f);
  if (!ok) { chem_ann_free(a); return set_error(CHEM_E_PARSE, "chem_ann_load: truncated checkpoint"); }
  a->step = hdr[2];
  if ((rc = chem_ann_set_norm(a, norm.data()))) { chem_ann_free(a); return rc; }
  *out = a;
  return cuda_check(cudaDeviceSynchronize(), "chem_ann_load");
}

}  // extern "C"
