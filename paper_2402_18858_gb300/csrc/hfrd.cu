// Random augmentation of training states by the hybrid flamelet/random data method (Sec. 2.2,
// Eqs. 3-6): temperature, pressure and N2 shifted by a random fraction of their data-set
// range, every other mass fraction raised to a random power near one, the result
// renormalised and filtered by the element-ratio and equivalence-ratio constraints.
//
// Two launches: one block reduces the data-set ranges of T, p and Y_N2 (min and max are
// order-independent, so the result is deterministic), then one thread per state applies
// Eqs. 3-6 in FP64 and writes the augmented state and its keep flag.  The random numbers are
// inputs (gamma), so the result is a pure function of the arguments.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdint>

#include "internal.h"

namespace chem {

__global__ void __launch_bounds__(1024) hfrd_ranges_kernel(int64_t n, const double* __restrict__ T,
                                                           const double* __restrict__ p,
                                                           const double* __restrict__ yn2, double* out) {
  __shared__ double red[6][32];
  double v[6] = {DBL_MAX, -DBL_MAX, DBL_MAX, -DBL_MAX, DBL_MAX, -DBL_MAX};
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double a = T[i], b = p[i], c = yn2[i];
    v[0] = fmin(v[0], a); v[1] = fmax(v[1], a);
    v[2] = fmin(v[2], b); v[3] = fmax(v[3], b);
    v[4] = fmin(v[4], c); v[5] = fmax(v[5], c);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    double x = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_down_sync(0xffffffffu, x, o);
      x = (q & 1) ? fmax(x, y) : fmin(x, y);
    }
    if (lane == 0) red[q][wid] = x;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      double x = lane < nw ? red[q][lane] : ((q & 1) ? -DBL_MAX : DBL_MAX);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double y = __shfl_down_sync(0xffffffffu, x, o);
        x = (q & 1) ? fmax(x, y) : fmin(x, y);
      }
      if (lane == 0) out[q] = x;
    }
  }
}

__global__ void __launch_bounds__(256) hfrd_kernel(DevMech m, int64_t n, int64_t ld, const double* __restrict__ T,
                                                  const double* __restrict__ p, const double* __restrict__ Y,
                                                  const double* __restrict__ gamma, chem_hfrd_opts o, HfrdIdx ix,
                                                  const double* __restrict__ rng, double* __restrict__ T_out,
                                                  double* __restrict__ p_out, double* __restrict__ Y_out,
                                                  int32_t* __restrict__ keep) {
  const int K = m.K, E = m.E;
  const double dT = rng[1] - rng[0], dp = rng[3] - rng[2], dn2 = rng[5] - rng[4];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double Tn = T[i] + o.alpha * gamma[i] * dT;                          // Eq. 3
    const double pn = p[i] + o.beta * gamma[(size_t)ld + i] * dp;             // Eq. 4
    double s = 0.0, yn2 = 0.0;
    for (int k = 0; k < K; ++k) {
      const double y = Y[(size_t)k * ld + i];
      double v;
      if (k == ix.i_n2) {
        v = y + o.alpha * gamma[2 * (size_t)ld + i] * dn2;                     // Eq. 5
        yn2 = v;
      } else {
        v = y > 0.0 ? pow(y, 1.0 + o.theta * gamma[(size_t)(3 + k) * ld + i]) : 0.0;   // Eq. 6
      }
      Y_out[(size_t)k * ld + i] = v;
      s += v;
    }
    bool ok = Tn > 0.0 && pn > 0.0 && yn2 >= 0.0 && s > 0.0;
    const double sd = s > 0.0 ? s : 1.0;
    double nC = 0.0, nH = 0.0, nO = 0.0, nN = 0.0;
    for (int k = 0; k < K; ++k) {
      const double y = Y_out[(size_t)k * ld + i] / sd;
      Y_out[(size_t)k * ld + i] = y;
      const double* cw = m.compW + (size_t)k * E;
      if (ix.el_C >= 0) nC += __ldg(cw + ix.el_C) * y;
      nH += __ldg(cw + ix.el_H) * y;
      nO += __ldg(cw + ix.el_O) * y;
      nN += __ldg(cw + ix.el_N) * y;
    }
    double num = 0.5 * nH;
    if (ix.el_C >= 0) {
      const double r = nH / nC;
      ok = ok && nC > 0.0 && r >= o.hc[0] && r <= o.hc[1];
      num += 2.0 * nC;
    }
    const double on = nO / nN, phi = num / nO;
    ok = ok && nN > 0.0 && on >= o.on[0] && on <= o.on[1];
    ok = ok && nO > 0.0 && phi >= o.phi[0] && phi <= o.phi[1];
    T_out[i] = Tn;
    p_out[i] = pn;
    keep[i] = ok ? 1 : 0;
  }
}

int launch_hfrd(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p, const double* Y,
                const double* gamma, const chem_hfrd_opts& o, const HfrdIdx& ix, double* T_out, double* p_out,
                double* Y_out, int32_t* keep, double* ranges, cudaStream_t s) {
  hfrd_ranges_kernel<<<1, 1024, 0, s>>>(n, T, p, Y + (size_t)ix.i_n2 * ld, ranges);
  int rc = cuda_check(cudaGetLastError(), "hfrd_ranges_kernel launch");
  if (rc) return rc;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
  hfrd_kernel<<<blocks, 256, 0, s>>>(m, n, ld, T, p, Y, gamma, o, ix, ranges, T_out, p_out, Y_out, keep);
  return cuda_check(cudaGetLastError(), "hfrd_kernel launch");
}

}  // namespace chem
