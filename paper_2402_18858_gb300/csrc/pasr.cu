// PaSR filtered reaction source from one chemistry step (the paper couples the learned step
// or DI to turbulence through the partially stirred reactor model, Sec. 3): per cell
//   kappa   = tau_c / (tau_c + tau_mix),
//   tau_mix = sqrt(sqrt(nu / eps) * k / eps)      (Kolmogorov time x sub-grid time k / eps),
//   tau_c   = max over species formed during the step (Y(t+dt) >= y_min and a gain
//             Y(t+dt) - Y(t) > r_min Y(t+dt)) of Y(t+dt) / ((Y(t+dt) - Y(t)) / dt)
//             (the slowest formation; r_min keeps rounding-level changes out),
//   omega_k = kappa rho (Y_k(t+dt) - Y_k(t)) / dt.
//
// One thread per cell over the species-major SoA state (coalesced loads and stores).  The
// kernel moves (3K + 5) doubles per cell, so it should be HBM-bound; on GB300 the K FP64
// differences and K products already cost about as much FP64 issue as the bytes cost HBM
// time, so everything else stays off the FP64 pipe: the formed/present decisions compare FP64
// bit patterns on the integer pipe (exact for the non-negative operands they see, after one
// IEEE product r_min Y(t+dt)), the search for the slowest formation compares
// cross products in FP32 (only the winner's time is formed, in FP64), and the mixing time is
// FP32 from correctly rounded inputs (relative error below 1e-6).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "internal.h"

namespace chem {

template <int KC>
__global__ void __launch_bounds__(256) pasr_kernel(int Kr, int64_t n, int64_t ld, double dt, double inv_dt,
                                                   const double* __restrict__ rho, const double* __restrict__ Y0,
                                                   const double* __restrict__ Y1, const double* __restrict__ ksgs,
                                                   const double* __restrict__ eps, const double* __restrict__ nu,
                                                   long long ymin_bits, double r_min, double* __restrict__ omega,
                                                   double* __restrict__ kappa) {
  const int K = KC ? KC : Kr;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double d[KC ? KC : CHEM_MAX_SPECIES];
    // slowest formation: the largest y1 / d over formed, present species, tracked as the
    // pair (yb, db) and compared by cross products (all candidates have d > 0)
    double yb = 0.0, dbest = 1.0;
    float ybf = 0.0f, dbf = 1.0f;
    bool any = false;
#pragma unroll
    for (int k = 0; k < (KC ? KC : K); ++k) {
      const double y1 = Y1[(size_t)k * ld + i];
      const double dk = y1 - Y0[(size_t)k * ld + i];
      d[k] = dk;
      // y1 >= y_min >= 0 makes r_min y1 >= 0, so dk > r_min y1 orders like the bit patterns
      if (__double_as_longlong(y1) >= ymin_bits &&
          __double_as_longlong(dk) > __double_as_longlong(__dmul_rn(r_min, y1))) {
        const float yf = narrow_f32(y1), df = narrow_f32(dk);
        if (!any || yf * dbf > ybf * df) {
          any = true;
          yb = y1;
          dbest = dk;
          ybf = yf;
          dbf = df;
        }
      }
    }
    const double tau_c = any ? dt * yb * rcp_nr(dbest) : 0.0;
    float tau_mix = 0.0f;
    const double kk = ksgs[i], ee = eps[i];
    if (__double_as_longlong(kk) > 0 && __double_as_longlong(ee) > 0) {
      const float ie = __frcp_rn(__double2float_rn(ee));
      tau_mix = sqrtf(sqrtf(__double2float_rn(nu[i]) * ie) * (__double2float_rn(kk) * ie));
    }
    const double tot = tau_c + (double)tau_mix;
    const double kap = tot > 0.0 ? tau_c * rcp_nr(tot) : 1.0;
    if (kappa) kappa[i] = kap;
    const double s = kap * rho[i] * inv_dt;
#pragma unroll
    for (int k = 0; k < (KC ? KC : K); ++k) omega[(size_t)k * ld + i] = s * d[k];
  }
}

int launch_pasr(const DevMech& m, int64_t n, int64_t ld, double dt, const double* rho, const double* Y0,
                const double* Y1, const double* ksgs, const double* eps, const double* nu, double y_min,
                double r_min, double* omega, double* kappa, cudaStream_t s) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
  long long yb = 0;
  std::memcpy(&yb, &y_min, sizeof yb);
  const double inv_dt = 1.0 / dt;
#define CHEM_PASR_K(KV)                                                                                 \
  if (m.K == KV) {                                                                                      \
    pasr_kernel<KV><<<blocks, 256, 0, s>>>(m.K, n, ld, dt, inv_dt, rho, Y0, Y1, ksgs, eps, nu, yb, r_min, \
                                           omega, kappa);                                                   \
    return cuda_check(cudaGetLastError(), "pasr_kernel launch");                                        \
  }
  CHEM_PASR_K(9)
  CHEM_PASR_K(30)
  CHEM_PASR_K(53)
#undef CHEM_PASR_K
  pasr_kernel<0><<<blocks, 256, 0, s>>>(m.K, n, ld, dt, inv_dt, rho, Y0, Y1, ksgs, eps, nu, yb, r_min, omega,
                                        kappa);
  return cuda_check(cudaGetLastError(), "pasr_kernel launch");
}

}  // namespace chem
