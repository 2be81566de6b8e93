// Warp-per-cell FP64 chemistry kernels for sm_103a: reaction rates (Eq. 1 right-hand side),
// the analytic Jacobian, and direct integration over one flow step (Eq. 2) by a
// variable-order BDF with a modified Newton iteration.
//
// Design (GB300): FP64 issue is the bottleneck (two FP64 lanes per clock per SM, so a warp
// FP64 instruction occupies the pipe for 16 cycles and idle lanes cost the same as busy
// ones).  One warp integrates one cell: lane k owns species k (and k + 32) and row k of the
// n x n Newton matrix; lane j evaluates reactions j, j + 32, ...; reductions are warp
// shuffles in a fixed order (results are bit-identical across lanes and runs).  Per-warp
// shared memory holds the Jacobian, its LU factors and the per-reaction terms; the BDF
// history lives in registers.  Step-control arithmetic that only steers heuristics (error
// norms, step-size factors) runs in FP32, the solution, the rates, the equilibrium
// constants and the LU stay FP64.  Every loop is bounded and every failure becomes a
// per-cell status code.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "internal.h"

namespace chem {

#define FULLMASK 0xffffffffu

// ------------------------------------------------------------------------------------------
// warp helpers
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ double wsum(double v) {
  // fixed-order tree into lane 0, then broadcast: every lane sees the same bits
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULLMASK, v, o);
  return __shfl_sync(FULLMASK, v, 0);
}

// the sums of a and b over the warp with one addition per tree level: the first level adds a
// in lanes 0-15 and b in lanes 16-31 (each lane keeps one value and sends the other across the
// halves), the next four reduce each half into its first lane, which is broadcast
__device__ __forceinline__ void wsum2(double a, double b, int lane, double& sa, double& sb) {
  const bool lo = lane < 16;
  double v = (lo ? a : b) + __shfl_xor_sync(FULLMASK, lo ? b : a, 16);
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_down_sync(FULLMASK, v, o, 16);
  sa = __shfl_sync(FULLMASK, v, 0);
  sb = __shfl_sync(FULLMASK, v, 16);
}

// a < b and a > b for non-negative doubles (not -0), on their bit patterns (integer pipe)
__device__ __forceinline__ bool pos_lt(double a, double b) { return __double_as_longlong(a) < __double_as_longlong(b); }
__device__ __forceinline__ bool pos_gt(double a, double b) { return __double_as_longlong(a) > __double_as_longlong(b); }

// x is finite, tested on its exponent bits (integer pipe)
__device__ __forceinline__ bool finite_bits(double x) {
  return ((unsigned int)((unsigned long long)__double_as_longlong(x) >> 32) & 0x7ff00000u) != 0x7ff00000u;
}

__device__ __forceinline__ float wsumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULLMASK, v, o);
  return __shfl_sync(FULLMASK, v, 0);
}

template <int NPL>
__device__ __forceinline__ double comp_get(const double (&x)[NPL], int i) {
  // value of component i (owned by lane i & 31, slot i >> 5), on every lane
  double v = x[0];
  if (NPL > 1 && (i >> 5) == 1) v = x[NPL > 1 ? 1 : 0];
  return __shfl_sync(FULLMASK, v, i & 31);
}

// ------------------------------------------------------------------------------------------
// per-warp shared memory
// ------------------------------------------------------------------------------------------
struct WarpMem {
  double* J;      // n x ld (Jacobian; rows 0..K-1 first hold dwdot/dC); in the compact layout
                  // the Jacobian is assembled in the LU region and kept as J32
  float* J32;     // n x ld compact layout only: the Jacobian rounded to FP32 (else null)
  double* LU;     // n x ld (factors of I - c J)
  double* C;      // K concentrations
  double* hRT;    // K
  double* g;      // K   run slots of the production rates (with eg and ieg, which follow it)
  double* eg;     // K   exp(-(g/RT - shift)) p0/RT, shift = element-potential term
  double* ieg;    // K   exp(+(g/RT - shift)) RT/p0
  double* q;      // I   net rates of progress
  double* kfe;    // I   effective forward coefficient (third-body factor included)
  double* kre;    // I   effective reverse coefficient
  double* aux;    // I   d q / d [M] factor (third-body: q0, Troe: dk/dM (fwd - rev/Kc))
  double* qT;     // I   d q / d T at fixed C
  double* tr;     // 14 per Troe reaction: [0..4] the exponentials of the rounds, [10] k,
                  // [11] dk/d[M], [12] dln k/dT (the other slots are spare)
  double* invd;   // n   reciprocal pivots
  double* ru;     // 64  step-size change matrix (0..24) and R(f) (32..56)
  int* perm;      // n   row permutation of the LU
  int ld;
};

__host__ __device__ inline int pad_ld(int n) { return n | 1; }

constexpr int kTroeSlots = 14;

// doubles per warp: matrices (optional) + species + reactions + Troe scratch + small vectors
// The per-reaction Jacobian terms (kfe, kre, aux, qT) are live only between rhs_eval<true> and
// jac_assemble, when the LU factors are stale (they are refactored right after), so with the
// matrices present they share the LU region whenever it is large enough.
// Compact layout (j32, for large mechanisms where it saves shared memory): the Jacobian is
// assembled in FP64 in the LU region and stored rounded to FP32 between refactorisations (it
// only shapes the Newton iteration matrix, which is approximate anyway: it is reused for up to
// 50 steps; the LU and every solve stay FP64); the Jacobian terms then share the FP32 region.
__host__ __device__ inline bool jac_terms_in_lu(int I, int n) {
  return 4 * (size_t)(I > 0 ? I : 1) <= (size_t)n * pad_ld(n);
}
__host__ __device__ inline size_t j32_doubles(int n) { return ((size_t)n * pad_ld(n) + 1) / 2; }
__host__ __device__ inline bool jac_terms_in_j32(int I, int n) {
  return 4 * (size_t)(I > 0 ? I : 1) <= j32_doubles(n);
}

__host__ __device__ inline size_t warp_doubles(int K, int I, int n, int nT, bool mats, bool jac, bool j32 = false) {
  size_t ld = pad_ld(n);
  size_t d;
  bool alias;
  if (mats && j32) {
    d = (size_t)n * ld + j32_doubles(n);
    alias = jac_terms_in_j32(I, n);
  } else {
    d = (mats ? 2 * (size_t)n * ld : (jac ? (size_t)n * ld : 0));
    alias = mats && jac && jac_terms_in_lu(I, n);
  }
  d += 5 * (size_t)K + 3 + (jac && !alias ? 5 : 1) * (size_t)(I > 0 ? I : 1) + (size_t)kTroeSlots * nT;
  d += (size_t)n + 64 + (size_t)(n + 1) / 2 + 2;
  return (d + 1) & ~size_t(1);   // keep 16-byte alignment per warp
}

// the direct-integration kernel's layout: compact when that needs less shared memory (the
// kernel for n <= 32 always takes the FP64 layout: the compact one is larger there)
__host__ __device__ inline bool di_use_j32(int K, int I, int n, int nT) {
  return warp_doubles(K, I, n, nT, true, true, true) < warp_doubles(K, I, n, nT, true, true, false);
}

__device__ __forceinline__ WarpMem carve(double* base, int K, int I, int n, int nT, bool mats, bool jac,
                                         bool j32 = false) {
  WarpMem w;
  w.ld = pad_ld(n);
  double* p = base;
  w.J = nullptr;
  w.J32 = nullptr;
  w.LU = nullptr;
  double* alias_at = nullptr;
  if (mats && j32) {
    w.LU = p; p += (size_t)n * w.ld;
    w.J = w.LU;
    w.J32 = (float*)p;
    if (jac && jac_terms_in_j32(I, n)) alias_at = p;
    p += j32_doubles(n);
  } else {
    if (mats || jac) { w.J = p; p += (size_t)n * w.ld; }
    if (mats) { w.LU = p; p += (size_t)n * w.ld; }
    if (jac && mats && jac_terms_in_lu(I, n)) alias_at = w.LU;
  }
  w.C = p; p += K + 1;
  w.hRT = p; p += K;
  w.g = p; p += K;
  w.eg = p; p += K + 1;
  w.ieg = p; p += K + 1;
  const int Ir = I > 0 ? I : 1;
  w.q = p; p += Ir;
  if (alias_at) {
    w.kfe = alias_at;
    w.kre = alias_at + Ir;
    w.aux = alias_at + 2 * Ir;
    w.qT = alias_at + 3 * Ir;
  } else if (jac) {
    w.kfe = p; p += Ir;
    w.kre = p; p += Ir;
    w.aux = p; p += Ir;
    w.qT = p; p += Ir;
  } else {
    w.kfe = w.kre = w.aux = w.qT = nullptr;
  }
  w.tr = p; p += (size_t)kTroeSlots * nT;
  w.invd = p; p += n;
  w.ru = p; p += 64;
  w.perm = (int*)p;
  return w;
}

// per-lane species values kept between the RHS and the Jacobian
template <int NPL>
struct LaneSp {
  double cpR[NPL], dcpR[NPL], hRT[NPL], wdot[NPL];
};

struct CellSc {
  double T, lnT, invT, RT, rho, Wbar, cp, Q;
};

// per-cell constants of the right-hand side: p / R and R / p (constant pressure)
struct CellP {
  double pR, Rp;
};
__device__ __forceinline__ CellP cell_p(double p) {
  CellP c;
  c.pR = p * (1.0 / kR);
  c.Rp = kR / p;
  return c;
}

// ------------------------------------------------------------------------------------------
// Troe falloff (Lindemann form with the Troe broadening factor, Gilbert, Luther & Troe 1983)
// for all falloff reactions of a cell.  The exponential rounds of rhs_eval have already put
// [0] k_inf, [1] k_0/k_inf, [2] exp(-T/T***), [3] exp(-T/T*), [4] exp(-T**/T) into w.tr.
// Reaction jt is worked by the lane pair t = 2 jt + q in rounds of 32 lanes, both lanes running
// one instruction stream on selected operands: lane q = 0 forms F_cent, lane q = 1 forms
// P_r = (k_0/k_inf)[M]; each takes the logarithm of its own value; after an exchange both
// have ln F_cent and ln P_r, form c, n and x = log10 P_r + c, and take one reciprocal: lane 0
// of 1/(den^2 + x^2) (den = n - 0.14 x), lane 1 of 1/(1 + P_r).  Lane 0 then forms
// F = exp(ln F_cent den^2 / (den^2 + x^2)) (the base-10 form of log10 F = log10 F_cent /
// (1 + (x/den)^2) with both sides times ln 10) and k = k_inf P_r/(1 + P_r) F.
// Results: [10] k, [11] dk/d[M], [12] d ln k/dT at fixed [M].
// ------------------------------------------------------------------------------------------
template <bool JAC>
__device__ __forceinline__ void troe_phase(const DevMech& m, const WarpMem& w, double invT, double ctot, int lane) {
  const int nT = m.I - m.n_tb_end;
  const double* __restrict__ et = m.exptab;
  const double kS = 0.4342944819032518;   // 1 / ln 10
  for (int t0 = 0; t0 < 2 * nT; t0 += 32) {
    const int t = t0 + lane, jt = t >> 1, q = t & 1;
    const bool act = t < 2 * nT;
    const int j = m.n_tb_end + jt;
    double* r = w.tr + kTroeSlots * (act ? jt : 0);
    // q = 0: F_cent = (1 - a) e_*** + a e_* + e_**;  q = 1: (k_0/k_inf) ([M] = ctot + sum_e
    // (alpha_e - 1) C_e), both as scale * (base + sum of four products)
    double c4[4] = {0.0, 0.0, 0.0, 0.0}, u4[4] = {0.0, 0.0, 0.0, 0.0}, base = 1.0, scale = 1.0;
    if (act) {
      if (q == 0) {
        const double a = __ldg(m.troe + 8 * (size_t)j + 3);
        c4[0] = 1.0 - a; u4[0] = r[2];
        c4[1] = a;       u4[1] = r[3];
        base = r[4];
      } else {
#pragma unroll
        for (int e = 0; e < kMaxEx; ++e) {
          const int se = __ldg(m.ex_sp + (size_t)j * kMaxEx + e);
          if (se >= 0) { c4[e] = __ldg(m.ex_a + (size_t)j * kMaxEx + e); u4[e] = w.C[se]; }
        }
        base = ctot;
        scale = r[1];
      }
    }
    const double v = fmax(scale * fma(c4[3], u4[3], fma(c4[2], u4[2], fma(c4[1], u4[1], fma(c4[0], u4[0], base)))), 1e-300);
    const double lv = log_t(v, m.logtab);
    const int l0 = lane & ~1, l1 = lane | 1;
    const double lc = __shfl_sync(FULLMASK, lv, l0);   // ln F_cent
    const double lp = __shfl_sync(FULLMASK, lv, l1);   // ln P_r
    const double Pr = __shfl_sync(FULLMASK, v, l1);
    const double c = fma(-0.67 * kS, lc, -0.4);
    const double nn = fma(-1.27 * kS, lc, 0.75);
    const double x = fma(kS, lp, c);
    const double den = fma(-0.14, x, nn);
    const double d2 = den * den;
    const double iS = rcp_nr(q ? 1.0 + Pr : fma(x, x, d2));
    const double ipr = __shfl_sync(FULLMASK, iS, l1);
    if (act && q == 0) {
      const double F = exp_t(lc * d2 * iS, et);
      const double kinf = r[0];
      r[10] = kinf * Pr * ipr * F;
      if (JAC) {
        const double L = kS * lc;   // log10 F_cent
        const double Fc = v;
        const double* tp = m.troe + 8 * (size_t)j;
        const double* ar = m.arr + 4 * (size_t)j;
        const double k0 = kinf * r[1];
        const double f1 = x / den;
        const double opf = 1.0 + f1 * f1;
        const double aa = __ldg(tp + 3), iT3 = __ldg(tp + 4), iT1 = __ldg(tp + 5);
        const double dFc = -(1.0 - aa) * iT3 * r[2] - aa * iT1 * r[3] + __ldg(tp + 6) * invT * invT * r[4];
        const double df1dx = nn / d2;
        const double gg = -L * 2.0 * f1 / (opf * opf) * df1dx;          // d log F / d log Pr
        r[11] = k0 * F * (ipr * ipr + gg * ipr);
        const double df1dL = df1dx * (-0.67) + (-x / d2) * (-1.27);
        const double dlogFdL = 1.0 / opf - L * 2.0 * f1 / (opf * opf) * df1dL;
        const double dlnkinf = __ldg(ar + 1) * invT + __ldg(ar + 2) * invT * invT;
        const double dlnk0 = __ldg(tp + 1) * invT + __ldg(tp + 2) * invT * invT;
        r[12] = dlnkinf + (ipr + gg) * (dlnk0 - dlnkinf) + dlogFdL * dFc / Fc;
      }
    }
  }
  __syncwarp();
}

// ------------------------------------------------------------------------------------------
// right-hand side f(z) of the reactor, z = (Y_1..Y_K, T)  [Eq. 1]
// ------------------------------------------------------------------------------------------
template <int NPL, bool JAC>
__device__ void rhs_eval(const DevMech& m, const WarpMem& w, const CellP& cp0, const double (&y)[NPL],
                         double (&f)[NPL], LaneSp<NPL>& sp, CellSc& cs, int lane) {
  const int K = m.K, I = m.I;
  const double T = comp_get<NPL>(y, K);
  const double lnT = log_t(T, m.logtab), RT = kR * T;
  const double* __restrict__ et = m.exptab;
  // T >= T_mid on the bit patterns (both positive: they order like the values)
  const int hi = __double_as_longlong(T) >= __double_as_longlong(m.Tmid) ? 1 : 0;
  // pass 1: c_p/R per species and the two mixture sums sum Y/W and sum Y c_p/(R W)
  double sYW = 0.0, cpp = 0.0, ywr[NPL];
#pragma unroll
  for (int s = 0; s < NPL; ++s) {
    const int k = lane + 32 * s;
    ywr[s] = 0.0;
    sp.cpR[s] = sp.dcpR[s] = sp.hRT[s] = 0.0;
    if (k < K) {
      const double* a = m.th + ((size_t)k * 2 + hi) * kThermoStride;
      const double a0 = __ldg(a + 0), a1 = __ldg(a + 1), a2 = __ldg(a + 2), a3 = __ldg(a + 3), a4 = __ldg(a + 4);
      const double cpR = a0 + T * (a1 + T * (a2 + T * (a3 + T * a4)));
      if (JAC) sp.dcpR[s] = a1 + T * (2.0 * a2 + T * (3.0 * a3 + T * 4.0 * a4));
      const double yw = y[s] * __ldg(m.invW + k);
      ywr[s] = yw;
      sYW += yw;
      cpp += yw * cpR;
      sp.cpR[s] = cpR;
    }
  }
  wsum2(sYW, cpp, lane, sYW, cpp);
  // one reciprocal gives 1/T, 1/(T sum Y/W) and 1/c_p (with p/R and R/p per cell: no division)
  const double TsY = T * sYW;
  const double inv = rcp_nr(TsY * cpp);
  const double invT = inv * (sYW * cpp);
  const double Wbar = JAC ? inv * (T * cpp) : 0.0;   // the mean molar mass and c_p: Jacobian only
  const double icp = inv * TsY * (1.0 / kR);
  const double rho = cp0.pR * (inv * cpp);           // p Wbar / (R T) = (p/R) / (T sum Y/W)
  const double irho = cp0.Rp * TsY;                  // 1 / rho
  const double ctot = cp0.pR * invT;                 // sum of the concentrations, p / (R T)
  const double cp = JAC ? cpp * kR : 0.0;
  // pass 2: h/RT and the concentrations (and the sentinel slots of the two-partner reactions,
  // which the production-rate runs of the previous call may have overwritten), and per species
  // e = exp(-g'/RT) with g' the free energy shifted by element potentials (one exp per species
  // instead of one per reaction; the shift cancels in every balanced reaction).
  // kr / kf = 1/K_c = prod_r e_r prod_p (1/e_p) (RT/p0)^(sum nu): the pressure factor goes
  // into the per-species values, p0/RT with every reactant and RT/p0 with every product
  const double P0RT = (kP0 / kR) * invT, RTP0 = RT * (1.0 / kP0);
  const bool two = !JAC && m.arity2;   // warp-uniform
#pragma unroll
  for (int s = 0; s < NPL; ++s) {
    const int k = lane + 32 * s;
    if (k == K) {
      w.C[K] = 1.0;
      w.eg[K] = 1.0;
      w.ieg[K] = 1.0;
    }
    if (k < K) {
      const double* a = m.th + ((size_t)k * 2 + hi) * kThermoStride;
      const double hRT = __ldg(a + 5) + T * (__ldg(a + 6) + T * (__ldg(a + 7) + T * (__ldg(a + 8) + T * __ldg(a + 9))))
                         + __ldg(a + 10) * invT;
      const double* gc = m.gneg + ((size_t)k * 2 + hi) * 8;
      const double2 g01 = __ldg((const double2*)gc), g23 = __ldg((const double2*)(gc + 2));
      const double2 g45 = __ldg((const double2*)(gc + 4));
      const double g6 = __ldg(gc + 6);
      const double ng = fma(T, T * fma(T, fma(T, g45.y, g45.x), g23.y) + g23.x, fma(g6, invT, fma(g01.y, lnT, g01.x)));
      const double Ck = rho * ywr[s];
      w.C[k] = Ck;
      w.hRT[k] = hRT;
      sp.hRT[s] = hRT;
      const double e = exp_s256(ng, et);
      w.eg[k] = e * P0RT;
      w.ieg[k] = rcp_nr(e) * (two ? RTP0 * Ck : RTP0);
    }
  }
  // exponential rounds: k_f of every non-falloff reaction (into w.q, read back by the same
  // lane below) and the five exponentials of each falloff reaction (into w.tr), all items
  // packed over the lanes
  const int nb = m.n_tb_end;
  // whole rounds before the first falloff item: k_f only, no T term in the argument
  const int n_plain = (nb / 32) * 32;
  for (int t = lane; t < n_plain; t += 32) {
    const double2 x01 = __ldg((const double2*)(m.xarg + 4 * (size_t)t));
    const double x2 = __ldg(m.xarg + 4 * (size_t)t + 2);
    w.q[t] = exp_s256(fma(-x2, invT, fma(x01.y, lnT, x01.x)), et);
  }
  for (int t = n_plain + lane; t < m.n_x; t += 32) {
    const double2 x01 = __ldg((const double2*)(m.xarg + 4 * (size_t)t));
    const double2 x23 = __ldg((const double2*)(m.xarg + 4 * (size_t)t + 2));
    const double e = exp_s256(fma(x23.y, T, fma(-x23.x, invT, fma(x01.y, lnT, x01.x))), et);
    if (t < nb) {
      w.q[t] = e;
    } else {
      const int u = t - nb, jt = u / 5;
      w.tr[kTroeSlots * jt + (u - 5 * jt)] = e;
    }
  }
  __syncwarp();
  if (I > nb) troe_phase<JAC>(m, w, invT, ctot, lane);
  if (two) {
    // q_j = k_f (C_a C_b - K_c^-1 C_c C_d) = k_f (C_a C_b - (e_a e_b)(u_c u_d)) with
    // e = exp(-g'/RT) p0/RT and u = exp(g'/RT) (RT/p0) C; a missing partner is the sentinel 1.
    // No predication on the reaction's arity, one rounding in the difference.
    for (int j = lane; j < I; j += 32) {
      const int4 rs = __ldg(m.rsp2 + j);
      double kf;
      if (j < nb) kf = w.q[j];
      else kf = w.tr[kTroeSlots * (j - nb) + 10];
      if (j >= m.n_elem && j < nb) {
        double M = ctot;
#pragma unroll
        for (int e = 0; e < kMaxEx; ++e) {
          const int se = __ldg(m.ex_sp + (size_t)j * kMaxEx + e);
          if (se >= 0) M += __ldg(m.ex_a + (size_t)j * kMaxEx + e) * w.C[se];
        }
        kf *= M;
      }
      w.q[j] = kf * fma(-(w.eg[rs.x] * w.eg[rs.y]), w.ieg[rs.z] * w.ieg[rs.w], w.C[rs.x] * w.C[rs.y]);
    }
  } else
  for (int j = lane; j < I; j += 32) {
    const int4 ra = __ldg((const int4*)(m.rsp + 8 * (size_t)j));
    const int4 rb = __ldg((const int4*)(m.rsp + 8 * (size_t)j + 4));
    const bool falloff = j >= nb;
    double kf, dlnkf = 0.0, dkdM = 0.0;
    if (!falloff) {
      kf = w.q[j];
      if (JAC) dlnkf = __ldg(m.arr + 4 * (size_t)j + 1) * invT + __ldg(m.arr + 4 * (size_t)j + 2) * invT * invT;
    } else {
      const double* r = w.tr + kTroeSlots * (j - nb);
      kf = r[10];
      if (JAC) { dkdM = r[11]; dlnkf = r[12]; }
    }
    double fwd = w.C[ra.x], ratio = w.eg[ra.x], sh = 0.0;
    if (JAC) sh = -w.hRT[ra.x];
    if (ra.w > 1) { fwd *= w.C[ra.y]; ratio *= w.eg[ra.y]; if (JAC) sh -= w.hRT[ra.y]; }
    if (ra.w > 2) { fwd *= w.C[ra.z]; ratio *= w.eg[ra.z]; if (JAC) sh -= w.hRT[ra.z]; }
    double rev = w.C[rb.x];
    ratio *= w.ieg[rb.x];
    if (JAC) sh += w.hRT[rb.x];
    if (rb.w > 1) { rev *= w.C[rb.y]; ratio *= w.ieg[rb.y]; if (JAC) sh += w.hRT[rb.y]; }
    if (rb.w > 2) { rev *= w.C[rb.z]; ratio *= w.ieg[rb.z]; if (JAC) sh += w.hRT[rb.z]; }
    double Mfac = 1.0;
    if (j >= m.n_elem && !falloff) {
      double M = ctot;
#pragma unroll
      for (int e = 0; e < kMaxEx; ++e) {
        const int se = __ldg(m.ex_sp + (size_t)j * kMaxEx + e);
        if (se >= 0) M += __ldg(m.ex_a + (size_t)j * kMaxEx + e) * w.C[se];
      }
      Mfac = M;
    }
    const double kr = kf * ratio;
    const double q0 = kf * fwd - kr * rev;
    w.q[j] = Mfac * q0;
    if (JAC) {
      w.kfe[j] = Mfac * kf;
      w.kre[j] = Mfac * kr;
      w.aux[j] = (j < m.n_elem) ? 0.0 : (j < nb ? q0 : dkdM * (fwd - ratio * rev));
      const double dlnKc = (sh - __ldg(m.arr + 4 * (size_t)j + 3)) * invT;
      w.qT[j] = Mfac * (kf * dlnkf * fwd - kr * (dlnkf - dlnKc) * rev);
    }
  }
  __syncwarp();
  // production rates wdot_k = sum_j nu_kj q_j
  const int P = m.bal_P;
  double* part = w.g;   // g, eg and ieg are dead from here on: 3K slots for the runs
  if (P > 0) {
    double acc = 0.0;
    for (int i = 0; i < P; ++i) {
      const unsigned int e = __ldg(m.bal + (size_t)i * 32 + lane);
      if (e & 3u) {
        // nu = +-1, +-2, +-3 built from its bits (no FP64 conversion)
        const unsigned int a = e & 3u;
        const unsigned int hw = (a == 1u ? 0x3ff00000u : a == 2u ? 0x40000000u : 0x40080000u) | ((e & 4u) << 29);
        acc = fma(__hiloint2double((int)hw, 0), w.q[e >> 12], acc);
        if (e & 8u) {
          part[(e >> 4) & 255u] = acc;
          acc = 0.0;
        }
      }
    }
    __syncwarp();
  }
  double Qp = 0.0;
#pragma unroll
  for (int s = 0; s < NPL; ++s) {
    const int k = lane + 32 * s;
    f[s] = 0.0;
    sp.wdot[s] = 0.0;
    if (k < K) {
      double wd = 0.0;
      if (P > 0) {
        const int r0 = __ldg(m.run_ptr + k), r1 = __ldg(m.run_ptr + k + 1);
        for (int r = r0; r < r1; ++r) wd += part[r];
      } else {
        const int e0 = __ldg(m.sp_ptr + k), e1 = __ldg(m.sp_ptr + k + 1);
        for (int e = e0; e < e1; ++e) wd += __ldg(m.sp_nu + e) * w.q[__ldg(m.sp_rxn + e)];
      }
      sp.wdot[s] = wd;
      f[s] = __ldg(m.W + k) * wd * irho;
      Qp += sp.hRT[s] * wd;
    }
  }
  const double Q = wsum(Qp) * RT;
  const double fT = -Q * irho * icp;
#pragma unroll
  for (int s = 0; s < NPL; ++s)
    if (lane + 32 * s == K) f[s] = fT;
  cs.T = T; cs.lnT = lnT; cs.invT = invT; cs.RT = RT; cs.rho = rho; cs.Wbar = Wbar;
  cs.cp = cp; cs.Q = Q;
}

// ------------------------------------------------------------------------------------------
// analytic Jacobian d f / d z into w.J (row-major, ld), after rhs_eval<NPL, true>
// ------------------------------------------------------------------------------------------
template <int NPL>
__device__ void jac_assemble(const DevMech& m, const WarpMem& w, const double (&y)[NPL],
                             const LaneSp<NPL>& sp, const CellSc& cs, int lane) {
  const int K = m.K, ld = w.ld;
  double dwdT[NPL], S[NPL], colH[NPL];
  // d wdot_k / d C_m at fixed T (rows of species k), and d wdot_k / dT at fixed C
#pragma unroll
  for (int s = 0; s < NPL; ++s) {
    const int k = lane + 32 * s;
    dwdT[s] = 0.0;
    if (k < K) {
      double* row = w.J + (size_t)k * ld;
      for (int c = 0; c < K; ++c) row[c] = 0.0;
      double acc = 0.0, dT = 0.0;
      const int e0 = __ldg(m.sp_ptr + k), e1 = __ldg(m.sp_ptr + k + 1);
      for (int e = e0; e < e1; ++e) {
        const int j = __ldg(m.sp_rxn + e);
        const double nu = __ldg(m.sp_nu + e);
        const int4 ra = __ldg((const int4*)(m.rsp + 8 * (size_t)j));
        const int4 rb = __ldg((const int4*)(m.rsp + 8 * (size_t)j + 4));
        const double kf = nu * w.kfe[j], kr = nu * w.kre[j];
        if (ra.w == 1) {
          row[ra.x] += kf;
        } else if (ra.w == 2) {
          row[ra.x] += kf * w.C[ra.y];
          row[ra.y] += kf * w.C[ra.x];
        } else {
          row[ra.x] += kf * w.C[ra.y] * w.C[ra.z];
          row[ra.y] += kf * w.C[ra.x] * w.C[ra.z];
          row[ra.z] += kf * w.C[ra.x] * w.C[ra.y];
        }
        if (rb.w == 1) {
          row[rb.x] -= kr;
        } else if (rb.w == 2) {
          row[rb.x] -= kr * w.C[rb.y];
          row[rb.y] -= kr * w.C[rb.x];
        } else {
          row[rb.x] -= kr * w.C[rb.y] * w.C[rb.z];
          row[rb.y] -= kr * w.C[rb.x] * w.C[rb.z];
          row[rb.z] -= kr * w.C[rb.x] * w.C[rb.y];
        }
        if (j >= m.n_elem) {
          const double a = nu * w.aux[j];
          acc += a;
#pragma unroll
          for (int x = 0; x < kMaxEx; ++x) {
            const int se = __ldg(m.ex_sp + (size_t)j * kMaxEx + x);
            if (se >= 0) row[se] += a * __ldg(m.ex_a + (size_t)j * kMaxEx + x);
          }
        }
        dT += nu * w.qT[j];
      }
      if (acc != 0.0)
        for (int c = 0; c < K; ++c) row[c] += acc;
      dwdT[s] = dT;
    }
  }
  __syncwarp();
  double hsp = 0.0;
#pragma unroll
  for (int s = 0; s < NPL; ++s) {
    const int k = lane + 32 * s;
    S[s] = 0.0;
    colH[s] = 0.0;
    if (k < K) {
      const double* row = w.J + (size_t)k * ld;
      double a = 0.0;
      for (int c = 0; c < K; ++c) a += row[c] * w.C[c];
      S[s] = a;
      hsp += sp.hRT[s] * a;
      double b = 0.0;   // column k: sum_r h_r/RT dwdot_r/dC_k
      for (int r = 0; r < K; ++r) b += w.hRT[r] * w.J[(size_t)r * ld + k];
      colH[s] = b;
    }
  }
  const double HS = wsum(hsp) * cs.RT;
  __syncwarp();
  const double rho = cs.rho, irho = 1.0 / rho, Wbar = cs.Wbar, cp = cs.cp, Q = cs.Q;
  const double rc = rho * cp, irc = 1.0 / rc, Qrc2 = Q * irc * irc;
  double dq = 0.0, dcp = 0.0;
#pragma unroll
  for (int s = 0; s < NPL; ++s) {
    const int k = lane + 32 * s;
    if (k < K) {
      double* row = w.J + (size_t)k * ld;
      const double Wk = __ldg(m.W + k), wd = sp.wdot[s];
      const double ak = Wbar * (wd - S[s]) * irho;
      for (int c = 0; c < K; ++c) row[c] = Wk * __ldg(m.invW + c) * (row[c] + ak);
      row[K] = Wk * irho * (dwdT[s] + (wd - S[s]) * cs.invT);
      // temperature row, column k
      const double iW = __ldg(m.invW + k);
      const double dQ = cs.RT * rho * colH[s] - Wbar * HS;   // HS already carries RT
      w.J[(size_t)K * ld + k] = iW * (-dQ * irc + Qrc2 * rho * (sp.cpR[s] * kR - cp * Wbar));
      dq += sp.cpR[s] * kR * wd + sp.hRT[s] * cs.RT * (dwdT[s] - S[s] * cs.invT);
      dcp += y[s] * sp.dcpR[s] * kR * iW;
    }
  }
  wsum2(dq, dcp, lane, dq, dcp);
  if (lane == 0) w.J[(size_t)K * ld + K] = -dq * irc + Qrc2 * (-rc * cs.invT + rho * dcp);
  __syncwarp();
  if (NPL > 1 && w.J32) {
    // compact layout (large mechanisms only): keep the Jacobian as FP32 (integer-pipe narrowing; the per-reaction
    // terms that shared this region are dead now)
    const int n = K + 1;
    for (int e = lane; e < n * ld; e += 32) w.J32[e] = narrow_f32(w.J[e]);
    __syncwarp();
  }
}

// ------------------------------------------------------------------------------------------
// dense LU of M = I - c J with partial pivoting (ties: lowest row), lane = row.  The pivot
// search runs on the warp's integer reductions (the bit pattern of a non-negative double
// orders like its value), the row permutation lives in shared memory, and each row of U is
// left scaled by its reciprocal pivot (unit upper factor) so that a solve multiplies by the
// pivots once instead of once per column.
// ------------------------------------------------------------------------------------------
template <int NPL>
__device__ bool lu_factor(const WarpMem& w, int n, double c, int lane) {
  const int ld = w.ld;
#pragma unroll
  for (int s = 0; s < NPL; ++s) {
    const int r = lane + 32 * s;
    if (r < n) {
      double* lr = w.LU + (size_t)r * ld;
      if (NPL > 1 && w.J32) {
        const float* jr = w.J32 + (size_t)r * ld;
        for (int cc = 0; cc < n; ++cc) lr[cc] = (r == cc ? 1.0 : 0.0) - c * widen_f64(jr[cc]);
      } else {
        const double* jr = w.J + (size_t)r * ld;
        for (int cc = 0; cc < n; ++cc) lr[cc] = (r == cc ? 1.0 : 0.0) - c * jr[cc];
      }
      w.perm[r] = r;
    }
  }
  __syncwarp();
  bool ok = true;
  for (int col = 0; col < n; ++col) {
    // this lane's best candidate (largest |v|, lower row on ties), then the warp's
    unsigned long long key = 0ull;
    unsigned int row = 0xffffffffu;
#pragma unroll
    for (int s = 0; s < NPL; ++s) {
      const int r = lane + 32 * s;
      if (r >= col && r < n) {
        const unsigned long long kv =
            (unsigned long long)__double_as_longlong(w.LU[(size_t)r * ld + col]) & 0x7fffffffffffffffull;   // |v|
        if (row == 0xffffffffu || kv > key) { key = kv; row = (unsigned int)r; }
      }
    }
    const unsigned int hi = (unsigned int)(key >> 32), lo = (unsigned int)key;
    const unsigned int mhi = __reduce_max_sync(FULLMASK, hi);
    const unsigned int mlo = __reduce_max_sync(FULLMASK, hi == mhi ? lo : 0u);
    const unsigned int bi = __reduce_min_sync(FULLMASK, (hi == mhi && lo == mlo) ? row : 0xffffffffu);
    // a pivot that is zero or not finite (its |value| bits: zero, or exponent all ones)
    if ((mhi | mlo) == 0u || mhi >= 0x7ff00000u || bi >= (unsigned int)n) { ok = false; break; }
    if ((int)bi != col) {
      for (int cc = lane; cc < n; cc += 32) {
        const double t = w.LU[(size_t)col * ld + cc];
        w.LU[(size_t)col * ld + cc] = w.LU[(size_t)bi * ld + cc];
        w.LU[(size_t)bi * ld + cc] = t;
      }
      if (lane == 0) {
        const int t = w.perm[col];
        w.perm[col] = w.perm[bi];
        w.perm[bi] = t;
      }
    }
    __syncwarp();
    const double inv = rcp_nr(w.LU[(size_t)col * ld + col]);
    if (lane == 0) w.invd[col] = inv;
    // multipliers (lane = row), then the trailing (n-col-1)^2 update spread over all lanes
    // (element e of the block at row e / m, column e % m, stepped incrementally)
#pragma unroll
    for (int s = 0; s < NPL; ++s) {
      const int r = lane + 32 * s;
      if (r > col && r < n) w.LU[(size_t)r * ld + col] *= inv;
    }
    __syncwarp();
    const int md = n - col - 1;
    if (md > 0) {
      const int q = 32 / md, rm = 32 - q * md;
      int rr = lane / md, cc = lane - rr * md;
      double* base = w.LU + (size_t)(col + 1) * ld + (col + 1);
      const double* pr = w.LU + (size_t)col * ld + (col + 1);
      for (int e = lane; e < md * md; e += 32) {
        double* a = base + (size_t)rr * ld + cc;
        *a = fma(-base[(size_t)rr * ld - 1], pr[cc], *a);
        rr += q;
        cc += rm;
        if (cc >= md) { cc -= md; ++rr; }
      }
    }
    __syncwarp();
  }
  if (ok) {
#pragma unroll
    for (int s = 0; s < NPL; ++s) {
      const int r = lane + 32 * s;
      if (r < n) {
        const double d = w.invd[r];
        double* lr = w.LU + (size_t)r * ld;
        for (int cc = r + 1; cc < n; ++cc) lr[cc] *= d;
      }
    }
    __syncwarp();
  }
  return ok;
}

// x <- M^{-1} x with the factors of lu_factor (x distributed: lane = row)
template <int NPL>
__device__ void lu_solve(const WarpMem& w, int n, double (&x)[NPL], int lane) {
  const int ld = w.ld;
  double b[NPL];
#pragma unroll
  for (int s = 0; s < NPL; ++s) {
    const int r = lane + 32 * s;
    const int src = r < n ? w.perm[r] : r;
    double v0 = __shfl_sync(FULLMASK, x[0], src & 31);
    double v = v0;
    if (NPL > 1) {
      const double v1 = __shfl_sync(FULLMASK, x[NPL > 1 ? 1 : 0], src & 31);
      v = (src >> 5) ? v1 : v0;
    }
    b[s] = r < n ? v : 0.0;
  }
  // L (unit lower) forward substitution
  for (int col = 0; col < n - 1; ++col) {
    const double xc = comp_get<NPL>(b, col);
#pragma unroll
    for (int s = 0; s < NPL; ++s) {
      const int r = lane + 32 * s;
      if (r > col && r < n) b[s] -= w.LU[(size_t)r * ld + col] * xc;
    }
  }
  // diag(1/u_kk), then the unit upper factor backward
#pragma unroll
  for (int s = 0; s < NPL; ++s) {
    const int r = lane + 32 * s;
    if (r < n) b[s] *= w.invd[r];
  }
  for (int col = n - 1; col > 0; --col) {
    const double xc = comp_get<NPL>(b, col);
#pragma unroll
    for (int s = 0; s < NPL; ++s) {
      const int r = lane + 32 * s;
      if (r < col) b[s] -= w.LU[(size_t)r * ld + col] * xc;
    }
  }
#pragma unroll
  for (int s = 0; s < NPL; ++s) x[s] = b[s];
}

// ------------------------------------------------------------------------------------------
// BDF (Shampine & Reichelt backward-difference form, orders 1..5) with modified Newton
// ------------------------------------------------------------------------------------------
constexpr int kMaxOrd = 5;
constexpr int kNewtonMax = 3;

__device__ __forceinline__ double bdf_gamma(int k) {
  // gamma_k = sum_{i=1..k} 1/i
  switch (k) {
    case 1: return 1.0;
    case 2: return 1.5;
    case 3: return 1.8333333333333333;
    case 4: return 2.0833333333333333;
    case 5: return 2.2833333333333333;
    default: return 2.45;
  }
}

__device__ __forceinline__ double bdf_inv_gamma(int k) {
  switch (k) {
    case 1: return 1.0;
    case 2: return 1.0 / 1.5;
    case 3: return 6.0 / 11.0;
    case 4: return 12.0 / 25.0;
    case 5: return 60.0 / 137.0;
    default: return 1.0 / 2.45;
  }
}

// wrms norm of x / scale in FP32 (an error-control heuristic; never feeds the solution)
template <int NPL>
__device__ __forceinline__ float wrms(const double (&x)[NPL], const float (&isc)[NPL], int n, int lane) {
  float a = 0.0f;
#pragma unroll
  for (int s = 0; s < NPL; ++s) {
    if (lane + 32 * s < n) {
      float v = fminf(fabsf(narrow_f32(x[s])) * isc[s], 1e15f);
      a += v * v;
    }
  }
  return sqrtf(wsumf(a) / (float)n);
}

// Step-size change of the backward differences (Shampine & Reichelt): D[1..order] <-
// (R(f) U)^T D[1..order] with R(f)_il = prod_{m=1..i} (m - 1 - f l) / m and U = R(1), i.e.
// U_lj = (-1)^l C(j, l); row and column 0 of R U are (1, 0, ...), so D[0] is untouched.
// Lanes 0..24 hold entry (i, l) = (1 + lane / 5, 1 + lane % 5): first R(f) (one product chain
// per lane), then (R U)_ij = sum_l R_il U_lj with U from a constant table.
// The update of D is specialised per order so that only order^2 FMAs are issued.
struct RescaleLane {
  int i;             // 1 + lane / 5
  int j;             // 1 + lane % 5
  double l;          // 1 + lane % 5 as a double (l in phase 1)
  double inv_fact;   // 1 / i!
};

// U_lj = (-1)^l C(j, l), l, j = 1..5 (row l - 1, column j - 1)
__device__ const double kRescaleU[25] = {-1, -2, -3, -4, -5,  0, 1, 3, 6, 10,  0, 0, -1, -4, -10,
                                         0, 0, 0, 1, 5,  0, 0, 0, 0, -1};

__device__ __forceinline__ RescaleLane rescale_lane(int lane) {
  RescaleLane rc;
  rc.i = 1 + lane / 5;
  rc.j = 1 + lane % 5;
  rc.l = (double)rc.j;
  rc.inv_fact = rc.i == 1 ? 1.0 : rc.i == 2 ? 0.5 : rc.i == 3 ? 1.0 / 6.0 : rc.i == 4 ? 1.0 / 24.0 : 1.0 / 120.0;
  return rc;
}

template <int ORD, int NPL>
__device__ __forceinline__ void rescale_apply(double (&D)[kMaxOrd + 3][NPL], const double* __restrict__ ru) {
  double Dn[ORD][NPL];
#pragma unroll
  for (int j = 1; j <= ORD; ++j)
#pragma unroll
    for (int s = 0; s < NPL; ++s) {
      double a = ru[j - 1] * D[1][s];
#pragma unroll
      for (int i = 2; i <= ORD; ++i) a = fma(ru[(i - 1) * 5 + (j - 1)], D[i][s], a);
      Dn[j - 1][s] = a;
    }
#pragma unroll
  for (int j = 1; j <= ORD; ++j)
#pragma unroll
    for (int s = 0; s < NPL; ++s) D[j][s] = Dn[j - 1][s];
}

template <int NPL>
__device__ void rescale_D(double (&D)[kMaxOrd + 3][NPL], int order, double fct, const WarpMem& w,
                          const RescaleLane& rc, int lane) {
  if (lane < 25) {
    const double fl = fct * rc.l;
    double r = -fl;                                   // m = 1
#pragma unroll
    for (int mm = 2; mm <= kMaxOrd; ++mm)
      if (mm <= rc.i) r *= (double)(mm - 1) - fl;
    w.ru[32 + lane] = r * rc.inv_fact;
  }
  __syncwarp();
  if (lane < 25) {
    const double* Ri = w.ru + 32 + (rc.i - 1) * 5;
    const double* Uj = kRescaleU + (rc.j - 1);
    double a = Ri[0] * __ldg(Uj);
#pragma unroll
    for (int l = 2; l <= kMaxOrd; ++l) a = fma(Ri[l - 1], __ldg(Uj + 5 * (l - 1)), a);
    w.ru[lane] = a;
  }
  __syncwarp();
  switch (order) {
    case 1: rescale_apply<1, NPL>(D, w.ru); break;
    case 2: rescale_apply<2, NPL>(D, w.ru); break;
    case 3: rescale_apply<3, NPL>(D, w.ru); break;
    case 4: rescale_apply<4, NPL>(D, w.ru); break;
    default: rescale_apply<5, NPL>(D, w.ru); break;
  }
  __syncwarp();
}

// predictor y = sum_{j<=order} D[j] and history term psi = sum_j gamma_j D[j] / gamma_order
template <int ORD, int NPL>
__device__ __forceinline__ void bdf_predict(const double (&D)[kMaxOrd + 3][NPL], double (&y)[NPL],
                                            double (&psi)[NPL], double ig) {
#pragma unroll
  for (int s = 0; s < NPL; ++s) {
    double yp = D[0][s] + D[1][s], ps = D[1][s];
#pragma unroll
    for (int j = 2; j <= ORD; ++j) {
      yp += D[j][s];
      ps = fma(bdf_gamma(j), D[j][s], ps);
    }
    y[s] = yp;
    psi[s] = ps * ig;
  }
}

// accepted step: D[order+2] = d - D[order+1], D[order+1] = d, D[j] += D[j+1] (j = order..0)
template <int ORD, int NPL>
__device__ __forceinline__ void bdf_accept(double (&D)[kMaxOrd + 3][NPL], const double (&d)[NPL]) {
#pragma unroll
  for (int s = 0; s < NPL; ++s) {
    D[ORD + 2][s] = d[s] - D[ORD + 1][s];
    D[ORD + 1][s] = d[s];
#pragma unroll
    for (int j = ORD; j >= 0; --j) D[j][s] += D[j + 1][s];
  }
}

struct DiOpts {
  double rtol, atol_Y, atol_T, newton_tol;
  int max_steps, jac_max_age;   // Jacobian reuse: a Newton failure with a stale one refreshes it
};

template <int NPL>
__device__ int integrate_cell(const DevMech& m, const WarpMem& w, double pc, double (&z)[NPL],
                              double dt, const DiOpts& o, int lane, int (&cnt)[4]) {
  const int n = m.n, K = m.K;
  cnt[0] = cnt[1] = cnt[2] = cnt[3] = 0;
  LaneSp<NPL> sp;
  CellSc cs;
  // error weights 1 / (atol + rtol |y|) in FP32 (they only steer step control)
  float atolf[NPL];
  float isc[NPL];
  const float rtolf = (float)o.rtol;
  bool fin = true;
#pragma unroll
  for (int s = 0; s < NPL; ++s) {
    const int i = lane + 32 * s;
    atolf[s] = (float)((i == K) ? o.atol_T : o.atol_Y);
    if (i < n && !isfinite(z[s])) fin = false;
  }
  if (__any_sync(FULLMASK, !fin)) return CHEM_CELL_NONFINITE;
  if (!(dt > 0.0)) return CHEM_CELL_OK;
  {
    const double T0 = comp_get<NPL>(z, K);
    if (!(T0 > 0.0)) return CHEM_CELL_OUT_OF_RANGE;
  }
  const double EPS = 2.220446049250313e-16;
  const float ntol = (float)o.newton_tol;
  const RescaleLane rc = rescale_lane(lane);
  const CellP pp = cell_p(pc);

  double D[kMaxOrd + 3][NPL];
  double f[NPL], y[NPL], d[NPL], dy[NPL], psi[NPL];
  // initial step (Hairer, Norsett & Wanner, Sec. II.4, order 1)
  rhs_eval<NPL, false>(m, w, pp, z, f, sp, cs, lane);
  cnt[1]++;
#pragma unroll
  for (int s = 0; s < NPL; ++s) isc[s] = __frcp_rn(fmaf(rtolf, fabsf(narrow_f32(z[s])), atolf[s]));
  const float d0 = wrms<NPL>(z, isc, n, lane), d1 = wrms<NPL>(f, isc, n, lane);
  double h0 = (d0 < 1e-5f || d1 < 1e-5f) ? 1e-6 : 0.01 * (double)d0 / (double)d1;
  h0 = fmin(h0, dt);
#pragma unroll
  for (int s = 0; s < NPL; ++s) y[s] = z[s] + h0 * f[s];
  rhs_eval<NPL, false>(m, w, pp, y, dy, sp, cs, lane);
  cnt[1]++;
#pragma unroll
  for (int s = 0; s < NPL; ++s) dy[s] -= f[s];
  const float d2 = (float)((double)wrms<NPL>(dy, isc, n, lane) / h0);
  const float dm = fmaxf(d1, d2);
  double h = (dm <= 1e-15f) ? fmax(1e-6, h0 * 1e-3) : (double)sqrtf(0.01f / dm);
  h = fmin(fmin(100.0 * h0, h), dt);
  if (!(h > 0.0)) h = 1e-12 * dt;

#pragma unroll
  for (int s = 0; s < NPL; ++s) {
    D[0][s] = z[s];
    D[1][s] = h * f[s];
#pragma unroll
    for (int j = 2; j < kMaxOrd + 3; ++j) D[j][s] = 0.0;
  }
  int order = 1, n_equal = 0, newton_iters = 0, fails = 0;
  bool need_jac = true, have_lu = false;
  int jac_age = 0;
  double c_lu = 0.0, ic_lu = 0.0;
  float crate = 0.5f;
  double t = 0.0;
  int status = CHEM_CELL_OK;

  // t, h, dt and hmin are positive (t starts at +0): their comparisons run on the bit patterns
  while (pos_lt(t, dt)) {
    if (cnt[0] >= o.max_steps) { status = CHEM_CELL_MAX_STEPS; break; }
    const double hmin = fma(10.0 * EPS, t, 1e-300);
    if (pos_gt(t + h, dt)) {
      const double hn = dt - t;
      rescale_D<NPL>(D, order, hn / h, w, rc, lane);
      h = hn;
      n_equal = 0;
    }
    if (pos_lt(h, hmin) || fails > 60) { status = CHEM_CELL_STEP_FAIL; break; }
    double t_new = t + h;
    if (pos_gt(t_new, dt) || pos_lt(dt - t_new, hmin)) t_new = dt;
    // predictor and the history term psi
    const double ig = bdf_inv_gamma(order);
    switch (order) {
      case 1: bdf_predict<1, NPL>(D, y, psi, ig); break;
      case 2: bdf_predict<2, NPL>(D, y, psi, ig); break;
      case 3: bdf_predict<3, NPL>(D, y, psi, ig); break;
      case 4: bdf_predict<4, NPL>(D, y, psi, ig); break;
      default: bdf_predict<5, NPL>(D, y, psi, ig); break;
    }
#pragma unroll
    for (int s = 0; s < NPL; ++s) {
      d[s] = 0.0;
      isc[s] = __frcp_rn(fmaf(rtolf, fabsf(narrow_f32(y[s])), atolf[s]));
    }
    const double c = h * ig;
    bool f_at_pred = false;
    if (need_jac) {
      rhs_eval<NPL, true>(m, w, pp, y, f, sp, cs, lane);
      jac_assemble<NPL>(m, w, y, sp, cs, lane);
      cnt[1]++;
      cnt[2]++;
      need_jac = false;
      jac_age = 0;
      have_lu = false;
      f_at_pred = true;   // f(ypred) doubles as the first Newton residual
    }
    // c / c_lu in FP32 (it only steers the refactorisation and the correction scale)
    float cr = narrow_f32(c * ic_lu);
    if (!have_lu || fabsf(cr - 1.0f) > 0.3f) {
      if (!lu_factor<NPL>(w, n, c, lane)) {
        // singular Newton matrix: shrink the step
        fails++;
        rescale_D<NPL>(D, order, 0.25, w, rc, lane);
        h *= 0.25;
        n_equal = 0;
        have_lu = false;
        continue;
      }
      cnt[3]++;
      c_lu = c;
      ic_lu = 1.0 / c;
      have_lu = true;
      crate = 0.5f;
    }
    // modified Newton with a stale h/gamma: scale the correction by 2 / (1 + c / c_lu)
    const bool rescale = c != c_lu;
    if (!rescale) cr = 1.0f;
    const double lscale = widen_f64(2.0f / (1.0f + cr));
    bool converged = false;
    float dn_old = 0.0f;
    newton_iters = 0;
    for (int it = 0; it < kNewtonMax; ++it) {
      if (!(it == 0 && f_at_pred)) {
        rhs_eval<NPL, false>(m, w, pp, y, f, sp, cs, lane);
        cnt[1]++;
      }
      bool ok = true;
#pragma unroll
      for (int s = 0; s < NPL; ++s) {
        if (!finite_bits(f[s])) ok = false;
        dy[s] = c * f[s] - psi[s] - d[s];
      }
      if (__any_sync(FULLMASK, !ok)) break;
      lu_solve<NPL>(w, n, dy, lane);
      if (rescale) {
#pragma unroll
        for (int s = 0; s < NPL; ++s) dy[s] *= lscale;
      }
      const float dn = wrms<NPL>(dy, isc, n, lane);
      ++newton_iters;
      if (it > 0) crate = fmaxf(0.3f * crate, dn / fmaxf(dn_old, 1e-30f));
#pragma unroll
      for (int s = 0; s < NPL; ++s) { y[s] += dy[s]; d[s] += dy[s]; }
      if (dn == 0.0f || (crate < 1.0f && crate / (1.0f - crate) * dn < ntol)) { converged = true; break; }
      if (it > 0 && dn > 2.0f * dn_old) break;
      dn_old = dn;
    }
    if (!converged) {
      fails++;
      if (jac_age > 0) {
        need_jac = true;       // retry this step with a fresh Jacobian
      } else {
        rescale_D<NPL>(D, order, 0.25, w, rc, lane);
        h *= 0.25;
        n_equal = 0;
      }
      continue;
    }
    // local error test
    const float safety = 0.9f * (2 * kNewtonMax + 1) / (float)(2 * kNewtonMax + newton_iters);
#pragma unroll
    for (int s = 0; s < NPL; ++s) isc[s] = __frcp_rn(fmaf(rtolf, fabsf(narrow_f32(y[s])), atolf[s]));
    const float en = wrms<NPL>(d, isc, n, lane) / (float)(order + 1);
    if (!(en <= 1.0f)) {
      fails++;
      const float fac = fmaxf(0.2f, safety * exp2f(-log2f(fmaxf(en, 1e-30f)) / (float)(order + 1)));
      const double facd = widen_f64(fac);
      rescale_D<NPL>(D, order, facd, w, rc, lane);
      h *= facd;
      n_equal = 0;
      continue;
    }
    // accept: D[order+2] = d - D[order+1]; D[order+1] = d; D[i] += D[i+1]
    fails = 0;
    t = t_new;
    cnt[0]++;
    n_equal++;
    jac_age++;
    switch (order) {
      case 1: bdf_accept<1, NPL>(D, d); break;
      case 2: bdf_accept<2, NPL>(D, d); break;
      case 3: bdf_accept<3, NPL>(D, d); break;
      case 4: bdf_accept<4, NPL>(D, d); break;
      default: bdf_accept<5, NPL>(D, d); break;
    }
    if (jac_age >= o.jac_max_age) need_jac = true;
    if (n_equal < order + 1) continue;
    // order and step-size selection
    double em[NPL], ep[NPL];
#pragma unroll
    for (int s = 0; s < NPL; ++s) {
      em[s] = 0.0;
      ep[s] = 0.0;
#pragma unroll
      for (int j = 0; j <= kMaxOrd + 2; ++j) {
        if (j == order) em[s] = D[j][s];
        if (j == order + 2) ep[s] = D[j][s];
      }
    }
    const float nm = order > 1 ? wrms<NPL>(em, isc, n, lane) / (float)order : 0.0f;
    const float np = order < kMaxOrd ? wrms<NPL>(ep, isc, n, lane) / (float)(order + 2) : 0.0f;
    const float fm = order > 1 ? (nm == 0.0f ? 1e30f : exp2f(-log2f(nm) / (float)order)) : 0.0f;
    const float f0 = en == 0.0f ? 1e30f : exp2f(-log2f(en) / (float)(order + 1));
    const float fp = order < kMaxOrd ? (np == 0.0f ? 1e30f : exp2f(-log2f(np) / (float)(order + 2))) : 0.0f;
    int delta = 0;
    float best = f0;
    if (fm > best) { best = fm; delta = -1; }
    if (fp > best) { best = fp; delta = 1; }
    order += delta;
    const float facf = fminf(10.0f, safety * best);
    n_equal = 0;
    // every proposed factor is taken, small growth included: a factor up to 1.3 reuses the
    // LU (the refactorisation test above), and keeping h below CVODE's 1.5 threshold cost
    // 16 % more steps on the 30-species workload
    const double fac = widen_f64(facf);
    rescale_D<NPL>(D, order, fac, w, rc, lane);
    h *= fac;
  }
  if (status == CHEM_CELL_OK) {
    bool okv = true;
#pragma unroll
    for (int s = 0; s < NPL; ++s) {
      if (lane + 32 * s < n && !isfinite(D[0][s])) okv = false;
    }
    if (__any_sync(FULLMASK, !okv)) status = CHEM_CELL_NONFINITE;
    else {
#pragma unroll
      for (int s = 0; s < NPL; ++s) z[s] = D[0][s];
    }
  }
  return status;
}

// ------------------------------------------------------------------------------------------
// kernels
// ------------------------------------------------------------------------------------------
template <int NPL>
__device__ __forceinline__ void load_cell(const DevMech& m, int64_t col, int64_t ld, const double* T,
                                          const double* Y, double (&z)[NPL], int lane) {
#pragma unroll
  for (int s = 0; s < NPL; ++s) {
    const int k = lane + 32 * s;
    z[s] = 0.0;
    if (k < m.K) z[s] = Y[(size_t)k * ld + col];
    else if (k == m.K) z[s] = T[col];
  }
}

template <int NPL>
__global__ void __launch_bounds__(NPL == 1 ? 160 : 128, 2) di_kernel(DevMech m, int64_t n, int64_t ld, double dt, double* T,
                                                 const double* p, double* Y, const int32_t* idx, DiOpts o,
                                                 int32_t* status, int32_t* stats, unsigned int* queue,
                                                 size_t warp_bytes, const int32_t* n_dev) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nT = m.I - m.n_tb_end;
  const WarpMem w = carve((double*)((char*)smem + wid * warp_bytes), m.K, m.I, m.n, nT, true, true,
                          NPL > 1 && di_use_j32(m.K, m.I, m.n, nT));
  // n_dev (optional): the number of entries of idx actually filled, known only on the device
  const int64_t n_eff = n_dev ? min(n, (int64_t)max(*n_dev, 0)) : n;
  while (true) {
    unsigned int slot = 0;
    if (lane == 0) slot = atomicAdd(queue, 1u);
    slot = __shfl_sync(FULLMASK, slot, 0);
    if ((int64_t)slot >= n_eff) break;
    const int64_t col = idx ? (int64_t)idx[slot] : (int64_t)slot;
    double z[NPL];
    int cnt[4];
    int st;
    if (col < 0 || col >= ld) {
      st = CHEM_CELL_OUT_OF_RANGE;
      cnt[0] = cnt[1] = cnt[2] = cnt[3] = 0;
    } else {
      load_cell<NPL>(m, col, ld, T, Y, z, lane);
      st = integrate_cell<NPL>(m, w, p[col], z, dt, o, lane, cnt);
      if (st == CHEM_CELL_OK) {
#pragma unroll
        for (int s = 0; s < NPL; ++s) {
          const int k = lane + 32 * s;
          if (k < m.K) Y[(size_t)k * ld + col] = z[s];
          else if (k == m.K) T[col] = z[s];
        }
      }
    }
    if (lane == 0) {
      status[slot] = st;
      if (stats) {
        stats[slot] = cnt[0];
        stats[n + slot] = cnt[1];
        stats[2 * n + slot] = cnt[2];
        stats[3 * n + slot] = cnt[3];
      }
    }
  }
}

template <int NPL>
__global__ void __launch_bounds__(128) rates_kernel(DevMech m, int64_t n, int64_t ld, const double* T,
                                                    const double* p, const double* Y, double* wdot,
                                                    double* hrr, size_t warp_bytes) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const WarpMem w = carve((double*)((char*)smem + wid * warp_bytes), m.K, m.I, m.n, m.I - m.n_tb_end, false, false);
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t col = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid; col < n; col += nw) {
    double z[NPL], f[NPL];
    LaneSp<NPL> sp;
    CellSc cs;
    load_cell<NPL>(m, col, ld, T, Y, z, lane);
    const double pc = p[col];
    rhs_eval<NPL, false>(m, w, cell_p(pc), z, f, sp, cs, lane);
#pragma unroll
    for (int s = 0; s < NPL; ++s) {
      const int k = lane + 32 * s;
      if (k < m.K) wdot[(size_t)k * ld + col] = sp.wdot[s];
    }
    if (hrr && lane == 0) hrr[col] = -cs.Q;
  }
}

template <int NPL>
__global__ void __launch_bounds__(128) jacobian_kernel(DevMech m, int64_t n, int64_t ld, const double* T,
                                                       const double* p, const double* Y, double* jac,
                                                       size_t warp_bytes) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const WarpMem w = carve((double*)((char*)smem + wid * warp_bytes), m.K, m.I, m.n, m.I - m.n_tb_end, false, true);
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int nn = m.n;
  for (int64_t col = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid; col < n; col += nw) {
    double z[NPL], f[NPL];
    LaneSp<NPL> sp;
    CellSc cs;
    load_cell<NPL>(m, col, ld, T, Y, z, lane);
    const double pc = p[col];
    rhs_eval<NPL, true>(m, w, cell_p(pc), z, f, sp, cs, lane);
    jac_assemble<NPL>(m, w, z, sp, cs, lane);
    double* out = jac + (size_t)col * nn * nn;
    for (int e = lane; e < nn * nn; e += 32) out[e] = w.J[(size_t)(e / nn) * w.ld + (e % nn)];
    __syncwarp();
  }
}

__global__ void exp_selftest_kernel(const double* __restrict__ tab, int64_t n, const double* x, double* y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = exp_t(x[i], tab);
}

__global__ void exp256_selftest_kernel(const double* __restrict__ tab, int64_t n, const double* x, double* y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = exp_s256(x[i], tab);
}

__global__ void log_selftest_kernel(const double* __restrict__ tab, int64_t n, const double* x, double* y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = log_t(x[i], tab);
}

__global__ void rcp_selftest_kernel(int64_t n, const double* x, double* y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = rcp_nr(x[i]);
}

// ------------------------------------------------------------------------------------------
// launches
// ------------------------------------------------------------------------------------------
int launch_rcp_selftest(int64_t n, const double* x, double* y, cudaStream_t s) {
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
  rcp_selftest_kernel<<<(int)blocks, 256, 0, s>>>(n, x, y);
  return cuda_check(cudaGetLastError(), "rcp_selftest_kernel launch");
}

int launch_exp_selftest(const DevMech& m, int64_t n, const double* x, double* y, cudaStream_t s) {
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
  exp_selftest_kernel<<<(int)blocks, 256, 0, s>>>(m.exptab, n, x, y);
  return cuda_check(cudaGetLastError(), "exp_selftest_kernel launch");
}

int launch_exp256_selftest(const DevMech& m, int64_t n, const double* x, double* y, cudaStream_t s) {
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
  exp256_selftest_kernel<<<(int)blocks, 256, 0, s>>>(m.exptab, n, x, y);
  return cuda_check(cudaGetLastError(), "exp256_selftest_kernel launch");
}

int launch_log_selftest(const DevMech& m, int64_t n, const double* x, double* y, cudaStream_t s) {
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
  log_selftest_kernel<<<(int)blocks, 256, 0, s>>>(m.logtab, n, x, y);
  return cuda_check(cudaGetLastError(), "log_selftest_kernel launch");
}

static int sm_count() {
  static int cached = 0;
  if (!cached) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev);
    if (cached <= 0) cached = 1;
  }
  return cached;
}

static int smem_optin() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

size_t di_smem_per_warp(const DevMech& m) {
  const int nT = m.I - m.n_tb_end;
  return warp_doubles(m.K, m.I, m.n, nT, true, true, m.n > 32 && di_use_j32(m.K, m.I, m.n, nT)) * sizeof(double);
}

template <typename KernelT>
static int configure(KernelT kern, size_t warp_bytes, int& warps_per_block, size_t& smem) {
  const int optin = smem_optin();
  warps_per_block = 4;
  while (warps_per_block > 1 && (size_t)warps_per_block * warp_bytes > (size_t)optin) --warps_per_block;
  smem = (size_t)warps_per_block * warp_bytes;
  if (smem > (size_t)optin)
    return set_error(CHEM_E_UNSUPPORTED, "mechanism needs more shared memory per warp than the device has");
  return cuda_check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                    "cudaFuncSetAttribute");
}

int launch_rates(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                 const double* Y, double* wdot, double* hrr, cudaStream_t s) {
  const size_t wb = warp_doubles(m.K, m.I, m.n, m.I - m.n_tb_end, false, false) * sizeof(double);
  int wpb;
  size_t smem;
  int rc;
  const int64_t want = (n + 3) / 4;
  if (m.n <= 32) {
    if ((rc = configure(rates_kernel<1>, wb, wpb, smem))) return rc;
    const int grid = (int)std::min<int64_t>((n + wpb - 1) / wpb, (int64_t)sm_count() * 64);
    rates_kernel<1><<<grid, 32 * wpb, smem, s>>>(m, n, ld, T, p, Y, wdot, hrr, wb);
  } else {
    if ((rc = configure(rates_kernel<2>, wb, wpb, smem))) return rc;
    const int grid = (int)std::min<int64_t>((n + wpb - 1) / wpb, (int64_t)sm_count() * 64);
    rates_kernel<2><<<grid, 32 * wpb, smem, s>>>(m, n, ld, T, p, Y, wdot, hrr, wb);
  }
  (void)want;
  return cuda_check(cudaGetLastError(), "rates_kernel launch");
}

int launch_jacobian(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                    const double* Y, double* jac, cudaStream_t s) {
  const size_t wb = warp_doubles(m.K, m.I, m.n, m.I - m.n_tb_end, false, true) * sizeof(double);
  int wpb;
  size_t smem;
  int rc;
  if (m.n <= 32) {
    if ((rc = configure(jacobian_kernel<1>, wb, wpb, smem))) return rc;
    const int grid = (int)std::min<int64_t>((n + wpb - 1) / wpb, (int64_t)sm_count() * 32);
    jacobian_kernel<1><<<grid, 32 * wpb, smem, s>>>(m, n, ld, T, p, Y, jac, wb);
  } else {
    if ((rc = configure(jacobian_kernel<2>, wb, wpb, smem))) return rc;
    const int grid = (int)std::min<int64_t>((n + wpb - 1) / wpb, (int64_t)sm_count() * 32);
    jacobian_kernel<2><<<grid, 32 * wpb, smem, s>>>(m, n, ld, T, p, Y, jac, wb);
  }
  return cuda_check(cudaGetLastError(), "jacobian_kernel launch");
}

int launch_di(const DevMech& m, int64_t n, int64_t ld, double dt, double* T, const double* p,
              double* Y, const int32_t* idx, const chem_di_opts& opts, int32_t* status,
              int32_t* stats, unsigned int* queue, cudaStream_t s, const int32_t* n_dev) {
  const size_t wb = di_smem_per_warp(m);
  DiOpts o{opts.rtol, opts.atol_Y, opts.atol_T, opts.newton_tol, opts.max_steps, opts.jac_max_age};
  int wpb;
  size_t smem;
  int rc;
  if (n > (int64_t)0x7fffffff) return set_error(CHEM_E_ARG, "chem_step_di: too many cells in one call");
  int dev = 0, per_sm = 0, max_threads_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_threads_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  // persistent grid: the block shape (1..5 warps) that keeps the most warps resident per SM
  auto best_shape = [&](auto kern) -> int {
    int best_w = 0;
    const int optin = smem_optin();
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return cuda_check(cudaGetLastError(), "di_kernel attributes");
    for (int cand = 5; cand >= 1; --cand) {
      if ((size_t)cand * wb > (size_t)optin || 32 * cand > fa.maxThreadsPerBlock) continue;
      int blocks = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, 32 * cand, (size_t)cand * wb);
      if (blocks * cand > best_w) { best_w = blocks * cand; wpb = cand; per_sm = blocks; }
    }
    smem = (size_t)wpb * wb;
    return best_w > 0 ? CHEM_OK : set_error(CHEM_E_UNSUPPORTED, "mechanism needs more shared memory per warp than the device has");
  };
  if (m.n <= 32) {
    if ((rc = best_shape(di_kernel<1>))) return rc;
    const int64_t grid = std::min<int64_t>((n + wpb - 1) / wpb, (int64_t)sm_count() * per_sm);
    di_kernel<1><<<(int)grid, 32 * wpb, smem, s>>>(m, n, ld, dt, T, p, Y, idx, o, status, stats, queue, wb, n_dev);
  } else {
    if ((rc = best_shape(di_kernel<2>))) return rc;
    const int64_t grid = std::min<int64_t>((n + wpb - 1) / wpb, (int64_t)sm_count() * per_sm);
    di_kernel<2><<<(int)grid, 32 * wpb, smem, s>>>(m, n, ld, dt, T, p, Y, idx, o, status, stats, queue, wb, n_dev);
  }
  return cuda_check(cudaGetLastError(), "di_kernel launch");
}

}  // namespace chem
