// Internal declarations shared by the libchem translation units (not part of the C ABI).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/chem.h"

namespace chem {

constexpr double kR = 8.314462618;    // J/mol/K
constexpr double kP0 = 101325.0;      // standard pressure of the NASA-7 entropies, Pa
constexpr int kMaxEx = 4;             // non-unit third-body efficiencies kept per reaction
constexpr int kThermoStride = 17;     // per species and range: cp(5) h(6) s(6)
constexpr double kDefaultNewtonTol = 0.2;   // Newton stop, in units of the local error test
// accepted steps between Jacobian evaluations (CVODE's default is 51; with the Newton stop at
// 0.2, 100 steps cost 2.9 % less time on the 30-species workload at unchanged parity)
constexpr int kDefaultJacMaxAge = 100;

// Device-resident mechanism tables.  Reactions are stored sorted by kind:
// [0, n_elem) elementary, [n_elem, n_tb_end) third-body, [n_tb_end, I) Troe falloff.
struct DevMech {
  int K, I, E, n;          // species, reactions, elements, unknowns per cell (K + 1)
  int n_elem, n_tb_end;
  int nnz;                 // entries of the species -> reaction incidence lists
  double Tmid;
  const double* W;         // [K] kg/mol
  const double* invW;      // [K]
  const double* th;        // [K][2][17]: low/high range; cp/R(5), h/RT(6: a1 a2/2 a3/3 a4/4 a5/5 a6),
                           //   s/R(6: a1 a2 a3/2 a4/3 a5/4 a7)
  const double* tr;        // [K][8]: ln mu fit (4), ln lambda fit (4)
  const double* wA;        // [K][K] 1/sqrt(8 (1 + W_k/W_j))
  const double* wB;        // [K][K] (W_j/W_k)^(1/4)
  const int* rsp;          // [I][8]: r0 r1 r2 nr p0 p1 p2 np
  const double* arr;       // [I][4]: ln A, b, Ea/R, sum nu (products - reactants)
  const int* ex_sp;        // [I][kMaxEx] species with non-unit efficiency (-1: none)
  const double* ex_a;      // [I][kMaxEx] efficiency - 1
  const double* troe;      // [I][8]: ln A0, b0, Ea0/R, a, 1/T***, 1/T*, T**, has T**
  const int* sp_ptr;       // [K+1]
  const int* sp_rxn;       // [nnz]
  const double* sp_nu;     // [nnz]
  // -g'_k/RT for the equilibrium constants, g' = g_k - sum_r P[k][r] g_{ref_r} the free
  // energy shifted by element potentials (P = composition x pinv(reference compositions));
  // balanced reactions cancel the shift exactly, and it keeps exp(-g') products in range.
  // Per species and range one polynomial: [0] + [1] ln T + T ([2] + T ([3] + T ([4] + T [5])))
  // + [6] / T ([7] unused), times 256/ln 2 (exp_s256's argument unit).
  const double* gneg;      // [K][2][8]
  const double* exptab;    // [256] 2^(j/256), the table of the FP64 exponential below
  const double* logtab;    // [97][3] F = j/128, 1/F, log F (j = 96..192): the table of log_t below
  const double* compW;     // [K][E] element counts divided by the molar mass (mol/kg)
  // the same rounded to FP32, for the learned step's FP32 parts
  const float* th32;       // [K][2][16]: c_p/R (5: a1..a5), h/RT (6: a1 a2/2 .. a5/5 a6), pad
  const float* invW32;     // [K]
  const float* compW32;    // [K][E]
  // Exponentials of one right-hand side, in lane rounds: item t < n_tb_end is k_f of reaction
  // t, then 5 per falloff reaction (k_inf, k_0/k_inf, the three F_cent terms).  Item t is
  // exp(x) with x = xarg[4t] + xarg[4t+1] ln T - xarg[4t+2] / T + xarg[4t+3] T, the
  // coefficients stored times 256/ln 2 (exp_s256's argument unit).
  int n_x;
  const double* xarg;      // [n_x][4]
  // Lane-balanced species production rates: lane L walks entries bal[i*32 + L], i < bal_P,
  // each |nu| (bits 0-1), nu < 0 (bit 2), last entry of its run (bit 3), run slot (bits 4-11),
  // reaction (bits 12-31); 0 = padding.  wdot_k = sum of the run slots run_ptr[k] ..
  // run_ptr[k+1] - 1 in order.  bal_P = 0: walk the incidence lists instead.
  int bal_P;
  const unsigned int* bal;   // [bal_P][32]
  const int* run_ptr;        // [K+1]
  // Two-partner form of the reactions, used when every reaction has at most two reactants and
  // two products (arity2 = 1): (r0, r1, p0, p1), a missing partner pointing at the sentinel
  // slot K of the per-species shared-memory vectors, which holds 1.
  int arity2;
  const int4* rsp2;          // [I]
};

// FP64 -> FP32 on the integer pipe for values that only steer heuristics or feed FP32 sums
// (exponent rebias, mantissa truncated: relative error below 2^-23).  |x| < 2^-126 gives a
// signed zero, |x| >= 2^128, inf and NaN give a signed inf.
__device__ __forceinline__ float narrow_f32(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int hi = (unsigned int)(b >> 32), lo = (unsigned int)b;
  const unsigned int e = (hi >> 20) & 0x7ffu, sgn = hi & 0x80000000u;
  const unsigned int f = ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  return __uint_as_float(e > 896u ? (e < 1151u ? (sgn | f) : (sgn | 0x7f800000u)) : sgn);
}

// FP32 -> FP64 on the integer pipe, exact for zero and normal numbers (sign kept, exponent
// rebiased by 1023 - 127, mantissa widened); used for small integers held in FP32.
__device__ __forceinline__ double widen_f64(float f) {
  const unsigned int b = __float_as_uint(f);
  const unsigned int mag = b & 0x7fffffffu, sgn = b & 0x80000000u;
  const unsigned int hi = mag ? (sgn | ((mag >> 3) + 0x38000000u)) : sgn;
  return __hiloint2double((int)hi, (int)(b << 29));
}

// FP64 exponential by the table-driven method (P. T. P. Tang, "Table-driven implementation of
// the exponential function in IEEE floating-point arithmetic", ACM TOMS 15, 1989), here with a
// 256-entry table: x = (256 k + j) ln2/256 + r, exp(x) = 2^k 2^(j/256) e^r, e^r - 1 from its
// degree-4 Taylor polynomial.  The split n = 256 k + j only has to keep r small, so it is
// taken from the FP32 value of x (integer-pipe narrowing, one FP32 FMA against 1.5 * 2^23,
// which rounds to an integer): for |x| < 709.8, |x 256/ln2 - n| <= 0.5 + 0.05, so |r| <=
// 1.49e-3 and the truncation |r|^5/120 < 6e-17 relative stays below an ulp.  n goes back to
// FP64 exactly through FP32 (|n| < 2^18) on the integer pipe, and n ln2/256 is split so that
// n times its high part is exact.  7 FP64 instructions (against ~22 FP64-pipe slots for the
// library exp on GB300); within 2 ulp of a correctly rounded exp (tested).
// Arguments below -708 return 0, above 709.78 return +inf, NaN propagates.
__device__ __forceinline__ double exp_t(double x, const double* __restrict__ tab) {
  const float kInvLf = 369.329930467574f;            // 256 / ln 2
  const float kMagicf = 12582912.0f;                 // 1.5 * 2^23: rounds to an integer
  const double kL1 = 0x1.62e42ff000000p-9;           // ln 2 / 256, high part (29 bits: nd kL1 exact)
  const double kL2 = -1.6409824502660487e-13;        // ln 2 / 256 - kL1
  const float tf = fmaf(narrow_f32(x), kInvLf, kMagicf);
  const int nn = (int)(__float_as_uint(tf) - 0x4B400000u);   // tf = 1.5 * 2^23 + n
  const double nd = widen_f64(tf - kMagicf);                 // n, exactly
  const double r = fma(-nd, kL2, fma(-nd, kL1, x));
  double q = fma(r, 1.0 / 24.0, 1.0 / 6.0);
  q = fma(q, r, 0.5);
  q = fma(q, r, 1.0);
  const double tj = __ldg(tab + (nn & 255));
  double res = fma(tj * r, q, tj);                   // 2^(j/256) (1 + r q)
  res = __longlong_as_double(__double_as_longlong(res) + ((long long)(nn >> 8) << 52));
  // |x| >= 708, inf and NaN, detected on the exponent bits (integer pipe, rare branch)
  if (((unsigned int)((unsigned long long)__double_as_longlong(x) >> 32) & 0x7fffffffu) >= 0x40862000u) {
    if (x != x) res = x;
    else if (x < -708.0) res = 0.0;
    else if (x > 709.78) res = __longlong_as_double(0x7ff0000000000000LL);
  }
  return res;
}
// exp of an argument given in units of ln2/256: exp_s256(y) = 2^(y/256) = exp(y ln2/256), the
// same table-driven method as exp_t for callers whose arguments are linear in tabulated
// coefficients (the rate constants and free energies of the chemistry kernels), which are
// stored pre-scaled by 256/ln 2.  y = 256 k + j + r_s with n = 256 k + j rounded from the FP32
// value of y (|y - n| <= 0.53) and r_s = y - n exact (Sterbenz); e^(r_s ln2/256) - 1 from
// its degree-4 Taylor polynomial in r_s, whose coefficients carry the powers of ln2/256
// (truncation below 5e-17 relative).  6 FP64 instructions; within 2 ulp of 2^(y/256)
// (tested).  y below -261485.59 (x < -708) returns 0, y >= 2^18 (x > 709.78) +inf, NaN
// propagates.
__device__ __forceinline__ double exp_s256(double y, const double* __restrict__ tab) {
  const float kMagicf = 12582912.0f;                 // 1.5 * 2^23: rounds to an integer
  const double c1 = 0.0027076061740622863;           // ln 2 / 256
  const double c2 = 3.6655655969101062e-06;          // c1^2 / 2
  const double c3 = 3.3083026805413713e-09;          // c1^3 / 6
  const double c4 = 2.239395190875157e-12;           // c1^4 / 24
  const float tf = narrow_f32(y) + kMagicf;
  const int nn = (int)(__float_as_uint(tf) - 0x4B400000u);   // tf = 1.5 * 2^23 + n
  const double rs = y - widen_f64(tf - kMagicf);             // y - n, exactly
  double q = fma(rs, c4, c3);
  q = fma(q, rs, c2);
  q = fma(q, rs, c1);
  const double tj = __ldg(tab + (nn & 255));
  double res = fma(tj * rs, q, tj);                  // 2^(j/256) (1 + r_s q)
  res = __longlong_as_double(__double_as_longlong(res) + ((long long)(nn >> 8) << 52));
  // |y| >= 261485, inf and NaN, detected on the exponent bits (integer pipe, rare branch)
  if (((unsigned int)((unsigned long long)__double_as_longlong(y) >> 32) & 0x7fffffffu) >= 0x410feb68u) {
    if (y != y) res = y;
    else if (y < -261485.59077104286) res = 0.0;
    else if (y >= 262144.0) res = __longlong_as_double(0x7ff0000000000000LL);
  }
  return res;
}

// FP64 natural logarithm by the table-driven method (P. T. P. Tang, "Table-driven
// implementation of the logarithm function in IEEE floating-point arithmetic", ACM TOMS 16,
// 1990): x = 2^k m with m in [0.75, 1.5), F = j/128 the grid point nearest m (j = 96..192),
// log x = k ln2 + log F + log1p(u), u = (m - F)/F (m - F exact), |u| <= 1/192, log1p(u) from
// its degree-7 Taylor polynomial (truncation < |u|^8/8: < 1.7e-18 |u| at F = 1, where u is
// exact, and < 3e-17 of the result elsewhere).  Centring m on 1 keeps log x accurate near
// x = 1; k ln2 is split (32-bit high part, exact product).
// tab[3(j-96) + {0, 1, 2}] = F_j, 1/F_j, log F_j.  Positive normal x only: zero, negative,
// subnormal, inf and NaN take the library log.
__device__ __forceinline__ double log_t(double x, const double* __restrict__ tab) {
  const long long b = __double_as_longlong(x);
  const unsigned int hw = (unsigned int)((unsigned long long)b >> 32);
  if (hw - 0x00100000u >= 0x7fe00000u) return log(x);
  const long long frac = b & 0x000fffffffffffffLL;
  const int up = (int)(frac >> 51);                 // m >= 1.5: use m/2 and k + 1
  const int j = (int)((frac + (1LL << 52) + (1LL << (44 + up))) >> (45 + up));     // round(128 m)
  const double* t = tab + 3 * (j - 96);
  const double m = __longlong_as_double(frac | ((long long)(1023 - up) << 52));
  const double u = (m - __ldg(t)) * __ldg(t + 1);
  double pl = fma(u, 1.0 / 7.0, -1.0 / 6.0);
  pl = fma(pl, u, 0.2);
  pl = fma(pl, u, -0.25);
  pl = fma(pl, u, 1.0 / 3.0);
  pl = fma(pl, u, -0.5);
  // k as a double without an FP64 instruction: 1.5 * 2^23 + k (any sign) has k in its low
  // bits, one FP32 subtraction leaves k exactly, and the integer pipe widens it
  const int k = (int)(hw >> 20) - 1023 + up;
  const double kd = widen_f64(__uint_as_float(0x4B400000u + (unsigned int)k) - 12582912.0f);
  const double kLn2Hi = 0x1.62e42fee00000p-1, kLn2Lo = 1.9082149292705877e-10;
  return fma(kd, kLn2Hi, __ldg(t + 2)) + fma(kd, kLn2Lo, fma(pl, u * u, u));
}
constexpr int kMaxElem = 8;

// 1/x from the hardware reciprocal estimate and one third-order step of the Newton-Raphson
// family for f(y) = 1/y - x (the series 1/x = y / (1 - e) = y (1 + e + e^2 + ...) with
// e = 1 - x y, truncated after e^2; e.g. Muller et al., Handbook of Floating-Point Arithmetic,
// ch. on iterative division): the relative error goes from eps to about eps^3.  The estimate
// was measured within 2^-19.9 relative on 2e8 random x, so one step reaches the rounding
// level: within 1 ulp of 1/x there.  3 FP64 instructions against 4 for two quadratic steps and
// about twice that for a correctly rounded division.  Zero, subnormal or infinite x give NaN
// (every caller treats that as a failed evaluation).
__device__ __forceinline__ double rcp_nr(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x, y, 1.0);
  return fma(y, fma(e, e, e), y);
}

struct HostMech;   // parsed mechanism (host)
const DevMech& mech_dev(chem_mech m);

// error reporting (thread-local message)
int set_error(int code, const std::string& msg);
int cuda_check(cudaError_t e, const char* what);

// launches (di.cu)
int launch_rates(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                 const double* Y, double* wdot, double* hrr, cudaStream_t s);
int launch_jacobian(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                    const double* Y, double* jac, cudaStream_t s);
int launch_di(const DevMech& m, int64_t n, int64_t ld, double dt, double* T, const double* p,
              double* Y, const int32_t* idx, const chem_di_opts& o, int32_t* status,
              int32_t* stats, unsigned int* queue, cudaStream_t s, const int32_t* n_dev = nullptr);
void di_fill_defaults(chem_di_opts& o);

// mlp.cu: C = A B^T on the tensor cores with a fused epilogue
struct GemmEpi {
  const float* bias;           // [N] or null
  void* out;                   // [M, ldo] BF16 or FP32
  int ldo;
  const __nv_bfloat16* z;      // epilogue 2: pre-activations [M, ldz]
  int ldz;
  __nv_bfloat16* zout;         // epilogue 0: optional copy of the pre-activations [M, ldo]
  // groups > 1: that many independent GEMMs of the same M, N, K in one launch.  Group g reads
  // its A tiles at coordinates offset by (row g a_row, column g a_col) and its B tiles by
  // (g b_row, g b_col), and writes out/zout at + g out_goff, reads z at + g z_goff and bias at
  // + g bias_goff (elements).  Column offsets are multiples of 8 (16-byte TMA coordinates).
  int groups;
  int a_row, a_col, b_row, b_col;
  int64_t out_goff, z_goff;
  int bias_goff;
};
int gemm_bf16(int epi, const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* B, int64_t ldb, int M, int N,
              int K, const GemmEpi& e, int* err, cudaStream_t s);
// output layer of per-species networks, backward to the last hidden layer: dZ[b, g h + j] =
// dU[b, g] W[g, j] GELU'(Z[b, g h + j]) (BF16 in and out, FP32 arithmetic)
int launch_group_out_dgrad(const __nv_bfloat16* dU, int ldu, const __nv_bfloat16* W, const __nv_bfloat16* Z,
                           int64_t B, int G, int h, __nv_bfloat16* dZ, cudaStream_t s);
size_t di_smem_per_warp(const DevMech& m);

int launch_rcp_selftest(int64_t n, const double* x, double* y, cudaStream_t s);
int launch_exp_selftest(const DevMech& m, int64_t n, const double* x, double* y, cudaStream_t s);
int launch_exp256_selftest(const DevMech& m, int64_t n, const double* x, double* y, cudaStream_t s);
int launch_log_selftest(const DevMech& m, int64_t n, const double* x, double* y, cudaStream_t s);

// thermo.cu
int launch_thermo(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* Y,
                  double* cp, double* h, double* mu, double* kappa, const double* h_in,
                  double* T_out, int mixed, cudaStream_t s);

// pasr.cu
int launch_pasr(const DevMech& m, int64_t n, int64_t ld, double dt, const double* rho, const double* Y0,
                const double* Y1, const double* ksgs, const double* eps, const double* nu, double y_min,
                double r_min, double* omega, double* kappa, cudaStream_t s);

// hfrd.cu
struct HfrdIdx {
  int i_n2, el_C, el_H, el_O, el_N;
};
int launch_hfrd(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p, const double* Y,
                const double* gamma, const chem_hfrd_opts& o, const HfrdIdx& ix, double* T_out, double* p_out,
                double* Y_out, int32_t* keep, double* ranges, cudaStream_t s);

// probe.cu
int launch_fp64_probe(double* gflops, cudaStream_t s);

}  // namespace chem
