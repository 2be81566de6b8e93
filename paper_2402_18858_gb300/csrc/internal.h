// Internal declarations shared by the libchem translation units (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/chem.h"

namespace chem {

constexpr double kR = 8.314462618;    // J/mol/K
constexpr double kP0 = 101325.0;      // standard pressure of the NASA-7 entropies, Pa
constexpr int kMaxEx = 4;             // non-unit third-body efficiencies kept per reaction
constexpr int kThermoStride = 17;     // per species and range: cp(5) h(6) s(6)

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
  // Element-potential shift of g/RT for the equilibrium constants: species k uses
  // g_k - sum_r P[k][r] g_{ref_r}, with P = composition x pinv(reference compositions).
  // Balanced reactions cancel the shift exactly; it keeps exp(-g) products in range.
  int n_ref;               // number of reference species (rank of the composition matrix)
  const int* ref_sp;       // [n_ref]
  const double* P;         // [K][n_ref]
};
constexpr int kMaxElem = 8;

struct HostMech;   // parsed mechanism (host)

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
              int32_t* stats, unsigned int* queue, cudaStream_t s);
size_t di_smem_per_warp(const DevMech& m);

// thermo.cu
int launch_thermo(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* Y,
                  double* cp, double* h, double* mu, double* kappa, const double* h_in,
                  double* T_out, int mixed, cudaStream_t s);

// probe.cu
int launch_fp64_probe(double* gflops, cudaStream_t s);

}  // namespace chem
