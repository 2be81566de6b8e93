// libchem C ABI: mechanism loading and the host side of every entry point.
//
// The mechanism loader turns the plain-text SI mechanism file into device tables laid out
// for the warp-per-cell kernels: reactions sorted by kind (elementary, third-body, Troe) so
// that the lanes of a warp take the same branch, NASA-7 coefficients pre-divided for the
// h/RT and s/R polynomials, sparse third-body efficiency exceptions, the Wilke constants
// that depend only on molar masses, and a species -> reaction incidence list so that the
// production rates are gathered per species in a fixed order (deterministic, no atomics).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "internal.h"

namespace chem {

static thread_local std::string g_last_error;

int set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return CHEM_OK;
  return set_error(CHEM_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

struct HostRxn {
  int kind = 0;                 // 0 elementary, 1 third-body, 2 Troe
  std::vector<int> reac, prod;
  double A = 0, b = 0, Ea = 0;
  std::vector<std::pair<int, double>> eff;
  double A0 = 0, b0 = 0, Ea0 = 0;
  std::vector<double> troe;
};

struct HostMech {
  std::vector<std::string> elements, species;
  std::vector<double> W;
  std::vector<int> comp;          // [K][E]
  double Tlow = 0, Tmid = 0, Thigh = 0;
  std::vector<double> nasa;       // [K][14]
  std::vector<double> transport;  // [K][8]
  std::vector<HostRxn> rxn;
};

static int parse_mech(const char* path, HostMech& hm) {
  std::ifstream in(path);
  if (!in) return set_error(CHEM_E_PARSE, std::string("cannot open mechanism file ") + path);
  std::map<std::string, int> sp_index;
  std::string tok;
  int K = -1, I = -1;
  bool saw_thermo = false, saw_end = false;
  std::vector<int> have_nasa, have_tr;
  auto species_of = [&](const std::string& s) -> int {
    auto it = sp_index.find(s);
    return it == sp_index.end() ? -1 : it->second;
  };
  auto bad = [&](const std::string& why) { return set_error(CHEM_E_PARSE, std::string(path) + ": " + why); };
  while (in >> tok) {
    if (tok == "mech") {
      std::string name;
      if (!(in >> name)) return bad("missing mechanism name");
    } else if (tok == "elements") {
      while (in >> tok && tok != "species") hm.elements.push_back(tok);
      if (tok != "species" || !(in >> K) || K <= 0) return bad("bad species count");
      if (K > CHEM_MAX_SPECIES)
        return set_error(CHEM_E_UNSUPPORTED, "mechanism has more species than the kernels support");
      const int E = (int)hm.elements.size();
      if (E < 1 || E > kMaxElem) return set_error(CHEM_E_UNSUPPORTED, "between 1 and 8 elements are supported");
      hm.species.resize(K);
      hm.W.resize(K);
      hm.comp.assign((size_t)K * E, 0);
      hm.nasa.assign((size_t)K * 14, 0.0);
      hm.transport.assign((size_t)K * 8, 0.0);
      have_nasa.assign(K, 0);
      have_tr.assign(K, 0);
      for (int k = 0; k < K; ++k) {
        if (!(in >> tok) || tok != "sp") return bad("expected 'sp'");
        if (!(in >> hm.species[k] >> hm.W[k]) || !(hm.W[k] > 0)) return bad("bad species line");
        if (sp_index.count(hm.species[k])) return bad("duplicate species " + hm.species[k]);
        sp_index[hm.species[k]] = k;
        for (int e = 0; e < E; ++e)
          if (!(in >> hm.comp[(size_t)k * E + e]) || hm.comp[(size_t)k * E + e] < 0) return bad("bad composition");
      }
    } else if (tok == "thermo_ranges") {
      if (!(in >> hm.Tlow >> hm.Tmid >> hm.Thigh) || !(hm.Tmid > 0)) return bad("bad thermo ranges");
      saw_thermo = true;
    } else if (tok == "nasa7" || tok == "transport") {
      const bool nasa = tok == "nasa7";
      std::string s;
      if (!(in >> s)) return bad("truncated line");
      int k = species_of(s);
      if (k < 0) return bad("unknown species " + s);
      for (int i = 0; i < (nasa ? 14 : 8); ++i) {
        double v;
        if (!(in >> v) || !std::isfinite(v)) return bad("bad coefficient for " + s);
        (nasa ? hm.nasa[(size_t)k * 14 + i] : hm.transport[(size_t)k * 8 + i]) = v;
      }
      (nasa ? have_nasa : have_tr)[k] = 1;
    } else if (tok == "reactions") {
      if (!(in >> I) || I < 0) return bad("bad reaction count");
      if (I > CHEM_MAX_REACTIONS)
        return set_error(CHEM_E_UNSUPPORTED, "mechanism has more reactions than the kernels support");
      hm.rxn.reserve(I);
    } else if (tok == "rxn") {
      if ((int)hm.rxn.size() >= I) return bad("more reactions than declared");
      HostRxn r;
      std::string kind;
      in >> kind;
      r.kind = kind == "elem" ? 0 : kind == "threebody" ? 1 : kind == "troe" ? 2 : -1;
      if (r.kind < 0) return bad("unknown reaction kind " + kind);
      for (int side = 0; side < 2; ++side) {
        int cnt;
        if (!(in >> cnt) || cnt < 1 || cnt > 3) return bad("bad stoichiometry count");
        for (int t = 0; t < cnt; ++t) {
          std::string s;
          in >> s;
          int k = species_of(s);
          if (k < 0) return bad("unknown species " + s + " in reaction");
          (side ? r.prod : r.reac).push_back(k);
        }
      }
      if (!(in >> r.A >> r.b >> r.Ea) || !(r.A > 0)) return bad("bad Arrhenius parameters");
      hm.rxn.push_back(r);
    } else if (tok == "eff") {
      int cnt;
      if (hm.rxn.empty() || !(in >> cnt) || cnt < 0) return bad("bad efficiency line");
      for (int t = 0; t < cnt; ++t) {
        std::string s;
        double a;
        if (!(in >> s >> a) || !(a >= 0)) return bad("bad efficiency entry");
        int k = species_of(s);
        if (k < 0) return bad("unknown species " + s + " in efficiencies");
        hm.rxn.back().eff.push_back({k, a});
      }
    } else if (tok == "low") {
      HostRxn& r = hm.rxn.back();
      if (hm.rxn.empty() || !(in >> r.A0 >> r.b0 >> r.Ea0) || !(r.A0 > 0)) return bad("bad low-pressure limit");
    } else if (tok == "troe") {
      int cnt;
      if (hm.rxn.empty() || !(in >> cnt) || cnt < 3 || cnt > 4) return bad("bad Troe line");
      HostRxn& r = hm.rxn.back();
      r.troe.resize(cnt);
      for (int t = 0; t < cnt; ++t)
        if (!(in >> r.troe[t])) return bad("bad Troe parameter");
      if (!(r.troe[1] > 0) || !(r.troe[2] > 0)) return bad("Troe T*** and T* must be positive");
    } else if (tok == "end") {
      saw_end = true;
      break;
    } else {
      return bad("unknown keyword '" + tok + "'");
    }
  }
  if (!saw_end || K <= 0 || I < 0 || !saw_thermo) return bad("incomplete mechanism");
  if ((int)hm.rxn.size() != I) return bad("fewer reactions than declared");
  for (int k = 0; k < K; ++k)
    if (!have_nasa[k] || !have_tr[k]) return bad("missing thermo or transport data for " + hm.species[k]);
  const int E = (int)hm.elements.size();
  for (int j = 0; j < I; ++j) {
    const HostRxn& r = hm.rxn[j];
    if (r.kind == 2 && (r.troe.empty() || !(r.A0 > 0))) return bad("Troe reaction without low/troe data");
    if ((int)r.eff.size() > kMaxEx) return set_error(CHEM_E_UNSUPPORTED, "too many third-body efficiencies");
    for (int e = 0; e < E; ++e) {
      int s = 0;
      for (int k : r.reac) s += hm.comp[(size_t)k * E + e];
      for (int k : r.prod) s -= hm.comp[(size_t)k * E + e];
      if (s != 0) return bad("reaction " + std::to_string(j) + " is not element balanced");
    }
  }
  return CHEM_OK;
}

}  // namespace chem

struct chem_mech_s {
  chem::DevMech dev{};
  void* dmem = nullptr;
  int device = 0;
  int K = 0, I = 0, E = 0;
  int i_n2 = -1;                          // species N2 (-1: none)
  int el_C = -1, el_H = -1, el_O = -1, el_N = -1;   // element indices (-1: absent)
};

using namespace chem;

const DevMech& chem::mech_dev(chem_mech m) { return m->dev; }

// Pack the host mechanism into one device allocation and point DevMech at its pieces.
static int upload(const HostMech& hm, chem_mech_s* cm) {
  const int K = (int)hm.species.size(), I = (int)hm.rxn.size();
  // order reactions by kind
  std::vector<int> order(I);
  for (int j = 0; j < I; ++j) order[j] = j;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return hm.rxn[a].kind < hm.rxn[b].kind; });
  int n_elem = 0, n_tb_end = 0;
  for (int j = 0; j < I; ++j) {
    if (hm.rxn[j].kind == 0) ++n_elem;
    if (hm.rxn[j].kind <= 1) ++n_tb_end;
  }
  std::vector<double> W(K), invW(K), th((size_t)K * 2 * kThermoStride), tr((size_t)K * 8);
  std::vector<double> wA((size_t)K * K), wB((size_t)K * K);
  for (int k = 0; k < K; ++k) {
    W[k] = hm.W[k];
    invW[k] = 1.0 / hm.W[k];
    for (int rg = 0; rg < 2; ++rg) {
      const double* a = &hm.nasa[(size_t)k * 14 + 7 * rg];
      double* o = &th[((size_t)k * 2 + rg) * kThermoStride];
      for (int i = 0; i < 5; ++i) o[i] = a[i];                   // cp/R
      for (int i = 0; i < 5; ++i) o[5 + i] = a[i] / (i + 1);     // h/RT polynomial
      o[10] = a[5];
      o[11] = a[0];                                              // s/R: a1 ln T + ...
      o[12] = a[1];
      o[13] = a[2] / 2;
      o[14] = a[3] / 3;
      o[15] = a[4] / 4;
      o[16] = a[6];
    }
    for (int i = 0; i < 8; ++i) tr[(size_t)k * 8 + i] = hm.transport[(size_t)k * 8 + i];
    for (int j = 0; j < K; ++j) {
      wA[(size_t)k * K + j] = 1.0 / std::sqrt(8.0 * (1.0 + hm.W[k] / hm.W[j]));
      wB[(size_t)k * K + j] = std::pow(hm.W[j] / hm.W[k], 0.25);
    }
  }
  std::vector<int> rsp((size_t)std::max(I, 1) * 8, -1), ex_sp((size_t)std::max(I, 1) * kMaxEx, -1);
  std::vector<double> arr((size_t)std::max(I, 1) * 4, 0.0), ex_a((size_t)std::max(I, 1) * kMaxEx, 0.0);
  std::vector<double> troe((size_t)std::max(I, 1) * 8, 0.0);
  std::vector<std::vector<std::pair<int, double>>> inc(K);
  for (int jj = 0; jj < I; ++jj) {
    const HostRxn& r = hm.rxn[order[jj]];
    int* s = &rsp[(size_t)jj * 8];
    for (size_t t = 0; t < r.reac.size(); ++t) s[t] = r.reac[t];
    s[3] = (int)r.reac.size();
    for (size_t t = 0; t < r.prod.size(); ++t) s[4 + t] = r.prod[t];
    s[7] = (int)r.prod.size();
    arr[(size_t)jj * 4 + 0] = std::log(r.A);
    arr[(size_t)jj * 4 + 1] = r.b;
    arr[(size_t)jj * 4 + 2] = r.Ea / kR;
    arr[(size_t)jj * 4 + 3] = (double)r.prod.size() - (double)r.reac.size();
    for (size_t t = 0; t < r.eff.size(); ++t) {
      ex_sp[(size_t)jj * kMaxEx + t] = r.eff[t].first;
      ex_a[(size_t)jj * kMaxEx + t] = r.eff[t].second - 1.0;
    }
    if (r.kind == 2) {
      double* tp = &troe[(size_t)jj * 8];
      tp[0] = std::log(r.A0);
      tp[1] = r.b0;
      tp[2] = r.Ea0 / kR;
      tp[3] = r.troe[0];
      tp[4] = 1.0 / r.troe[1];
      tp[5] = 1.0 / r.troe[2];
      tp[6] = r.troe.size() == 4 ? r.troe[3] : 0.0;
      tp[7] = r.troe.size() == 4 ? 1.0 : 0.0;
    }
    // net stoichiometric coefficient per species
    std::map<int, double> nu;
    for (int k : r.reac) nu[k] -= 1.0;
    for (int k : r.prod) nu[k] += 1.0;
    for (auto& kv : nu)
      if (kv.second != 0.0) inc[kv.first].push_back({jj, kv.second});
  }
  // Reference species for the element potentials: greedily, the species with the fewest
  // atoms that raise the rank of the composition matrix.  lambda = Linv g_ref solves
  // sum_e a_re lambda_e = g_r in the least-squares sense over the chosen rows, so that
  // g_k - sum_e a_ke lambda_e is centred; balanced reactions cancel the shift exactly.
  const int E = (int)hm.elements.size();
  std::vector<int> by_atoms(K);
  for (int k = 0; k < K; ++k) by_atoms[k] = k;
  auto atoms = [&](int k) { int a = 0; for (int e = 0; e < E; ++e) a += hm.comp[(size_t)k * E + e]; return a; };
  std::stable_sort(by_atoms.begin(), by_atoms.end(), [&](int a, int b) { return atoms(a) < atoms(b); });
  std::vector<int> refs;
  std::vector<std::vector<double>> basis;   // Gram-Schmidt rows of the chosen compositions
  for (int k : by_atoms) {
    if ((int)refs.size() == E) break;
    std::vector<double> v(E);
    for (int e = 0; e < E; ++e) v[e] = hm.comp[(size_t)k * E + e];
    for (auto& b : basis) {
      double d = 0, bb = 0;
      for (int e = 0; e < E; ++e) { d += v[e] * b[e]; bb += b[e] * b[e]; }
      for (int e = 0; e < E; ++e) v[e] -= d / bb * b[e];
    }
    double nv = 0;
    for (int e = 0; e < E; ++e) nv += v[e] * v[e];
    if (nv > 1e-9) { basis.push_back(v); refs.push_back(k); }
  }
  const int R = (int)refs.size();
  // Linv = pinv(A) with A = comp rows of refs (R x E): Linv = A^T (A A^T)^{-1}  (E x R)
  std::vector<double> AAt((size_t)R * R, 0.0), inv((size_t)R * R, 0.0), Linv((size_t)E * std::max(R, 1), 0.0);
  for (int a = 0; a < R; ++a)
    for (int b = 0; b < R; ++b)
      for (int e = 0; e < E; ++e) AAt[(size_t)a * R + b] += (double)hm.comp[(size_t)refs[a] * E + e] * hm.comp[(size_t)refs[b] * E + e];
  for (int a = 0; a < R; ++a) inv[(size_t)a * R + a] = 1.0;
  for (int c = 0; c < R; ++c) {   // Gauss-Jordan with partial pivoting
    int pr = c;
    for (int r = c + 1; r < R; ++r) if (std::fabs(AAt[(size_t)r * R + c]) > std::fabs(AAt[(size_t)pr * R + c])) pr = r;
    for (int j = 0; j < R; ++j) { std::swap(AAt[(size_t)c * R + j], AAt[(size_t)pr * R + j]); std::swap(inv[(size_t)c * R + j], inv[(size_t)pr * R + j]); }
    const double d = AAt[(size_t)c * R + c];
    for (int j = 0; j < R; ++j) { AAt[(size_t)c * R + j] /= d; inv[(size_t)c * R + j] /= d; }
    for (int r = 0; r < R; ++r) {
      if (r == c) continue;
      const double f = AAt[(size_t)r * R + c];
      for (int j = 0; j < R; ++j) { AAt[(size_t)r * R + j] -= f * AAt[(size_t)c * R + j]; inv[(size_t)r * R + j] -= f * inv[(size_t)c * R + j]; }
    }
  }
  for (int e = 0; e < E; ++e)
    for (int b = 0; b < R; ++b) {
      double acc = 0;
      for (int a = 0; a < R; ++a) acc += (double)hm.comp[(size_t)refs[a] * E + e] * inv[(size_t)a * R + b];
      Linv[(size_t)e * R + b] = acc;
    }
  std::vector<double> Pm((size_t)K * std::max(R, 1), 0.0);
  for (int k = 0; k < K; ++k)
    for (int r = 0; r < R; ++r) {
      double acc = 0;
      for (int e = 0; e < E; ++e) acc += (double)hm.comp[(size_t)k * E + e] * Linv[(size_t)e * R + r];
      Pm[(size_t)k * R + r] = acc;
    }
  // exponent arguments of the kernels' exponential are kept in units of ln2/256
  const long double kExpScale = 256.0L / 0.693147180559945309417232121458176568L;
  // -g'_k/RT per species and range as one polynomial in (1, ln T, T, T^2, T^3, T^4, 1/T):
  // g/RT = h/RT - s/R = (a1 - a7) - a1 ln T - a2 T/2 - a3 T^2/6 - a4 T^3/12 - a5 T^4/20 + a6/T
  // of the NASA-7 fit (coefficients a1..a7), shifted by the element potentials,
  // g' = g - sum_r P[k][r] g_ref_r (formed in long double, rounded once)
  std::vector<double> gneg((size_t)K * 2 * 8, 0.0);
  for (int rg = 0; rg < 2; ++rg) {
    auto gcoef = [&](int k, long double* c) {
      const double* a = &hm.nasa[(size_t)k * 14 + 7 * rg];
      c[0] = (long double)a[0] - (long double)a[6];
      c[1] = -(long double)a[0];
      c[2] = -(long double)a[1] / 2;
      c[3] = -(long double)a[2] / 6;
      c[4] = -(long double)a[3] / 12;
      c[5] = -(long double)a[4] / 20;
      c[6] = (long double)a[5];
    };
    for (int k = 0; k < K; ++k) {
      long double c[7], cr[7];
      gcoef(k, c);
      for (int r = 0; r < R; ++r) {
        gcoef(refs[r], cr);
        for (int i = 0; i < 7; ++i) c[i] -= (long double)Pm[(size_t)k * R + r] * cr[i];
      }
      for (int i = 0; i < 7; ++i) gneg[((size_t)k * 2 + rg) * 8 + i] = (double)(-c[i] * kExpScale);
    }
  }
  std::vector<double> exptab(256);
  for (int j = 0; j < 256; ++j) exptab[j] = (double)std::exp2((long double)j / 256.0L);
  std::vector<double> logtab(3 * 97);
  for (int j = 96; j <= 192; ++j) {
    const long double F = (long double)j / 128.0L;
    logtab[3 * (j - 96)] = (double)F;
    logtab[3 * (j - 96) + 1] = (double)(1.0L / F);
    logtab[3 * (j - 96) + 2] = (double)std::log(F);
  }
  // FP32 copies for the learned step's update (its enthalpy, element sums and T(h) run in
  // FP32): NASA-7 c_p/R (5) and h/RT (6) per species and range, 1/W, composition / W
  std::vector<float> th32((size_t)K * 2 * 16, 0.0f), invW32(K), compW32((size_t)K * E);
  for (int k = 0; k < K; ++k) {
    invW32[k] = (float)(1.0 / hm.W[k]);
    for (int rg = 0; rg < 2; ++rg)
      for (int c = 0; c < 11; ++c)
        th32[((size_t)k * 2 + rg) * 16 + c] = (float)th[((size_t)k * 2 + rg) * kThermoStride + c];
    for (int e = 0; e < E; ++e) compW32[(size_t)k * E + e] = (float)(hm.comp[(size_t)k * E + e] / hm.W[k]);
  }
  std::vector<double> compW((size_t)K * E);
  for (int k = 0; k < K; ++k)
    for (int e = 0; e < E; ++e) compW[(size_t)k * E + e] = hm.comp[(size_t)k * E + e] / hm.W[k];
  // exponential items of the right-hand side (see DevMech::xarg)
  const int nT = I - n_tb_end;
  const int n_x = n_tb_end + 5 * nT;
  std::vector<double> xarg((size_t)std::max(n_x, 1) * 4, 0.0);
  for (int jj = 0; jj < n_tb_end; ++jj)
    for (int c = 0; c < 3; ++c) xarg[(size_t)jj * 4 + c] = arr[(size_t)jj * 4 + c];
  for (int jt = 0; jt < nT; ++jt) {
    const int jj = n_tb_end + jt;
    const double* a = &arr[(size_t)jj * 4];
    const double* tp = &troe[(size_t)jj * 8];
    double* x = &xarg[(size_t)(n_tb_end + 5 * jt) * 4];
    x[0] = a[0]; x[1] = a[1]; x[2] = a[2];                            // k_inf
    x[4] = tp[0] - a[0]; x[5] = tp[1] - a[1]; x[6] = tp[2] - a[2];    // k_0 / k_inf
    x[11] = -tp[4];                                                   // exp(-T / T***)
    x[15] = -tp[5];                                                   // exp(-T / T*)
    if (tp[7] != 0.0) x[18] = tp[6];                                  // exp(-T** / T)
    else x[16] = -1e300;                                              // absent term: 0
  }
  for (auto& v : xarg) v = (double)((long double)v * kExpScale);

  std::vector<int> sp_ptr(K + 1, 0), sp_rxn;
  std::vector<double> sp_nu;
  for (int k = 0; k < K; ++k) {
    sp_ptr[k] = (int)sp_rxn.size();
    for (auto& e : inc[k]) {
      sp_rxn.push_back(e.first);
      sp_nu.push_back(e.second);
    }
  }
  sp_ptr[K] = (int)sp_rxn.size();
  // Lane-balanced schedule of the species production rates (see DevMech::bal): the incidence
  // entries in species order, cut into 32 equal segments, one per lane; a segment's
  // consecutive entries of one species form a run whose partial sum goes to its own slot.
  const int E_inc = (int)sp_rxn.size();
  int bal_P = (E_inc + 31) / 32;
  std::vector<unsigned int> bal((size_t)std::max(bal_P, 1) * 32, 0u);
  std::vector<int> run_ptr(K + 1, 0);
  {
    int runs = 0;
    bool ok = bal_P > 0 && I < (1 << 20);
    std::vector<int> run_of_entry(E_inc, -1), sp_of(E_inc);
    for (int k = 0; k < K; ++k)
      for (int e = sp_ptr[k]; e < sp_ptr[k + 1]; ++e) sp_of[e] = k;
    for (int e = 0; e < E_inc && ok; ++e) {
      const bool first = e == 0 || sp_of[e] != sp_of[e - 1] || e % bal_P == 0;
      if (first) ++runs;
      run_of_entry[e] = runs - 1;
      const double nu = sp_nu[e];
      const int a = (int)std::fabs(nu);
      if ((double)a != std::fabs(nu) || a < 1 || a > 3) ok = false;
    }
    if (runs > 3 * K || runs > 255) ok = false;   // the runs' slots reuse 3K dead doubles
    if (ok) {
      for (int k = 0; k < K; ++k) run_ptr[k] = sp_ptr[k] < sp_ptr[k + 1] ? run_of_entry[sp_ptr[k]] : -1;
      run_ptr[K] = runs;
      for (int k = K - 1; k >= 0; --k) if (run_ptr[k] < 0) run_ptr[k] = run_ptr[k + 1];
      for (int e = 0; e < E_inc; ++e) {
        const int lane = e / bal_P, i = e % bal_P;
        const bool last = e + 1 == E_inc || run_of_entry[e + 1] != run_of_entry[e];
        const double nu = sp_nu[e];
        bal[(size_t)i * 32 + lane] = (unsigned int)std::fabs(nu) | (nu < 0 ? 4u : 0u) | (last ? 8u : 0u) |
                                     ((unsigned int)run_of_entry[e] << 4) | ((unsigned int)sp_rxn[e] << 12);
      }
    } else {
      bal_P = 0;
    }
  }
  // two-partner reaction table (see DevMech::rsp2)
  std::vector<int> rsp2((size_t)std::max(I, 1) * 4, K);
  int arity2 = 1;
  for (int jj = 0; jj < I; ++jj) {
    const int* s = &rsp[(size_t)jj * 8];
    if (s[3] > 2 || s[7] > 2) arity2 = 0;
    rsp2[(size_t)jj * 4 + 0] = s[0];
    rsp2[(size_t)jj * 4 + 1] = s[3] > 1 ? s[1] : K;
    rsp2[(size_t)jj * 4 + 2] = s[4];
    rsp2[(size_t)jj * 4 + 3] = s[7] > 1 ? s[5] : K;
  }
  const int nnz = std::max((int)sp_rxn.size(), 1);
  sp_rxn.resize(nnz, 0);
  sp_nu.resize(nnz, 0.0);

  // one allocation, 256-byte aligned pieces
  struct Piece { const void* src; size_t bytes; size_t off; };
  std::vector<Piece> pieces;
  size_t total = 0;
  auto add = [&](const void* src, size_t bytes) {
    size_t off = total;
    pieces.push_back({src, bytes, off});
    total += (bytes + 255) & ~size_t(255);
    return off;
  };
  size_t oW = add(W.data(), W.size() * 8), oiW = add(invW.data(), invW.size() * 8);
  size_t oth = add(th.data(), th.size() * 8), otr = add(tr.data(), tr.size() * 8);
  size_t owA = add(wA.data(), wA.size() * 8), owB = add(wB.data(), wB.size() * 8);
  size_t orsp = add(rsp.data(), rsp.size() * 4), oarr = add(arr.data(), arr.size() * 8);
  size_t oexs = add(ex_sp.data(), ex_sp.size() * 4), oexa = add(ex_a.data(), ex_a.size() * 8);
  size_t otroe = add(troe.data(), troe.size() * 8), optr = add(sp_ptr.data(), sp_ptr.size() * 4);
  size_t orxn = add(sp_rxn.data(), sp_rxn.size() * 4), onu = add(sp_nu.data(), sp_nu.size() * 8);
  size_t ogn = add(gneg.data(), gneg.size() * 8);
  size_t oth32 = add(th32.data(), th32.size() * 4), oiw32 = add(invW32.data(), invW32.size() * 4);
  size_t ocw32 = add(compW32.data(), compW32.size() * 4);
  size_t oexp = add(exptab.data(), exptab.size() * 8), ocw = add(compW.data(), compW.size() * 8);
  size_t oxa = add(xarg.data(), xarg.size() * 8), olog = add(logtab.data(), logtab.size() * 8);
  size_t obal = add(bal.data(), bal.size() * 4), orun = add(run_ptr.data(), run_ptr.size() * 4);
  size_t orsp2 = add(rsp2.data(), rsp2.size() * 4);
  std::vector<char> blob(total, 0);
  for (auto& p : pieces) std::memcpy(blob.data() + p.off, p.src, p.bytes);
  void* d = nullptr;
  if (cudaMalloc(&d, total) != cudaSuccess) {
    cudaGetLastError();
    return set_error(CHEM_E_NOMEM, "cudaMalloc of mechanism tables failed");
  }
  int rc = cuda_check(cudaMemcpy(d, blob.data(), total, cudaMemcpyHostToDevice), "mechanism upload");
  if (rc) { cudaFree(d); return rc; }
  char* b = (char*)d;
  DevMech& m = cm->dev;
  m.K = K; m.I = I; m.E = (int)hm.elements.size(); m.n = K + 1;
  m.n_elem = n_elem; m.n_tb_end = n_tb_end; m.nnz = (int)sp_ptr[K];
  m.Tmid = hm.Tmid;
  m.W = (const double*)(b + oW); m.invW = (const double*)(b + oiW);
  m.th = (const double*)(b + oth); m.tr = (const double*)(b + otr);
  m.wA = (const double*)(b + owA); m.wB = (const double*)(b + owB);
  m.rsp = (const int*)(b + orsp); m.arr = (const double*)(b + oarr);
  m.ex_sp = (const int*)(b + oexs); m.ex_a = (const double*)(b + oexa);
  m.troe = (const double*)(b + otroe); m.sp_ptr = (const int*)(b + optr);
  m.sp_rxn = (const int*)(b + orxn); m.sp_nu = (const double*)(b + onu);
  m.gneg = (const double*)(b + ogn);
  m.exptab = (const double*)(b + oexp);
  m.logtab = (const double*)(b + olog);
  m.compW = (const double*)(b + ocw);
  m.th32 = (const float*)(b + oth32);
  m.invW32 = (const float*)(b + oiw32);
  m.compW32 = (const float*)(b + ocw32);
  m.n_x = n_x;
  m.xarg = (const double*)(b + oxa);
  m.bal_P = bal_P;
  m.bal = (const unsigned int*)(b + obal);
  m.run_ptr = (const int*)(b + orun);
  m.arity2 = arity2;
  m.rsp2 = (const int4*)(b + orsp2);
  cm->dmem = d;
  cm->K = K; cm->I = I; cm->E = m.E;
  for (int k = 0; k < K; ++k)
    if (hm.species[k] == "N2") cm->i_n2 = k;
  for (int e = 0; e < (int)hm.elements.size(); ++e) {
    const std::string& nm = hm.elements[e];
    if (nm == "C") cm->el_C = e;
    if (nm == "H") cm->el_H = e;
    if (nm == "O") cm->el_O = e;
    if (nm == "N") cm->el_N = e;
  }
  return CHEM_OK;
}

static int check_mech(chem_mech m) {
  if (!m || !m->dmem) return set_error(CHEM_E_ARG, "null or freed mechanism handle");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != m->device)
    return set_error(CHEM_E_ARG, "mechanism was loaded on another device");
  return CHEM_OK;
}

extern "C" {

int chem_load_mech(const char* path, chem_mech* out) {
  if (!path || !out) return set_error(CHEM_E_ARG, "chem_load_mech: null argument");
  *out = nullptr;
  HostMech hm;
  int rc = parse_mech(path, hm);
  if (rc) return rc;
  chem_mech_s* cm = new chem_mech_s();
  if ((rc = cuda_check(cudaGetDevice(&cm->device), "cudaGetDevice"))) { delete cm; return rc; }
  if ((rc = upload(hm, cm))) { delete cm; return rc; }
  *out = cm;
  return CHEM_OK;
}

void chem_free_mech(chem_mech m) {
  if (!m) return;
  if (m->dmem) cudaFree(m->dmem);
  m->dmem = nullptr;
  delete m;
}

int chem_mech_info(chem_mech m, int* n_species, int* n_reactions, int* n_elements) {
  if (!m) return set_error(CHEM_E_ARG, "null mechanism handle");
  if (n_species) *n_species = m->K;
  if (n_reactions) *n_reactions = m->I;
  if (n_elements) *n_elements = m->E;
  return CHEM_OK;
}

const char* chem_last_error(void) { return g_last_error.c_str(); }

int chem_rates(chem_mech m, int64_t n, int64_t ld, const double* T, const double* p,
               const double* Y, double* wdot, double* hrr, chem_stream stream) {
  int rc = check_mech(m);
  if (rc) return rc;
  if (n < 0 || ld < n) return set_error(CHEM_E_ARG, "chem_rates: need 0 <= n <= ld");
  if (n == 0) return CHEM_OK;
  if (!T || !p || !Y || !wdot) return set_error(CHEM_E_ARG, "chem_rates: null array");
  return launch_rates(m->dev, n, ld, T, p, Y, wdot, hrr, (cudaStream_t)stream);
}

int chem_jacobian(chem_mech m, int64_t n, int64_t ld, const double* T, const double* p,
                  const double* Y, double* jac, chem_stream stream) {
  int rc = check_mech(m);
  if (rc) return rc;
  if (n < 0 || ld < n) return set_error(CHEM_E_ARG, "chem_jacobian: need 0 <= n <= ld");
  if (n == 0) return CHEM_OK;
  if (!T || !p || !Y || !jac) return set_error(CHEM_E_ARG, "chem_jacobian: null array");
  return launch_jacobian(m->dev, n, ld, T, p, Y, jac, (cudaStream_t)stream);
}

}  // extern "C"

void chem::di_fill_defaults(chem_di_opts& o) {
  if (!(o.rtol > 0)) o.rtol = 1e-9;
  if (!(o.atol_Y > 0)) o.atol_Y = 1e-18;
  if (!(o.atol_T > 0)) o.atol_T = 1e-9;
  if (o.max_steps <= 0) o.max_steps = 20000;
  if (!(o.newton_tol > 0)) o.newton_tol = kDefaultNewtonTol;
  if (o.jac_max_age <= 0) o.jac_max_age = kDefaultJacMaxAge;
}

extern "C" {

size_t chem_workspace_bytes(chem_mech m, int64_t n) {
  (void)m;
  (void)n;
  return 256;   // the cell work-queue counter, padded to one 256-byte line
}

int chem_step_di(chem_mech m, int64_t n, int64_t ld, double dt, double* T, const double* p,
                 double* Y, const int32_t* idx, const chem_di_opts* opts, int32_t* status,
                 int32_t* stats, void* workspace, size_t ws_bytes, chem_stream stream) {
  int rc = check_mech(m);
  if (rc) return rc;
  if (n < 0 || ld < n) return set_error(CHEM_E_ARG, "chem_step_di: need 0 <= n <= ld");
  if (!(dt >= 0) || !std::isfinite(dt)) return set_error(CHEM_E_ARG, "chem_step_di: dt must be finite and >= 0");
  if (n == 0) return CHEM_OK;
  if (!T || !p || !Y || !status) return set_error(CHEM_E_ARG, "chem_step_di: null array");
  if (!workspace || ws_bytes < chem_workspace_bytes(m, n))
    return set_error(CHEM_E_WORKSPACE, "chem_step_di: workspace missing or smaller than chem_workspace_bytes()");
  chem_di_opts o{};
  if (opts) o = *opts;
  di_fill_defaults(o);
  if (!(o.rtol < 1) || !std::isfinite(o.atol_Y) || !std::isfinite(o.atol_T))
    return set_error(CHEM_E_ARG, "chem_step_di: bad tolerances");
  if ((rc = cuda_check(cudaMemsetAsync(workspace, 0, sizeof(unsigned int), (cudaStream_t)stream),
                       "chem_step_di: queue reset")))
    return rc;
  return launch_di(m->dev, n, ld, dt, T, p, Y, idx, o, status, stats, (unsigned int*)workspace,
                   (cudaStream_t)stream);
}

int thermo_props(chem_mech m, int64_t n, int64_t ld, const double* T, const double* Y,
                 double* cp, double* h, double* mu, double* kappa, const double* h_in,
                 double* T_out, int mixed_precision, chem_stream stream) {
  int rc = check_mech(m);
  if (rc) return rc;
  if (n < 0 || ld < n) return set_error(CHEM_E_ARG, "thermo_props: need 0 <= n <= ld");
  if (n == 0) return CHEM_OK;
  if (!T || !Y) return set_error(CHEM_E_ARG, "thermo_props: null T or Y");
  if (h_in && !T_out) return set_error(CHEM_E_ARG, "thermo_props: h_in given without T_out");
  if (mixed_precision != 0 && mixed_precision != 1)
    return set_error(CHEM_E_ARG, "thermo_props: mixed_precision must be 0 or 1");
  return launch_thermo(m->dev, n, ld, T, Y, cp, h, mu, kappa, h_in, T_out, mixed_precision,
                       (cudaStream_t)stream);
}

int chem_pasr_source(chem_mech m, int64_t n, int64_t ld, double dt, const double* rho, const double* Y0,
                     const double* Y1, const double* k_sgs, const double* eps, const double* nu, double y_min,
                     double r_min, double* omega, double* kappa, chem_stream stream) {
  int rc = check_mech(m);
  if (rc) return rc;
  if (n < 0 || ld < n) return set_error(CHEM_E_ARG, "chem_pasr_source: need 0 <= n <= ld");
  if (!(dt > 0.0) || !(dt < 1e300)) return set_error(CHEM_E_ARG, "chem_pasr_source: dt must be positive and finite");
  if (n == 0) return CHEM_OK;
  if (!rho || !Y0 || !Y1 || !k_sgs || !eps || !nu || !omega)
    return set_error(CHEM_E_ARG, "chem_pasr_source: null array argument");
  if (!(y_min == y_min)) return set_error(CHEM_E_ARG, "chem_pasr_source: y_min is NaN");
  if (!(r_min == r_min)) return set_error(CHEM_E_ARG, "chem_pasr_source: r_min is NaN");
  if (y_min < 0.0) y_min = 1e-10;
  if (r_min < 0.0) r_min = 1e-9;
  return launch_pasr(m->dev, n, ld, dt, rho, Y0, Y1, k_sgs, eps, nu, y_min, r_min, omega, kappa,
                     (cudaStream_t)stream);
}

size_t chem_hfrd_workspace_bytes(void) { return 256; }

int chem_hfrd_augment(chem_mech m, int64_t n, int64_t ld, const double* T, const double* p, const double* Y,
                      const double* gamma, const chem_hfrd_opts* opts, double* T_out, double* p_out,
                      double* Y_out, int32_t* keep, void* workspace, size_t ws_bytes, chem_stream stream) {
  int rc = check_mech(m);
  if (rc) return rc;
  if (n < 0 || ld < n) return set_error(CHEM_E_ARG, "chem_hfrd_augment: need 0 <= n <= ld");
  if (n == 0) return CHEM_OK;
  if (!T || !p || !Y || !gamma || !T_out || !p_out || !Y_out || !keep)
    return set_error(CHEM_E_ARG, "chem_hfrd_augment: null array argument");
  if (!workspace || ws_bytes < chem_hfrd_workspace_bytes())
    return set_error(CHEM_E_WORKSPACE, "chem_hfrd_augment: workspace missing or smaller than chem_hfrd_workspace_bytes()");
  if (m->i_n2 < 0 || m->el_H < 0 || m->el_O < 0 || m->el_N < 0)
    return set_error(CHEM_E_UNSUPPORTED, "chem_hfrd_augment: the mechanism needs species N2 and elements H, O, N");
  chem_hfrd_opts o{0.125, 10.0, 0.1, {2.65, 4.67}, {0.254, 0.320}, {0.20, 1.15}};
  if (opts) o = *opts;
  HfrdIdx ix{m->i_n2, m->el_C, m->el_H, m->el_O, m->el_N};
  return launch_hfrd(m->dev, n, ld, T, p, Y, gamma, o, ix, T_out, p_out, Y_out, keep, (double*)workspace,
                     (cudaStream_t)stream);
}

int chem_selftest_exp(chem_mech m, int64_t n, const double* x, double* y, chem_stream stream) {
  int rc = check_mech(m);
  if (rc) return rc;
  if (n < 0 || (n > 0 && (!x || !y))) return set_error(CHEM_E_ARG, "chem_selftest_exp: bad arguments");
  if (n == 0) return CHEM_OK;
  return launch_exp_selftest(m->dev, n, x, y, (cudaStream_t)stream);
}

int chem_selftest_exp256(chem_mech m, int64_t n, const double* x, double* y, chem_stream stream) {
  int rc = check_mech(m);
  if (rc) return rc;
  if (n < 0 || (n > 0 && (!x || !y))) return set_error(CHEM_E_ARG, "chem_selftest_exp256: bad arguments");
  if (n == 0) return CHEM_OK;
  return launch_exp256_selftest(m->dev, n, x, y, (cudaStream_t)stream);
}

int chem_selftest_log(chem_mech m, int64_t n, const double* x, double* y, chem_stream stream) {
  int rc = check_mech(m);
  if (rc) return rc;
  if (n < 0 || (n > 0 && (!x || !y))) return set_error(CHEM_E_ARG, "chem_selftest_log: bad arguments");
  if (n == 0) return CHEM_OK;
  return launch_log_selftest(m->dev, n, x, y, (cudaStream_t)stream);
}

int chem_selftest_rcp(int64_t n, const double* x, double* y, chem_stream stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return set_error(CHEM_E_ARG, "chem_selftest_rcp: bad arguments");
  if (n == 0) return CHEM_OK;
  return launch_rcp_selftest(n, x, y, (cudaStream_t)stream);
}

int chem_fp64_peak_gflops(double* gflops, chem_stream stream) {
  if (!gflops) return set_error(CHEM_E_ARG, "chem_fp64_peak_gflops: null output");
  return launch_fp64_probe(gflops, (cudaStream_t)stream);
}

}  // extern "C"
