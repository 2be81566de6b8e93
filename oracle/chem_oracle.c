/*
 * CPU FP64 oracle for the per-cell chemistry step.  TEST INFRASTRUCTURE ONLY: it is called by
 * the tests, by the package's smoke check and by the benchmark's CPU-baseline leg, never by the
 * GPU library.  It shares no code with the CUDA path (its own parser, its own formulas).
 *
 * What it computes (the paper's Sec. 2.2):
 *   Eq. 1 -- the reaction ODE of a closed, adiabatic, constant-pressure cell, state
 *            z = (Y_1..Y_K, T):  dY_k/dt = W_k wdot_k / rho,
 *                                dT/dt   = -sum_k h_k wdot_k / (rho c_p);
 *   Eq. 2 -- the map z(t) -> z(t + dt) obtained by integrating Eq. 1 over one flow step.
 * The paper gives no kinetics formulas (it runs Cantera + CVODE); the textbook forms used here
 * follow Kee, Coltrin & Glarborg, "Chemically Reacting Flow" (Chemkin conventions):
 *   NASA-7 polynomials (two ranges), k = A T^b exp(-Ea/RT), third-body [M] = sum alpha_k C_k,
 *   Lindemann falloff with the Troe broadening factor (Gilbert, Luther & Troe 1983),
 *   K_c = exp(-sum nu g/RT) (p0/RT)^{sum nu}, k_r = k_f / K_c.
 * The integrator is the three-stage Radau IIA method (order 5, L-stable; Hairer & Wanner,
 * "Solving ODEs II", Sec. IV.5) with a FULL Newton iteration on its stage equations (the
 * analytic Jacobian at every stage value and a fresh LU at every iterate) and step-size
 * control by step doubling -- a one-step implicit Runge-Kutta method, deliberately unrelated
 * to the multistep BDF scheme of the paper's CVODE (Sec. 2.2) and of the GPU kernel.
 * A fixed-step classical RK4 is the second, independent path for small checks.
 * Mixture properties: c_p, h mass-weighted; Wilke's rule for viscosity; the Mathur-Saxena
 * average for conductivity; T from h by Newton (the paper's Sec. 2.1 "Newton's method and
 * high-order temperature polynomials").
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_R 8.314462618
#define OR_P0 101325.0
#define OR_NAME 24

typedef struct {
  int K, I, E;
  char (*name)[OR_NAME];
  char (*elem)[8];
  double* W;      /* [K] kg/mol */
  int* comp;      /* [K*E] */
  double Tlow, Tmid, Thigh;
  double* alow;   /* [K*7] */
  double* ahigh;  /* [K*7] */
  double* mufit;  /* [K*4] */
  double* lamfit; /* [K*4] */
  int* kind;      /* [I] 0 elementary, 1 third body, 2 Troe */
  int* nreac;     /* [I] */
  int* nprod;     /* [I] */
  int* reac;      /* [I*3] */
  int* prod;      /* [I*3] */
  double *A, *b, *Ea;    /* [I] SI */
  double* eff;           /* [I*K] third-body efficiencies (1 by default) */
  double *A0, *b0, *Ea0; /* [I] low-pressure limit of Troe reactions */
  int* ntroe;            /* [I] 3 or 4 */
  double* troe;          /* [I*4] a, T3, T1, T2 */
} omech;

/* ------------------------------------------------------------------------------------ */
/* parsing                                                                              */
/* ------------------------------------------------------------------------------------ */
static int find_species(const omech* m, const char* s) {
  for (int k = 0; k < m->K; ++k)
    if (strcmp(m->name[k], s) == 0) return k;
  return -1;
}

static void or_free_fields(omech* m) {
  if (!m) return;
  free(m->name); free(m->elem); free(m->W); free(m->comp); free(m->alow); free(m->ahigh);
  free(m->mufit); free(m->lamfit); free(m->kind); free(m->nreac); free(m->nprod);
  free(m->reac); free(m->prod); free(m->A); free(m->b); free(m->Ea); free(m->eff);
  free(m->A0); free(m->b0); free(m->Ea0); free(m->ntroe); free(m->troe);
}

void or_mech_free(void* h) {
  omech* m = (omech*)h;
  or_free_fields(m);
  free(m);
}

#define FAIL(msg) do { snprintf(err, errlen, "%s", msg); goto bad; } while (0)

void* or_mech_load(const char* path, char* err, int errlen) {
  FILE* f = fopen(path, "r");
  if (!f) { snprintf(err, errlen, "cannot open %s", path); return NULL; }
  omech* m = (omech*)calloc(1, sizeof(omech));
  char tok[256];
  int ir = -1;
  while (fscanf(f, "%255s", tok) == 1) {
    if (strcmp(tok, "mech") == 0) {
      if (fscanf(f, "%255s", tok) != 1) FAIL("bad mech line");
    } else if (strcmp(tok, "elements") == 0) {
      /* the element list ends at the 'species' keyword */
      char names[16][8]; int ne = 0;
      while (fscanf(f, "%255s", tok) == 1 && strcmp(tok, "species") != 0) {
        if (ne >= 16) FAIL("too many elements");
        snprintf(names[ne++], 8, "%.7s", tok);
      }
      m->E = ne;
      m->elem = (char(*)[8])calloc(ne, 8);
      for (int e = 0; e < ne; ++e) memcpy(m->elem[e], names[e], 8);
      if (fscanf(f, "%d", &m->K) != 1 || m->K <= 0) FAIL("bad species count");
      int K = m->K;
      m->name = (char(*)[OR_NAME])calloc(K, OR_NAME);
      m->W = (double*)calloc(K, sizeof(double));
      m->comp = (int*)calloc(K * m->E, sizeof(int));
      m->alow = (double*)calloc(K * 7, sizeof(double));
      m->ahigh = (double*)calloc(K * 7, sizeof(double));
      m->mufit = (double*)calloc(K * 4, sizeof(double));
      m->lamfit = (double*)calloc(K * 4, sizeof(double));
      for (int k = 0; k < K; ++k) {
        if (fscanf(f, "%255s", tok) != 1 || strcmp(tok, "sp") != 0) FAIL("expected sp");
        if (fscanf(f, "%23s %lf", m->name[k], &m->W[k]) != 2) FAIL("bad sp");
        for (int e = 0; e < m->E; ++e)
          if (fscanf(f, "%d", &m->comp[k * m->E + e]) != 1) FAIL("bad composition");
      }
    } else if (strcmp(tok, "thermo_ranges") == 0) {
      if (fscanf(f, "%lf %lf %lf", &m->Tlow, &m->Tmid, &m->Thigh) != 3) FAIL("bad ranges");
    } else if (strcmp(tok, "nasa7") == 0 || strcmp(tok, "transport") == 0) {
      int is_nasa = tok[0] == 'n';
      if (fscanf(f, "%255s", tok) != 1) FAIL("bad line");
      int k = find_species(m, tok);
      if (k < 0) FAIL("unknown species in thermo/transport");
      for (int i = 0; i < (is_nasa ? 14 : 8); ++i) {
        double v;
        if (fscanf(f, "%lf", &v) != 1) FAIL("bad coefficient");
        if (is_nasa) { if (i < 7) m->alow[k * 7 + i] = v; else m->ahigh[k * 7 + i - 7] = v; }
        else { if (i < 4) m->mufit[k * 4 + i] = v; else m->lamfit[k * 4 + i - 4] = v; }
      }
    } else if (strcmp(tok, "reactions") == 0) {
      if (fscanf(f, "%d", &m->I) != 1 || m->I < 0) FAIL("bad reaction count");
      int I = m->I, K = m->K;
      m->kind = (int*)calloc(I, sizeof(int));
      m->nreac = (int*)calloc(I, sizeof(int));
      m->nprod = (int*)calloc(I, sizeof(int));
      m->reac = (int*)calloc(I * 3, sizeof(int));
      m->prod = (int*)calloc(I * 3, sizeof(int));
      m->A = (double*)calloc(I, sizeof(double));
      m->b = (double*)calloc(I, sizeof(double));
      m->Ea = (double*)calloc(I, sizeof(double));
      m->eff = (double*)calloc((size_t)I * K, sizeof(double));
      m->A0 = (double*)calloc(I, sizeof(double));
      m->b0 = (double*)calloc(I, sizeof(double));
      m->Ea0 = (double*)calloc(I, sizeof(double));
      m->ntroe = (int*)calloc(I, sizeof(int));
      m->troe = (double*)calloc(I * 4, sizeof(double));
      for (int i = 0; i < I * K; ++i) m->eff[i] = 1.0;
    } else if (strcmp(tok, "rxn") == 0) {
      ++ir;
      if (ir >= m->I) FAIL("too many reactions");
      if (fscanf(f, "%255s", tok) != 1) FAIL("bad rxn");
      m->kind[ir] = strcmp(tok, "elem") == 0 ? 0 : strcmp(tok, "threebody") == 0 ? 1
                  : strcmp(tok, "troe") == 0 ? 2 : -1;
      if (m->kind[ir] < 0) FAIL("unknown reaction kind");
      for (int side = 0; side < 2; ++side) {
        int cnt;
        if (fscanf(f, "%d", &cnt) != 1 || cnt < 1 || cnt > 3) FAIL("bad stoichiometry count");
        for (int t = 0; t < cnt; ++t) {
          if (fscanf(f, "%255s", tok) != 1) FAIL("bad species");
          int k = find_species(m, tok);
          if (k < 0) FAIL("unknown species in reaction");
          if (side == 0) m->reac[ir * 3 + t] = k; else m->prod[ir * 3 + t] = k;
        }
        if (side == 0) m->nreac[ir] = cnt; else m->nprod[ir] = cnt;
      }
      if (fscanf(f, "%lf %lf %lf", &m->A[ir], &m->b[ir], &m->Ea[ir]) != 3) FAIL("bad Arrhenius");
    } else if (strcmp(tok, "eff") == 0) {
      int cnt;
      if (ir < 0 || fscanf(f, "%d", &cnt) != 1) FAIL("bad eff");
      for (int t = 0; t < cnt; ++t) {
        double a;
        if (fscanf(f, "%255s %lf", tok, &a) != 2) FAIL("bad eff entry");
        int k = find_species(m, tok);
        if (k < 0) FAIL("unknown species in eff");
        m->eff[(size_t)ir * m->K + k] = a;
      }
    } else if (strcmp(tok, "low") == 0) {
      if (ir < 0 || fscanf(f, "%lf %lf %lf", &m->A0[ir], &m->b0[ir], &m->Ea0[ir]) != 3) FAIL("bad low");
    } else if (strcmp(tok, "troe") == 0) {
      int cnt;
      if (ir < 0 || fscanf(f, "%d", &cnt) != 1 || cnt < 3 || cnt > 4) FAIL("bad troe");
      m->ntroe[ir] = cnt;
      for (int t = 0; t < cnt; ++t)
        if (fscanf(f, "%lf", &m->troe[ir * 4 + t]) != 1) FAIL("bad troe value");
    } else if (strcmp(tok, "end") == 0) {
      break;
    } else {
      FAIL("unknown keyword");
    }
  }
  fclose(f);
  if (m->K <= 0 || ir + 1 != m->I) { snprintf(err, errlen, "incomplete mechanism"); or_mech_free(m); return NULL; }
  for (int i = 0; i < m->I; ++i) {
    if (m->kind[i] == 2 && m->ntroe[i] == 0) { snprintf(err, errlen, "troe reaction without parameters"); or_mech_free(m); return NULL; }
    /* element balance */
    for (int e = 0; e < m->E; ++e) {
      int s = 0;
      for (int t = 0; t < m->nreac[i]; ++t) s += m->comp[m->reac[i * 3 + t] * m->E + e];
      for (int t = 0; t < m->nprod[i]; ++t) s -= m->comp[m->prod[i * 3 + t] * m->E + e];
      if (s != 0) { snprintf(err, errlen, "reaction %d is not element balanced", i); or_mech_free(m); return NULL; }
    }
  }
  return m;
bad:
  fclose(f);
  or_mech_free(m);
  return NULL;
}

void or_mech_dims(const void* h, int* K, int* I, int* E) {
  const omech* m = (const omech*)h;
  *K = m->K; *I = m->I; *E = m->E;
}

void or_mech_W(const void* h, double* W) {
  const omech* m = (const omech*)h;
  for (int k = 0; k < m->K; ++k) W[k] = m->W[k];
}

void or_mech_comp(const void* h, int* comp) {
  const omech* m = (const omech*)h;
  for (int i = 0; i < m->K * m->E; ++i) comp[i] = m->comp[i];
}

/* ------------------------------------------------------------------------------------ */
/* species thermo (NASA-7)                                                               */
/* ------------------------------------------------------------------------------------ */
/* cp/R, h/(RT), s/R and d(cp/R)/dT of species k at T */
static void nasa7(const omech* m, int k, double T, double* cpR, double* hRT, double* sR, double* dcpR) {
  const double* a = (T < m->Tmid) ? &m->alow[k * 7] : &m->ahigh[k * 7];
  *cpR = a[0] + a[1] * T + a[2] * T * T + a[3] * T * T * T + a[4] * T * T * T * T;
  *hRT = a[0] + a[1] * T / 2 + a[2] * T * T / 3 + a[3] * T * T * T / 4 + a[4] * T * T * T * T / 5
       + a[5] / T;
  *sR = a[0] * log(T) + a[1] * T + a[2] * T * T / 2 + a[3] * T * T * T / 3 + a[4] * T * T * T * T / 4
      + a[6];
  if (dcpR) *dcpR = a[1] + 2 * a[2] * T + 3 * a[3] * T * T + 4 * a[4] * T * T * T;
}

void or_species_thermo(const void* h, double T, double* cpR, double* hRT, double* sR) {
  const omech* m = (const omech*)h;
  for (int k = 0; k < m->K; ++k) nasa7(m, k, T, &cpR[k], &hRT[k], &sR[k], NULL);
}

/* ------------------------------------------------------------------------------------ */
/* kinetics                                                                              */
/* ------------------------------------------------------------------------------------ */
typedef struct {
  double kf, kr;      /* effective forward/reverse rate constants (falloff included) */
  double M;           /* third-body concentration (1 if none) */
  double q;           /* net rate of progress, mol/m^3/s */
} rxn_state;

/* Troe falloff: returns k and, if asked, dk/d[M] and dln k/dT at fixed [M] */
static double troe_k(const omech* m, int i, double T, double M, double kinf, double dlnkinf,
                     double* dk_dM, double* dlnk_dT) {
  double k0 = m->A0[i] * pow(T, m->b0[i]) * exp(-m->Ea0[i] / (OR_R * T));
  double dlnk0 = m->b0[i] / T + m->Ea0[i] / (OR_R * T * T);
  const double* tp = &m->troe[i * 4];
  double a = tp[0], T3 = tp[1], T1 = tp[2];
  double Fc = (1 - a) * exp(-T / T3) + a * exp(-T / T1);
  double dFc = -(1 - a) / T3 * exp(-T / T3) - a / T1 * exp(-T / T1);
  if (m->ntroe[i] == 4) {
    double T2 = tp[3];
    Fc += exp(-T2 / T);
    dFc += T2 / (T * T) * exp(-T2 / T);
  }
  double Pr = k0 * M / kinf;
  if (Pr < 1e-300) Pr = 1e-300;
  double L = log10(Fc);
  double c = -0.4 - 0.67 * L;
  double n = 0.75 - 1.27 * L;
  double x = log10(Pr) + c;
  double den = n - 0.14 * x;
  double f1 = x / den;
  double logF = L / (1 + f1 * f1);
  double F = pow(10.0, logF);
  double k = kinf * Pr / (1 + Pr) * F;
  /* g = d log10 F / d log10 Pr at fixed T */
  double df1_dx = n / (den * den);
  double g = -L * 2 * f1 / ((1 + f1 * f1) * (1 + f1 * f1)) * df1_dx;
  if (dk_dM) *dk_dM = k0 * F * (1.0 / ((1 + Pr) * (1 + Pr)) + g / (1 + Pr));
  if (dlnk_dT) {
    double df1_dn = -x / (den * den);
    double df1_dL = df1_dx * (-0.67) + df1_dn * (-1.27);
    double dlogF_dL = 1 / (1 + f1 * f1) - L * 2 * f1 / ((1 + f1 * f1) * (1 + f1 * f1)) * df1_dL;
    double dlnPr = dlnk0 - dlnkinf;
    *dlnk_dT = dlnkinf + (1 / (1 + Pr) + g) * dlnPr + dlogF_dL * dFc / Fc;
  }
  return k;
}

/* Concentrations from (T, p, Y): rho = p Wbar/(R T), C_k = rho Y_k / W_k */
static double concentrations(const omech* m, double T, double p, const double* Y, double* C) {
  double s = 0;
  for (int k = 0; k < m->K; ++k) s += Y[k] / m->W[k];
  double rho = p / (OR_R * T * s);
  for (int k = 0; k < m->K; ++k) C[k] = rho * Y[k] / m->W[k];
  return rho;
}

/* Rates of progress of every reaction (and optionally their T- and C-derivatives). */
static void reaction_rates(const omech* m, double T, const double* C, const double* hRT,
                           const double* sR, rxn_state* rs,
                           double* dq_dC /* [I*K] or NULL */, double* dq_dT /* [I] or NULL */) {
  int K = m->K;
  double lnT = log(T);
  for (int i = 0; i < m->I; ++i) {
    double kf = m->A[i] * exp(m->b[i] * lnT - m->Ea[i] / (OR_R * T));
    double dlnkf = m->b[i] / T + m->Ea[i] / (OR_R * T * T);
    /* third-body concentration */
    double M = 1.0;
    if (m->kind[i] >= 1) {
      M = 0;
      for (int k = 0; k < K; ++k) M += m->eff[(size_t)i * K + k] * C[k];
    }
    double dk_dM = 0;
    if (m->kind[i] == 2) {
      double dlnk;
      kf = troe_k(m, i, T, M, kf, dlnkf, &dk_dM, &dlnk);
      dlnkf = dlnk;
    }
    /* equilibrium constant */
    int dnu = m->nprod[i] - m->nreac[i];
    double sum_g = 0, sum_h = 0;
    for (int t = 0; t < m->nprod[i]; ++t) {
      int k = m->prod[i * 3 + t];
      sum_g += hRT[k] - sR[k];
      sum_h += hRT[k];
    }
    for (int t = 0; t < m->nreac[i]; ++t) {
      int k = m->reac[i * 3 + t];
      sum_g -= hRT[k] - sR[k];
      sum_h -= hRT[k];
    }
    double Kc = exp(-sum_g) * pow(OR_P0 / (OR_R * T), dnu);
    double kr = kf / Kc;
    /* d ln Kc / dT = sum nu h/(R T^2) - dnu / T */
    double dlnKc = sum_h / T - dnu / T;
    double fwd = 1, rev = 1;
    for (int t = 0; t < m->nreac[i]; ++t) fwd *= C[m->reac[i * 3 + t]];
    for (int t = 0; t < m->nprod[i]; ++t) rev *= C[m->prod[i * 3 + t]];
    double q0 = kf * fwd - kr * rev;
    double Mfac = (m->kind[i] == 1) ? M : 1.0;
    rs[i].kf = kf; rs[i].kr = kr; rs[i].M = M; rs[i].q = Mfac * q0;
    if (dq_dT) dq_dT[i] = Mfac * (kf * dlnkf * fwd - kr * (dlnkf - dlnKc) * rev);
    if (dq_dC) {
      double* row = &dq_dC[(size_t)i * K];
      for (int k = 0; k < K; ++k) row[k] = 0;
      /* derivative of the concentration products: one term per occurrence */
      for (int t = 0; t < m->nreac[i]; ++t) {
        double d = kf;
        for (int u = 0; u < m->nreac[i]; ++u) if (u != t) d *= C[m->reac[i * 3 + u]];
        row[m->reac[i * 3 + t]] += Mfac * d;
      }
      for (int t = 0; t < m->nprod[i]; ++t) {
        double d = kr;
        for (int u = 0; u < m->nprod[i]; ++u) if (u != t) d *= C[m->prod[i * 3 + u]];
        row[m->prod[i * 3 + t]] -= Mfac * d;
      }
      if (m->kind[i] == 1) {
        for (int k = 0; k < K; ++k) row[k] += m->eff[(size_t)i * K + k] * q0;
      } else if (m->kind[i] == 2) {
        /* q = k(M) (fwd - rev/Kc): dq/dC_k += dk/dM alpha_k (fwd - rev/Kc) */
        double base = fwd - rev / Kc;
        for (int k = 0; k < K; ++k) row[k] += dk_dM * m->eff[(size_t)i * K + k] * base;
      }
    }
  }
}

/* Net production rates wdot [K] (mol/m^3/s) and heat release rate (W/m^3) at (T, p, Y) */
int or_rates(const void* h, double T, double p, const double* Y, double* wdot, double* hrr,
             double* q_out, double* kf_out, double* kr_out) {
  const omech* m = (const omech*)h;
  int K = m->K, I = m->I;
  double* C = (double*)malloc(sizeof(double) * K * 4);
  double *cpR = C + K, *hRT = C + 2 * K, *sR = C + 3 * K;
  rxn_state* rs = (rxn_state*)malloc(sizeof(rxn_state) * (I > 0 ? I : 1));
  concentrations(m, T, p, Y, C);
  for (int k = 0; k < K; ++k) nasa7(m, k, T, &cpR[k], &hRT[k], &sR[k], NULL);
  reaction_rates(m, T, C, hRT, sR, rs, NULL, NULL);
  for (int k = 0; k < K; ++k) wdot[k] = 0;
  for (int i = 0; i < I; ++i) {
    for (int t = 0; t < m->nreac[i]; ++t) wdot[m->reac[i * 3 + t]] -= rs[i].q;
    for (int t = 0; t < m->nprod[i]; ++t) wdot[m->prod[i * 3 + t]] += rs[i].q;
    if (q_out) q_out[i] = rs[i].q;
    if (kf_out) kf_out[i] = rs[i].kf;
    if (kr_out) kr_out[i] = rs[i].kr;
  }
  if (hrr) {
    double s = 0;
    for (int k = 0; k < K; ++k) s += hRT[k] * OR_R * T * wdot[k];
    *hrr = -s;
  }
  free(rs);
  free(C);
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* reactor right-hand side and analytic Jacobian, z = (Y_1..Y_K, T)                      */
/* ------------------------------------------------------------------------------------ */
typedef struct {
  double *C, *cpR, *hRT, *sR, *dcpR, *wdot, *dq_dC, *dq_dT, *JC, *dwdT;
  rxn_state* rs;
} work;

static void work_alloc(const omech* m, work* w) {
  int K = m->K, I = m->I;
  w->C = (double*)calloc(K * 7, sizeof(double));
  w->cpR = w->C + K; w->hRT = w->C + 2 * K; w->sR = w->C + 3 * K; w->dcpR = w->C + 4 * K;
  w->wdot = w->C + 5 * K; w->dwdT = w->C + 6 * K;
  w->dq_dC = (double*)calloc((size_t)(I > 0 ? I : 1) * K, sizeof(double));
  w->dq_dT = (double*)calloc(I > 0 ? I : 1, sizeof(double));
  w->JC = (double*)calloc((size_t)K * K, sizeof(double));
  w->rs = (rxn_state*)calloc(I > 0 ? I : 1, sizeof(rxn_state));
}

static void work_free(work* w) {
  free(w->C); free(w->dq_dC); free(w->dq_dT); free(w->JC); free(w->rs);
}

/* f = dz/dt.  Returns rho. */
static double rhs_w(const omech* m, double p, const double* z, double* f, work* w) {
  int K = m->K;
  double T = z[K];
  double rho = concentrations(m, T, p, z, w->C);
  for (int k = 0; k < K; ++k) nasa7(m, k, T, &w->cpR[k], &w->hRT[k], &w->sR[k], &w->dcpR[k]);
  reaction_rates(m, T, w->C, w->hRT, w->sR, w->rs, NULL, NULL);
  for (int k = 0; k < K; ++k) w->wdot[k] = 0;
  for (int i = 0; i < m->I; ++i) {
    for (int t = 0; t < m->nreac[i]; ++t) w->wdot[m->reac[i * 3 + t]] -= w->rs[i].q;
    for (int t = 0; t < m->nprod[i]; ++t) w->wdot[m->prod[i * 3 + t]] += w->rs[i].q;
  }
  double cp = 0, Q = 0;
  for (int k = 0; k < K; ++k) {
    cp += z[k] * w->cpR[k] * OR_R / m->W[k];
    Q += w->hRT[k] * OR_R * T * w->wdot[k];
  }
  for (int k = 0; k < K; ++k) f[k] = m->W[k] * w->wdot[k] / rho;
  f[K] = -Q / (rho * cp);
  return rho;
}

int or_rhs(const void* h, double p, const double* z, double* f) {
  const omech* m = (const omech*)h;
  work w;
  work_alloc(m, &w);
  rhs_w(m, p, z, f, &w);
  work_free(&w);
  return 0;
}

/* J[i*n + j] = d f_i / d z_j, n = K + 1.  Also returns f. */
static void jac_w(const omech* m, double p, const double* z, double* f, double* J, work* w) {
  int K = m->K, n = K + 1, I = m->I;
  double T = z[K];
  double s = 0;
  for (int k = 0; k < K; ++k) s += z[k] / m->W[k];
  double Wbar = 1.0 / s;
  double rho = concentrations(m, T, p, z, w->C);
  for (int k = 0; k < K; ++k) nasa7(m, k, T, &w->cpR[k], &w->hRT[k], &w->sR[k], &w->dcpR[k]);
  reaction_rates(m, T, w->C, w->hRT, w->sR, w->rs, w->dq_dC, w->dq_dT);
  for (int k = 0; k < K; ++k) { w->wdot[k] = 0; w->dwdT[k] = 0; }
  for (int k = 0; k < K * K; ++k) w->JC[k] = 0;
  /* JC[k][mm] = d wdot_k / d C_mm at fixed T; dwdT[k] = d wdot_k / dT at fixed C */
  for (int i = 0; i < I; ++i) {
    for (int side = 0; side < 2; ++side) {
      int cnt = side ? m->nprod[i] : m->nreac[i];
      const int* sp = side ? &m->prod[i * 3] : &m->reac[i * 3];
      double sg = side ? 1.0 : -1.0;
      for (int t = 0; t < cnt; ++t) {
        int k = sp[t];
        w->wdot[k] += sg * w->rs[i].q;
        w->dwdT[k] += sg * w->dq_dT[i];
        for (int mm = 0; mm < K; ++mm) w->JC[k * K + mm] += sg * w->dq_dC[(size_t)i * K + mm];
      }
    }
  }
  double cp = 0, Q = 0, dcp_dT = 0;
  for (int k = 0; k < K; ++k) {
    cp += z[k] * w->cpR[k] * OR_R / m->W[k];
    dcp_dT += z[k] * w->dcpR[k] * OR_R / m->W[k];
    Q += w->hRT[k] * OR_R * T * w->wdot[k];
  }
  for (int k = 0; k < K; ++k) f[k] = m->W[k] * w->wdot[k] / rho;
  f[K] = -Q / (rho * cp);
  /* S_k = sum_m JC[k][m] C_m */
  double* S = (double*)malloc(sizeof(double) * K * 3);
  double* dwdY = S + K;   /* scratch column: d wdot_k / d Y_i for fixed i */
  double* dwdT_tot = S + 2 * K;
  for (int k = 0; k < K; ++k) {
    double acc = 0;
    for (int mm = 0; mm < K; ++mm) acc += w->JC[k * K + mm] * w->C[mm];
    S[k] = acc;
    /* total T-derivative at fixed Y: C_m depends on T through rho ~ 1/T */
    dwdT_tot[k] = w->dwdT[k] - acc / T;
  }
  /* Y columns */
  for (int i = 0; i < K; ++i) {
    /* d C_m / d Y_i = delta_mi rho/W_m - C_m Wbar/W_i */
    for (int k = 0; k < K; ++k) dwdY[k] = w->JC[k * K + i] * rho / m->W[i] - S[k] * Wbar / m->W[i];
    double drho = -rho * Wbar / m->W[i];
    for (int k = 0; k < K; ++k)
      J[k * n + i] = m->W[k] * dwdY[k] / rho - m->W[k] * w->wdot[k] / (rho * rho) * drho;
    /* temperature row */
    double dQ = 0;
    for (int k = 0; k < K; ++k) dQ += w->hRT[k] * OR_R * T * dwdY[k];
    double drhocp = cp * drho + rho * w->cpR[i] * OR_R / m->W[i];
    J[K * n + i] = -dQ / (rho * cp) + Q / ((rho * cp) * (rho * cp)) * drhocp;
  }
  /* T column */
  for (int k = 0; k < K; ++k)
    J[k * n + K] = m->W[k] * dwdT_tot[k] / rho + m->W[k] * w->wdot[k] / (rho * T);
  double dQdT = 0;
  for (int k = 0; k < K; ++k) dQdT += w->cpR[k] * OR_R * w->wdot[k] + w->hRT[k] * OR_R * T * dwdT_tot[k];
  double drhocp_dT = -rho * cp / T + rho * dcp_dT;
  J[K * n + K] = -dQdT / (rho * cp) + Q / ((rho * cp) * (rho * cp)) * drhocp_dT;
  (void)n;
  free(S);
}

int or_jacobian(const void* h, double p, const double* z, double* J) {
  const omech* m = (const omech*)h;
  work w;
  work_alloc(m, &w);
  double* f = (double*)malloc(sizeof(double) * (m->K + 1));
  jac_w(m, p, z, f, J, &w);
  free(f);
  work_free(&w);
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* dense LU with partial pivoting (ties: lowest row index)                               */
/* ------------------------------------------------------------------------------------ */
static int lu_factor(double* A, int n, int* piv) {
  for (int c = 0; c < n; ++c) {
    int best = c;
    double bv = fabs(A[c * n + c]);
    for (int r = c + 1; r < n; ++r)
      if (fabs(A[r * n + c]) > bv) { bv = fabs(A[r * n + c]); best = r; }
    piv[c] = best;
    if (bv == 0.0 || !isfinite(bv)) return -1;
    if (best != c)
      for (int j = 0; j < n; ++j) { double t = A[c * n + j]; A[c * n + j] = A[best * n + j]; A[best * n + j] = t; }
    for (int r = c + 1; r < n; ++r) {
      double l = A[r * n + c] / A[c * n + c];
      A[r * n + c] = l;
      for (int j = c + 1; j < n; ++j) A[r * n + j] -= l * A[c * n + j];
    }
  }
  return 0;
}

/* Solve with the factors of P A = L U.  lu_factor swaps whole rows (the multipliers move with
 * their rows), so all interchanges are applied to x first, then forward and back substitution. */
static void lu_solve(const double* A, int n, const int* piv, double* x) {
  for (int c = 0; c < n; ++c)
    if (piv[c] != c) { double t = x[c]; x[c] = x[piv[c]]; x[piv[c]] = t; }
  for (int c = 0; c < n; ++c)
    for (int r = c + 1; r < n; ++r) x[r] -= A[r * n + c] * x[c];
  for (int c = n - 1; c >= 0; --c) {
    for (int j = c + 1; j < n; ++j) x[c] -= A[c * n + j] * x[j];
    x[c] /= A[c * n + c];
  }
}

/* Dense solve A x = b (A row-major n x n, overwritten by its factors; b overwritten by x).
 * Returns 0, or -1 for a singular matrix. */
int or_dense_solve(int n, double* A, double* b) {
  int* piv = (int*)malloc(sizeof(int) * n);
  int s = lu_factor(A, n, piv);
  if (s == 0) lu_solve(A, n, piv, b);
  free(piv);
  return s;
}

/* ------------------------------------------------------------------------------------ */
/* Radau IIA integrator                                                                  */
/* ------------------------------------------------------------------------------------ */
/* The three-stage Radau IIA collocation method (Ehle 1969; Hairer & Wanner, "Solving
 * Ordinary Differential Equations II", Sec. IV.5): order 5, stage order 3, L-stable, stiffly
 * accurate (the new state is the last stage).  Chosen as the oracle's method because it is a
 * one-step implicit Runge-Kutta method, unrelated to the multistep (BDF) scheme the GPU
 * kernel uses, so the two agree only through the solution of Eq. 2 itself.
 *
 * Nodes c_i are the zeros of the Radau right polynomial d^2/dx^2 [x^2 (x - 1)^3]:
 * c = ((4 - sqrt 6)/10, (4 + sqrt 6)/10, 1); the coefficients a_ij = int_0^{c_i} l_j(s) ds
 * integrate the Lagrange basis l_j of those nodes (collocation). */
typedef struct {
  double rtol, atol_Y, atol_T;
  int max_steps;
} or_opts;

typedef struct {
  int steps, rhs_evals, jac_evals, lu, failed_err, failed_newton;
} or_stats;

static void radau_tableau(double A[3][3], double c[3]) {
  const double s6 = sqrt(6.0);
  c[0] = (4.0 - s6) / 10.0;
  c[1] = (4.0 + s6) / 10.0;
  c[2] = 1.0;
  A[0][0] = (88.0 - 7.0 * s6) / 360.0;
  A[0][1] = (296.0 - 169.0 * s6) / 1800.0;
  A[0][2] = (-2.0 + 3.0 * s6) / 225.0;
  A[1][0] = (296.0 + 169.0 * s6) / 1800.0;
  A[1][1] = (88.0 + 7.0 * s6) / 360.0;
  A[1][2] = (-2.0 - 3.0 * s6) / 225.0;
  A[2][0] = (16.0 - s6) / 36.0;
  A[2][1] = (16.0 + s6) / 36.0;
  A[2][2] = 1.0 / 9.0;
}

/* Testing hook: the tableau, A row-major [9], c [3]. */
void or_radau_tableau(double* A, double* c) {
  double a[3][3];
  radau_tableau(a, c);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) A[i * 3 + j] = a[i][j];
}

static double wrms(const double* x, const double* scale, int n) {
  double s = 0;
  for (int i = 0; i < n; ++i) { double v = x[i] / scale[i]; s += v * v; }
  return sqrt(s / n);
}

typedef struct {
  double *Z, *Ys, *F, *J, *M, *G;
  int* piv;
} radau_buf;

static void radau_alloc(int n, radau_buf* r) {
  r->Z = (double*)calloc((size_t)3 * n, sizeof(double));
  r->Ys = (double*)calloc((size_t)3 * n, sizeof(double));
  r->F = (double*)calloc((size_t)3 * n, sizeof(double));
  r->G = (double*)calloc((size_t)3 * n, sizeof(double));
  r->J = (double*)calloc((size_t)3 * n * n, sizeof(double));
  r->M = (double*)calloc((size_t)9 * n * n, sizeof(double));
  r->piv = (int*)calloc((size_t)3 * n, sizeof(int));
}

static void radau_free(radau_buf* r) {
  free(r->Z); free(r->Ys); free(r->F); free(r->G); free(r->J); free(r->M); free(r->piv);
}

#define RADAU_NEWTON_MAXIT 12

/* One Radau IIA step of length h from y into ynew.  The stage increments Z_i = Y_i - y solve
 *   Z_i = h sum_j a_ij f(y + Z_j),   i = 1..3,
 * by a full Newton iteration from Z = 0: at every iterate the exact Jacobian of this 3n
 * system (block (i, j) = delta_ij I - h a_ij J(y + Z_j)) is formed from the analytic Jacobian
 * at the three stage values and factored afresh.  The iteration stops when the correction's
 * weighted RMS norm (weights `scale`, repeated per stage) is below kappa, or when it has
 * stalled at the rounding floor (from the third iterate on, no longer halving) below a tenth
 * of the error tolerance.  ynew = y + Z_3.  Returns 0, or -1 when the iteration fails (no
 * convergence in RADAU_NEWTON_MAXIT iterates, growing corrections, a singular matrix or a
 * non-finite value). */
static int radau_step(const omech* m, double p, const double* y, double h, const double* scale,
                      double kappa, double* ynew, radau_buf* r, or_stats* st, work* w) {
  const int n = m->K + 1, N = 3 * n;
  double A[3][3], c[3];
  radau_tableau(A, c);
  for (int i = 0; i < N; ++i) r->Z[i] = 0.0;
  double prev = INFINITY;
  for (int it = 0; it < RADAU_NEWTON_MAXIT; ++it) {
    for (int j = 0; j < 3; ++j) {
      for (int q = 0; q < n; ++q) r->Ys[j * n + q] = y[q] + r->Z[j * n + q];
      jac_w(m, p, &r->Ys[j * n], &r->F[j * n], &r->J[(size_t)j * n * n], w);
      st->jac_evals++;
      st->rhs_evals++;
    }
    for (int i = 0; i < N; ++i) if (!isfinite(r->F[i])) return -1;
    /* residual G_i = Z_i - h sum_j a_ij F_j  and matrix delta_ij I - h a_ij J_j */
    for (int i = 0; i < 3; ++i)
      for (int q = 0; q < n; ++q) {
        double s = 0;
        for (int j = 0; j < 3; ++j) s += A[i][j] * r->F[j * n + q];
        r->G[i * n + q] = -(r->Z[i * n + q] - h * s);
      }
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        for (int q = 0; q < n; ++q)
          for (int u = 0; u < n; ++u) {
            double v = -h * A[i][j] * r->J[(size_t)j * n * n + (size_t)q * n + u];
            if (i == j && q == u) v += 1.0;
            r->M[(size_t)(i * n + q) * N + (j * n + u)] = v;
          }
    if (lu_factor(r->M, N, r->piv) != 0) return -1;
    st->lu++;
    lu_solve(r->M, N, r->piv, r->G);   /* G now holds the correction */
    double s2 = 0;
    for (int i = 0; i < 3; ++i)
      for (int q = 0; q < n; ++q) {
        const double v = r->G[i * n + q] / scale[q];
        s2 += v * v;
        r->Z[i * n + q] += r->G[i * n + q];
      }
    const double nrm = sqrt(s2 / N);
    if (!isfinite(nrm)) return -1;
    if (nrm <= kappa || (it >= 2 && nrm <= 0.1 && nrm >= 0.5 * prev)) {
      for (int q = 0; q < n; ++q) ynew[q] = y[q] + r->Z[2 * n + q];
      for (int q = 0; q < n; ++q) if (!isfinite(ynew[q])) return -1;
      return 0;
    }
    if (it >= 3 && nrm > prev) return -1;
    prev = nrm;
  }
  return -1;
}

/* z(t + tend) from z(t) by Radau IIA steps with step-size control by step doubling
 * (Richardson extrapolation, Hairer, Norsett & Wanner, "Solving ODEs I", Sec. II.4): every
 * step of length h is taken once whole (y1) and once as two halves (y2); y2 is kept, and its
 * error is estimated by the whole difference |y2 - y1| -- the extrapolated estimate
 * |y2 - y1|/(2^5 - 1) assumes the full order 5, which stiff components do not reach (stage
 * order 3), so the undivided difference is the safe bound.  The step is accepted when the
 * weighted RMS norm of that estimate, weights atol + rtol max(|y|, |y2|), is at most 1; the
 * next step is h * min(4, max(0.2, 0.9 err^(-1/6))) (no growth right after a rejection).
 * Newton failures halve h.  Status: 0 ok, 1 max steps, 2 step size underflow, 3 non-finite. */
static int integrate_w(const omech* m, double p, double* z, double tend, const or_opts* o,
                       or_stats* st, work* w) {
  const int K = m->K, n = K + 1;
  const double EPS = 2.220446049250313e-16;
  memset(st, 0, sizeof(*st));
  for (int i = 0; i < n; ++i) if (!isfinite(z[i])) return 3;
  if (tend <= 0) return 0;
  radau_buf r;
  radau_alloc(n, &r);
  double* buf = (double*)malloc(sizeof(double) * (size_t)n * 6);
  double *y1 = buf, *ym = buf + n, *y2 = buf + 2 * n, *scale = buf + 3 * n, *d = buf + 4 * n;
  double* atol = buf + 5 * n;
  for (int i = 0; i < K; ++i) atol[i] = o->atol_Y;
  atol[K] = o->atol_T;
  /* Newton stop: 1e-3 of the error tolerance, but not below what rounding allows */
  const double kappa = fmax(1e-3, 100.0 * EPS / o->rtol);
  int status = 0, rejected = 0;
  double t = 0.0, h = fmin(tend, 1e-10);
  while (t < tend) {
    if (st->steps >= o->max_steps) { status = 1; break; }
    if (h < 1e-22 * tend || h < 1e-300) { status = 2; break; }
    const int last = t + h >= tend;
    if (last) h = tend - t;
    for (int i = 0; i < n; ++i) scale[i] = atol[i] + o->rtol * fabs(z[i]);
    int ok = radau_step(m, p, z, h, scale, kappa, y1, &r, st, w) == 0;
    if (ok) ok = radau_step(m, p, z, 0.5 * h, scale, kappa, ym, &r, st, w) == 0;
    if (ok) {
      for (int i = 0; i < n; ++i) scale[i] = atol[i] + o->rtol * fabs(ym[i]);
      ok = radau_step(m, p, ym, 0.5 * h, scale, kappa, y2, &r, st, w) == 0;
    }
    if (!ok) {
      st->failed_newton++;
      h *= 0.5;
      rejected = 1;
      continue;
    }
    for (int i = 0; i < n; ++i) {
      scale[i] = atol[i] + o->rtol * fmax(fabs(z[i]), fabs(y2[i]));
      d[i] = y2[i] - y1[i];
    }
    const double err = wrms(d, scale, n);
    double fac = err > 0 ? 0.9 * pow(err, -1.0 / 6.0) : 4.0;
    fac = fmin(4.0, fmax(0.2, fac));
    if (err <= 1.0) {
      for (int i = 0; i < n; ++i) z[i] = y2[i];
      t = last ? tend : t + h;
      st->steps++;
      if (rejected) fac = fmin(fac, 1.0);
      rejected = 0;
    } else {
      st->failed_err++;
      rejected = 1;
    }
    h *= fac;
  }
  if (status == 0)
    for (int i = 0; i < n; ++i) if (!isfinite(z[i])) status = 3;
  radau_free(&r);
  free(buf);
  return status;
}

/* Testing hook: nsteps fixed Radau IIA steps of length h (no error control), Newton stop at
 * 1e-14 relative.  Returns 0, or -1 if a step's Newton iteration failed. */
int or_radau_fixed(const void* hd, double p, double* z, double h, int nsteps) {
  const omech* m = (const omech*)hd;
  const int n = m->K + 1;
  work w;
  work_alloc(m, &w);
  radau_buf r;
  radau_alloc(n, &r);
  or_stats st;
  memset(&st, 0, sizeof(st));
  double* buf = (double*)malloc(sizeof(double) * (size_t)n * 2);
  double *scale = buf, *y = buf + n;
  int s = 0;
  for (int k = 0; k < nsteps && s == 0; ++k) {
    for (int i = 0; i < n; ++i) scale[i] = 1e-30 + 1e-14 * fabs(z[i]);
    s = radau_step(m, p, z, h, scale, 1.0, y, &r, &st, &w);
    if (s == 0) memcpy(z, y, sizeof(double) * n);
  }
  free(buf);
  radau_free(&r);
  work_free(&w);
  return s;
}

int or_integrate(const void* h, double p, double* z, double dt, double rtol, double atol_Y,
                 double atol_T, int max_steps, int* stats /* [6] or NULL */) {
  const omech* m = (const omech*)h;
  or_opts o = {rtol, atol_Y, atol_T, max_steps};
  or_stats st;
  work w;
  work_alloc(m, &w);
  int s = integrate_w(m, p, z, dt, &o, &st, &w);
  work_free(&w);
  if (stats) {
    stats[0] = st.steps; stats[1] = st.rhs_evals; stats[2] = st.jac_evals; stats[3] = st.lu;
    stats[4] = st.failed_err; stats[5] = st.failed_newton;
  }
  return s;
}

/* Batch over cells, species-major SoA: T[i], p[i], Y[k*ld + i]; OpenMP over cells. */
int or_integrate_batch(const void* h, int64_t n, int64_t ld, double dt, double* T, const double* p,
                       double* Y, double rtol, double atol_Y, double atol_T, int max_steps,
                       int* status, int* steps, int nthreads) {
  const omech* m = (const omech*)h;
  int K = m->K;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel
  {
    work w;
    work_alloc(m, &w);
    double* z = (double*)malloc(sizeof(double) * (K + 1));
    or_opts o = {rtol, atol_Y, atol_T, max_steps};
    or_stats st;
#pragma omp for schedule(dynamic, 1)
    for (int64_t c = 0; c < n; ++c) {
      for (int k = 0; k < K; ++k) z[k] = Y[k * ld + c];
      z[K] = T[c];
      int s = integrate_w(m, p[c], z, dt, &o, &st, &w);
      status[c] = s;
      if (steps) steps[c] = st.steps;
      if (s == 0) {
        for (int k = 0; k < K; ++k) Y[k * ld + c] = z[k];
        T[c] = z[K];
      }
    }
    free(z);
    work_free(&w);
  }
  return 0;
}

int or_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Fixed-step classical RK4 (second, independent integration path). */
int or_rk4(const void* h, double p, double* z, double dt, int64_t nsub) {
  const omech* m = (const omech*)h;
  int n = m->K + 1;
  work w;
  work_alloc(m, &w);
  double* b = (double*)malloc(sizeof(double) * n * 6);
  double *k1 = b, *k2 = b + n, *k3 = b + 2 * n, *k4 = b + 3 * n, *y = b + 4 * n;
  double hh = dt / (double)nsub;
  for (int64_t s = 0; s < nsub; ++s) {
    rhs_w(m, p, z, k1, &w);
    for (int i = 0; i < n; ++i) y[i] = z[i] + 0.5 * hh * k1[i];
    rhs_w(m, p, y, k2, &w);
    for (int i = 0; i < n; ++i) y[i] = z[i] + 0.5 * hh * k2[i];
    rhs_w(m, p, y, k3, &w);
    for (int i = 0; i < n; ++i) y[i] = z[i] + hh * k3[i];
    rhs_w(m, p, y, k4, &w);
    for (int i = 0; i < n; ++i) z[i] += hh / 6.0 * (k1[i] + 2 * k2[i] + 2 * k3[i] + k4[i]);
  }
  free(b);
  work_free(&w);
  for (int i = 0; i < n; ++i) if (!isfinite(z[i])) return 3;
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* mixture thermo and transport properties                                               */
/* ------------------------------------------------------------------------------------ */
static double poly_lnT(const double* b, double lnT) {
  return b[0] + b[1] * lnT + b[2] * lnT * lnT + b[3] * lnT * lnT * lnT;
}

/* cp [J/kg/K], h [J/kg], Wilke viscosity mu [Pa s], mixture conductivity [W/m/K] */
int or_thermo_props(const void* h, double T, const double* Y, double* cp, double* hm,
                    double* mu, double* kappa) {
  const omech* m = (const omech*)h;
  int K = m->K;
  double* X = (double*)malloc(sizeof(double) * K * 3);
  double *muk = X + K, *lamk = X + 2 * K;
  double cps = 0, hs = 0, s = 0;
  for (int k = 0; k < K; ++k) {
    double cpR, hRT, sR;
    nasa7(m, k, T, &cpR, &hRT, &sR, NULL);
    cps += Y[k] * cpR * OR_R / m->W[k];
    hs += Y[k] * hRT * OR_R * T / m->W[k];
    s += Y[k] / m->W[k];
  }
  double lnT = log(T);
  for (int k = 0; k < K; ++k) {
    X[k] = Y[k] / m->W[k] / s;
    muk[k] = exp(poly_lnT(&m->mufit[k * 4], lnT));
    lamk[k] = exp(poly_lnT(&m->lamfit[k * 4], lnT));
  }
  double mus = 0;
  for (int k = 0; k < K; ++k) {
    double den = 0;
    for (int j = 0; j < K; ++j) {
      double t = 1 + sqrt(muk[k] / muk[j]) * pow(m->W[j] / m->W[k], 0.25);
      double phi = t * t / sqrt(8.0 * (1 + m->W[k] / m->W[j]));
      den += X[j] * phi;
    }
    mus += X[k] * muk[k] / den;
  }
  double l1 = 0, l2 = 0;
  for (int k = 0; k < K; ++k) { l1 += X[k] * lamk[k]; l2 += X[k] / lamk[k]; }
  if (cp) *cp = cps;
  if (hm) *hm = hs;
  if (mu) *mu = mus;
  if (kappa) *kappa = 0.5 * (l1 + 1.0 / l2);
  free(X);
  return 0;
}

/* T such that h(T, Y) = h_target, by Newton from T0; bracketed to [200, 6000] K. */
int or_T_from_h(const void* hd, double h_target, const double* Y, double T0, double* T_out) {
  const omech* m = (const omech*)hd;
  double T = T0;
  for (int it = 0; it < 50; ++it) {
    double cp, h;
    or_thermo_props(m, T, Y, &cp, &h, NULL, NULL);
    double dT = (h - h_target) / cp;
    double Tn = T - dT;
    if (Tn < 200) Tn = 200;
    if (Tn > 6000) Tn = 6000;
    if (fabs(Tn - T) < 1e-10) { *T_out = Tn; return 0; }
    T = Tn;
  }
  *T_out = T;
  return 1;
}
