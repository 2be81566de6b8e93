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
 * The integrator is a variable-order (1..5), variable-step BDF in backward-difference form
 * with quasi-constant step size (Shampine & Reichelt, "The MATLAB ODE Suite", SIAM J. Sci.
 * Comput. 18, 1997), the family CVODE/VODE belong to (the paper's integrator, Sec. 2.2),
 * here with a FULL Newton iteration: the analytic Jacobian and a fresh LU at every iterate.
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
/* BDF integrator                                                                        */
/* ------------------------------------------------------------------------------------ */
typedef struct {
  double rtol, atol_Y, atol_T;
  int max_steps;
} or_opts;

typedef struct {
  int steps, rhs_evals, jac_evals, lu, failed_err, failed_newton;
} or_stats;

#define MAXORD 5
#define NEWTON_MAXIT 4

static double wrms(const double* x, const double* scale, int n) {
  double s = 0;
  for (int i = 0; i < n; ++i) { double v = x[i] / scale[i]; s += v * v; }
  return sqrt(s / n);
}

/* Rescale the difference array D[0..order] for a step-size change by `factor`:
 * D <- (R(factor) U)^T D, with R(r)_{ij} = prod_{l=1..i} (l - 1 - r j)/l (row 0 = 1). */
static void rescale_differences(double* D, int n, int order, double factor) {
  double R[MAXORD + 1][MAXORD + 1], U[MAXORD + 1][MAXORD + 1], RU[MAXORD + 1][MAXORD + 1];
  for (int j = 0; j <= order; ++j) { R[0][j] = 1; U[0][j] = 1; }
  for (int i = 1; i <= order; ++i)
    for (int j = 0; j <= order; ++j) {
      if (j == 0) { R[i][j] = 0; U[i][j] = 0; continue; }
      R[i][j] = R[i - 1][j] * (i - 1 - factor * j) / i;
      U[i][j] = U[i - 1][j] * (i - 1 - 1.0 * j) / i;
    }
  for (int i = 0; i <= order; ++i)
    for (int j = 0; j <= order; ++j) {
      double s = 0;
      for (int l = 0; l <= order; ++l) s += R[i][l] * U[l][j];
      RU[i][j] = s;
    }
  double* tmp = (double*)malloc(sizeof(double) * (order + 1) * n);
  for (int j = 0; j <= order; ++j)
    for (int c = 0; c < n; ++c) {
      double s = 0;
      for (int i = 0; i <= order; ++i) s += RU[i][j] * D[i * n + c];
      tmp[j * n + c] = s;
    }
  memcpy(D, tmp, sizeof(double) * (order + 1) * n);
  free(tmp);
}

/* status: 0 ok, 1 max steps, 2 step-size/Newton failure, 3 non-finite */
static int integrate_w(const omech* m, double p, double* z, double tend, const or_opts* o,
                       or_stats* st, work* w) {
  int K = m->K, n = K + 1;
  const double EPS = 2.220446049250313e-16;
  double gamma[MAXORD + 2], errc[MAXORD + 2];
  gamma[0] = 0;
  for (int k = 1; k <= MAXORD + 1; ++k) gamma[k] = gamma[k - 1] + 1.0 / k;
  for (int k = 0; k <= MAXORD + 1; ++k) errc[k] = 1.0 / (k + 1);
  double newton_tol = fmax(10 * EPS / o->rtol, fmin(0.03, sqrt(o->rtol)));
  memset(st, 0, sizeof(*st));
  for (int i = 0; i < n; ++i) if (!isfinite(z[i])) return 3;
  if (tend <= 0) return 0;

  double* D = (double*)calloc((size_t)(MAXORD + 3) * n, sizeof(double));
  double* buf = (double*)calloc((size_t)n * 8 + (size_t)n * n, sizeof(double));
  double *f = buf, *y = buf + n, *ypred = buf + 2 * n, *psi = buf + 3 * n, *d = buf + 4 * n;
  double *dy = buf + 5 * n, *scale = buf + 6 * n, *tmp = buf + 7 * n, *Mx = buf + 8 * n;
  int* piv = (int*)calloc(n, sizeof(int));
  double* atol = (double*)malloc(sizeof(double) * n);
  for (int i = 0; i < K; ++i) atol[i] = o->atol_Y;
  atol[K] = o->atol_T;
  int status = 0;

  /* initial step (Hairer, Norsett & Wanner, Sec. II.4) for order 1 */
  rhs_w(m, p, z, f, w); st->rhs_evals++;
  for (int i = 0; i < n; ++i) scale[i] = atol[i] + o->rtol * fabs(z[i]);
  double d0 = wrms(z, scale, n), d1 = wrms(f, scale, n);
  double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
  if (h0 > tend) h0 = tend;
  for (int i = 0; i < n; ++i) y[i] = z[i] + h0 * f[i];
  rhs_w(m, p, y, tmp, w); st->rhs_evals++;
  for (int i = 0; i < n; ++i) dy[i] = tmp[i] - f[i];
  double d2 = wrms(dy, scale, n) / h0;
  double h1 = (d1 <= 1e-15 && d2 <= 1e-15) ? fmax(1e-6, h0 * 1e-3) : pow(0.01 / fmax(d1, d2), 0.5);
  double h = fmin(100 * h0, h1);
  if (!(h > 0) || !isfinite(h)) h = 1e-12 * tend;
  if (h > tend) h = tend;

  for (int i = 0; i < n; ++i) { D[i] = z[i]; D[n + i] = h * f[i]; }
  int order = 1, n_equal = 0;
  double t = 0;
  while (t < tend) {
    if (st->steps >= o->max_steps) { status = 1; break; }
    double hmin = 10 * EPS * fabs(t) + 1e-300;
    if (t + h > tend) {
      double hn = tend - t;
      rescale_differences(D, n, order, hn / h);
      h = hn;
      n_equal = 0;
    }
    int accepted = 0, newton_iters = 0;
    double err_norm = 0;
    while (!accepted) {
      if (h < hmin) { status = 2; goto done; }
      double t_new = t + h;
      if (t_new > tend || tend - t_new < hmin) t_new = tend;
      for (int i = 0; i < n; ++i) {
        double s = 0;
        for (int j = 0; j <= order; ++j) s += D[j * n + i];
        ypred[i] = s;
        scale[i] = atol[i] + o->rtol * fabs(s);
        double ps = 0;
        for (int j = 1; j <= order; ++j) ps += gamma[j] * D[j * n + i];
        psi[i] = ps / gamma[order];
      }
      double c = h / gamma[order];
      /* full Newton on  d - c f(ypred + d) + psi = 0 */
      for (int i = 0; i < n; ++i) { d[i] = 0; y[i] = ypred[i]; }
      int converged = 0;
      double dy_old = 0;
      newton_iters = 0;
      for (int it = 0; it < NEWTON_MAXIT; ++it) {
        jac_w(m, p, y, f, Mx, w); st->jac_evals++; st->rhs_evals++;
        int finite = 1;
        for (int i = 0; i < n; ++i) if (!isfinite(f[i])) finite = 0;
        if (!finite) break;
        for (int i = 0; i < n * n; ++i) Mx[i] = -c * Mx[i];
        for (int i = 0; i < n; ++i) Mx[i * n + i] += 1.0;
        if (lu_factor(Mx, n, piv) != 0) break;
        st->lu++;
        for (int i = 0; i < n; ++i) dy[i] = c * f[i] - psi[i] - d[i];
        lu_solve(Mx, n, piv, dy);
        double dn = wrms(dy, scale, n);
        ++newton_iters;
        double rate = (it > 0) ? dn / dy_old : -1;
        if (it > 0 && (rate >= 1 || pow(rate, NEWTON_MAXIT - it) / (1 - rate) * dn > newton_tol)) break;
        for (int i = 0; i < n; ++i) { y[i] += dy[i]; d[i] += dy[i]; }
        if (dn == 0 || (it > 0 && rate / (1 - rate) * dn < newton_tol)) { converged = 1; break; }
        if (it == 0 && dn < newton_tol * 1e-3) { converged = 1; break; }
        dy_old = dn;
      }
      if (!converged) {
        st->failed_newton++;
        rescale_differences(D, n, order, 0.5);
        h *= 0.5;
        n_equal = 0;
        continue;
      }
      double safety = 0.9 * (2 * NEWTON_MAXIT + 1) / (2 * NEWTON_MAXIT + newton_iters);
      for (int i = 0; i < n; ++i) {
        scale[i] = atol[i] + o->rtol * fabs(y[i]);
        tmp[i] = errc[order] * d[i];
      }
      err_norm = wrms(tmp, scale, n);
      if (err_norm > 1) {
        st->failed_err++;
        double fac = fmax(0.2, safety * pow(err_norm, -1.0 / (order + 1)));
        rescale_differences(D, n, order, fac);
        h *= fac;
        n_equal = 0;
        continue;
      }
      accepted = 1;
      t = t_new;
      st->steps++;
      n_equal++;
      /* update differences: D[order+2] = d - D[order+1]; D[order+1] = d; D[i] += D[i+1] */
      for (int i = 0; i < n; ++i) {
        D[(order + 2) * n + i] = d[i] - D[(order + 1) * n + i];
        D[(order + 1) * n + i] = d[i];
      }
      for (int j = order; j >= 0; --j)
        for (int i = 0; i < n; ++i) D[j * n + i] += D[(j + 1) * n + i];
      if (n_equal < order + 1) break;
      /* order and step selection */
      double em = INFINITY, ep = INFINITY;
      if (order > 1) {
        for (int i = 0; i < n; ++i) tmp[i] = errc[order - 1] * D[order * n + i];
        em = wrms(tmp, scale, n);
      }
      if (order < MAXORD) {
        for (int i = 0; i < n; ++i) tmp[i] = errc[order + 1] * D[(order + 2) * n + i];
        ep = wrms(tmp, scale, n);
      }
      double fm = (em == INFINITY) ? 0 : (em == 0 ? 1e30 : pow(em, -1.0 / order));
      double f0 = (err_norm == 0) ? 1e30 : pow(err_norm, -1.0 / (order + 1));
      double fp = (ep == INFINITY) ? 0 : (ep == 0 ? 1e30 : pow(ep, -1.0 / (order + 2)));
      int delta = 0;
      double best = f0;
      if (fm > best) { best = fm; delta = -1; }
      if (fp > best) { best = fp; delta = 1; }
      order += delta;
      double fac = fmin(10.0, safety * best);
      rescale_differences(D, n, order, fac);
      h *= fac;
      n_equal = 0;
    }
  }
done:
  if (status == 0) {
    for (int i = 0; i < n; ++i) z[i] = D[i];
    for (int i = 0; i < n; ++i) if (!isfinite(z[i])) status = 3;
  }
  free(D); free(buf); free(piv); free(atol);
  return status;
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
