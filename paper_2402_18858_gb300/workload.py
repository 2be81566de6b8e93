"""Seeded synthetic inputs for the per-cell chemistry step: mechanisms and cell states.

This module is shared by the CPU oracle's tests and by the GPU library's tests and benchmark.
It holds only input generation (random draws, element bookkeeping, least-squares fits of the
synthetic heat capacity, file writing); none of the chemistry step's own arithmetic (no rate
constants, no equilibrium constants, no NASA-7 evaluation, no integration) lives here.

The paper integrates the reaction system of Eq. 1 over one flow step (Eq. 2) with a detailed
mechanism (DRM19, Sec. 2.2) that is not available here, so mechanisms are synthetic:

* species are real element compositions (formula names) over H/O/N or C/H/O/N; N2 is inert;
* reactions are random element-balanced A+B<=>C+D, A+B(+M)<=>C(+M) third-body and
  A+B(+M)<=>C(+M) Troe falloff reactions;
* A is log-uniform in [1e8, 1e14] (cm-mol-s), b uniform in [-1, 2], Ea uniform in 0-200 kJ/mol;
* NASA-7 coefficients are least-squares fits (two ranges, continuous value and slope at
  T_mid) of a smooth synthetic cp(T)/R = c_inf - (c_inf - c_0) exp(-T/theta);
* formation enthalpies are class-based draws, rescaled so that complete combustion of the
  stoichiometric fuel-air mixture from 300 K reaches an adiabatic temperature near 2300 K;
* transport fits are ln mu_k = sum_n b_n (ln T)^n (and the same for lambda_k), n = 0..3.

Cell states follow the paper's mixing of lean products with fresh gas (Sec. 2.2, the
interpolation between the leanest equilibrium and ambient air): Y on mixing lines between the
unburnt lean mixture and its burnt state, with a log-normal perturbation, T drawn
independently. The burnt endpoint is the complete-combustion product state plus a seeded
radical pool (no equilibrium solve here).

The file format is this project's own plain text, in SI units (kg/mol, m-mol-s, J/mol).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

R_GAS = 8.314462618  # J/mol/K (exact SI value of N_A * k_B)
P_ATM = 101325.0
ATOMIC_MASS = {"H": 1.008e-3, "C": 12.011e-3, "O": 15.999e-3, "N": 14.007e-3}  # kg/mol
VALENCE = {"H": 1, "C": 4, "O": 2, "N": 3}

# ----------------------------------------------------------------------------------------
# species sets (element compositions only; no published mechanism is reproduced)
# ----------------------------------------------------------------------------------------
_SP9 = ["H2", "O2", "H2O", "H", "O", "OH", "HO2", "H2O2", "N2"]
_SP30 = ["H2", "H", "O", "O2", "OH", "H2O", "HO2", "H2O2", "C", "CH", "CH2", "CH3", "CH4",
         "CO", "CO2", "HCO", "CH2O", "CH3O", "CH3OH", "C2H", "C2H2", "C2H3", "C2H4", "C2H5",
         "C2H6", "HCCO", "CH2CO", "N", "NO", "N2"]
_SP53_EXTRA = ["C3H8", "C3H7", "C3H6", "C3H5", "C3H4", "C3H3", "C2H4O", "C2H3O", "C2H6O",
               "CH3O2", "CHO2", "CH2O2", "NH", "NH2", "NH3", "N2H", "N2O", "NO2", "HNO", "CN",
               "HCN", "HNCO", "NCO"]
_SP53 = _SP30 + _SP53_EXTRA

# name -> (species list, elements, fuel, n_reactions, n_thirdbody, n_troe)
MECH_KINDS = {
    "h2_9": (_SP9, ["H", "O", "N"], "H2", 24, 3, 0),
    "c_30": (_SP30, ["C", "H", "O", "N"], "CH4", 180, 6, 8),
    "c_53": (_SP53, ["C", "H", "O", "N"], "CH4", 320, 10, 12),
}

INERT = ("N2",)
REFERENCE = ("H2", "O2", "N2")  # elements in their standard state: zero formation enthalpy


def parse_formula(name: str) -> Dict[str, int]:
    """Element counts of a formula name such as 'CH2CO' or 'C2H6O'."""
    out: Dict[str, int] = {}
    i = 0
    while i < len(name):
        el = name[i]
        if el not in ATOMIC_MASS:
            raise ValueError(f"bad element in {name!r}")
        i += 1
        j = i
        while j < len(name) and name[j].isdigit():
            j += 1
        cnt = int(name[i:j]) if j > i else 1
        out[el] = out.get(el, 0) + cnt
        i = j
    return out


# ----------------------------------------------------------------------------------------
# data classes
# ----------------------------------------------------------------------------------------
@dataclasses.dataclass
class Reaction:
    kind: int                      # 0 elementary, 1 third-body, 2 Troe falloff
    reactants: List[int]           # species indices, repeated for stoichiometric 2
    products: List[int]
    A: float                       # SI (m, mol, s)
    b: float
    Ea: float                      # J/mol
    eff: Dict[int, float] = dataclasses.field(default_factory=dict)   # non-unit efficiencies
    low: Optional[Tuple[float, float, float]] = None                  # k0 (A SI, b, Ea)
    troe: Optional[Tuple[float, ...]] = None                          # (a, T3, T1[, T2])


@dataclasses.dataclass
class Mechanism:
    name: str
    elements: List[str]
    species: List[str]
    comp: np.ndarray               # [K, E] element counts
    W: np.ndarray                  # [K] kg/mol
    T_low: float
    T_mid: float
    T_high: float
    nasa_low: np.ndarray           # [K, 7]
    nasa_high: np.ndarray          # [K, 7]
    mu_fit: np.ndarray             # [K, 4] ln(mu) = sum b_n (lnT)^n, mu in Pa s
    lam_fit: np.ndarray            # [K, 4] ln(lambda) = sum b_n (lnT)^n, lambda in W/m/K
    reactions: List[Reaction]
    fuel: str
    T_ad_stoich: float = float("nan")   # complete-combustion adiabatic T of the phi=1 mixture

    @property
    def n_species(self) -> int:
        return len(self.species)

    @property
    def n_reactions(self) -> int:
        return len(self.reactions)

    def index(self, name: str) -> int:
        return self.species.index(name)


# ----------------------------------------------------------------------------------------
# synthetic thermochemistry (the generator's own smooth cp model, closed-form integrals)
# ----------------------------------------------------------------------------------------
def _cp_model(c0, cinf, theta, T):
    return cinf - (cinf - c0) * np.exp(-T / theta)


def _h_model_R(c0, cinf, theta, T, T0=298.15):
    """integral_{T0}^{T} cp/R dT of the synthetic model (K)."""
    return cinf * (T - T0) + (cinf - c0) * theta * (np.exp(-T / theta) - np.exp(-T0 / theta))


def _s_model_R(c0, cinf, theta, T, T0=298.15, n_quad=400):
    """integral_{T0}^{T} cp/(R T) dT of the synthetic model (Gauss-Legendre quadrature)."""
    x, w = np.polynomial.legendre.leggauss(n_quad)
    a, b = T0, T
    t = 0.5 * (b - a) * x + 0.5 * (b + a)
    return 0.5 * (b - a) * np.sum(w * _cp_model(c0, cinf, theta, t) / t)


def _fit_nasa7(c0, cinf, theta, dHf_R, s298_R, T_low, T_mid, T_high):
    """Two-range NASA-7 fit of the synthetic cp with value and slope continuity at T_mid.

    The quartic cp/R polynomials are least-squares fits in the scaled variable t = T/1000 on
    each range; the low range carries two equality constraints (cp and dcp/dT equal to the
    high-range fit at T_mid), solved through the KKT system. a6 and a7 are set from the
    formation enthalpy and standard entropy at 298.15 K and continuity at T_mid.
    """
    S = 1000.0
    th = np.linspace(T_mid, T_high, 200)
    tl = np.linspace(T_low, T_mid, 200)
    Vh = np.vander(th / S, 5, increasing=True)
    ch, *_ = np.linalg.lstsq(Vh, _cp_model(c0, cinf, theta, th), rcond=None)
    tm = T_mid / S
    val = sum(ch[i] * tm ** i for i in range(5))
    der = sum(i * ch[i] * tm ** (i - 1) for i in range(1, 5))
    Vl = np.vander(tl / S, 5, increasing=True)
    Cst = np.array([[tm ** i for i in range(5)], [i * tm ** (i - 1) if i else 0.0 for i in range(5)]])
    kkt = np.zeros((7, 7))
    kkt[:5, :5] = 2 * Vl.T @ Vl
    kkt[:5, 5:] = Cst.T
    kkt[5:, :5] = Cst
    rhs = np.concatenate([2 * Vl.T @ _cp_model(c0, cinf, theta, tl), [val, der]])
    cl = np.linalg.solve(kkt, rhs)[:5]
    a_low = np.zeros(7)
    a_high = np.zeros(7)
    for i in range(5):
        a_low[i] = cl[i] / S ** i
        a_high[i] = ch[i] / S ** i

    def h_poly_noa6(a, T):   # h/R without the a6 term (K)
        return sum(a[i] * T ** (i + 1) / (i + 1) for i in range(5))

    def s_poly_noa7(a, T):   # s/R without the a7 term
        return a[0] * math.log(T) + sum(a[i] * T ** i / i for i in range(1, 5))

    a_low[5] = dHf_R - h_poly_noa6(a_low, 298.15)
    a_high[5] = h_poly_noa6(a_low, T_mid) + a_low[5] - h_poly_noa6(a_high, T_mid)
    a_low[6] = s298_R - s_poly_noa7(a_low, 298.15)
    a_high[6] = s_poly_noa7(a_low, T_mid) + a_low[6] - s_poly_noa7(a_high, T_mid)
    return a_low, a_high


def _is_radical(comp: Dict[str, int]) -> bool:
    atoms = sum(comp.values())
    val = sum(VALENCE[e] * c for e, c in comp.items())
    return atoms == 1 or (val % 2 == 1)


# ----------------------------------------------------------------------------------------
# mixture bookkeeping used by the generator (element counting only)
# ----------------------------------------------------------------------------------------
def _fuel_air_moles(comp_fuel: Dict[str, int], phi: np.ndarray):
    """Moles of fuel per mole O2 at equivalence ratio phi (element based, O2 from air only)."""
    c, h, o = comp_fuel.get("C", 0), comp_fuel.get("H", 0), comp_fuel.get("O", 0)
    o2_stoich = c + h / 4.0 - o / 2.0      # mol O2 per mol fuel at phi = 1
    return phi / o2_stoich, o2_stoich


def unburnt_and_burnt_moles(mech: Mechanism, phi: np.ndarray):
    """Mole numbers [K, N] of the fresh fuel-air mixture and its complete-combustion products.

    Air is O2:N2 = 1:3.76 molar; lean or stoichiometric only (phi <= 1).
    """
    phi = np.atleast_1d(np.asarray(phi, dtype=np.float64))
    if np.any(phi > 1.0 + 1e-12):
        raise ValueError("complete-combustion endpoint is defined for phi <= 1 only")
    K = mech.n_species
    cf = parse_formula(mech.fuel)
    nf, o2s = _fuel_air_moles(cf, phi)
    nu = np.zeros((K, phi.size))
    nb = np.zeros((K, phi.size))
    iF, iO2, iN2 = mech.index(mech.fuel), mech.index("O2"), mech.index("N2")
    nu[iF] = nf
    nu[iO2] = 1.0
    nu[iN2] = 3.76
    nb[iO2] = 1.0 - nf * o2s
    nb[iN2] = 3.76
    if cf.get("C", 0):
        nb[mech.index("CO2")] += nf * cf["C"]
    if cf.get("H", 0):
        nb[mech.index("H2O")] += nf * cf["H"] / 2.0
    return nu, nb


def moles_to_mass_fractions(mech: Mechanism, n: np.ndarray) -> np.ndarray:
    m = n * mech.W[:, None]
    return m / m.sum(axis=0, keepdims=True)


# ----------------------------------------------------------------------------------------
# mechanism generation
# ----------------------------------------------------------------------------------------
def _candidates(species: Sequence[str], comps: List[Dict[str, int]], elements: Sequence[str]):
    """All element-balanced A+B<=>C+D and A+B<=>C sets among reactive species."""
    key = [tuple(c.get(e, 0) for e in elements) for c in comps]
    reactive = [i for i, s in enumerate(species) if s not in INERT]
    pairs: Dict[Tuple[int, ...], List[Tuple[int, int]]] = {}
    for ai, a in enumerate(reactive):
        for b in reactive[ai:]:
            s = tuple(x + y for x, y in zip(key[a], key[b]))
            pairs.setdefault(s, []).append((a, b))
    bimol = []
    for s, lst in pairs.items():
        for i in range(len(lst)):
            for j in range(i + 1, len(lst)):
                if set(lst[i]) & set(lst[j]):
                    continue
                bimol.append((lst[i], lst[j]))
    single = {key[i]: i for i in reactive}
    assoc = []
    for s, lst in pairs.items():
        if s in single:
            c = single[s]
            for (a, b) in lst:
                if c not in (a, b):
                    assoc.append(((a, b), c))
    return bimol, assoc


def make_mechanism(kind: str, seed: int) -> Mechanism:
    """Seeded synthetic mechanism of the given kind ('h2_9', 'c_30', 'c_53')."""
    species, elements, fuel, n_rxn, n_tb, n_troe = MECH_KINDS[kind]
    rng = np.random.default_rng(seed)
    comps = [parse_formula(s) for s in species]
    K = len(species)
    comp = np.array([[c.get(e, 0) for e in elements] for c in comps], dtype=np.int64)
    W = np.array([sum(ATOMIC_MASS[e] * n for e, n in c.items()) for c in comps])

    # --- synthetic cp model parameters per species
    c0 = np.empty(K)
    cinf = np.empty(K)
    theta = rng.uniform(400.0, 1500.0, K)
    for k, c in enumerate(comps):
        na = sum(c.values())
        if na == 1:
            c0[k], cinf[k] = 2.5, 2.5
        elif na == 2:
            c0[k], cinf[k] = 3.5, 4.5 + rng.uniform(-0.1, 0.1)
        else:
            c0[k], cinf[k] = 4.0, 0.8 * (3 * na - 2) + rng.uniform(-0.3, 0.3)
    s298 = np.array([15.0 + 3.0 * sum(c.values()) + rng.uniform(0, 3) for c in comps])

    # --- class-based formation enthalpies (J/mol), later scaled for the flame temperature
    dHf0 = np.zeros(K)
    for k, (s, c) in enumerate(zip(species, comps)):
        heavy = sum(n for e, n in c.items() if e != "H")
        if s in REFERENCE:
            dHf0[k] = 0.0
        elif _is_radical(c):
            dHf0[k] = rng.uniform(30e3, 250e3)
        else:
            dHf0[k] = -rng.uniform(60e3, 130e3) * max(heavy, 1)
    for prod in ("H2O", "CO2", "CO"):
        if prod in species:
            k = species.index(prod)
            dHf0[k] = {"H2O": -240e3, "CO2": -390e3, "CO": -110e3}[prod] * rng.uniform(0.95, 1.05)

    T_low, T_mid, T_high = 300.0, 1000.0, 5000.0
    mech_tmp = Mechanism(kind, elements, species, comp, W, T_low, T_mid, T_high,
                         np.zeros((K, 7)), np.zeros((K, 7)), np.zeros((K, 4)), np.zeros((K, 4)),
                         [], fuel)

    # scale non-reference formation enthalpies so that the stoichiometric complete-combustion
    # adiabatic temperature from 300 K is 2300 K (bisection on the closed-form model enthalpy)
    nu, nb = unburnt_and_burnt_moles(mech_tmp, np.array([1.0]))
    nu, nb = nu[:, 0], nb[:, 0]

    def h_mix(n, T, scale):
        return sum(n[k] * (scale * dHf0[k] + R_GAS * _h_model_R(c0[k], cinf[k], theta[k], T))
                   for k in range(K))

    def T_ad(scale):
        target = h_mix(nu, 300.0, scale)
        lo, hi = 300.0, 6000.0
        for _ in range(100):
            mid = 0.5 * (lo + hi)
            if h_mix(nb, mid, scale) > target:
                hi = mid
            else:
                lo = mid
        return 0.5 * (lo + hi)

    lo, hi = 0.05, 5.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if T_ad(mid) > 2300.0:
            hi = mid
        else:
            lo = mid
    scale = 0.5 * (lo + hi)
    dHf = scale * dHf0

    nasa_low = np.zeros((K, 7))
    nasa_high = np.zeros((K, 7))
    for k in range(K):
        nasa_low[k], nasa_high[k] = _fit_nasa7(c0[k], cinf[k], theta[k], dHf[k] / R_GAS, s298[k],
                                               T_low, T_mid, T_high)

    # --- transport fits: ln(mu) and ln(lambda) cubic in ln T around ln 300
    mu_fit = np.zeros((K, 4))
    lam_fit = np.zeros((K, 4))
    L0 = math.log(300.0)
    for k in range(K):
        for fit, ref, expo in ((mu_fit, 1.8e-5 * math.sqrt(W[k] / 0.028) * rng.uniform(0.8, 1.2),
                                rng.uniform(0.65, 0.80)),
                               (lam_fit, 0.025 * math.sqrt(0.028 / W[k]) * rng.uniform(0.8, 1.2),
                                rng.uniform(0.70, 0.90))):
            c2 = rng.uniform(-0.02, 0.02)
            c3 = rng.uniform(-0.003, 0.003)
            # ln f = ln ref + expo u + c2 u^2 + c3 u^3 with u = lnT - L0, expanded in lnT
            fit[k, 0] = math.log(ref) - expo * L0 + c2 * L0 ** 2 - c3 * L0 ** 3
            fit[k, 1] = expo - 2 * c2 * L0 + 3 * c3 * L0 ** 2
            fit[k, 2] = c2 - 3 * c3 * L0
            fit[k, 3] = c3

    # --- reactions
    bimol, assoc = _candidates(species, comps, elements)
    n_el = n_rxn - n_tb - n_troe
    reactions: List[Reaction] = []
    used_b = set()
    used_a = set()

    T_REF = 1000.0

    def draw_arrh():
        # A is the prefactor at T_REF: k = A (T/T_REF)^b exp(-Ea/RT); returned in the
        # standard form A' T^b exp(-Ea/RT) with A' = A / T_REF^b
        A = 10.0 ** rng.uniform(8.0, 14.0)
        b = rng.uniform(-1.0, 2.0)
        return A / T_REF ** b, b, rng.uniform(0.0, 200e3)

    def exothermic_first(lhs, rhs):
        # write the reaction in its exothermic direction (298 K formation enthalpies), so the
        # drawn Ea belongs to that direction and the endothermic reverse follows from K_c
        dH = sum(dHf[k] for k in rhs) - sum(dHf[k] for k in lhs)
        return (lhs, rhs) if dH <= 0 else (rhs, lhs)

    def eff_for():
        e = {}
        for s in ("H2O", "CO2"):
            if s in species:
                e[species.index(s)] = float(rng.uniform(2.0, 12.0))
        return e

    def add_bimol(ci):
        lhs, rhs = exothermic_first(list(bimol[ci][0]), list(bimol[ci][1]))
        A, bb, Ea = draw_arrh()
        reactions.append(Reaction(0, lhs, rhs, A * 1e-6, bb, Ea))
        used_b.add(ci)

    def add_assoc(ci, kind_):
        (a, b), c = assoc[ci]
        A, bb, Ea = draw_arrh()
        if kind_ == 1:
            reactions.append(Reaction(1, [a, b], [c], A * 1e-12, bb, Ea, eff=eff_for()))
        else:
            A0 = A * 10.0 ** rng.uniform(4.0, 6.0)
            b0 = bb - rng.uniform(0.0, 1.0)
            Ea0 = Ea * rng.uniform(0.0, 1.0)
            tro = [float(rng.uniform(0.3, 0.9)), float(10 ** rng.uniform(1, 3)),
                   float(10 ** rng.uniform(math.log10(500), math.log10(5000)))]
            if rng.random() < 0.5:
                tro.append(float(10 ** rng.uniform(3, 4)))
            reactions.append(Reaction(2, [a, b], [c], A * 1e-6, bb, Ea, eff=eff_for(),
                                      low=(A0 * 1e-12, b0, Ea0), troe=tuple(tro)))
        used_a.add(ci)

    # association reactions first (third-body, then Troe)
    # recombinations used as third-body/falloff reactions are the exothermic ones
    order_a = [int(i) for i in rng.permutation(len(assoc))]
    order_a = ([i for i in order_a if dHf[assoc[i][1]] - dHf[assoc[i][0][0]] - dHf[assoc[i][0][1]] <= 0]
               + [i for i in order_a if dHf[assoc[i][1]] - dHf[assoc[i][0][0]] - dHf[assoc[i][0][1]] > 0])
    if len(order_a) < n_tb + n_troe:
        raise RuntimeError("not enough association candidates")
    for t in range(n_tb):
        add_assoc(int(order_a[t]), 1)
    for t in range(n_troe):
        add_assoc(int(order_a[n_tb + t]), 2)
    # cover every reactive species with at least one reaction
    covered = set()
    for r in reactions:
        covered.update(r.reactants + r.products)
    for k in rng.permutation(K):
        k = int(k)
        if species[k] in INERT or k in covered or len(reactions) >= n_rxn:
            continue
        cand = [i for i, ((a, b), (c, d)) in enumerate(bimol)
                if i not in used_b and k in (a, b, c, d)]
        if not cand:
            continue
        ci = cand[int(rng.integers(len(cand)))]
        add_bimol(ci)
        covered.update(reactions[-1].reactants + reactions[-1].products)
    free = [i for i in rng.permutation(len(bimol)) if int(i) not in used_b]
    free_a = [i for i in rng.permutation(len(assoc)) if int(i) not in used_a]
    while len(reactions) < n_rxn:
        if free:
            add_bimol(int(free.pop()))
        else:
            # fewer balanced A+B<=>C+D sets exist than requested (9-species H/O/N set):
            # the rest are elementary A+B<=>C associations without a third body
            (a, b), c = assoc[int(free_a.pop())]
            lhs, rhs = exothermic_first([a, b], [c])
            A, bb, Ea = draw_arrh()
            reactions.append(Reaction(0, lhs, rhs, A * (1e-6 if len(lhs) == 2 else 1.0), bb, Ea))
    # final order: shuffle so kinds are interleaved
    perm = rng.permutation(len(reactions))
    reactions = [reactions[int(i)] for i in perm]

    mech = Mechanism(kind, elements, species, comp, W, T_low, T_mid, T_high, nasa_low, nasa_high,
                     mu_fit, lam_fit, reactions, fuel)
    mech.T_ad_stoich = T_ad(scale)
    return mech


# ----------------------------------------------------------------------------------------
# file format
# ----------------------------------------------------------------------------------------
def write_mechanism(mech: Mechanism, path: str) -> None:
    """Write the mechanism in this project's plain-text format (SI units)."""
    L = []
    L.append(f"mech {mech.name}")
    L.append("elements " + " ".join(mech.elements))
    L.append(f"species {mech.n_species}")
    for k, s in enumerate(mech.species):
        L.append(f"sp {s} {mech.W[k]:.17g} " + " ".join(str(int(x)) for x in mech.comp[k]))
    L.append(f"thermo_ranges {mech.T_low:.17g} {mech.T_mid:.17g} {mech.T_high:.17g}")
    for k, s in enumerate(mech.species):
        L.append(f"nasa7 {s} " + " ".join(f"{x:.17g}" for x in mech.nasa_low[k]) + " "
                 + " ".join(f"{x:.17g}" for x in mech.nasa_high[k]))
    for k, s in enumerate(mech.species):
        L.append(f"transport {s} " + " ".join(f"{x:.17g}" for x in mech.mu_fit[k]) + " "
                 + " ".join(f"{x:.17g}" for x in mech.lam_fit[k]))
    L.append(f"reactions {mech.n_reactions}")
    for j, r in enumerate(mech.reactions):
        kind = ("elem", "threebody", "troe")[r.kind]
        lhs = " ".join(mech.species[i] for i in r.reactants)
        rhs = " ".join(mech.species[i] for i in r.products)
        L.append(f"rxn {kind} {len(r.reactants)} {lhs} {len(r.products)} {rhs} "
                 f"{r.A:.17g} {r.b:.17g} {r.Ea:.17g}")
        if r.kind >= 1:
            L.append(f"eff {len(r.eff)} " + " ".join(f"{mech.species[i]} {a:.17g}" for i, a in
                                                      sorted(r.eff.items())))
        if r.kind == 2:
            L.append(f"low {r.low[0]:.17g} {r.low[1]:.17g} {r.low[2]:.17g}")
            L.append(f"troe {len(r.troe)} " + " ".join(f"{x:.17g}" for x in r.troe))
    L.append("end")
    with open(path, "w") as f:
        f.write("\n".join(L) + "\n")


# ----------------------------------------------------------------------------------------
# cell states
# ----------------------------------------------------------------------------------------
@dataclasses.dataclass
class States:
    T: np.ndarray      # [N] K
    p: np.ndarray      # [N] Pa
    Y: np.ndarray      # [K, N] mass fractions, species-major (SoA)


def make_states(mech: Mechanism, n: int, seed: int, T_range=(300.0, 2500.0), p=P_ATM,
                phi_range=(0.6, 1.0), sigma=0.05) -> States:
    """Seeded cell states on fresh-gas / burnt-gas mixing lines.

    phi ~ U(phi_range), xi ~ U[0, 1]; Y = (1 - xi) Y_u + xi Y_b + radical pool; then
    Y_k *= exp(sigma N(0, 1)) and renormalise; T ~ U(T_range) independently; p fixed.
    The radical pool gives every species that is absent from both endpoints a seeded mass
    fraction xi * 10^U[-7, -3] + 10^U[-12, -9].
    """
    rng = np.random.default_rng(seed)
    K = mech.n_species
    phi = rng.uniform(phi_range[0], phi_range[1], n)
    xi = rng.uniform(0.0, 1.0, n)
    T = rng.uniform(T_range[0], T_range[1], n)
    nu, nb = unburnt_and_burnt_moles(mech, phi)
    Yu = moles_to_mass_fractions(mech, nu)
    Yb = moles_to_mass_fractions(mech, nb)
    Y = (1.0 - xi) * Yu + xi * Yb
    major = (nu.sum(axis=1) > 0) | (nb.sum(axis=1) > 0)
    pool_hi = xi * 10.0 ** rng.uniform(-7.0, -3.0, (K, n))
    pool_lo = 10.0 ** rng.uniform(-12.0, -9.0, (K, n))
    Y = np.where(major[:, None], Y, pool_hi + pool_lo)
    Y = Y * np.exp(sigma * rng.standard_normal((K, n)))
    Y = Y / Y.sum(axis=0, keepdims=True)
    return States(T=np.ascontiguousarray(T), p=np.full(n, float(p)), Y=np.ascontiguousarray(Y))


# ----------------------------------------------------------------------------------------
# named workloads (mechanism kind, mechanism seed, cells, dt, state seed)
# ----------------------------------------------------------------------------------------
WORKLOADS = {
    "di_h2_9sp_4k": dict(kind="h2_9", mech_seed=0, n=4096, dt=1e-6, state_seed=100),
    "di_c_30sp_1m": dict(kind="c_30", mech_seed=1, n=1_000_000, dt=5e-6, state_seed=101),
    "di_c_53sp_8m": dict(kind="c_53", mech_seed=5, n=8_000_000, dt=1e-5, state_seed=105),
}


def uniform_draws(rows: int, n: int, seed: int) -> np.ndarray:
    """Seeded uniform numbers in [-1, 1], shape [rows, n] (the gamma of the random
    augmentation of training states)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=(rows, n))


@dataclasses.dataclass
class TurbulenceFields:
    """Per-cell LES sub-grid quantities for the PaSR source: density (kg/m^3), sub-grid kinetic
    energy k (m^2/s^2), its dissipation rate eps (m^2/s^3) and kinematic viscosity nu (m^2/s)."""
    rho: np.ndarray
    k: np.ndarray
    eps: np.ndarray
    nu: np.ndarray


def make_turbulence(n: int, seed: int, laminar_fraction: float = 0.05) -> TurbulenceFields:
    """Seeded synthetic sub-grid fields with swirl-flame LES magnitudes: rho log-uniform in
    [0.12, 1.2] (2500 K to 300 K at 1 atm), k log-uniform in [1e-3, 10], eps log-uniform in
    [1, 1e6], nu log-uniform in [1.5e-5, 4e-4]; a fraction of cells has k = 0 (no sub-grid
    turbulence, e.g. near walls or in the fresh gas core)."""
    rng = np.random.default_rng(seed)
    lu = lambda lo, hi: np.exp(rng.uniform(np.log(lo), np.log(hi), n))  # noqa: E731
    rho, k, eps, nu = lu(0.12, 1.2), lu(1e-3, 10.0), lu(1.0, 1e6), lu(1.5e-5, 4e-4)
    k[rng.random(n) < laminar_fraction] = 0.0
    return TurbulenceFields(rho=rho, k=k, eps=eps, nu=nu)


def mechanism_file(kind: str, seed: int, directory: str) -> str:
    """Generate (once) and return the path of a mechanism file in `directory`."""
    import os
    os.makedirs(directory, exist_ok=True)
    path = os.path.join(directory, f"{kind}_seed{seed}.mech")
    if not os.path.exists(path):
        tmp = path + f".tmp{os.getpid()}"
        write_mechanism(make_mechanism(kind, seed), tmp)
        os.replace(tmp, path)
    return path
