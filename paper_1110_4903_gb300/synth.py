"""Seeded synthetic inputs: reaction mechanisms shaped like the paper's two
cases and initial (T, P, Y) fields.

This module builds input arrays only.  It evaluates no thermodynamic
function, rate, source term or Jacobian: converting (T, P, Y) to the
chemistry state (rho_s, e) and everything after it is done separately by the
CUDA library and by the CPU oracle.  Both consume exactly the arrays made
here.

Mechanism shapes (Le & Cambier, arXiv 1110.4903):
  * 9 species / 38 reversible reactions: the 19-reaction H2-air topology of
    Appendix A (six +M reactions: 5, 6, 7, 8, 10, 15) plus 19 more
    element-balanced reactions over the same species, with N2 as an inert
    ninth species (3 elements H, O, N).  Sec. 5.2 reports this case.
  * 36 species / 308 reversible reactions, 4 elements (H, O, N, C): 40
    third-body recombinations, 12 pressure-independent unimolecular
    decompositions, 256 bimolecular exchanges.  Sec. 5.2 reports a case of
    this size.
All coefficients are synthetic (the paper prints none): log10 A ~ U[8, 14]
(CGS), beta ~ U[-1, 1], Ea ~ U[0, 2e5] J/mol, NASA-7 polynomials built so
that cp/R >= 1.3 on [0, 6000] K and cp, h, s are continuous at 1000 K.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

# Standard atomic weights, kg/mol.
ELEMENT_MASS = {"H": 1.00794e-3, "O": 15.9994e-3, "N": 14.0067e-3, "C": 12.0107e-3}
# Gas-phase atom enthalpies of formation at 298 K, J/mol (scale of the
# bond-additive formation enthalpies below).
ATOM_ENTHALPY = {"H": 2.18e5, "O": 2.49e5, "N": 4.73e5, "C": 7.17e5}

T_MID = 1000.0
T_LOW = 200.0
T_HIGH = 6000.0

# Appendix A of the paper: H2-air detonation mechanism (topology only).
# Each entry: (reactants, products, third_body); species with multiplicity.
APPENDIX_A = [
    (("H", "O2"), ("O", "OH"), 0),
    (("O", "H2"), ("H", "OH"), 0),
    (("H2", "OH"), ("H", "H2O"), 0),
    (("OH", "OH"), ("H2O", "O"), 0),
    (("H", "OH"), ("H2O",), 1),
    (("H", "H"), ("H2",), 1),
    (("H", "O"), ("OH",), 1),
    (("O", "O"), ("O2",), 1),
    (("H2", "O2"), ("HO2", "H"), 0),
    (("H", "O2"), ("HO2",), 1),
    (("H", "HO2"), ("OH", "OH"), 0),
    (("H", "HO2"), ("O", "H2O"), 0),
    (("O", "HO2"), ("O2", "OH"), 0),
    (("OH", "HO2"), ("O2", "H2O"), 0),
    (("H2O2",), ("OH", "OH"), 1),
    (("HO2", "HO2"), ("H2O2", "O2"), 0),
    (("H", "H2O2"), ("H2", "HO2"), 0),
    (("O", "H2O2"), ("OH", "HO2"), 0),
    (("OH", "H2O2"), ("H2O", "HO2"), 0),
]

H2AIR_SPECIES = {
    "H": {"H": 1}, "O2": {"O": 2}, "O": {"O": 1}, "OH": {"O": 1, "H": 1},
    "H2": {"H": 2}, "H2O": {"H": 2, "O": 1}, "HO2": {"H": 1, "O": 2},
    "H2O2": {"H": 2, "O": 2}, "N2": {"N": 2},
}


@dataclass
class Mechanism:
    """Flat mechanism arrays, the layout both the library and the oracle take."""
    name: str
    species: list
    elements: list
    molar_mass: np.ndarray      # [ns] kg/mol
    elem_comp: np.ndarray       # [ns, ne] int32
    nasa7: np.ndarray           # [ns, 2, 7] low range, high range
    t_range: np.ndarray         # [ns, 3] T_low, T_mid, T_high
    arr_A: np.ndarray           # [nr] CGS
    arr_beta: np.ndarray        # [nr]
    arr_Ea: np.ndarray          # [nr] J/mol
    reac_sp: np.ndarray         # [nr, 3] int32, -1 unused
    reac_nu: np.ndarray         # [nr, 3] int32
    prod_sp: np.ndarray         # [nr, 3] int32
    prod_nu: np.ndarray         # [nr, 3] int32
    third_body: np.ndarray      # [nr] int32
    tb_eff: np.ndarray          # [nr, ns]
    extra: dict = field(default_factory=dict)

    @property
    def ns(self):
        return len(self.species)

    @property
    def nr(self):
        return int(self.arr_A.shape[0])

    @property
    def ne(self):
        return len(self.elements)


def _counts(names):
    out = {}
    for s in names:
        out[s] = out.get(s, 0) + 1
    return out


def _pack_side(side_counts, index):
    sp = np.full(3, -1, np.int32)
    nu = np.zeros(3, np.int32)
    for j, (name, k) in enumerate(sorted(side_counts.items(), key=lambda kv: index[kv[0]])):
        sp[j] = index[name]
        nu[j] = k
    return sp, nu


def make_mechanism(name, species, compositions, elements, reactions, nasa7,
                   arr_A, arr_beta, arr_Ea, tb_eff=None, t_mid=T_MID):
    """Build a Mechanism from explicit lists.

    species: names; compositions: {name: {element: count}};
    reactions: list of (reactant_names, product_names, third_body) with names
    repeated for multiplicity; nasa7: array [ns, 2, 7].
    """
    index = {s: i for i, s in enumerate(species)}
    ns, nr, ne = len(species), len(reactions), len(elements)
    comp = np.zeros((ns, ne), np.int32)
    for i, s in enumerate(species):
        for el, k in compositions[s].items():
            comp[i, elements.index(el)] = k
    W = np.array([sum(ELEMENT_MASS[el] * k for el, k in compositions[s].items())
                  for s in species], np.float64)
    reac_sp = np.full((nr, 3), -1, np.int32)
    reac_nu = np.zeros((nr, 3), np.int32)
    prod_sp = np.full((nr, 3), -1, np.int32)
    prod_nu = np.zeros((nr, 3), np.int32)
    tb = np.zeros(nr, np.int32)
    for r, (re, pr, m) in enumerate(reactions):
        reac_sp[r], reac_nu[r] = _pack_side(_counts(re), index)
        prod_sp[r], prod_nu[r] = _pack_side(_counts(pr), index)
        tb[r] = int(m)
    if tb_eff is None:
        tb_eff = np.ones((nr, ns), np.float64)
    t_range = np.tile(np.array([T_LOW, t_mid, T_HIGH], np.float64), (ns, 1))
    return Mechanism(name=name, species=list(species), elements=list(elements),
                     molar_mass=W, elem_comp=comp,
                     nasa7=np.ascontiguousarray(nasa7, np.float64),
                     t_range=t_range,
                     arr_A=np.ascontiguousarray(arr_A, np.float64),
                     arr_beta=np.ascontiguousarray(arr_beta, np.float64),
                     arr_Ea=np.ascontiguousarray(arr_Ea, np.float64),
                     reac_sp=reac_sp, reac_nu=reac_nu, prod_sp=prod_sp,
                     prod_nu=prod_nu, third_body=tb,
                     tb_eff=np.ascontiguousarray(tb_eff, np.float64))


# ---------------------------------------------------------------------------
# NASA-7 coefficient construction
# ---------------------------------------------------------------------------
def _nasa7_draw(rng, n_atoms):
    """Low-range coefficients with cp/R >= 1.5 on [0, 6000] K by construction,
    and a high range that differs by c (T - Tm)^2 + d (T - Tm)^3 (|.| <= 0.2
    above Tm), with a6, a7 shifted by the closed-form constants that keep h and
    s continuous at Tm.  Returns a [2, 7] array."""
    kappa = 0.05 if n_atoms == 1 else 0.25
    if n_atoms == 1:
        a1 = 2.5
    else:
        a1 = rng.uniform(2.5 + 0.5 * (n_atoms - 1), 2.5 + 1.5 * (n_atoms - 1))
    Tb = T_HIGH
    a2 = rng.uniform(0.0, 1.0) * kappa / Tb
    a3 = rng.uniform(-1.0, 1.0) * kappa / Tb ** 2
    a4 = rng.uniform(-1.0, 1.0) * kappa / Tb ** 3
    a5 = rng.uniform(-1.0, 1.0) * kappa / Tb ** 4
    return a1, a2, a3, a4, a5


def _nasa7_pair(a1, a2, a3, a4, a5, a6, a7, c, d, m=T_MID):
    low = np.array([a1, a2, a3, a4, a5, a6, a7], np.float64)
    # coefficient shifts of c (T-m)^2 + d (T-m)^3 in monomials
    d1 = c * m * m - d * m ** 3
    d2 = -2.0 * c * m + 3.0 * d * m * m
    d3 = c - 3.0 * d * m
    d4 = d
    d6 = -c * m ** 3 / 3.0 + d * m ** 4 / 4.0
    d7 = -(c * m * m - d * m ** 3) * np.log(m) + 1.5 * c * m * m - (11.0 / 6.0) * d * m ** 3
    high = low + np.array([d1, d2, d3, d4, 0.0, d6, d7])
    return np.stack([low, high])


def _species_thermo(rng, comps):
    """NASA-7 for every species.  Formation enthalpies are bond-additive: the
    atoms' enthalpies minus one bond energy U[3.5e5, 4.5e5] J/mol per bond of
    a chain molecule, plus U[-2e4, 2e4] J/mol; standard entropies grow with
    size, s/R(298 K) ~ 13 + 3.5 atoms + U[-1.5, 1.5].  This keeps every rate
    bounded like a physical mechanism: a dissociation needs about a bond
    energy, so no reverse rate outruns its forward rate by many decades."""
    out = []
    for name, comp in comps:
        n_atoms = sum(comp.values())
        a1, a2, a3, a4, a5 = _nasa7_draw(rng, n_atoms)
        dHf = sum(ATOM_ENTHALPY[el] * k for el, k in comp.items())
        dHf -= rng.uniform(3.5e5, 4.5e5, n_atoms - 1).sum()
        dHf += rng.uniform(-2e4, 2e4)
        a6 = dHf / 8.314462618 - 298.15 * a1
        a7 = 13.0 + 3.5 * n_atoms + rng.uniform(-1.5, 1.5) - a1 * 5.7
        c = rng.uniform(-1.0, 1.0) * 0.1 / 5000.0 ** 2
        d = rng.uniform(-1.0, 1.0) * 0.1 / 5000.0 ** 3
        out.append(_nasa7_pair(a1, a2, a3, a4, a5, a6, a7, c, d))
    return np.stack(out)


def _enthalpy_proxy(nasa7, idx):
    """Dominant part of h(298 K)/R of a species: a6 + 298.15 a1 (the
    generator's own formation-enthalpy draw).  Used only to orient reactions
    so the forward direction is the exothermic one."""
    return nasa7[idx, 0, 5] + 298.15 * nasa7[idx, 0, 0]


def _orient(reactions, nasa7, index):
    out = []
    for re, pr, m in reactions:
        dh = sum(_enthalpy_proxy(nasa7, index[s]) for s in pr) - \
            sum(_enthalpy_proxy(nasa7, index[s]) for s in re)
        out.append((pr, re, m) if dh > 0 else (re, pr, m))
    return out


def _arrhenius(rng, nr):
    A = 10.0 ** rng.uniform(8.0, 14.0, nr)
    beta = rng.uniform(-1.0, 1.0, nr)
    Ea = rng.uniform(0.0, 2e5, nr)
    return A, beta, Ea


def _efficiencies(rng, reactions, ns):
    eff = np.ones((len(reactions), ns), np.float64)
    for r, (_, _, m) in enumerate(reactions):
        if m:
            k = int(rng.integers(2, 4))
            for s in rng.choice(ns, size=k, replace=False):
                eff[r, s] = rng.uniform(0.4, 5.0)
    return eff


def _vec(comp, elements):
    return tuple(comp.get(e, 0) for e in elements)


def _balanced_pairs(species, comps, elements, sizes_left, sizes_right, exclude=()):
    """All element-balanced (left, right) multiset pairs with no common species."""
    by_vec = {}
    for size in sorted(set(sizes_left) | set(sizes_right)):
        for ms in itertools.combinations_with_replacement(species, size):
            v = tuple(sum(x) for x in zip(*[_vec(comps[s], elements) for s in ms]))
            by_vec.setdefault(v, []).append(ms)
    ex = set(exclude)
    pairs = []
    for v, group in by_vec.items():
        for a in group:
            for b in group:
                if len(a) not in sizes_left or len(b) not in sizes_right:
                    continue
                if set(a) & set(b):
                    continue
                key = frozenset([tuple(sorted(a)), tuple(sorted(b))])
                if key in ex:
                    continue
                ex.add(key)
                pairs.append((a, b))
    return pairs


def h2_air_9sp(seed: int = 9038) -> Mechanism:
    """9 species / 38 reversible reactions: Appendix A (19 reactions, six +M)
    plus 19 element-balanced exchanges drawn over the same species."""
    rng = np.random.default_rng(seed)
    species = ["H", "O2", "O", "OH", "H2", "H2O", "HO2", "H2O2", "N2"]
    elements = ["H", "O", "N"]
    comps = H2AIR_SPECIES
    reactions = [(tuple(re), tuple(pr), m) for re, pr, m in APPENDIX_A]
    existing = {frozenset([tuple(sorted(re)), tuple(sorted(pr))]) for re, pr, _ in reactions}
    reactive = [s for s in species if s != "N2"]
    cand = _balanced_pairs(reactive, comps, elements, (1, 2, 3), (1, 2, 3), exclude=existing)
    cand = [(a, b) for a, b in cand if len(a) + len(b) >= 3]
    cand.sort()
    pick = rng.choice(len(cand), size=19, replace=False)
    for i in sorted(pick):
        reactions.append((cand[i][0], cand[i][1], 0))
    nasa = _species_thermo(rng, [(s, comps[s]) for s in species])
    index = {s: i for i, s in enumerate(species)}
    reactions = _orient(reactions, nasa, index)
    A, beta, Ea = _arrhenius(rng, len(reactions))
    eff = _efficiencies(rng, reactions, len(species))
    return make_mechanism("h2air-9sp-38r", species, comps, elements, reactions, nasa,
                          A, beta, Ea, tb_eff=eff)


def _formula(comp, elements):
    s = ""
    for el in elements:
        k = comp.get(el, 0)
        if k:
            s += el + (str(k) if k > 1 else "")
    return s


def hydrocarbon_36sp(seed: int = 36308) -> Mechanism:
    """36 species / 308 reversible reactions over H, O, N, C: 40 third-body
    recombinations A + B + M = AB + M, 12 pressure-independent unimolecular
    decompositions AB = A + B, 256 bimolecular exchanges A + B = C + D."""
    return hydrocarbon_mechanism(36, 40, 12, 256, seed, "hc-36sp-308r")


def hydrocarbon_mechanism(ns: int, n_tb: int, n_uni: int, n_ex: int, seed: int, name: str) -> Mechanism:
    """ns species over H, O, N, C grown from atoms and diatomics (at most 6
    atoms), with n_tb third-body recombinations, n_uni pressure-independent
    unimolecular decompositions and n_ex bimolecular exchanges."""
    rng = np.random.default_rng(seed)
    elements = ["H", "O", "N", "C"]
    comps = [{"H": 1}, {"O": 1}, {"N": 1}, {"C": 1}, {"H": 2}, {"O": 2}, {"N": 2}]
    seen = {_vec(c, elements) for c in comps}
    # grow the species set by joining an existing species with an atom or a
    # diatomic (<= 6 atoms), so that every new species has at least one
    # recombination channel; no homonuclear species beyond diatomics
    while len(comps) < ns:
        i = int(rng.integers(0, len(comps)))
        j = 0 if rng.uniform() < 0.5 else int(rng.integers(0, 7))
        v = tuple(a + b for a, b in zip(_vec(comps[i], elements), _vec(comps[j], elements)))
        if sum(v) > 6 or v in seen or (sum(1 for k in v if k) == 1 and sum(v) > 2):
            continue
        seen.add(v)
        comps.append({el: int(k) for el, k in zip(elements, v) if k})
    names = [_formula(c, elements) for c in comps]
    comp_map = dict(zip(names, comps))

    # recombination candidates (A, B, AB): comp(A) + comp(B) = comp(AB)
    vecs = {n: np.array(_vec(comp_map[n], elements)) for n in names}
    recomb = []
    for i, a in enumerate(names):
        for b in names[i:]:
            v = vecs[a] + vecs[b]
            for ab in names:
                if ab not in (a, b) and np.array_equal(vecs[ab], v):
                    recomb.append(((a, b), (ab,)))
    recomb.sort()
    if len(recomb) < n_tb + n_uni:
        raise RuntimeError("species draw leaves too few recombination channels")
    pick = rng.choice(len(recomb), size=n_tb + n_uni, replace=False)
    tb_set = [recomb[i] for i in pick[:n_tb]]
    uni_set = [recomb[i] for i in pick[n_tb:]]
    reactions = [(re, pr, 1) for re, pr in tb_set]
    reactions += [(pr, re, 0) for re, pr in uni_set]
    used = {frozenset([tuple(sorted(re)), tuple(sorted(pr))]) for re, pr, _ in reactions}
    ex = _balanced_pairs(names, comp_map, elements, (2,), (2,), exclude=used)
    ex.sort()
    if len(ex) < n_ex:
        raise RuntimeError("species draw leaves too few exchange channels")
    pick = rng.choice(len(ex), size=n_ex, replace=False)
    for i in sorted(pick):
        reactions.append((ex[i][0], ex[i][1], 0))
    nasa = _species_thermo(rng, [(n, comp_map[n]) for n in names])
    index = {s: i for i, s in enumerate(names)}
    reactions = _orient(reactions, nasa, index)
    A, beta, Ea = _arrhenius(rng, len(reactions))
    eff = _efficiencies(rng, reactions, len(names))
    return make_mechanism(name, names, comp_map, elements, reactions, nasa,
                          A, beta, Ea, tb_eff=eff)


# ---------------------------------------------------------------------------
# Initial fields: T, P, Y (mass fractions, SoA [ns, n])
# ---------------------------------------------------------------------------
@dataclass
class Field:
    T: np.ndarray
    P: np.ndarray
    Y: np.ndarray   # [ns, n]

    @property
    def n(self):
        return int(self.T.shape[0])


def uniform_field(ns: int, n: int, T_lo: float, T_hi: float, seed: int,
                  P: float = 101325.0) -> Field:
    """T ~ U[T_lo, T_hi], constant P, Y ~ Dirichlet(1, ..., 1)."""
    rng = np.random.default_rng(seed)
    T = rng.uniform(T_lo, T_hi, n)
    Y = np.ascontiguousarray(rng.dirichlet(np.ones(ns), size=n).T)
    return Field(T=T, P=np.full(n, P), Y=Y)


def _stable_order(mech):
    """Species indices from most to least stable per atom by the generator's
    own formation-enthalpy draw (a6 + 298.15 a1, the same proxy that orients
    the reactions)."""
    atoms = mech.elem_comp.sum(1)
    proxy = (mech.nasa7[:, 0, 5] + 298.15 * mech.nasa7[:, 0, 0]) / atoms
    return np.argsort(proxy, kind="stable")


def front_field(mech, nx: int = 2048, ny: int = 1024, seed: int = 4,
                P: float = 101325.0, band: int = 64, T_band: float = 2800.0) -> Field:
    """2-D field, x fastest: unburnt gas at 300-1200 K (T linear in y plus a
    smooth seeded perturbation) and a vertical band `band` columns wide at
    T_band with tanh edges.  Outside the band the gas is a stable reactant
    mixture (N2, O2, H2 and the two most stable polyatomic species); inside
    it is product-rich (the most stable species per atom) with a small
    radical pool; the edges mix the two."""
    ns = mech.ns
    rng = np.random.default_rng(seed)
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    k1, k2 = rng.integers(1, 4, size=2)
    p1, p2 = rng.uniform(0, 2 * np.pi, size=2)
    T_gas = 300.0 + 900.0 * y / (ny - 1) + 40.0 * np.sin(2 * np.pi * k1 * x / nx + p1) * \
        np.sin(2 * np.pi * k2 * y / ny + p2)
    T_gas = np.clip(T_gas, 300.0, 1200.0)
    xc = nx / 2 + rng.uniform(-nx / 8, nx / 8)
    wgt = 0.5 * (np.tanh((x - (xc - band / 2)) / 4.0) - np.tanh((x - (xc + band / 2)) / 4.0))
    wgt = np.broadcast_to(wgt, (ny, nx))
    T = T_gas * (1.0 - wgt) + T_band * wgt
    names = list(mech.species)
    order = [int(i) for i in _stable_order(mech)]
    poly = [i for i in order if mech.elem_comp[i].sum() > 2][:2]
    Y_out = np.zeros(ns)
    for nm, v in (("N2", 0.70), ("O2", 0.20), ("H2", 0.04)):
        Y_out[names.index(nm)] = v
    for i in poly:
        Y_out[i] += 0.03
    Y_in = np.zeros(ns)
    Y_in[names.index("N2")] = 0.70
    stable = [i for i in order if names[i] != "N2"][:4]
    Y_in[stable] += rng.dirichlet(np.full(len(stable), 4.0)) * 0.29
    radicals = [i for i in range(ns) if mech.elem_comp[i].sum() == 1]
    Y_in[radicals] += 0.01 / len(radicals)
    Y_out /= Y_out.sum()
    Y_in /= Y_in.sum()
    w = wgt.reshape(-1)
    Y = Y_out[:, None] * (1.0 - w)[None, :] + Y_in[:, None] * w[None, :]
    return Field(T=T.reshape(-1).copy(), P=np.full(nx * ny, P), Y=np.ascontiguousarray(Y))


# Named workloads (mechanism, field) with their sizes.
def workload(name: str):
    if name == "h2air-1k":
        m = h2_air_9sp()
        return m, uniform_field(m.ns, 1024, 1000.0, 2500.0, seed=1), 1e-7
    if name == "h2air-1M":
        m = h2_air_9sp()
        return m, uniform_field(m.ns, 1 << 20, 900.0, 2800.0, seed=2), 1e-6
    if name == "hc36-256k":
        m = hydrocarbon_36sp()
        return m, uniform_field(m.ns, 1 << 18, 900.0, 2800.0, seed=3), 1e-6
    if name == "hc36-front-2M":
        m = hydrocarbon_36sp()
        return m, front_field(m, seed=4), 1e-6
    raise KeyError(name)


def subsample(f: Field, idx: np.ndarray) -> Field:
    return Field(T=f.T[idx].copy(), P=f.P[idx].copy(), Y=np.ascontiguousarray(f.Y[:, idx]))


def poisson_requests(n_req: int, rate_hz: float, seed: int = 5,
                     min_cells: int = 1024, max_cells: int = 262144,
                     dt_lo: float = 1e-8, dt_hi: float = 1e-5):
    """Request stream: Poisson arrivals, log-uniform sizes and dt, mechanism
    0 or 1 with probability 1/2 each."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, n_req)
    t = np.cumsum(gaps)
    sizes = np.exp(rng.uniform(np.log(min_cells), np.log(max_cells), n_req)).astype(np.int64)
    mech = rng.integers(0, 2, n_req)
    dts = np.exp(rng.uniform(np.log(dt_lo), np.log(dt_hi), n_req))
    seeds = rng.integers(0, 2 ** 31 - 1, n_req)
    return [dict(t=float(t[i]), n=int(sizes[i]), mech=int(mech[i]), dt=float(dts[i]),
                 seed=int(seeds[i])) for i in range(n_req)]
