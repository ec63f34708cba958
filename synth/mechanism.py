"""Seeded synthetic reaction mechanisms.

A mechanism is a dict of numpy arrays with this layout (SI units throughout):

    ns, nr, ne         species, reactions, elements
    names              list of species names (shaped after real species)
    elements           list of element symbols
    elem   [ns, ne]    int32 atom counts
    W      [ns]        float64 molar mass, kg/mol (from the atomic weights)
    thermo [ns, 9]     float64 NASA-7 coefficients a1..a7 (cp/R = a1 + a2 T + ... + a5 T^4,
                       h/R = a1 T + a2 T^2/2 + ... + a5 T^5/5 + a6,
                       s/R = a1 ln T + a2 T + ... + a5 T^4/4 + a7), then T_lo, T_hi (K)
    nu_f, nu_r [nr, ns] int8 reactant / product coefficients (0..2)
    A, b, Ea   [nr]    k_f = A T^b exp(-Ea / (R T)); A in SI (mol, m^3, s), Ea in J/mol
    reversible [nr]    uint8
    third_body [nr]    uint8
    eff    [nr, ns]    float64 third-body collision efficiencies (1.0 by default)
    fuel, oxidizer, inert, product   species indices of the premix roles

Readings of the mechanism recipe (the paper gives no mechanism data, only shapes):
  * species carry real element compositions, so every drawn reaction is element balanced;
  * a reaction side holds 1..3 molecules (1..2 for third-body reactions), coefficients 0..2,
    no species on both sides, no duplicate reactions, the inert species only as collider;
  * A is drawn log-uniform in CGS units and converted to SI with the forward molecularity
    n (+1 for a third body): A_SI = A_CGS * (1e-6)^(n-1);
  * cp/R is a quartic fitted through 5 seeded nodes on [300, 3500] K, rejected unless
    1.5 <= cp/R <= 12 on the whole range; outside [T_lo, T_hi] cp is held constant;
  * formation enthalpy at 300 K is 0 for the element-reference species (H2, O2, N2),
    uniform in [0, 3e5] J/mol for open-shell species (atoms and odd-electron species) and
    uniform in [-3e5, 0] J/mol for closed-shell molecules; entropy at 300 K is drawn by atom
    count (1: [110, 165], 2: [130, 225], 3: [185, 245], >= 4: [200, 280] J/mol/K);
  * every reaction is written in its exothermic direction at 300 K before A, b, Ea are drawn,
    so the endothermic direction, whose rate comes from K_c, carries the reaction enthalpy as
    an activation barrier.  Without this, reverse rate constants k_f / K_c reach 1e30 and
    q_f - q_r cancels below FP64 resolution, so no integrator could compute the solution.
"""
import itertools
import numpy as np

R_GAS = 8.314462618      # J/mol/K
P_ATM = 101325.0         # Pa

ATOMIC_WEIGHT = {"H": 1.008e-3, "C": 12.011e-3, "N": 14.007e-3, "O": 15.999e-3}
T_LO, T_HI = 300.0, 3500.0
T_REF = 300.0            # reference temperature of the drawn formation enthalpy / entropy

H2_AIR_SPECIES = [
    ("H2", {"H": 2}), ("O2", {"O": 2}), ("H", {"H": 1}), ("O", {"O": 1}),
    ("OH", {"H": 1, "O": 1}), ("H2O", {"H": 2, "O": 1}), ("HO2", {"H": 1, "O": 2}),
    ("H2O2", {"H": 2, "O": 2}), ("N2", {"N": 2}),
]
ELEMENT_REFERENCES = ("H2", "O2", "N2")


VALENCE_ELECTRONS = {"H": 1, "C": 4, "N": 5, "O": 6}
S_RANGE = {1: (110.0, 165.0), 2: (130.0, 225.0), 3: (185.0, 245.0), 4: (200.0, 280.0)}


def _open_shell(comp):
    """Atoms and odd-electron species are treated as radicals."""
    n_atoms = sum(comp.values())
    electrons = sum(VALENCE_ELECTRONS[e] * n for e, n in comp.items())
    return n_atoms == 1 or electrons % 2 == 1


def _formula(name_counts):
    return "".join(f"{el}{n if n > 1 else ''}" for el, n in name_counts if n > 0)


def _hydrocarbon_species(ns):
    """Deterministic C/H/O(/N) species list of size ns, shaped like a C2 combustion set."""
    base = [s for s in H2_AIR_SPECIES if s[0] != "N2"]
    seen = {tuple(sorted(c.items())) for _, c in base}
    extra = []
    for c in range(1, 4):
        for o in range(0, 3):
            for h in range(0, 2 * c + 3):
                comp = {"C": c, "H": h, "O": o}
                comp = {k: v for k, v in comp.items() if v > 0}
                key = tuple(sorted(comp.items()))
                if key in seen:
                    continue
                # keep near-valence species: H <= 2C+2, at most one more O than C
                if h > 2 * c + 2 or o > c + 1:
                    continue
                seen.add(key)
                name = _formula([("C", c), ("H", h), ("O", o)])
                extra.append((name, comp))
    # nitrogen-bearing minor species
    for comp in ({"N": 1}, {"N": 1, "O": 1}, {"N": 1, "O": 2}, {"N": 1, "H": 1}, {"N": 1, "H": 2},
                 {"N": 1, "H": 3}, {"H": 1, "C": 1, "N": 1}, {"N": 2, "O": 1}, {"C": 1, "N": 1}):
        key = tuple(sorted(comp.items()))
        if key not in seen:
            seen.add(key)
            extra.append((_formula([(e, comp.get(e, 0)) for e in "CHNO"]), comp))
    # order: small species first so truncation keeps the light ones
    extra.sort(key=lambda s: (sum(s[1].values()), s[0]))
    need = ns - len(base) - 1
    if need > len(extra):
        raise ValueError(f"cannot build {ns} species")
    return base + extra[:need] + [("N2", {"N": 2})]


def _thermo_fit(rng, n_atoms, h_f, s_ref):
    """Draw cp/R nodes shaped by atom count, fit a quartic, fix a6/a7 from h_f and s_ref."""
    if n_atoms == 1:
        lo, hi = 2.5, 2.6
    elif n_atoms == 2:
        lo, hi = 3.5, 4.6
    else:
        lo, hi = 4.0 + 0.3 * (n_atoms - 3), min(11.5, 3.0 * n_atoms - 1.5)
    nodes = np.linspace(T_LO, T_HI, 5)
    x = nodes / 1000.0
    vand = np.vander(x, 5, increasing=True)
    for _ in range(1000):
        tau = rng.uniform(600.0, 1500.0)
        shape = 1.0 - np.exp(-(nodes - T_LO) / tau)
        cp_nodes = lo + (hi - lo) * shape * rng.uniform(0.85, 1.0)
        cp_nodes *= 1.0 + rng.uniform(-0.02, 0.02, size=5)
        c = np.linalg.solve(vand, cp_nodes)
        grid = np.linspace(T_LO, T_HI, 321) / 1000.0
        cp_grid = np.polynomial.polynomial.polyval(grid, c)
        if cp_grid.min() >= 1.5 and cp_grid.max() <= 12.0:
            break
    else:  # pragma: no cover
        raise RuntimeError("thermo fit rejection did not terminate")
    a = np.zeros(9)
    a[0:5] = c / 1000.0 ** np.arange(5)
    T = T_REF
    poly_h = a[0] * T + a[1] * T**2 / 2 + a[2] * T**3 / 3 + a[3] * T**4 / 4 + a[4] * T**5 / 5
    poly_s = a[0] * np.log(T) + a[1] * T + a[2] * T**2 / 2 + a[3] * T**3 / 3 + a[4] * T**4 / 4
    a[5] = h_f / R_GAS - poly_h
    a[6] = s_ref / R_GAS - poly_s
    a[7], a[8] = T_LO, T_HI
    return a


def _draw_reactions(rng, elem, reactive, nr, n_tb, seen=None):
    """Element-balanced reactions by rejection; returns list of (reactants, products, tb)."""
    nre = len(reactive)
    sides_by_m = {}
    for m in (1, 2, 3):
        ss = []
        for comb in itertools.combinations_with_replacement(range(nre), m):
            if m == 3 and comb[0] == comb[2]:
                continue  # coefficient 3 not allowed
            ss.append(tuple(reactive[i] for i in comb))
        sides_by_m[m] = ss
    by_elem = {}
    for m, ss in sides_by_m.items():
        for s in ss:
            key = tuple(np.sum(elem[list(s)], axis=0))
            by_elem.setdefault(key, []).append(s)
    seen = set() if seen is None else seen
    out = []
    tb_flags = [True] * n_tb + [False] * (nr - n_tb)
    for tb in tb_flags:
        for _ in range(100000):
            max_m = 2 if tb else 3
            m = int(rng.choice([1, 2, 3][:max_m], p=[0.2, 0.6, 0.2][:max_m] / np.sum([0.2, 0.6, 0.2][:max_m])))
            ss = sides_by_m[m]
            lhs = ss[rng.integers(len(ss))]
            key = tuple(np.sum(elem[list(lhs)], axis=0))
            cand = [s for s in by_elem[key]
                    if s != lhs and not (set(s) & set(lhs)) and len(s) <= max_m]
            if not cand:
                continue
            rhs = cand[rng.integers(len(cand))]
            pair = frozenset((lhs, rhs))
            if pair in seen:
                continue
            seen.add(pair)
            out.append((lhs, rhs, tb))
            break
        else:  # pragma: no cover
            raise RuntimeError("reaction rejection did not terminate")
    return out


def _build(species, nr, n_tb, seed, fuel, oxidizer, product):
    rng = np.random.default_rng(seed)
    elements = sorted({e for _, comp in species for e in comp}, key=lambda e: "CHON".index(e))
    ns, ne = len(species), len(elements)
    names = [s[0] for s in species]
    elem = np.zeros((ns, ne), dtype=np.int32)
    for k, (_, comp) in enumerate(species):
        for e, n in comp.items():
            elem[k, elements.index(e)] = n
    W = elem @ np.array([ATOMIC_WEIGHT[e] for e in elements])
    inert = names.index("N2")
    reactive = [k for k in range(ns) if k != inert]

    thermo = np.zeros((ns, 9))
    h_form = np.zeros(ns)
    for k, (name, comp) in enumerate(species):
        n_atoms = int(sum(comp.values()))
        if name in ELEMENT_REFERENCES:
            h_f = 0.0
        elif _open_shell(comp):
            h_f = rng.uniform(0.0, 3e5)
        else:
            h_f = rng.uniform(-3e5, 0.0)
        s_ref = rng.uniform(*S_RANGE[min(n_atoms, 4)])
        h_form[k] = h_f
        thermo[k] = _thermo_fit(rng, n_atoms, h_f, s_ref)

    rank_target = len(reactive) - np.linalg.matrix_rank(elem[reactive].astype(float))
    for attempt in range(1000):
        rx = _draw_reactions(rng, elem, reactive, nr, n_tb)
        nu_f = np.zeros((nr, ns), dtype=np.int8)
        nu_r = np.zeros((nr, ns), dtype=np.int8)
        for r, (lhs, rhs, _) in enumerate(rx):
            for k in lhs:
                nu_f[r, k] += 1
            for k in rhs:
                nu_r[r, k] += 1
        dnu = (nu_r - nu_f).astype(float)
        used = np.any(nu_f[:, reactive] + nu_r[:, reactive] > 0, axis=0)
        if used.all() and np.linalg.matrix_rank(dnu) == min(rank_target, nr):
            break
    else:  # pragma: no cover
        raise RuntimeError("no connected reaction set found")
    tb = np.array([t for _, _, t in rx], dtype=np.uint8)
    # orient every reaction in its exothermic direction at the reference temperature
    dH = (nu_r.astype(float) - nu_f) @ h_form
    swap = dH > 0
    nu_f[swap], nu_r[swap] = nu_r[swap].copy(), nu_f[swap].copy()
    perm = rng.permutation(nr)          # mix third-body reactions into the list
    nu_f, nu_r, tb = nu_f[perm], nu_r[perm], tb[perm]

    molecularity = nu_f.sum(axis=1).astype(float) + tb
    A_cgs = 10.0 ** rng.uniform(6.0, 16.0, size=nr)
    A = A_cgs * (1e-6) ** (molecularity - 1.0)
    b = rng.uniform(-1.5, 2.0, size=nr)
    Ea = rng.uniform(0.0, 2e5, size=nr)
    eff = np.ones((nr, ns))
    for r in np.nonzero(tb)[0]:
        pick = rng.choice(ns, size=min(5, ns), replace=False)
        eff[r, pick] = np.exp(rng.uniform(np.log(0.5), np.log(12.0), size=len(pick)))
    return dict(ns=ns, nr=nr, ne=ne, names=names, elements=elements, elem=elem, W=W,
                thermo=thermo, nu_f=nu_f, nu_r=nu_r, A=A, b=b, Ea=Ea, A_cgs=A_cgs,
                reversible=np.ones(nr, dtype=np.uint8), third_body=tb, eff=eff,
                fuel=names.index(fuel), oxidizer=names.index(oxidizer), inert=inert,
                product=names.index(product), seed=seed)


def h2_air_mechanism(seed=0, nr=21, n_third_body=4):
    """H2-air-shaped mechanism: 9 species (8 reactive + inert N2), 21 reversible reactions.

    Four of the reactions are third-body reactions (the recipe does not fix the count; H2-air
    mechanisms carry a handful of dissociation/recombination reactions)."""
    return _build(H2_AIR_SPECIES, nr, n_third_body, seed, "H2", "O2", "H2O")


def hydrocarbon_mechanism(seed=0, ns=53, nr=325, n_third_body=30):
    """Hydrocarbon-air-shaped mechanism: 53 C/H/O/N species incl. inert N2, 325 reversible
    reactions of which 30 are third-body reactions."""
    species = _hydrocarbon_species(ns)
    names = [s[0] for s in species]
    fuel = "C2H4" if "C2H4" in names else "H2"
    return _build(species, nr, n_third_body, seed, fuel, "O2", "H2O")


def toy_mechanism(kind, A=1.0e6, b=0.0, Ea=0.0, cp_R=2.5, eff_inert=1.0):
    """Hand-built mechanisms with closed-form solutions (used to pin the oracle).

    kind = "AB"      A <=> B, identical thermo and W (K_c = 1, T constant)
           "A->B"    irreversible A -> B, identical thermo and W
           "2A->B"   irreversible 2 A -> B, W_B = 2 W_A, per-mass energies equal (T constant)
           "A+M->B"  irreversible A + M -> B + M with an inert collider I of efficiency eff_inert
    """
    W0 = 0.02
    def th(cp, h0, s0):
        a = np.zeros(9)
        a[0] = cp
        a[5] = h0
        a[6] = s0
        a[7], a[8] = T_LO, T_HI
        return a
    if kind in ("AB", "A->B"):
        names, elem, W = ["A", "B"], np.array([[1], [1]], np.int32), np.array([W0, W0])
        thermo = np.stack([th(cp_R, -1000.0, 20.0), th(cp_R, -1000.0, 20.0)])
        nu_f = np.array([[1, 0]], np.int8)
        nu_r = np.array([[0, 1]], np.int8)
        tb = np.array([0], np.uint8)
        rev = np.array([1 if kind == "AB" else 0], np.uint8)
        eff = np.ones((1, 2))
    elif kind == "2A->B":
        names, elem, W = ["A", "B"], np.array([[1], [2]], np.int32), np.array([W0, 2 * W0])
        thermo = np.stack([th(cp_R, -1000.0, 20.0), th(2 * cp_R - 1.0, -2000.0, 30.0)])
        nu_f = np.array([[2, 0]], np.int8)
        nu_r = np.array([[0, 1]], np.int8)
        tb = np.array([0], np.uint8)
        rev = np.array([0], np.uint8)
        eff = np.ones((1, 2))
    elif kind == "A+M->B":
        names = ["A", "B", "I"]
        elem, W = np.array([[1, 0], [1, 0], [0, 1]], np.int32), np.array([W0, W0, W0])
        thermo = np.stack([th(cp_R, -1000.0, 20.0)] * 3)
        nu_f = np.array([[1, 0, 0]], np.int8)
        nu_r = np.array([[0, 1, 0]], np.int8)
        tb = np.array([1], np.uint8)
        rev = np.array([0], np.uint8)
        eff = np.array([[1.0, 1.0, eff_inert]])
    else:
        raise ValueError(kind)
    ns = len(names)
    return dict(ns=ns, nr=1, ne=elem.shape[1], names=names, elements=["X", "Y"][:elem.shape[1]],
                elem=elem, W=W, thermo=thermo, nu_f=nu_f, nu_r=nu_r,
                A=np.array([A]), b=np.array([b]), Ea=np.array([Ea]), A_cgs=np.array([A]),
                reversible=rev, third_body=tb, eff=eff,
                fuel=0, oxidizer=0, inert=ns - 1, product=1, seed=-1)
