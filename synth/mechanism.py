"""Seeded synthetic reaction mechanisms over the elements C/H/O/N.

The paper's workloads use GRI-3.0 (53 species, 325 reactions), a 30-species
DME mechanism and Burke's H2 mechanism (Sec. 4.4 and the 1-D/3-D DME cases);
none of them is available here, so mechanisms of matching size are drawn from a
seed.  The construction makes every reaction element-balanced by enumeration and
bounds thermodynamics and stiffness by construction:

* Species are distinct formulas C_c H_h O_o N_n with small counts.  W_k is the
  sum of element masses, so mass balance follows from element balance.
* NASA-7 coefficients are an element-additive reference (the same coefficient
  vector in both temperature ranges) plus a per-species perturbation: a
  constant heat-capacity offset ``dc``, enthalpy and entropy offsets ``dh``,
  ``ds`` and, above T_mid only, a heat-capacity slope ``e`` whose integration
  constants are chosen so that cp, h and s are continuous at T_mid.  For an
  element-balanced reaction the element-additive part cancels from
  Delta G, so reaction free energies are set by the perturbations alone.
* Arrhenius parameters are drawn from the stated ranges (A log-uniform, b and
  Ea uniform) and redrawn while the pseudo-first-order forward or reverse rate
  at the ideal-gas concentration over the temperature window exceeds
  ``k_cap``.  This keeps the substep counts of a 1e-6..1e-7 s split step in a
  practical range; the paper's real mechanisms are stiff in the same sense.

The generator draws and assembles parameters.  It evaluates nothing the method
computes at a cell state (no rates of a state, no right-hand side, no step).
"""

from __future__ import annotations

import dataclasses
import itertools

import numpy as np

ELEMENTS = ("C", "H", "O", "N")
# kg/mol
ELEMENT_MASS = np.array([12.011e-3, 1.008e-3, 15.999e-3, 14.007e-3])

_R = 8.314462618
_P_REF = 101325.0

# Element-additive reference thermo (per atom): cp/R polynomial a1..a5 and the
# integration constants a6 (K) and a7.  Chosen so |g/RT| per atom stays small
# over 200..3500 K; it cancels from every reaction's Delta G.
_ELEMENT_REF = {
    "C": (2.10, 4.0e-4, -1.0e-7, 1.2e-11, -5.0e-16, -600.0, -13.5),
    "H": (1.60, 2.0e-4, 3.0e-8, -8.0e-12, 4.0e-16, -300.0, -11.0),
    "O": (1.90, 3.0e-4, -5.0e-8, 6.0e-12, -2.0e-16, -450.0, -12.5),
    "N": (1.80, 2.5e-4, -4.0e-8, 5.0e-12, -1.5e-16, -400.0, -12.0),
}


@dataclasses.dataclass
class Mechanism:
    """Plain array description of a gas-phase mechanism (SI except A: cm-mol-s).

    species arrays (Ns rows):
      names  list[str]
      elem   int32  [Ns, 4]   atom counts of C, H, O, N
      W      f64    [Ns]      molar mass, kg/mol
      nasa   f64    [Ns, 17]  T_lo, T_mid, T_hi, low a1..a7, high a1..a7
    reaction arrays (Nr rows):
      rxn_sp int32  [Nr, 4]   reactant species in slots 0,1 and product species
                              in slots 2,3; -1 marks an empty slot
      rxn_nu int32  [Nr, 4]   signed stoichiometric coefficients of those slots
                              (reactants < 0, products > 0, empty 0)
      arrh   f64    [Nr, 3]   A (cm, mol, s units), b, Ea (J/mol); for a Troe
                              reaction this is the high-pressure limit
      reversible u8 [Nr]
      kind   int32  [Nr]      0 elementary, 1 third body (+M), 2 Troe falloff (+M)
      eff    f64    [Nr, Ns]  third-body efficiencies (1 where unused)
      falloff f64   [Nr, 7]   A0 (cm, mol, s), b0, Ea0 (J/mol), a, T***, T*, T**
                              (T** <= 0 omits that term); zeros when unused
    """

    names: list
    elem: np.ndarray
    W: np.ndarray
    nasa: np.ndarray
    rxn_sp: np.ndarray
    rxn_nu: np.ndarray
    arrh: np.ndarray
    reversible: np.ndarray
    kind: np.ndarray
    eff: np.ndarray
    falloff: np.ndarray

    @property
    def n_species(self) -> int:
        return int(self.W.shape[0])

    @property
    def n_reactions(self) -> int:
        return int(self.arrh.shape[0])

    @property
    def n_state(self) -> int:
        return self.n_species + 1

    def copy(self) -> "Mechanism":
        return Mechanism(**{f.name: (list(getattr(self, f.name)) if f.name == "names"
                                     else np.array(getattr(self, f.name), copy=True))
                            for f in dataclasses.fields(self)})


def _formula_name(c: int, h: int, o: int, n: int) -> str:
    out = ""
    for sym, cnt in zip(ELEMENTS, (c, h, o, n)):
        if cnt == 1:
            out += sym
        elif cnt > 1:
            out += f"{sym}{cnt}"
    return out


def _pick_species(rng, n_species):
    """Species are sums of one to three "building blocks" (small formulas that
    together cover C, H, O and N), so that association, dissociation and
    exchange reactions between them are element-balanced by construction."""
    small = [f for f in itertools.product(range(2), range(3), range(2), range(2))
             if 1 <= sum(f) <= 2]
    n_blocks = 2 if n_species <= 12 else (6 if n_species <= 40 else 8)
    for _ in range(1000):
        idx = rng.choice(len(small), size=n_blocks, replace=False)
        blocks = np.array([small[i] for i in idx], dtype=np.int32)
        if not np.all(blocks.sum(axis=0) > 0):
            continue
        pool = {}
        for size in (1, 2, 3, 4):
            for ms in itertools.combinations_with_replacement(range(n_blocks), size):
                f = tuple(int(x) for x in blocks[list(ms)].sum(axis=0))
                if sum(f) <= 9 and f not in pool:
                    pool[f] = size
        if len(pool) < n_species:
            continue
        forms = list(pool.keys())
        w = np.array([{1: 6.0, 2: 3.0, 3: 1.0, 4: 0.5}[pool[f]] for f in forms])
        sel = rng.choice(len(forms), size=n_species, replace=False, p=w / w.sum())
        comp = np.array([forms[i] for i in sel], dtype=np.int32)
        if not np.all(comp.sum(axis=0) > 0):
            continue
        order = np.lexsort((comp[:, 3], comp[:, 2], comp[:, 1], comp[:, 0]))
        return comp[order]
    raise RuntimeError("could not draw a species set")


def _candidate_reactions(elem, rng, max_candidates=200000):
    """All element-balanced (<=2) <-> (<=2) reactions with no spectator species."""
    ns = elem.shape[0]
    groups: dict = {}
    multisets = [(i,) for i in range(ns)] + [(i, j) for i in range(ns) for j in range(i, ns)]
    for ms in multisets:
        key = tuple(int(x) for x in elem[list(ms)].sum(axis=0))
        groups.setdefault(key, []).append(ms)
    cands = []
    for key, members in groups.items():
        if len(members) < 2:
            continue
        for a, b in itertools.combinations(members, 2):
            if set(a) & set(b):
                continue
            cands.append((a, b))
    if len(cands) > max_candidates:
        sel = rng.choice(len(cands), size=max_candidates, replace=False)
        cands = [cands[i] for i in sel]
    return cands


def _slots(reac, prod):
    """Pack multisets into the 4-slot (species, signed nu) form."""
    sp = [-1, -1, -1, -1]
    nu = [0, 0, 0, 0]
    for side, ms, sign in ((0, reac, -1), (2, prod, 1)):
        uniq = sorted(set(ms))
        for k, s in enumerate(uniq):
            sp[side + k] = s
            nu[side + k] = sign * ms.count(s)
    return sp, nu


def generate_mechanism(
    n_species: int,
    n_reactions: int,
    *,
    seed: int,
    n_third_body: int = 0,
    n_troe: int = 0,
    k_cap: float = 1.0e8,
    T_window: tuple = (300.0, 3000.0),
    p_window: float = 101325.0,
    dg_max: float = 20.0,
    frac_irreversible: float = 0.0,
) -> Mechanism:
    """Draw a mechanism.  See the module docstring for the construction."""
    rng = np.random.default_rng(seed)
    best = None
    for _ in range(60):  # keep the draw with the richest reaction network
        e_try = _pick_species(rng, n_species)
        c_try = _candidate_reactions(e_try, rng)
        if best is None or len(c_try) > len(best[1]):
            best = (e_try, c_try)
        if len(c_try) >= 3 * n_reactions:
            break
    elem, cands = best
    W = elem @ ELEMENT_MASS
    names = [_formula_name(*row) for row in elem]

    # ---- thermo: element-additive reference + perturbations ---------------
    ref = np.array([_ELEMENT_REF[e] for e in ELEMENTS])  # [4, 7]
    base = elem @ ref  # [Ns, 7]
    t_mid = rng.uniform(900.0, 1100.0, n_species)
    dc = rng.uniform(0.0, 1.5, n_species)
    dh = rng.uniform(-15000.0, 15000.0, n_species)  # K
    ds = rng.uniform(-2.0, 2.0, n_species)
    slope = rng.uniform(-3.0e-4, 3.0e-4, n_species)
    low = base.copy()
    low[:, 0] += dc
    low[:, 5] += dh
    low[:, 6] += ds
    high = base.copy()
    high[:, 0] += dc - slope * t_mid
    high[:, 1] += slope
    high[:, 5] += dh + slope * t_mid**2 / 2.0
    high[:, 6] += ds + slope * t_mid * np.log(t_mid) - slope * t_mid
    nasa = np.zeros((n_species, 17))
    nasa[:, 0] = 200.0
    nasa[:, 1] = t_mid
    nasa[:, 2] = 3500.0
    nasa[:, 3:10] = low
    nasa[:, 10:17] = high

    # Free-energy offset of each species relative to the element reference,
    # as a function of T (the perturbation terms above), used only to shape
    # the reaction set and the reverse-rate bound.
    def dg_rt(T):
        T = np.asarray(T, dtype=float)[..., None]
        lo = dc + dh / T - dc * np.log(T) - ds
        a1 = dc - slope * t_mid
        a6 = dh + slope * t_mid**2 / 2.0
        a7 = ds + slope * t_mid * np.log(t_mid) - slope * t_mid
        hi = a1 + slope * T / 2.0 + a6 / T - (a1 * np.log(T) + slope * T + a7)
        return np.where(T < t_mid, lo, hi)

    # ---- reactions ----------------------------------------------------------
    rng.shuffle(cands)
    t_grid = np.linspace(T_window[0], T_window[1], 24)
    g_grid = dg_rt(t_grid)  # [nT, Ns]
    c_tot = p_window / (_R * t_grid)

    def net_dg(reac, prod):
        return sum(g_grid[:, s] for s in prod) - sum(g_grid[:, s] for s in reac)

    n_special = n_third_body + n_troe
    special_ok = [i for i, (a, b) in enumerate(cands) if len(a) + len(b) == 3]
    chosen = []
    kinds = []
    used = set()

    def try_add(idx, kind):
        a, b = cands[idx]
        # orientation: recombination direction (2 -> 1) for pressure-dependent
        if kind > 0:
            reac, prod = (a, b) if len(a) == 2 else (b, a)
        else:
            reac, prod = (a, b) if rng.random() < 0.5 else (b, a)
        dgg = net_dg(reac, prod)
        if np.max(np.abs(dgg[np.abs(t_grid - 1200.0).argmin()])) > dg_max:
            return False
        sp, nu = _slots(list(reac), list(prod))
        key = (tuple(sorted(reac)), tuple(sorted(prod)))
        if key in used or (key[1], key[0]) in used:
            return False
        n_r = len(reac)
        n_p = len(prod)
        dnu = n_p - n_r
        rev = rng.random() >= frac_irreversible
        for _attempt in range(400):
            A = 10.0 ** rng.uniform(6.0, 14.0)
            b_ = rng.uniform(-1.0, 2.0)
            Ea = rng.uniform(0.0, 200.0e3)
            order = n_r + (1 if kind == 1 else 0)
            kf = A * 1e-6 ** (order - 1) * t_grid**b_ * np.exp(-Ea / (_R * t_grid))
            eff_f = kf * c_tot ** (order - 1)
            kc = np.exp(-dgg) * (_P_REF / (_R * t_grid)) ** dnu
            eff_r = (kf / kc) * c_tot ** (n_p + (1 if kind == 1 else 0) - 1) if rev else 0.0 * kf
            fo = np.zeros(7)
            if kind == 2:
                A0 = 10.0 ** rng.uniform(10.0, 18.0)
                b0 = rng.uniform(-2.0, 0.5)
                Ea0 = rng.uniform(0.0, 100.0e3)
                k0 = A0 * 1e-6**n_r * t_grid**b0 * np.exp(-Ea0 / (_R * t_grid))
                e0 = k0 * c_tot**n_r  # k0 [M] C^(n_r-1)
                kinf_eff = eff_f
                eff_f = np.minimum(kinf_eff, e0)
                eff_r = (eff_f / kc) * c_tot ** (n_p - 1) / c_tot ** (n_r - 1) if rev else 0.0 * kf
                fo[:] = (A0, b0, Ea0, rng.uniform(0.1, 0.9), rng.uniform(50.0, 500.0),
                         rng.uniform(500.0, 5000.0), rng.uniform(3000.0, 9000.0))
                if np.max(kinf_eff) > 1e3 * k_cap or np.max(e0) > 1e3 * k_cap:
                    continue
            if np.max(eff_f) <= k_cap and np.max(eff_r) <= k_cap:
                used.add(key)
                chosen.append((sp, nu, (A, b_, Ea), rev, fo))
                kinds.append(kind)
                return True
        return False

    order_special = list(special_ok)
    for idx in order_special:
        if sum(1 for k in kinds if k == 1) < n_third_body:
            try_add(idx, 1)
        elif sum(1 for k in kinds if k == 2) < n_troe:
            try_add(idx, 2)
        else:
            break
    if len(chosen) < n_special:
        raise RuntimeError("not enough recombination candidates for third-body/Troe reactions")
    for idx in range(len(cands)):
        if len(chosen) >= n_reactions:
            break
        try_add(idx, 0)
    if len(chosen) < n_reactions:
        raise RuntimeError(
            f"only {len(chosen)} admissible reactions for {n_species} species (wanted {n_reactions})")

    nr = n_reactions
    # put the pressure-dependent reactions at seeded positions
    perm = rng.permutation(nr)
    rxn_sp = np.full((nr, 4), -1, dtype=np.int32)
    rxn_nu = np.zeros((nr, 4), dtype=np.int32)
    arrh = np.zeros((nr, 3))
    reversible = np.zeros(nr, dtype=np.uint8)
    kind = np.zeros(nr, dtype=np.int32)
    eff = np.ones((nr, n_species))
    falloff = np.zeros((nr, 7))
    for src_i, dst in enumerate(perm):
        sp, nu, ar, rev, fo = chosen[src_i]
        rxn_sp[dst] = sp
        rxn_nu[dst] = nu
        arrh[dst] = ar
        reversible[dst] = 1 if rev else 0
        kind[dst] = kinds[src_i]
        falloff[dst] = fo
        if kinds[src_i] > 0:
            picks = rng.choice(n_species, size=min(3, n_species), replace=False)
            eff[dst, picks] = rng.uniform(0.3, 5.0, size=len(picks))
    return Mechanism(names=names, elem=elem.astype(np.int32), W=W, nasa=nasa, rxn_sp=rxn_sp,
                     rxn_nu=rxn_nu, arrh=arrh, reversible=reversible, kind=kind, eff=eff,
                     falloff=falloff)


def single_reaction_mechanism(reac, prod, formulas, A, b, Ea, *, reversible=True, nasa=None):
    """A hand-specified tiny mechanism (used by tests): ``formulas`` is a list of
    (c, h, o, n) tuples, ``reac``/``prod`` lists of species indices with repeats."""
    elem = np.array(formulas, dtype=np.int32)
    ns = elem.shape[0]
    W = elem @ ELEMENT_MASS
    if nasa is None:
        ref = np.array([_ELEMENT_REF[e] for e in ELEMENTS])
        base = elem @ ref
        nasa = np.zeros((ns, 17))
        nasa[:, 0], nasa[:, 1], nasa[:, 2] = 200.0, 1000.0, 3500.0
        nasa[:, 3:10] = base
        nasa[:, 10:17] = base
    sp, nu = _slots(list(reac), list(prod))
    return Mechanism(
        names=[_formula_name(*f) for f in formulas], elem=elem, W=W, nasa=np.asarray(nasa, float),
        rxn_sp=np.array([sp], dtype=np.int32), rxn_nu=np.array([nu], dtype=np.int32),
        arrh=np.array([[A, b, Ea]], float), reversible=np.array([1 if reversible else 0], np.uint8),
        kind=np.zeros(1, np.int32), eff=np.ones((1, ns)), falloff=np.zeros((1, 7)))


def mechanism_summary(m: Mechanism) -> str:
    kinds = np.bincount(m.kind, minlength=3)
    return (f"{m.n_species} species / {m.n_reactions} reactions "
            f"({kinds[1]} third-body, {kinds[2]} Troe, {int((m.reversible == 0).sum())} irreversible)")


def _self_check_balance(m: Mechanism) -> bool:
    """Integer element balance of every reaction (a property of the construction)."""
    for j in range(m.n_reactions):
        tot = np.zeros(4, dtype=np.int64)
        for s, n in zip(m.rxn_sp[j], m.rxn_nu[j]):
            if s >= 0:
                tot += int(n) * m.elem[s].astype(np.int64)
        if np.any(tot != 0):
            return False
    return True


__all__ = ["Mechanism", "generate_mechanism", "single_reaction_mechanism", "mechanism_summary",
           "ELEMENTS", "ELEMENT_MASS"]
