"""Seeded synthetic reaction networks shaped like the paper's workloads.

The paper integrates a 150-isotope / 1604-reaction thermonuclear network and
shows runs up to 365 isotopes (Sec. 6, Fig. 1); the real rate library is not
available, so these generators build stand-ins of the same size and the same
structure: every reaction conserves the mass number sum_i A_i Y_i, reactions
are 1-, 2- or 3-body with a rho^(r-1) density weighting, and the light species
(A = 1..4, the protons/neutrons/alphas of Sec. 11 item 5) are hubs with
hundreds of producing and consuming reactions while most species have few.

Rates are drawn as ln k0_j (log-uniform k0) and a temperature exponent n_j,
so that k_j(T9, rho) = k0_j * T9**n_j * rho**(r_j - 1).  This module only
draws inputs; it evaluates no rate, flux or update.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .rng import SplitMix64

MAX_REAC = 3
MAX_PROD = 3


@dataclass
class Network:
    """Reaction network description (the arrays a caller hands to the library).

    A       [N]     mass number of each species (float64)
    reac    [R, 3]  reactant species ids, -1 padded; a repeated id is a repeated
                    reactant (i + i -> k), each occurrence is one reactant slot
    prod    [R, 3]  product species ids, -1 padded (repeats allowed likewise)
    ln_k0   [R]     natural log of the rate prefactor k0_j
    t9_exp  [R]     temperature exponent n_j
    """
    name: str
    A: np.ndarray
    reac: np.ndarray
    prod: np.ndarray
    ln_k0: np.ndarray
    t9_exp: np.ndarray
    init_X: dict = field(default_factory=dict)  # mass-number -> mass fraction

    @property
    def n_species(self) -> int:
        return int(self.A.shape[0])

    @property
    def n_reactions(self) -> int:
        return int(self.ln_k0.shape[0])

    @property
    def n_reac(self) -> np.ndarray:
        return (self.reac >= 0).sum(axis=1).astype(np.int8)

    @property
    def n_prod(self) -> np.ndarray:
        return (self.prod >= 0).sum(axis=1).astype(np.int8)

    def initial_Y(self) -> np.ndarray:
        """Molar abundances Y_i = X_i / A_i for the network's initial composition.

        init_X maps a mass number to a mass fraction that is split evenly over
        all species with that mass number, so sum_i A_i Y_i = sum X = 1.
        """
        Y = np.zeros(self.n_species)
        for a, x in self.init_X.items():
            ids = np.nonzero(self.A == a)[0]
            Y[ids] = x / len(ids) / a
        return Y

    def slot_counts(self):
        """(reactant slots S_r, product slots S_p)."""
        return int((self.reac >= 0).sum()), int((self.prod >= 0).sum())

    def fan_in(self) -> np.ndarray:
        """Per species: number of reactant slots + product slots naming it."""
        c = np.zeros(self.n_species, dtype=np.int64)
        for arr in (self.reac, self.prod):
            ids = arr[arr >= 0]
            np.add.at(c, ids, 1)
        return c

    def summary(self) -> dict:
        nr = self.n_reac
        s_r, s_p = self.slot_counts()
        fi = self.fan_in()
        return {
            "name": self.name,
            "n_species": self.n_species,
            "n_reactions": self.n_reactions,
            "frac_1body": float((nr == 1).mean()),
            "frac_2body": float((nr == 2).mean()),
            "frac_3body": float((nr == 3).mean()),
            "reactant_slots": s_r,
            "product_slots": s_p,
            "max_fan_in": int(fi.max()),
            "median_fan_in": float(np.median(fi)),
        }


def _pack(rows, width):
    out = np.full((len(rows), width), -1, dtype=np.int32)
    for i, r in enumerate(rows):
        out[i, : len(r)] = r
    return out


def _make(name, A, reactions, rng, lnk_lo, lnk_hi, init_X):
    """reactions: list of (reactant tuple, product tuple); draws ln k0, n_j per reaction."""
    ln_k0 = np.empty(len(reactions))
    t9_exp = np.empty(len(reactions))
    for j in range(len(reactions)):
        ln_k0[j] = lnk_lo + rng.uniform() * (lnk_hi - lnk_lo)
        t9_exp[j] = 8.0 * rng.uniform()
    return Network(
        name=name,
        A=np.asarray(A, dtype=np.float64),
        reac=_pack([r for r, _ in reactions], MAX_REAC),
        prod=_pack([p for _, p in reactions], MAX_PROD),
        ln_k0=ln_k0,
        t9_exp=t9_exp,
        init_X=init_X,
    )


def chain_network(seed: int = 0) -> Network:
    """16-species / 48-reaction chain network (A_i = i).

    15 captures (A=a) + (A=1) -> (A=a+1), 15 breakups (A=a+1) -> (A=a) + (A=1)
    (the A-conserving reading of "i -> i+1"), and 18 distinct random 2-body
    captures i + j -> i+j with 2 <= i <= j, i + j <= 16.  k0 log-uniform in
    [1e-6, 1e8], n uniform in [0, 8].  Initial state: all mass in A = 1.
    """
    rng = SplitMix64(seed)
    n = 16
    A = list(range(1, n + 1))
    sp = {a: a - 1 for a in A}  # mass number -> species id
    reactions = []
    for a in range(1, n):
        reactions.append(((sp[1], sp[a]), (sp[a + 1],)))
    for a in range(1, n):
        reactions.append(((sp[a + 1],), (sp[a], sp[1])))
    pairs = [(i, j) for i in range(2, n + 1) for j in range(i, n + 1) if i + j <= n]
    rng.shuffle(pairs)
    for i, j in pairs[:18]:
        reactions.append(((sp[i], sp[j]), (sp[i + j],)))
    return _make("chain16_48", A, reactions, rng, math.log(1e-6), math.log(1e8), {1: 1.0})


def general_network(n_species: int, n_reactions: int, a_max: int, n_pairs: int,
                    seed: int = 0, name: str | None = None) -> Network:
    """Random A-conserving network with hub light species.

    Species 0..3 are light (A = 1..4); the other N-4 are spread round-robin over
    A = 5..a_max.  n_reactions - n_pairs base reactions are drawn 30/60/10 % as
    1-, 2-, 3-body:
      1-body: isobaric i -> i' (same A) half the time, else breakup i -> light + rest;
      2-body: first reactant light with probability 0.8, product an isobar of A_i + A_j;
      3-body: two light reactants plus any species, product an isobar of the sum.
    Then n_pairs distinct base reactions get their reverse appended (independent
    k0, n), so n_reactions counts the reverses.  k0 log-uniform in [1e-8, 1e10],
    n uniform in [0, 8].  Initial composition: X = 0.5 over A = 12, 0.5 over A = 16.
    """
    rng = SplitMix64(seed)
    light = [0, 1, 2, 3]
    A = [1, 2, 3, 4] + [5 + ((s - 4) % (a_max - 4)) for s in range(4, n_species)]
    by_A: dict[int, list[int]] = {}
    for s, a in enumerate(A):
        by_A.setdefault(a, []).append(s)
    heavy = list(range(4, n_species))
    n_base = n_reactions - n_pairs
    n1 = int(round(0.3 * n_base))
    n3 = int(round(0.1 * n_base))
    n2 = n_base - n1 - n3
    kinds = [1] * n1 + [2] * n2 + [3] * n3
    rng.shuffle(kinds)
    seen = set()
    reactions = []

    def key(r, p):
        return (tuple(sorted(r)), tuple(sorted(p)))

    for kind in kinds:
        while True:
            if kind == 1:
                if rng.uniform() < 0.5:
                    i = rng.choice(heavy)
                    others = [s for s in by_A[A[i]] if s != i]
                    r, p = (i,), (rng.choice(others),)
                else:
                    i = rng.randint(1, n_species - 1)  # any species with A >= 2
                    ls = [l for l in light if A[l] < A[i]]
                    l = rng.choice(ls)
                    rest = rng.choice(by_A[A[i] - A[l]])
                    r, p = (i,), (l, rest)
            elif kind == 2:
                i = rng.choice(light) if rng.uniform() < 0.8 else rng.randint(0, n_species - 1)
                j = rng.randint(0, n_species - 1)
                if A[i] + A[j] > a_max:
                    continue
                r, p = (i, j), (rng.choice(by_A[A[i] + A[j]]),)
            else:
                l1, l2 = rng.choice(light), rng.choice(light)
                x = rng.randint(0, n_species - 1)
                if A[l1] + A[l2] + A[x] > a_max:
                    continue
                r, p = (l1, l2, x), (rng.choice(by_A[A[l1] + A[l2] + A[x]]),)
            k = key(r, p)
            if k in seen:
                continue
            seen.add(k)
            reactions.append((r, p))
            break
    idx = list(range(n_base))
    rng.shuffle(idx)
    base_count = len(reactions)
    # draw the base reactions' rates first so the reverses' draws follow them
    net_base = _make("tmp", A, reactions, rng, math.log(1e-8), math.log(1e10), {})
    rev = [(reactions[b][1], reactions[b][0]) for b in idx[:n_pairs]]
    net_rev = _make("tmp", A, rev, rng, math.log(1e-8), math.log(1e10), {})
    assert base_count == n_base
    name = name or f"net{n_species}_{n_reactions}"
    return Network(
        name=name,
        A=net_base.A,
        reac=np.concatenate([net_base.reac, net_rev.reac]),
        prod=np.concatenate([net_base.prod, net_rev.prod]),
        ln_k0=np.concatenate([net_base.ln_k0, net_rev.ln_k0]),
        t9_exp=np.concatenate([net_base.t9_exp, net_rev.t9_exp]),
        init_X={12: 0.5, 16: 0.5},
    )


def net150(seed: int = 0) -> Network:
    """150 species / 1604 reactions (400 of them reverses), A_max = 56."""
    return general_network(150, 1604, 56, 400, seed, "net150_1604")


def net365(seed: int = 0) -> Network:
    """365 species / 4400 reactions, A_max = 100, reverse pairs scaled as round(400*4400/1604)."""
    return general_network(365, 4400, 100, int(round(400 * 4400 / 1604)), seed, "net365_4400")


SWEEP_SIZES = (16, 32, 64, 100, 150, 250, 365)


def sweep_network(n_species: int, seed: int = 0) -> Network:
    """The network of the size sweep with n_species species.

    16 is the 16/48 chain; 150 and 365 are net150 and net365.  Other sizes use
    general_network with the reaction count interpolated from those two
    (10.69 reactions per species at 150, 12.05 at 365, linear in N, and 10.69 per
    species below 150), reverse pairs in the same 400/1604 proportion, and
    A_max = 56 at 150 and 100 at 365, interpolated, capped at (N - 4)/2 + 4 so
    every mass number holds at least two species.
    """
    if n_species == 16:
        return chain_network(seed)
    if n_species == 150:
        return net150(seed)
    if n_species == 365:
        return net365(seed)
    if n_species < 24:
        raise ValueError("sweep networks other than the chain need at least 24 species")
    per = 1604 / 150 if n_species <= 150 else 1604 / 150 + (n_species - 150) * (4400 / 365 - 1604 / 150) / 215
    n_reac = int(round(n_species * per))
    a_max = int(round(56 + (n_species - 150) * 44 / 215)) if n_species > 150 else 56
    a_max = min(a_max, (n_species - 4) // 2 + 4)
    return general_network(n_species, n_reac, a_max, int(round(400 * n_reac / 1604)), seed,
                           f"net{n_species}_{n_reac}")


def custom_network(A, reactions, ln_k0, t9_exp, init_X=None, name="custom") -> Network:
    """Hand-built network from explicit reactions [(reactants, products), ...]."""
    return Network(
        name=name,
        A=np.asarray(A, dtype=np.float64),
        reac=_pack([tuple(r) for r, _ in reactions], MAX_REAC),
        prod=_pack([tuple(p) for _, p in reactions], MAX_PROD),
        ln_k0=np.asarray(ln_k0, dtype=np.float64),
        t9_exp=np.asarray(t9_exp, dtype=np.float64),
        init_X=init_X or {},
    )


def pair_network(kf: float, kr: float, A: float = 1.0) -> Network:
    """Two species of equal mass number with A <-> B (rates independent of T, rho)."""
    return custom_network([A, A], [((0,), (1,)), ((1,), (0,))],
                          [math.log(kf), math.log(kr)], [0.0, 0.0], name="pairAB")


def random_tiny_network(n_species: int, n_reactions: int, seed: int,
                        lnk_lo: float = math.log(1e-2), lnk_hi: float = math.log(1e4)) -> Network:
    """Small A-conserving random network (species A = 1..n) for brute-force checks.

    Reaction 0 is 1 + 1 -> 2; the rest are 1-body breakups a -> b + (a-b) and
    2-body captures a + b -> a+b drawn without duplicates; rate exponents
    n_j = 0 so k_j = k0_j rho^(r-1).  Initial state: all mass in A = 1.
    """
    rng = SplitMix64(seed)
    A = list(range(1, n_species + 1))
    cand = []
    for a in range(1, n_species + 1):
        for b in range(a, n_species + 1):
            if a + b <= n_species:
                cand.append(((a - 1, b - 1), (a + b - 1,)))
                cand.append(((a + b - 1,), (a - 1, b - 1)))
    rng.shuffle(cand)
    first = ((0, 0), (1,))  # 1 + 1 -> 2 always present so the initial A = 1 mass reacts
    reactions = [first] + [c for c in cand if c != first][: n_reactions - 1]
    ln_k0 = [lnk_lo + rng.uniform() * (lnk_hi - lnk_lo) for _ in reactions]
    return custom_network(A, reactions, ln_k0, [0.0] * len(reactions),
                          init_X={1: 1.0}, name=f"tiny{n_species}_{len(reactions)}_{seed}")


def binding_energies(net: Network, seed: int = 17) -> np.ndarray:
    """Synthetic per-species binding energies (MeV): A times a binding-per-nucleon
    curve peaking at A = 56 (8.8 MeV), with a seeded 1 % scatter.  Input data
    only (the rate library carries no energies)."""
    rng = SplitMix64(seed)
    A = net.A
    b = 8.8 - 2.0 * ((A - 56.0) / 56.0) ** 2 - 6.0 / np.sqrt(A)
    scatter = np.array([1.0 + 0.01 * (2.0 * rng.uniform() - 1.0) for _ in range(len(A))])
    return A * np.maximum(b, 0.5) * scatter
