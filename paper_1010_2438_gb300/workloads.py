"""Seeded synthetic inputs for the batched CWC / Gillespie simulator.

This module is the single place where inputs are generated; both the CUDA path
and the CPU oracle receive what it builds.  It contains no simulation
arithmetic: no propensities, no random streams of the method, no time
advance.  Random choices here use SplitMix64 (Steele, Lea, Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014), written out in pure
Python so that every machine builds identical models from the same seed.

Model representation (the restricted CWC rule language of Sec. 2.1-2.2):

* ``S`` atoms (species) ``0..S-1``; ``L`` compartment labels, label 0 is the
  top level (the root compartment, which has no wrap); ``C`` compartment
  slots per trajectory, slot 0 is the root.
* Rule ``j`` has a ``kind``:
  ``LOCAL``        ``l: p X -> p' X`` rewrites the content of a compartment of
                   label ``l`` (the paper's example ``l: a b X -> c X``);
  ``PARENT_CHILD`` ``l: p X (w x | q Y)^l' -> p' X (w' x | q' Y)^l'`` rewrites
                   a parent content of label ``l`` together with the wrap and
                   content of one child compartment of label ``l'`` (binding
                   to a wrap, transport in and out);
  ``CREATE``       ``l: p X -> p' X (w' | q')^l'`` makes a new compartment;
  ``DISSOLVE``     ``l: p X (w x | q Y)^l' -> p' X x Y`` removes a child and
                   releases its remaining wrap and content into the parent;
  ``FUSION``       ``l: p X (w1 x1 | q1 Y1)^l' (w2 x2 | q2 Y2)^l' ->
                   p' X (w' x1 x2 | q' Y1 Y2)^l'`` merges two sibling
                   compartments (two compartments in one left-hand side);
  ``NESTED``       ``l: p X (w x | q Y (v z | u Z)^l'')^l' ->
                   p' X (w' x | q' Y (v' z | u' Z)^l'')^l'`` rewrites a
                   compartment two levels down together with its parent and
                   grandparent (a pattern of depth two);
  ``PAIR``         ``l: p X (w1 x1 | q1 Y1)^l' (w2 x2 | q2 Y2)^l' ->
                   p' X (w1' x1 | q1' Y1)^l' (w2' x2 | q2' Y2)^l'`` rewrites
                   two sibling compartments, both kept (e.g. transport from
                   one to the other).
* ``lhs[j, 0/1/2, :]`` are the multiplicities of the parent (context)
  content, child wrap and child content patterns; ``rhs`` the same for the
  right-hand side.  ``lhs_ext[j, 0/1, :]`` (and ``rhs_ext``) are rows 3 and 4:
  the second child's wrap and content (FUSION, PAIR) or the grandchild's wrap
  and content (NESTED); ``grand_label[j]`` is NESTED's grandchild label.

Flat mass-action networks are the special case ``L = 1``, ``C = 1`` and only
``LOCAL`` rules on label 0.
"""
from __future__ import annotations

import dataclasses
import json
import math
import os
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

LOCAL, PARENT_CHILD, CREATE, DISSOLVE, FUSION, NESTED, PAIR = 0, 1, 2, 3, 4, 5, 6
KIND_NAMES = {LOCAL: "LOCAL", PARENT_CHILD: "PARENT_CHILD", CREATE: "CREATE", DISSOLVE: "DISSOLVE",
              FUSION: "FUSION", NESTED: "NESTED", PAIR: "PAIR"}

_MASK64 = (1 << 64) - 1

# Horizons T of the synthetic workloads, chosen so that the mean number of
# events per trajectory is near each workload's target (file written by
# oracle/calibrate_horizons.py).
HORIZONS_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workload_horizons.json")


def calibrated_horizon(name: str) -> Optional[float]:
    try:
        with open(HORIZONS_PATH) as f:
            return float(json.load(f)[name])
    except (OSError, KeyError, ValueError):
        return None


class SplitMix64:
    """SplitMix64 generator (input generation only)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Double in [0, 1) with 53 random bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def randint(self, lo: int, hi: int) -> int:
        """Integer uniform on [lo, hi] (inclusive); modulo bias is irrelevant here."""
        return lo + self.next_u64() % (hi - lo + 1)

    def log_uniform(self, lo_exp: float, hi_exp: float) -> float:
        return 10.0 ** (lo_exp + (hi_exp - lo_exp) * self.uniform())

    def choice_distinct(self, n: int, k: int) -> List[int]:
        pool = list(range(n))
        out = []
        for _ in range(k):
            i = self.randint(0, len(pool) - 1)
            out.append(pool.pop(i))
        return out


@dataclasses.dataclass
class Model:
    n_species: int
    n_labels: int
    max_compartments: int
    kind: np.ndarray          # int32 [M]
    ctx_label: np.ndarray     # int32 [M]
    child_label: np.ndarray   # int32 [M]  (-1 for LOCAL)
    lhs: np.ndarray           # int32 [M, 3, S]
    rhs: np.ndarray           # int32 [M, 3, S]
    name: str = ""
    grand_label: Optional[np.ndarray] = None   # int32 [M] (-1 unless NESTED), or None
    lhs_ext: Optional[np.ndarray] = None       # int32 [M, 2, S] rows 3 and 4, or None
    rhs_ext: Optional[np.ndarray] = None       # int32 [M, 2, S]
    rate_law: Optional[np.ndarray] = None      # int32 [M]: 0 mass action, 1 + s Michaelis-Menten of substrate s
    rate_par: Optional[np.ndarray] = None      # float64 [M]: the Michaelis constant K (molecules)

    @property
    def has_ext(self) -> bool:
        return self.lhs_ext is not None

    def rows5(self) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
        """(lhs [M, 5, S], rhs [M, 5, S], grand_label [M]) with rows 3-4 zero
        and grand labels -1 when the model has no FUSION / NESTED rule."""
        M, S = self.n_rules, self.n_species
        z = np.zeros((M, 2, S), np.int32)
        le = z if self.lhs_ext is None else np.asarray(self.lhs_ext, np.int32)
        re = z if self.rhs_ext is None else np.asarray(self.rhs_ext, np.int32)
        gl = np.full(M, -1, np.int32) if self.grand_label is None else np.asarray(self.grand_label, np.int32)
        return (np.ascontiguousarray(np.concatenate([self.lhs, le], axis=1), np.int32),
                np.ascontiguousarray(np.concatenate([self.rhs, re], axis=1), np.int32),
                np.ascontiguousarray(gl, np.int32))

    @property
    def n_rules(self) -> int:
        return int(self.kind.shape[0])

    @property
    def is_flat(self) -> bool:
        return self.n_labels == 1 and self.max_compartments == 1

    @property
    def n_observables(self) -> int:
        S, L = self.n_species, self.n_labels
        if self.is_flat:
            return S
        return L * S + (L - 1) * S + L

    def contiguous(self) -> "Model":
        def c(a):
            return None if a is None else np.ascontiguousarray(a, dtype=np.int32)
        return dataclasses.replace(
            self,
            kind=c(self.kind), ctx_label=c(self.ctx_label), child_label=c(self.child_label),
            lhs=c(self.lhs), rhs=c(self.rhs), grand_label=c(self.grand_label),
            lhs_ext=c(self.lhs_ext), rhs_ext=c(self.rhs_ext), rate_law=c(self.rate_law),
            rate_par=None if self.rate_par is None else np.ascontiguousarray(self.rate_par, dtype=np.float64),
        )


Reaction = Tuple[Dict[int, int], Dict[int, int]]


def flat_model(n_species: int, reactions: Sequence[Reaction], name: str = "",
               michaelis_menten: Optional[Dict[int, Tuple[int, float]]] = None) -> Model:
    """Flat network: every reaction is a LOCAL rule of the root, with mass-
    action kinetics unless ``michaelis_menten[j] = (substrate, K)`` makes
    reaction j's rate k_j n_E n_S / (K + n_S) (the enzyme E the other
    reactant, if any; both reactants of multiplicity 1)."""
    M = len(reactions)
    lhs = np.zeros((M, 3, n_species), np.int32)
    rhs = np.zeros((M, 3, n_species), np.int32)
    for j, (reac, prod) in enumerate(reactions):
        for s, c in reac.items():
            lhs[j, 0, s] += c
        for s, c in prod.items():
            rhs[j, 0, s] += c
    law = par = None
    if michaelis_menten:
        law = np.zeros(M, np.int32)
        par = np.zeros(M, np.float64)
        for j, (sub, K) in michaelis_menten.items():
            law[j] = 1 + sub
            par[j] = K
    return Model(n_species, 1, 1, np.zeros(M, np.int32), np.zeros(M, np.int32),
                 np.full(M, -1, np.int32), lhs, rhs, name, rate_law=law, rate_par=par)


@dataclasses.dataclass
class RuleSpec:
    kind: int
    ctx_label: int
    child_label: int = -1
    lhs_ctx: Dict[int, int] = dataclasses.field(default_factory=dict)
    lhs_wrap: Dict[int, int] = dataclasses.field(default_factory=dict)
    lhs_child: Dict[int, int] = dataclasses.field(default_factory=dict)
    rhs_ctx: Dict[int, int] = dataclasses.field(default_factory=dict)
    rhs_wrap: Dict[int, int] = dataclasses.field(default_factory=dict)
    rhs_child: Dict[int, int] = dataclasses.field(default_factory=dict)
    # rows 3 and 4: the second child (FUSION, PAIR) or the grandchild (NESTED)
    lhs_wrap2: Dict[int, int] = dataclasses.field(default_factory=dict)
    lhs_child2: Dict[int, int] = dataclasses.field(default_factory=dict)
    rhs_wrap2: Dict[int, int] = dataclasses.field(default_factory=dict)
    rhs_child2: Dict[int, int] = dataclasses.field(default_factory=dict)
    grand_label: int = -1


def cwc_model(n_species: int, n_labels: int, max_compartments: int,
              rules: Sequence[RuleSpec], name: str = "") -> Model:
    M = len(rules)
    lhs = np.zeros((M, 3, n_species), np.int32)
    rhs = np.zeros((M, 3, n_species), np.int32)
    kind = np.zeros(M, np.int32)
    ctx = np.zeros(M, np.int32)
    child = np.full(M, -1, np.int32)
    ext = any(r.kind in (FUSION, NESTED, PAIR) or r.lhs_wrap2 or r.lhs_child2 or r.rhs_wrap2 or r.rhs_child2
              for r in rules)
    lhs_ext = np.zeros((M, 2, n_species), np.int32)
    rhs_ext = np.zeros((M, 2, n_species), np.int32)
    grand = np.full(M, -1, np.int32)
    for j, r in enumerate(rules):
        kind[j], ctx[j], child[j] = r.kind, r.ctx_label, r.child_label
        grand[j] = r.grand_label
        for k, d in enumerate((r.lhs_ctx, r.lhs_wrap, r.lhs_child)):
            for s, c in d.items():
                lhs[j, k, s] += c
        for k, d in enumerate((r.rhs_ctx, r.rhs_wrap, r.rhs_child)):
            for s, c in d.items():
                rhs[j, k, s] += c
        for k, d in enumerate((r.lhs_wrap2, r.lhs_child2)):
            for s, c in d.items():
                lhs_ext[j, k, s] += c
        for k, d in enumerate((r.rhs_wrap2, r.rhs_child2)):
            for s, c in d.items():
                rhs_ext[j, k, s] += c
    if not ext:
        return Model(n_species, n_labels, max_compartments, kind, ctx, child, lhs, rhs, name)
    return Model(n_species, n_labels, max_compartments, kind, ctx, child, lhs, rhs, name,
                 grand_label=grand, lhs_ext=lhs_ext, rhs_ext=rhs_ext)


# ----------------------------------------------------------------------------
# Initial terms.  A flat model takes counts [S]; a compartmentalised model takes
# a slot image [C, 3 + 2S]: (alive, label, parent, wrap[S], content[S]).
# ----------------------------------------------------------------------------

def slot_image_width(n_species: int) -> int:
    return 3 + 2 * n_species


def empty_slot_image(model: Model) -> np.ndarray:
    S, C = model.n_species, model.max_compartments
    img = np.zeros((C, slot_image_width(S)), np.int32)
    img[:, 2] = -1
    img[0, 0] = 1  # root alive, label 0, parent -1
    return img


# ----------------------------------------------------------------------------
# Batches
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Batch:
    """One call's inputs: P sweep points x R replicas on a time grid."""
    model: Model
    rates: np.ndarray     # float64 [P, M]
    init: np.ndarray      # int32 [Pi, S] (flat) or [Pi, C, 3+2S]; Pi in {1, P}
    grid: np.ndarray      # float64 [G], 0 <= g0 < g1 < ...
    R: int
    seed: int
    max_events: int = (1 << 32) - 1
    name: str = ""

    @property
    def P(self) -> int:
        return int(self.rates.shape[0])

    @property
    def G(self) -> int:
        return int(self.grid.shape[0])

    @property
    def n_traj(self) -> int:
        return self.P * self.R


def uniform_grid(T: float, G: int) -> np.ndarray:
    """g_i = i*T/(G-1), i = 0..G-1 (g_0 = 0 records the initial term)."""
    if G == 1:
        return np.array([T], np.float64)
    return np.array([T * i / (G - 1) for i in range(G)], np.float64)


def crude_rate(model: Model, rates: np.ndarray, counts: np.ndarray) -> float:
    """Rough total event rate of a flat model at ``counts``: sum_j k_j prod_x n_x^nu.

    Used only to pick a time horizon that gives roughly the wanted number of
    events; it deliberately ignores the exact combinatorial count.
    """
    total = 0.0
    for j in range(model.n_rules):
        term = float(rates[j])
        for s in range(model.n_species):
            nu = int(model.lhs[j, 0, s])
            if nu:
                term *= float(counts[s]) ** nu
        total += term
    return total


def random_flat_network(rng: SplitMix64, S: int, n_order1: int, n_order2: int,
                        n_inflow_pairs: int = 0, name: str = "") -> Model:
    """Random mass-action network without sink species.

    * ``n_inflow_pairs`` pairs (0 -> X_i, X_i -> 0) on distinct species;
    * ``n_order1`` unimolecular conversions ``A -> B``; the first ``S`` of them
      form one directed cycle through all species (a random permutation), so
      every species has an outgoing reaction and molecules never pile up in a
      sink; the rest are random (B != A);
    * ``n_order2`` bimolecular reactions ``A + B -> C + D`` (alternately A != B
      and ``2A``), products drawn independently (``2C`` is possible).
    Apart from the inflow/outflow pairs every reaction conserves the molecule
    count.  The reaction order is shuffled with the same seeded stream.
    """
    if n_order1 < S:
        raise ValueError("need at least S unimolecular reactions for the cycle")
    reactions: List[Reaction] = []
    inflow_species = rng.choice_distinct(S, n_inflow_pairs)
    for s in inflow_species:
        reactions.append(({}, {s: 1}))
        reactions.append(({s: 1}, {}))
    perm = rng.choice_distinct(S, S)
    body: List[Reaction] = []
    for i in range(S):
        body.append(({perm[i]: 1}, {perm[(i + 1) % S]: 1}))
    for _ in range(n_order1 - S):
        a = rng.randint(0, S - 1)
        b = (a + rng.randint(1, S - 1)) % S
        body.append(({a: 1}, {b: 1}))
    for i in range(n_order2):
        if i % 2 == 0:
            a, b = rng.choice_distinct(S, 2)
            reac = {a: 1, b: 1}
        else:
            a = rng.randint(0, S - 1)
            reac = {a: 2}
        c = rng.randint(0, S - 1)
        d = rng.randint(0, S - 1)
        prod: Dict[int, int] = {}
        prod[c] = prod.get(c, 0) + 1
        prod[d] = prod.get(d, 0) + 1
        body.append((reac, prod))
    for i in range(len(body) - 1, 0, -1):
        k = rng.randint(0, i)
        body[i], body[k] = body[k], body[i]
    reactions.extend(body)
    return flat_model(S, reactions, name)


def reaction_order(model: Model, j: int) -> int:
    return int(model.lhs[j, 0].sum())


def _flat_batch(model: Model, rng: SplitMix64, P: int, R: int, G: int, x_lo: int, x_hi: int,
                target_events: float, seed: int, rate_decades: Tuple[float, float] = (-3.0, 0.0),
                name: str = "", use_calibrated: bool = True) -> Batch:
    """Rates, initial counts and horizon for a flat network.

    Rate constants are log-uniform over ``rate_decades`` in concentration
    units and converted to stochastic constants for a system of size
    Omega = (x_lo + x_hi) / 2 molecules (order 0: k*Omega, order 1: k,
    order 2: k/Omega), the usual volume scaling of mass-action kinetics.  The
    horizon is the calibrated one for ``name`` when available (and the
    default target), else T = target_events / crude_rate(x0).
    """
    M, S = model.n_rules, model.n_species
    omega = 0.5 * (x_lo + x_hi)
    base = np.empty(M, np.float64)
    for j in range(M):
        k = rng.log_uniform(*rate_decades)
        base[j] = k * omega ** (1 - reaction_order(model, j))
    x0 = np.array([rng.randint(x_lo, x_hi) for _ in range(S)], np.int32)
    T = target_events / crude_rate(model, base, x0)
    if use_calibrated:
        Tc = calibrated_horizon(name)
        if Tc is not None:
            T = Tc
    rates = np.tile(base, (P, 1))
    return Batch(model, rates, x0[None, :].copy(), uniform_grid(T, G), R, seed, name=name)


# ----------------------------------------------------------------------------
# The five benchmark workloads (shapes of the paper's multi-instance runs,
# Sec. 5.2: replicas and parameter sweeps of mass-action / CWC models).
# ----------------------------------------------------------------------------

def flat8x12(R: int = 64, G: int = 100, use_calibrated: bool = True) -> Batch:
    """8 species, 12 reactions (8-cycle of conversions + 4 bimolecular), 64 replicas,
    ~1e4 events, 100-point grid."""
    rng = SplitMix64(1)
    model = random_flat_network(rng, 8, 8, 4, 0, "flat8x12")
    return _flat_batch(model, rng, 1, R, G, 50, 500, 1e4, seed=101, name="flat8x12",
                       use_calibrated=use_calibrated)


def flat32x64(R: int = 65536, G: int = 1000, use_calibrated: bool = True) -> Batch:
    """32 species, 64 reactions (8 inflow/outflow pairs, 32 order-1, 16 order-2)."""
    rng = SplitMix64(2)
    model = random_flat_network(rng, 32, 32, 16, 8, "flat32x64")
    return _flat_batch(model, rng, 1, R, G, 100, 5000, 1e5, seed=102, name="flat32x64",
                       use_calibrated=use_calibrated)


def sweep256x256(P: int = 256, R: int = 256, G: int = 1000) -> Batch:
    """flat32x64's network under P rate vectors, R replicas each.

    Sweep point p scales every rate by a common factor 10^U(-1,1) (two
    decades, so trajectory lengths vary about 100x across points) times a
    per-rate jitter 10^U(-1/4,1/4) (so the vectors also differ in shape).
    """
    rng = SplitMix64(2)
    model = random_flat_network(rng, 32, 32, 16, 8, "flat32x64")
    b = _flat_batch(model, rng, 1, R, G, 100, 5000, 1e5, seed=104, name="flat32x64")
    srng = SplitMix64(204)
    rates = np.empty((P, model.n_rules), np.float64)
    for p in range(P):
        common = srng.log_uniform(-1.0, 1.0)
        rates[p] = b.rates[0] * common * np.array(
            [srng.log_uniform(-0.25, 0.25) for _ in range(model.n_rules)])
    return Batch(model, rates, b.init, b.grid, R, 104, name="sweep256x256")


def flat16x24(R: int = 131072, G: int = 100, use_calibrated: bool = True) -> Batch:
    """16 species, 24 reactions (2 inflow/outflow pairs, 16 order-1, 4 order-2)."""
    rng = SplitMix64(5)
    model = random_flat_network(rng, 16, 16, 4, 2, "flat16x24")
    return _flat_batch(model, rng, 1, R, G, 50, 500, 1e4, seed=105, name="flat16x24",
                       use_calibrated=use_calibrated)


# ----------------------------------------------------------------------------
# Small models with known laws (used to pin the oracle)
# ----------------------------------------------------------------------------

def birth_death() -> Model:
    """0 -> A (k1), A -> 0 (k2)."""
    return flat_model(1, [({}, {0: 1}), ({0: 1}, {})], "birth_death")


def isomerisation() -> Model:
    """A -> B (kf), B -> A (kb)."""
    return flat_model(2, [({0: 1}, {1: 1}), ({1: 1}, {0: 1})], "isomerisation")


def dimerisation() -> Model:
    """2A -> B (k1), B -> 2A (k2)."""
    return flat_model(2, [({0: 2}, {1: 1}), ({1: 1}, {0: 2})], "dimerisation")


def heterodimer() -> Model:
    """A + B -> C (k1), C -> A + B (k2)."""
    return flat_model(3, [({0: 1, 1: 1}, {2: 1}), ({2: 1}, {0: 1, 1: 1})], "heterodimer")


def paper_example_rule() -> Model:
    """The worked example of Sec. 2.2: l: a b X -> c X (species a=0, b=1, c=2)."""
    return flat_model(3, [({0: 1, 1: 1}, {2: 1})], "paper_example")


# ----------------------------------------------------------------------------
# Compartmentalised workload (labels top, 1, 2, 3; top contains 1 and 2, 1
# contains 3): intra-compartment reactions, transport in and out, binding to
# the wrap, creation and dissolution of compartments (Sec. 2.1 rule forms).
# ----------------------------------------------------------------------------

CWC_TOKEN = 23      # species that marks a compartment: one in every wrap


def _cwc3_rules(rng: SplitMix64, S: int) -> List[RuleSpec]:
    """48 rules: 24 LOCAL (6 per label: 4 conversions, 2 bimolecular), 12
    PARENT_CHILD (6 in, 4 out, 2 wrap binding), 6 CREATE, 6 DISSOLVE.  The
    token species is used only by CREATE (consumes one free token from the
    parent content, puts it in the new wrap) and DISSOLVE (matches the wrap
    token, released to the parent with the rest of the compartment)."""
    mol = S - 1          # molecular species 0..S-2
    rules: List[RuleSpec] = []
    for lab in range(4):
        for _ in range(4):
            a = rng.randint(0, mol - 1)
            b = (a + rng.randint(1, mol - 1)) % mol
            rules.append(RuleSpec(LOCAL, lab, lhs_ctx={a: 1}, rhs_ctx={b: 1}))
        for i in range(2):
            if i == 0:
                a, b = rng.choice_distinct(mol, 2)
                reac = {a: 1, b: 1}
            else:
                a = rng.randint(0, mol - 1)
                reac = {a: 2}
            c, d = rng.randint(0, mol - 1), rng.randint(0, mol - 1)
            prod: Dict[int, int] = {}
            prod[c] = prod.get(c, 0) + 1
            prod[d] = prod.get(d, 0) + 1
            rules.append(RuleSpec(LOCAL, lab, lhs_ctx=reac, rhs_ctx=prod))
    pairs_in = [(0, 1), (0, 1), (0, 2), (0, 2), (1, 3), (1, 3)]
    for par, ch in pairs_in:
        x = rng.randint(0, mol - 1)
        rules.append(RuleSpec(PARENT_CHILD, par, ch, lhs_ctx={x: 1}, rhs_child={x: 1}))
    for par, ch in [(0, 1), (0, 2), (1, 3), (1, 3)]:
        x = rng.randint(0, mol - 1)
        rules.append(RuleSpec(PARENT_CHILD, par, ch, lhs_child={x: 1}, rhs_ctx={x: 1}))
    for par, ch in [(0, 1), (0, 2)]:
        x, y = rng.choice_distinct(mol, 2)
        z = rng.randint(0, mol - 1)
        rules.append(RuleSpec(PARENT_CHILD, par, ch, lhs_ctx={x: 1}, lhs_wrap={y: 1}, rhs_wrap={z: 1, y: 1}))
    for par, ch in [(0, 1), (0, 1), (0, 2), (0, 2), (1, 3), (1, 3)]:
        x = rng.randint(0, mol - 1)
        rules.append(RuleSpec(CREATE, par, ch, lhs_ctx={CWC_TOKEN: 1}, rhs_wrap={CWC_TOKEN: 1}, rhs_child={x: 20}))
    for par, ch in [(0, 1), (0, 1), (0, 2), (0, 2), (1, 3), (1, 3)]:
        rules.append(RuleSpec(DISSOLVE, par, ch, lhs_wrap={CWC_TOKEN: 1}))
    return rules


def cwc3x24(R: int = 16384, G: int = 500, use_calibrated: bool = True) -> Batch:
    """3 labels below the top level (nesting depth 2), 24 species, 48 rules,
    at most 64 compartments per trajectory (63 tokens), 16,384 replicas,
    500-point grid.

    Initial term: the root holds U{10..200} of each molecular species and 31
    free tokens; 8 label-1 compartments (each containing 2 label-3 ones) and 8
    label-2 compartments, every one with one token in its wrap and U{10..200}
    of each molecular species inside: 33 compartments, 63 tokens in all, so
    CREATE can never run out of slots.  Molecular rate constants are
    log-uniform over three decades with volume scaling for Omega = 100
    molecules; creation and dissolution constants are log-uniform over
    [0.1, 1] per compartment or token, which keeps the compartment population
    stable and makes structural events about 0.6 % of all events."""
    S, L, C = 24, 4, 64
    rng = SplitMix64(3)
    rules = _cwc3_rules(rng, S)
    model = cwc_model(S, L, C, rules, "cwc3x24")
    omega = 100.0
    M = model.n_rules
    rates = np.empty(M, np.float64)
    for j in range(M):
        if model.kind[j] in (CREATE, DISSOLVE):
            rates[j] = rng.log_uniform(-1.0, 0.0)
        else:
            order = int(model.lhs[j].sum())
            rates[j] = rng.log_uniform(-3.0, 0.0) * omega ** (1 - order)
    img = empty_slot_image(model)
    W_ = slot_image_width(S)
    mol = S - 1

    def fill_content(slot):
        for x in range(mol):
            img[slot, 3 + S + x] = rng.randint(10, 200)

    fill_content(0)
    img[0, 3 + S + CWC_TOKEN] = 31
    slot = 1
    l1_slots = []
    for _ in range(8):
        img[slot, :3] = [1, 1, 0]
        img[slot, 3 + CWC_TOKEN] = 1
        fill_content(slot)
        l1_slots.append(slot)
        slot += 1
    for par in l1_slots:
        for _ in range(2):
            img[slot, :3] = [1, 3, par]
            img[slot, 3 + CWC_TOKEN] = 1
            fill_content(slot)
            slot += 1
    for _ in range(8):
        img[slot, :3] = [1, 2, 0]
        img[slot, 3 + CWC_TOKEN] = 1
        fill_content(slot)
        slot += 1
    assert img.shape[1] == W_
    T = 1.0
    if use_calibrated:
        Tc = calibrated_horizon("cwc3x24")
        if Tc is not None:
            T = Tc
    return Batch(model, rates[None, :], img[None], uniform_grid(T, G), R, 103, name="cwc3x24")


# ----------------------------------------------------------------------------
# n-species Lotka-Volterra chain: the model family of the paper's single-
# instance experiments (Sec. 5.1, n = 2 ... 32; n = 2 is prey-predator).  The
# paper gives neither rates nor counts; the reading here is the chain
# S1 -> 2 S1, S_i + S_(i+1) -> 2 S_(i+1) (i < n), S_n -> 0, with the constants
# of Gillespie's 1977 prey-predator example (c1 = 10 per prey, c2 = 0.01,
# c3 = 10) and 1000 molecules of every species.
# ----------------------------------------------------------------------------

# ----------------------------------------------------------------------------
# General patterns (Sec. 2.1: a left-hand side may hold several compartments,
# and compartments inside compartments): cells (label 1) in the top, vesicles
# (label 2) in cells; every rule kind, including fusion of cells and of
# vesicles and rules that reach two membranes down.
# ----------------------------------------------------------------------------

GEN_M, GEN_V = 5, 6   # cell and vesicle tokens (one in every wrap; merged wraps hold several)


def cwc_general(R: int = 256, G: int = 50, seed: int = 7) -> Batch:
    """Seven species (A..E = 0..4, the cell token M = 5, the vesicle token
    V = 6), labels top / cell / vesicle, 21 rules of all seven kinds:
    reactions in each compartment type, transport across the cell and the
    vesicle membranes, creation and dissolution of cells (token M) and
    vesicles (token V), fusion of two cells (identical patterns: one M in
    each wrap) and of two vesicles (different patterns: V in the first wrap,
    E in the second content), two depth-two rules (E taken out of a
    vesicle straight into the top with a B there; vesicle-membrane catalysis
    of A -> C in the cell), and two rules on two sibling compartments that
    keep both (a C passed from one cell to another: ordered pairs; both
    vesicles of a pair turning a D into an E: unordered pairs).  Tokens are
    conserved (10 M, 8 V), so at most 18
    compartments exist besides the root (24 slots).  Rates log-uniform over
    two decades with volume scaling for Omega = 50 (creation, dissolution and
    the two-compartment rules log-uniform in [10^-1.5, 10^-0.5] without
    scaling); initial term: the top with
    U{20..80} of A..E and 6 free M, 4 cells each with one M in the wrap,
    U{5..40} of A..E, one free V and one vesicle (one V in its wrap, U{2..10}
    of A..E)."""
    A, B, C_, D, E, M_, V = 0, 1, 2, 3, 4, GEN_M, GEN_V
    S, L, Cmax = 7, 3, 24
    rules = [
        RuleSpec(LOCAL, 0, lhs_ctx={A: 1}, rhs_ctx={B: 1}),
        RuleSpec(LOCAL, 0, lhs_ctx={B: 1, C_: 1}, rhs_ctx={D: 1}),
        RuleSpec(LOCAL, 0, lhs_ctx={D: 1}, rhs_ctx={A: 1, C_: 1}),
        RuleSpec(LOCAL, 1, lhs_ctx={A: 1}, rhs_ctx={C_: 1}),
        RuleSpec(LOCAL, 1, lhs_ctx={C_: 2}, rhs_ctx={E: 1}),
        RuleSpec(LOCAL, 2, lhs_ctx={E: 1}, rhs_ctx={D: 1}),
        RuleSpec(LOCAL, 2, lhs_ctx={D: 1}, rhs_ctx={E: 1}),
        RuleSpec(PARENT_CHILD, 0, 1, lhs_ctx={A: 1}, rhs_child={A: 1}),
        RuleSpec(PARENT_CHILD, 0, 1, lhs_child={C_: 1}, rhs_ctx={C_: 1}),
        RuleSpec(PARENT_CHILD, 1, 2, lhs_ctx={E: 1}, rhs_child={E: 1}),
        RuleSpec(PARENT_CHILD, 1, 2, lhs_child={D: 1}, rhs_ctx={D: 1}),
        RuleSpec(CREATE, 0, 1, lhs_ctx={M_: 1}, rhs_wrap={M_: 1}, rhs_child={A: 5}),
        RuleSpec(DISSOLVE, 0, 1, lhs_wrap={M_: 1}),
        RuleSpec(CREATE, 1, 2, lhs_ctx={V: 1}, rhs_wrap={V: 1}, rhs_child={E: 2}),
        RuleSpec(DISSOLVE, 1, 2, lhs_wrap={V: 1}),
        RuleSpec(FUSION, 0, 1, lhs_wrap={M_: 1}, lhs_wrap2={M_: 1}, rhs_wrap={M_: 2}),
        RuleSpec(FUSION, 1, 2, lhs_wrap={V: 1}, lhs_child2={E: 1}, rhs_wrap={V: 1}, rhs_child={E: 1}),
        RuleSpec(NESTED, 0, 1, grand_label=2, lhs_ctx={B: 1}, lhs_child2={E: 1}, rhs_ctx={C_: 1}),
        RuleSpec(NESTED, 0, 1, grand_label=2, lhs_child={A: 1}, lhs_wrap2={V: 1},
                 rhs_child={C_: 1}, rhs_wrap2={V: 1}),
        RuleSpec(PAIR, 0, 1, lhs_child={C_: 1}, rhs_child2={C_: 1}),
        RuleSpec(PAIR, 1, 2, lhs_child={D: 1}, lhs_child2={D: 1}, rhs_child={E: 1}, rhs_child2={E: 1}),
    ]
    model = cwc_model(S, L, Cmax, rules, "cwc_general")
    rng = SplitMix64(seed)
    omega = 50.0
    rates = np.empty(model.n_rules, np.float64)
    for j in range(model.n_rules):
        if model.kind[j] in (CREATE, DISSOLVE, FUSION, PAIR):
            rates[j] = rng.log_uniform(-1.5, -0.5)
        else:
            lhs5, _, _ = model.rows5()
            order = int(lhs5[j].sum())
            rates[j] = rng.log_uniform(-2.0, 0.0) * omega ** (1 - order)
    img = empty_slot_image(model)
    for x in range(5):
        img[0, 3 + S + x] = rng.randint(20, 80)
    img[0, 3 + S + M_] = 6
    slot = 1
    for _ in range(4):
        cell = slot
        img[cell, :3] = [1, 1, 0]
        img[cell, 3 + M_] = 1
        for x in range(5):
            img[cell, 3 + S + x] = rng.randint(5, 40)
        img[cell, 3 + S + V] = 1
        ves = slot + 1
        img[ves, :3] = [1, 2, cell]
        img[ves, 3 + V] = 1
        for x in range(5):
            img[ves, 3 + S + x] = rng.randint(2, 10)
        slot += 2
    T = 20.0
    return Batch(model, rates[None, :], img[None], uniform_grid(T, G), R, 1000 + seed, name="cwc_general")


def lotka_volterra_model(n: int) -> Model:
    reactions: List[Reaction] = [({0: 1}, {0: 2})]
    for i in range(n - 1):
        reactions.append(({i: 1, i + 1: 1}, {i + 1: 2}))
    reactions.append(({n - 1: 1}, {}))
    return flat_model(n, reactions, "lotka_volterra_%d" % n)


def lotka_volterra(n: int, R: int = 65536, G: int = 100, T: float = 1.0, seed: int = 300) -> Batch:
    model = lotka_volterra_model(n)
    rates = np.array([[10.0] + [0.01] * (n - 1) + [10.0]], np.float64)
    init = np.full((1, n), 1000, np.int32)
    return Batch(model, rates, init, uniform_grid(T, G), R, seed + n, name="lotka_volterra_%d" % n)


def mm_cascade_model(stages: int) -> Model:
    """A kinase cascade with Michaelis-Menten kinetics throughout (the usual
    enzyme-kinetics shape of signalling models): species 0 is the input
    kinase E; stage i (1..stages) has an inactive form 2i-1 and an active form
    2i.  Activation of stage i: X_i + E_i -> X_i* + E_i at k n_E n_X / (K +
    n_X), the enzyme E_1 = E and E_i = X_{i-1}* after it; deactivation
    X_i* -> X_i at k n_X* / (K + n_X*) (a saturating phosphatase).  Rule
    2(i-1) activates stage i, rule 2(i-1)+1 deactivates it."""
    reactions: List[Reaction] = []
    mm: Dict[int, Tuple[int, float]] = {}
    for i in range(1, stages + 1):
        x, xa = 2 * i - 1, 2 * i
        enz = 0 if i == 1 else 2 * (i - 1)
        mm[len(reactions)] = (x, 50.0)
        reactions.append(({x: 1, enz: 1}, {xa: 1, enz: 1}))
        mm[len(reactions)] = (xa, 50.0)
        reactions.append(({xa: 1}, {x: 1}))
    return flat_model(2 * stages + 1, reactions, "mm_cascade_%d" % stages, michaelis_menten=mm)


def mm_cascade(stages: int = 20, R: int = 16384, G: int = 100, T: float = 20.0, P: int = 1,
               seed: int = 400) -> Batch:
    """Seeded batch of the cascade: 10 input kinases, 100 molecules of each
    stage's inactive form; activation k = 1 and deactivation k = 20 (per
    unit time, the maximal rates of one enzyme and of the phosphatase), K = 50
    molecules.  P > 1 sweep points scale the activation constants by factors
    drawn log-uniformly from [0.5, 2] (SplitMix64 from the seed)."""
    model = mm_cascade_model(stages)
    M = model.n_rules
    base = np.tile(np.array([1.0, 20.0]), stages)
    rates = np.tile(base, (P, 1))
    if P > 1:
        rng = SplitMix64(seed)
        for p in range(P):
            f = 2.0 ** (2.0 * rng.uniform() - 1.0)
            rates[p, 0::2] *= f
    init = np.zeros((1, 2 * stages + 1), np.int32)
    init[0, 0] = 10
    init[0, 1::2] = 100
    assert rates.shape == (P, M)
    return Batch(model, rates, init, uniform_grid(T, G), R, seed + stages, name="mm_cascade_%d" % stages)
