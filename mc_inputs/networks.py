"""Reaction-network descriptions: Robertson's 3-species system and seeded
synthetic element-conserving chemistry networks.

The paper's networks come from pynucastro and nuclear rate libraries (Software
design section, paragraph on network/integrator separation); those are not
available, so synthetic chemical-kinetics networks stand in for them. A network
here is plain data: stoichiometry, Arrhenius parameters (A, b, C) for both
directions of each reaction, and the energy each forward reaction releases.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

# Boltzmann constant in eV/K (CODATA 2018, exact to the digits given).
K_B_EV = 8.617333262e-5


@dataclass
class Network:
    """Plain-data reaction network.

    Reaction r turns its reactants ``react[r]`` into products ``prod[r]``
    (each a pair of species indices, -1 for an empty slot). Rate coefficient
    of a direction: k = A * T**b * exp(-C/T). The forward direction releases
    ``dE_eV[r]`` electron-volts per reaction event (negative = absorbs).
    """
    name: str
    n_species: int
    n_elements: int
    energy_eq: bool
    react: np.ndarray          # int32 [R, 2]
    prod: np.ndarray           # int32 [R, 2]
    composition: np.ndarray    # int32 [S, E] element counts per species
    A_f: np.ndarray
    b_f: np.ndarray
    C_f: np.ndarray
    A_r: np.ndarray
    b_r: np.ndarray
    C_r: np.ndarray
    dE_eV: np.ndarray
    gamma: float = 5.0 / 3.0
    species_energy_eV: np.ndarray | None = None   # set under the species-energy reading
    seed: int | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n_reactions(self) -> int:
        return int(self.react.shape[0])

    @property
    def n_ode(self) -> int:
        return self.n_species + (1 if self.energy_eq else 0)

    def stoich(self) -> np.ndarray:
        """Net stoichiometric matrix nu [S, R] (products minus reactants)."""
        nu = np.zeros((self.n_species, self.n_reactions), dtype=np.int64)
        for r in range(self.n_reactions):
            for s in self.react[r]:
                if s >= 0:
                    nu[s, r] -= 1
            for s in self.prod[r]:
                if s >= 0:
                    nu[s, r] += 1
        return nu


def robertson_network() -> Network:
    """Robertson's stiff kinetics (Robertson 1966) written as three reactions:
    A -> B (k1), B + B -> B + C (k2), B + C -> A + C (k3), with
    k1 = 0.04, k2 = 3e7, k3 = 1e4, no reverse directions and no energy
    equation. One pseudo-element counts every species once, so its total is
    y1 + y2 + y3."""
    react = np.array([[0, -1], [1, 1], [1, 2]], dtype=np.int32)
    prod = np.array([[1, -1], [1, 2], [0, 2]], dtype=np.int32)
    z = np.zeros(3)
    return Network(
        name="robertson3", n_species=3, n_elements=1, energy_eq=False,
        react=react, prod=prod, composition=np.ones((3, 1), dtype=np.int32),
        A_f=np.array([0.04, 3.0e7, 1.0e4]), b_f=z.copy(), C_f=z.copy(),
        A_r=z.copy(), b_r=z.copy(), C_r=z.copy(), dE_eV=z.copy(), gamma=5.0 / 3.0,
    )


def _species_vectors(n_elements: int, n_species: int, rng: np.random.Generator) -> np.ndarray:
    """Element-count vectors in {0,1,2}^E without the zero vector: every
    monatomic species first, the rest drawn distinct from the remaining
    vectors (in the generator's order)."""
    unit = [tuple(int(i == e) for i in range(n_elements)) for e in range(n_elements)]
    others = [v for v in itertools.product((0, 1, 2), repeat=n_elements)
              if any(v) and v not in unit]
    if n_species - n_elements > len(others):
        raise ValueError("too many species for this element count")
    pick = rng.choice(len(others), size=n_species - n_elements, replace=False)
    vecs = unit + [others[i] for i in pick]
    return np.array(vecs, dtype=np.int32)


def _candidate_reactions(comp: np.ndarray):
    """All element-balanced reactions with at most two species a side, each
    unordered reaction listed once: exchange reactions A+B <=> C+D (A=B
    allowed) between distinct unordered species pairs, then association
    reactions A+B <=> C. A side is a tuple of species indices; -1 pads a
    one-species side."""
    S = comp.shape[0]
    pairs = [(a, b) for a in range(S) for b in range(a, S)]
    by_sum: dict[tuple, list] = {}
    for p in pairs:
        key = tuple((comp[p[0]] + comp[p[1]]).tolist())
        by_sum.setdefault(key, []).append(p)
    cands = []
    for key in sorted(by_sum):
        group = by_sum[key]
        for i in range(len(group)):
            for j in range(i + 1, len(group)):
                cands.append((group[i], group[j]))
    single = {tuple(v): i for i, v in enumerate(comp.tolist())}
    for p in pairs:
        key = tuple((comp[p[0]] + comp[p[1]]).tolist())
        if key in single:
            cands.append((p, (single[key], -1)))
    return cands


def synthetic_network(n_species: int, n_elements: int, n_reactions: int, seed: int,
                      energy_model: str = "species", name: str | None = None,
                      gamma: float = 5.0 / 3.0) -> Network:
    """Seeded synthetic element-conserving network with an energy equation.

    Species are element-count vectors in {0,1,2}^E (all monatomic species plus
    distinct draws). Reactions are drawn without replacement from every
    balanced exchange (A+B <=> C+D) and association (A+B <=> C) candidate, and
    each is given a random direction. A species set with fewer than
    ``n_reactions`` candidates is redrawn.

    Rate parameters per direction: A log-uniform in [1e-12, 1e-8] cm^3/s,
    b uniform in [-1, 1], C uniform in [0, 5e4] K (independent draws for the
    forward and reverse directions).

    energy_model:
      "species"  -- every species gets an energy eps_i ~ U[-2.5, 2.5] eV and a
                    reaction releases dE = eps(reactants) - eps(products);
                    candidates with |dE| > 5 eV are dropped, so dE lies in
                    [-5, 5] eV and total energy is a state function.
      "reaction" -- dE drawn per reaction, uniform in [-5, 5] eV (literal).
    """
    if energy_model not in ("species", "reaction"):
        raise ValueError(energy_model)
    rng = np.random.default_rng(seed)

    def side_energy(side, eps):
        return sum(eps[s] for s in side if s >= 0)

    # Species sets with too few balanced reactions are redrawn from the same
    # stream, so a seed still fixes the network.
    for _ in range(10000):
        comp = _species_vectors(n_elements, n_species, rng)
        eps = rng.uniform(-2.5, 2.5, size=n_species) if energy_model == "species" else None
        cands = _candidate_reactions(comp)
        if energy_model == "species":
            cands = [c for c in cands if abs(side_energy(c[0], eps) - side_energy(c[1], eps)) <= 5.0]
        if len(cands) >= n_reactions:
            break
    else:
        raise ValueError("no species set with enough balanced reactions")
    pick = rng.choice(len(cands), size=n_reactions, replace=False)
    flip = rng.random(n_reactions) < 0.5
    react = np.zeros((n_reactions, 2), dtype=np.int32)
    prod = np.zeros((n_reactions, 2), dtype=np.int32)
    for r, (ci, f) in enumerate(zip(pick, flip)):
        lhs, rhs = cands[ci]
        if f:
            lhs, rhs = rhs, lhs
        react[r] = lhs
        prod[r] = rhs
    R = n_reactions
    A_f = 10.0 ** rng.uniform(-12.0, -8.0, R)
    b_f = rng.uniform(-1.0, 1.0, R)
    C_f = rng.uniform(0.0, 5.0e4, R)
    A_r = 10.0 ** rng.uniform(-12.0, -8.0, R)
    b_r = rng.uniform(-1.0, 1.0, R)
    C_r = rng.uniform(0.0, 5.0e4, R)
    if energy_model == "species":
        dE = np.array([side_energy(react[r], eps) - side_energy(prod[r], eps) for r in range(R)])
    else:
        dE = rng.uniform(-5.0, 5.0, R)
    return Network(
        name=name or f"synthetic{n_species}_{n_elements}_{n_reactions}_s{seed}",
        n_species=n_species, n_elements=n_elements, energy_eq=True,
        react=react, prod=prod, composition=comp,
        A_f=A_f, b_f=b_f, C_f=C_f, A_r=A_r, b_r=b_r, C_r=C_r, dE_eV=dE,
        gamma=gamma, species_energy_eV=eps, seed=seed,
        meta={"energy_model": energy_model},
    )


def network_13(energy_model: str = "species") -> Network:
    """12 species from 3 elements plus the energy equation (13 ODEs), 40
    reversible reactions, network seed 2."""
    return synthetic_network(12, 3, 40, seed=2, energy_model=energy_model, name="net13")


def network_33(energy_model: str = "species") -> Network:
    """32 species from 4 elements plus the energy equation (33 ODEs), 120
    reversible reactions, network seed 5."""
    return synthetic_network(32, 4, 120, seed=5, energy_model=energy_model, name="net33")
