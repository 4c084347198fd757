"""Seeded synthetic geometries shaped like the paper's benchmark systems.

Every coordinate array is float32 [n, 3] in Angstrom; species are uint8
indices into the model's species list (H=0, C=1, N=2, O=3, S=4, F=5, Cl=6);
``box`` is an orthorhombic edge triple (float64) or None (non-periodic);
``mask`` marks the atoms that belong to the machine-learned region (None = all).

Recipes (the paper's systems are not available, so these stand in for them):
  gas24        24 atoms H12 C7 N3 O2 uniform in a 10 A cube, min pair distance
               0.9 A, non-periodic (small organic molecule scale)
  water9000    3000 rigid waters (O-H 0.96 A, H-O-H 104.5 deg, random
               orientation) on a jittered 15^3 lattice, periodic edge 44.77 A
               (1 g/cm^3), like the paper's water boxes
  solvated100k one 1000-atom branched organic-like solute (bonds 1.0-1.5 A)
               in 33,000 waters, periodic edge 99.9 A, 7 species
  molecules64  64 molecules of 20-60 atoms, 4 species drawn 12:7:3:2
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

H, C, N, O, S, F, CL = range(7)
# solute species distribution (C 35%, H 45%, N 7%, O 8%, S 2%, F 1.5%, Cl 1.5%)
SOLUTE_FRACTIONS = {C: 0.35, H: 0.45, N: 0.07, O: 0.08, S: 0.02, F: 0.015, CL: 0.015}
ORGANIC4_WEIGHTS = {H: 12, C: 7, N: 3, O: 2}

OH_BOND = 0.96
HOH_ANGLE = math.radians(104.5)


@dataclasses.dataclass
class System:
    name: str
    coords: np.ndarray                 # float32 [n, 3]
    species: np.ndarray                # uint8 [n]
    box: Optional[np.ndarray] = None   # float64 [3] or None
    mask: Optional[np.ndarray] = None  # uint8 [n] or None

    @property
    def n_atoms(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_ml(self) -> int:
        return self.n_atoms if self.mask is None else int(self.mask.sum())


def _rng(seed) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _random_rotations(rng, n):
    """Uniform random rotation matrices from normalised Gaussian quaternions."""
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _water_template():
    half = HOH_ANGLE / 2
    return np.array([[0.0, 0.0, 0.0],
                     [OH_BOND * math.sin(half), 0.0, OH_BOND * math.cos(half)],
                     [-OH_BOND * math.sin(half), 0.0, OH_BOND * math.cos(half)]])


def water_molecule_sites(rng, centres):
    """Place one rigid water at each centre (O at the centre), random orientation.
    Returns float64 [3*m, 3] (O, H, H per molecule) and species."""
    m = centres.shape[0]
    R = _random_rotations(rng, m)
    tmpl = _water_template()
    xyz = centres[:, None, :] + np.einsum("mij,kj->mki", R, tmpl)
    sp = np.tile(np.array([O, H, H], dtype=np.uint8), m)
    return xyz.reshape(-1, 3), sp


def gas_molecule(rng, n, species, density=0.024, min_dist=0.9, name="gas"):
    """n atoms uniform in a cube of edge (n/density)^(1/3) A with rejection so that
    no pair is closer than min_dist; non-periodic.  ``species``: uint8 array [n]."""
    edge = (n / density) ** (1.0 / 3.0)
    pts = np.empty((n, 3))
    k = 0
    tries = 0
    while k < n:
        p = rng.uniform(0.0, edge, size=3)
        tries += 1
        if k == 0 or np.min(np.sum((pts[:k] - p) ** 2, axis=1)) >= min_dist ** 2:
            pts[k] = p
            k += 1
        if tries > 1000000:
            raise RuntimeError("rejection sampling failed")
    return System(name, pts.astype(np.float32), np.asarray(species, dtype=np.uint8))


def _species_exact(fractions, n, rng):
    """Exact species counts from fractions (largest remainder), shuffled."""
    keys = list(fractions)
    raw = np.array([fractions[k] * n for k in keys])
    cnt = np.floor(raw).astype(int)
    rem = n - cnt.sum()
    order = np.argsort(-(raw - cnt), kind="stable")
    for t in range(rem):
        cnt[order[t]] += 1
    sp = np.concatenate([np.full(c, k, dtype=np.uint8) for k, c in zip(keys, cnt)])
    rng.shuffle(sp)
    return sp


def _species_drawn(weights, n, rng):
    keys = np.array(list(weights), dtype=np.uint8)
    p = np.array([weights[k] for k in weights], dtype=float)
    return rng.choice(keys, size=n, p=p / p.sum()).astype(np.uint8)


def branched_solute(rng, n, centre, min_dist=1.0, bond=(1.0, 1.5)):
    """Random branched chain: each new atom bonds to a random existing atom with
    fewer than 4 bonds, bond length U(bond), isotropic direction, rejected if
    closer than min_dist to any other solute atom."""
    pts = np.zeros((n, 3))
    pts[0] = centre
    nb = np.zeros(n, dtype=int)
    k = 1
    tries = 0
    while k < n:
        tries += 1
        if tries > 200000:
            raise RuntimeError("solute growth failed")
        cand = np.flatnonzero(nb[:k] < 4)
        parent = rng.choice(cand)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        p = pts[parent] + d * rng.uniform(*bond)
        dist2 = np.sum((pts[:k] - p) ** 2, axis=1)
        dist2[parent] = np.inf
        if np.min(dist2) < min_dist ** 2:
            continue
        pts[k] = p
        nb[parent] += 1
        nb[k] = 1
        k += 1
    return pts


def _lattice(n_side, edge):
    g = (np.arange(n_side) + 0.5) * (edge / n_side)
    return np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)


def water_box(n_mol, edge, n_side, seed, jitter=0.25, name="water"):
    """n_mol waters on a jittered n_side^3 lattice (random subset of sites),
    periodic cube of the given edge, coordinates wrapped into [0, edge)."""
    rng = _rng(seed)
    sites = _lattice(n_side, edge)
    pick = rng.choice(sites.shape[0], size=n_mol, replace=False)
    centres = sites[np.sort(pick)] + rng.uniform(-jitter, jitter, size=(n_mol, 3))
    xyz, sp = water_molecule_sites(rng, centres)
    xyz = np.mod(xyz, edge)
    return System(name, xyz.astype(np.float32), sp, np.array([edge] * 3, dtype=np.float64))


def solvated_solute(n_water, n_solute, edge, seed, min_water_dist=2.5, jitter=0.25,
                    name="solvated", mask_solute=False):
    """A branched solute at the box centre plus n_water waters on lattice sites
    farther than min_water_dist from every solute atom.  Solute atoms come first."""
    rng = _rng(seed)
    solute = branched_solute(rng, n_solute, np.full(3, edge / 2))
    sol_sp = _species_exact(SOLUTE_FRACTIONS, n_solute, rng)
    n_side = int(math.ceil(n_water ** (1.0 / 3.0)))
    while True:
        sites = _lattice(n_side, edge)
        # distance from each site to the nearest solute atom (chunked, min-image)
        keep = np.ones(sites.shape[0], dtype=bool)
        for c in range(0, sites.shape[0], 4096):
            d = sites[c:c + 4096, None, :] - solute[None, :, :]
            d -= edge * np.round(d / edge)
            keep[c:c + 4096] = np.min(np.sum(d * d, axis=2), axis=1) > min_water_dist ** 2
        free = np.flatnonzero(keep)
        if free.size >= n_water:
            break
        n_side += 1
    pick = np.sort(rng.choice(free, size=n_water, replace=False))
    centres = sites[pick] + rng.uniform(-jitter, jitter, size=(n_water, 3))
    wxyz, wsp = water_molecule_sites(rng, centres)
    xyz = np.mod(np.concatenate([solute, wxyz]), edge)
    sp = np.concatenate([sol_sp, wsp]).astype(np.uint8)
    mask = None
    if mask_solute:
        mask = np.zeros(sp.shape[0], dtype=np.uint8)
        mask[:n_solute] = 1
    return System(name, xyz.astype(np.float32), sp, np.array([edge] * 3, dtype=np.float64), mask)


def workload(name: str):
    """Named workloads.  Returns (list_of_systems, model_kind, weight_seed)."""
    if name == "gas24":
        rng = _rng(0)
        sp = np.array([H] * 12 + [C] * 7 + [N] * 3 + [O] * 2, dtype=np.uint8)
        rng.shuffle(sp)
        return [gas_molecule(rng, 24, sp, density=24 / 1000.0, name="gas24")], "ani4", 1
    if name == "water9000":
        return [water_box(3000, 44.77, 15, seed=1, name="water9000")], "ani4", 1
    if name == "water99k":
        # the water9000 recipe at the 100k scale with the 4-species model: 33,000
        # rigid waters (99,000 atoms) on a 33^3 lattice, periodic 99.6 A (1 g/cm^3)
        return [water_box(33000, 99.6, 33, seed=6, name="water99k")], "ani4", 1
    if name == "solvated100k":
        return [solvated_solute(33000, 1000, 99.9, seed=2, name="solvated100k")], "ani7x8", 1
    if name == "solvated20k":
        # the serving stream's resident box size (6,667 waters + a 30-80 atom solute,
        # 58.4 A) with the 8-network model; the whole box is the ML region
        return [solvated_solute(6667, 50, 58.4, seed=5, name="solvated20k")], "ani7x8", 1
    if name == "molecules64":
        rng = _rng(4)
        mols = []
        for m in range(64):
            n = int(rng.integers(20, 61))
            mols.append(gas_molecule(rng, n, _species_drawn(ORGANIC4_WEIGHTS, n, rng),
                                     name=f"mol{m}"))
        return mols, "ani4", 1
    raise ValueError(name)
