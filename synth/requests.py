"""Seeded request streams for the serving workload.

A stream of energy+force requests with Poisson arrivals, shaped like the many
short evaluations that free-energy lambda windows and replicas issue (the
paper's alchemical and binding free-energy studies):
  70% gas-phase molecules of 10-120 atoms (solute species distribution,
      density 0.024 atoms/A^3, non-periodic)
  30% hybrid requests: new solute coordinates for one of 8 resident solvated
      boxes (about 20k waters' atoms, edge 58.4 A, solute of 30-80 atoms); only
      the solute is in the machine-learned region (mask = solute), as in the
      hybrid potential V_ML(P) of the paper's hybrid model.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

from .systems import (System, gas_molecule, solvated_solute, _species_exact,
                      SOLUTE_FRACTIONS, _rng)


@dataclasses.dataclass
class Request:
    arrival_s: float                    # scheduled arrival time (seconds from t0)
    system: Optional[System] = None     # gas-phase request: the full system
    box_id: int = -1                    # hybrid request: which resident box
    solute_xyz: Optional[np.ndarray] = None   # new solute coordinates float32 [m,3]

    @property
    def n_ml(self) -> int:
        return self.system.n_atoms if self.system is not None else int(self.solute_xyz.shape[0])


def resident_boxes(seed=300, n_boxes=8):
    boxes = []
    rng = _rng(seed)
    for b in range(n_boxes):
        n_sol = int(rng.integers(30, 81))
        boxes.append(solvated_solute(6667, n_sol, 58.4, seed=seed + 1 + b,
                                     name=f"resident{b}", mask_solute=True))
    return boxes


def request_stream(rate_hz, n_requests, seed, boxes, hybrid_fraction=0.3,
                   perturb=0.02):
    rng = _rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n_requests))
    reqs = []
    for k in range(n_requests):
        if rng.uniform() < hybrid_fraction:
            b = int(rng.integers(0, len(boxes)))
            box = boxes[b]
            m = int(box.mask.sum())
            xyz = box.coords[:m].astype(np.float64) + rng.normal(0.0, perturb, size=(m, 3))
            reqs.append(Request(float(t[k]), box_id=b, solute_xyz=xyz.astype(np.float32)))
        else:
            n = int(rng.integers(10, 121))
            sp = _species_exact(SOLUTE_FRACTIONS, n, rng)
            reqs.append(Request(float(t[k]), system=gas_molecule(rng, n, sp, name=f"req{k}")))
    return reqs
