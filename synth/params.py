"""Model hyper-parameters (plain data) and seeded random network weights.

AEV hyper-parameters (Eqs. 3-4 of the paper):
  radial:  16 Gaussian shells, eta_r = 16 A^-2, centres spread over
           [0.9, 5.2) A (half-open: centre_r = 0.9 + r * 4.3/16), Rc_r = 5.2 A
  angular: 4 distance shells (eta_a = 8 A^-2, centres 0.9 + a*0.65),
           8 angle sections theta_z = (2z+1) pi/16, zeta = 32, Rc_a = 3.5 A
The angle sections are stored as theta values; any derived quantity (their
cosines and sines) is computed by each implementation on its own.

Network weights: one multilayer perceptron per (ensemble member, species),
layer l maps widths[l] -> widths[l+1], stored row-major W[out, in] then b[out].
Flat layout of the weight vector (the data contract both sides read):
  for e in range(n_ensemble): for s in range(n_species): for l in range(n_layers):
      W (widths[l+1] * widths[l] floats), then b (widths[l+1] floats)
Initialisation is PyTorch's nn.Linear default (Kaiming-uniform with a=sqrt(5)),
i.e. W, b ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)), drawn from numpy PCG64(seed).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SPECIES4 = (1, 6, 7, 8)              # H, C, N, O   (index order = AEV order)
SPECIES7 = (1, 6, 7, 8, 16, 9, 17)   # H, C, N, O, S, F, Cl


@dataclasses.dataclass(frozen=True)
class AevParams:
    n_species: int
    rc_r: float
    eta_r: float
    shf_r: tuple
    rc_a: float
    eta_a: float
    zeta: float
    shf_a: tuple
    shf_z: tuple          # angle-section centres theta_z (radians)
    cos_scale: float = 1.0


@dataclasses.dataclass(frozen=True)
class ModelSpec:
    aev: AevParams
    widths: tuple          # (D, h1, h2, h3, 1)
    n_ensemble: int
    celu_alpha: float = 0.1
    atomic_numbers: tuple = SPECIES4


def aev_params(n_species: int, cos_scale: float = 1.0) -> AevParams:
    shf_r = tuple(0.9 + r * (5.2 - 0.9) / 16.0 for r in range(16))
    shf_a = tuple(0.9 + a * (3.5 - 0.9) / 4.0 for a in range(4))
    shf_z = tuple((2 * z + 1) * math.pi / 16.0 for z in range(8))
    return AevParams(n_species=n_species, rc_r=5.2, eta_r=16.0, shf_r=shf_r,
                     rc_a=3.5, eta_a=8.0, zeta=32.0, shf_a=shf_a, shf_z=shf_z,
                     cos_scale=cos_scale)


def aev_dim(p: AevParams) -> int:
    S = p.n_species
    return S * len(p.shf_r) + (S * (S + 1) // 2) * len(p.shf_a) * len(p.shf_z)


def model_spec(kind: str) -> ModelSpec:
    """'ani4': 4 species, AEV 384, MLP 384-160-128-96-1, one network.
    'ani7': 7 species, AEV 1008, MLP 1008-256-192-160-1.
    'ani7x8': the 'ani7' layout with an ensemble of 8 networks (mean)."""
    if kind == "ani4":
        p = aev_params(4)
        return ModelSpec(p, (aev_dim(p), 160, 128, 96, 1), 1, 0.1, SPECIES4)
    if kind == "ani7":
        p = aev_params(7)
        return ModelSpec(p, (aev_dim(p), 256, 192, 160, 1), 1, 0.1, SPECIES7)
    if kind == "ani7x8":
        p = aev_params(7)
        return ModelSpec(p, (aev_dim(p), 256, 192, 160, 1), 8, 0.1, SPECIES7)
    raise ValueError(kind)


def n_weights(widths, n_species: int, n_ensemble: int) -> int:
    per = sum(widths[l + 1] * widths[l] + widths[l + 1] for l in range(len(widths) - 1))
    return per * n_species * n_ensemble


def make_weights(spec: ModelSpec, seed: int) -> np.ndarray:
    """Flat float32 weight vector in the layout described in the module docstring."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = spec.widths
    S = spec.aev.n_species
    out = []
    for _e in range(spec.n_ensemble):
        for _s in range(S):
            for l in range(len(w) - 1):
                bound = 1.0 / math.sqrt(w[l])
                out.append(rng.uniform(-bound, bound, size=w[l + 1] * w[l]))
                out.append(rng.uniform(-bound, bound, size=w[l + 1]))
    flat = np.concatenate(out).astype(np.float32)
    assert flat.size == n_weights(w, S, spec.n_ensemble)
    return flat
