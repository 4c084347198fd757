"""Helpers shared by the tests: seeded workloads, models on both sides, error norms."""
import numpy as np

import synth


def model_for(kind, seed=1, cos_scale=1.0):
    import dataclasses
    spec = synth.model_spec(kind)
    if cos_scale != 1.0:
        spec = dataclasses.replace(spec, aev=dataclasses.replace(spec.aev, cos_scale=cos_scale))
    return spec, synth.make_weights(spec, seed)


def force_errors(F, Fref):
    d = np.asarray(F, np.float64) - np.asarray(Fref, np.float64)
    return float(np.sqrt(np.mean(d * d))), float(np.abs(d).max())


def to_cuda(system):
    import torch
    out = {"coords": torch.from_numpy(np.ascontiguousarray(system.coords)).cuda(),
           "species": torch.from_numpy(np.ascontiguousarray(system.species)).cuda(),
           "box": None if system.box is None else [float(b) for b in system.box],
           "mask": None if system.mask is None else torch.from_numpy(system.mask).cuda()}
    return out
