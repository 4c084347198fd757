"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the FP64 oracle.

This module holds no arithmetic of the method (no cutoff, symmetry function,
network or force code).  It only draws geometries, species, network weights and
request streams from seeded numpy generators, and states the model
hyper-parameters as plain data.  Both the GPU library and the oracle receive
these arrays as inputs; neither imports the other.

Workloads follow the paper's benchmark systems (water boxes, solvated
solutes, small organic molecules; Sec. "Benchmark Systems") and the ANI model
layout of Eqs. 2-4 (4 species H,C,N,O for ANI-1x style models, 7 species
adding S,F,Cl for ANI-2x style models).
"""
from .params import (SPECIES4, SPECIES7, AevParams, ModelSpec, aev_params,
                     model_spec, make_weights, aev_dim)
from .systems import (System, gas_molecule, water_box, solvated_solute,
                      workload, water_molecule_sites)
from .requests import Request, request_stream, resident_boxes

__all__ = [
    "SPECIES4", "SPECIES7", "AevParams", "ModelSpec", "aev_params",
    "model_spec", "make_weights", "aev_dim", "System", "gas_molecule",
    "water_box", "solvated_solute", "workload", "water_molecule_sites",
    "Request", "request_stream", "resident_boxes",
]
