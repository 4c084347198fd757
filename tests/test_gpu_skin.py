"""Persistent neighbour lists with a Verlet skin.

A handle with a skin keeps its cell and neighbour lists between calls and
rebuilds them on the device only when an atom has moved more than skin/2 since
the last build.  Every result must equal a fresh evaluation (lists rebuilt at the
cutoffs) up to FP32 summation order, and the final state must also match the
FP64 oracle within the FP32 path's tolerances.
"""
import numpy as np
import pytest

import oracle
import synth
from tests._common import force_errors, model_for, to_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def _pair(kind="ani4", precision="fp32", skin=1.0):
    from paper_2207_14276_gb300 import Potential
    spec, w = model_for(kind)
    fresh = Potential(spec, w, precision=precision)
    kept = Potential(spec, w, precision=precision)
    kept.set_skin(skin)
    return fresh, kept, oracle.Model(spec, w)


def _same(a, b, e_rel=1e-6, f_atol=2e-4):
    (Ea, Fa), (Eb, Fb) = a, b
    Ea, Eb = float(Ea.cpu()[0]), float(Eb.cpu()[0])
    assert abs(Ea - Eb) <= e_rel * max(1.0, abs(Ea)), (Ea, Eb)
    d = np.abs(Fa.cpu().numpy().astype(np.float64) - Fb.cpu().numpy())
    assert d.max() <= f_atol, d.max()


def test_trajectory_matches_fresh_lists_and_rebuilds_only_when_needed(torch_cuda):
    torch = torch_cuda
    fresh, kept, orc = _pair()
    s = synth.water_box(300, 20.5, 7, seed=31)
    d = to_cuda(s)
    x = d["coords"].clone()
    gen = torch.Generator(device="cuda").manual_seed(5)
    builds = []
    for step in range(12):
        if step > 0:   # small thermal steps: 0.02 A per coordinate
            x = x + 0.02 * torch.randn(x.shape, device="cuda", generator=gen)
        _same(fresh.energy_forces(x, d["species"], d["box"]),
              kept.energy_forces(x, d["species"], d["box"]))
        builds.append(kept.list_stats()[0])
    # 0.5 A of allowed drift: the first call builds, the drift of a few steps
    # (|dr| ~ 0.035 A per step) stays under it for a while, then one rebuild
    assert builds[0] == 1
    assert builds[3] == 1
    assert builds[-1] < 12
    # a single atom moved by 0.6 A forces a rebuild on the next call
    b0 = kept.list_stats()[0]
    x[17] += torch.tensor([0.6, 0.0, 0.0], device="cuda")
    _same(fresh.energy_forces(x, d["species"], d["box"]),
          kept.energy_forces(x, d["species"], d["box"]))
    assert kept.list_stats()[0] == b0 + 1
    # and the kept-list result agrees with the FP64 oracle
    E, F = kept.energy_forces(x, d["species"], d["box"])
    ref = orc.energy_forces(x.cpu().numpy(), s.species, s.box)
    assert abs(float(E.cpu()[0]) - ref["energy"]) <= 1e-3
    rms, _ = force_errors(F.cpu().numpy(), ref["forces"])
    assert rms <= 1e-3


def test_wrapping_across_the_box_is_not_a_displacement(torch_cuda):
    torch = torch_cuda
    fresh, kept, _ = _pair()
    s = synth.water_box(200, 18.0, 6, seed=32)
    d = to_cuda(s)
    x = d["coords"].clone()
    kept.energy_forces(x, d["species"], d["box"])
    assert kept.list_stats()[0] == 1
    # every atom of the first 50 shifted by one box edge: same configuration
    x2 = x.clone()
    x2[:50] += 18.0
    _same(fresh.energy_forces(x2, d["species"], d["box"]),
          kept.energy_forces(x2, d["species"], d["box"]))
    assert kept.list_stats()[0] == 1


def test_new_layout_rebuilds(torch_cuda):
    torch = torch_cuda
    fresh, kept, _ = _pair()
    s = synth.water_box(200, 18.0, 6, seed=33)
    d = to_cuda(s)
    kept.energy_forces(d["coords"], d["species"], d["box"])
    # same values in a different species array: the layout changed, so rebuild
    sp2 = d["species"].clone()
    _same(fresh.energy_forces(d["coords"], sp2, d["box"]),
          kept.energy_forces(d["coords"], sp2, d["box"]))
    assert kept.list_stats()[0] == 2
    # a mask (hybrid partition) is part of the layout too
    mask = torch.zeros(s.n_atoms, dtype=torch.uint8, device="cuda")
    mask[:90] = 1
    _same(fresh.energy_forces(d["coords"], sp2, d["box"], mask),
          kept.energy_forces(d["coords"], sp2, d["box"], mask))
    assert kept.list_stats()[0] == 3
    # a system of another size
    s2 = synth.water_box(150, 18.0, 6, seed=34)
    d2 = to_cuda(s2)
    _same(fresh.energy_forces(d2["coords"], d2["species"], d2["box"]),
          kept.energy_forces(d2["coords"], d2["species"], d2["box"]))
    assert kept.list_stats()[0] == 4


def test_batch_and_molecules_with_skin(torch_cuda):
    torch = torch_cuda
    fresh, kept, _ = _pair()
    systems, _, _ = synth.workload("molecules64")
    batch = [to_cuda(m) for m in systems[:12]] + [to_cuda(synth.water_box(200, 18.0, 6, seed=35))]
    gen = torch.Generator(device="cuda").manual_seed(6)
    for step in range(4):
        if step > 0:
            for b in batch:
                b["coords"] = b["coords"] + 0.01 * torch.randn(b["coords"].shape, device="cuda",
                                                             generator=gen)
        ra = fresh.energy_forces_batch(batch)
        rb = kept.energy_forces_batch(batch)
        for a, b in zip(ra, rb):
            _same((a["energy"], a["forces"]), (b["energy"], b["forces"]))
    assert kept.list_stats()[0] == 1


def test_bf16_path_with_skin(torch_cuda):
    torch = torch_cuda
    fresh, kept, _ = _pair(kind="ani7", precision="bf16")
    systems, _, _ = synth.workload("molecules64")
    s = systems[3]
    d = to_cuda(s)
    x = d["coords"].clone()
    gen = torch.Generator(device="cuda").manual_seed(7)
    for step in range(4):
        if step > 0:
            x = x + 0.02 * torch.randn(x.shape, device="cuda", generator=gen)
        # the same BF16 arithmetic on both sides: only summation order differs
        _same(fresh.energy_forces(x, d["species"]), kept.energy_forces(x, d["species"]),
              e_rel=1e-5, f_atol=2e-3)


def test_force_vjp_between_skin_calls(torch_cuda):
    torch = torch_cuda
    fresh, kept, _ = _pair()
    systems, _, _ = synth.workload("molecules64")
    s = systems[5]
    d = to_cuda(s)
    kept.energy_forces(d["coords"], d["species"])
    dLdF = torch.ones((s.n_atoms, 3), dtype=torch.float32, device="cuda")
    kept.force_vjp_batch([{"coords": d["coords"], "species": d["species"]}], [1.0], [dLdF])
    torch.cuda.synchronize()
    _same(fresh.energy_forces(d["coords"], d["species"]),
          kept.energy_forces(d["coords"], d["species"]))


def test_dense_box_capacity_growth_with_skin(torch_cuda):
    # three times liquid density: ~90 angular and ~300 radial neighbours, far
    # above the initial list capacities; the first call overflows, reports it,
    # and the repeated call (with grown lists) matches fresh lists
    fresh, kept, _ = _pair(skin=0.5)
    s = synth.water_box(1000, 18.0, 10, seed=36)
    d = to_cuda(s)
    _same(fresh.energy_forces(d["coords"], d["species"], d["box"]),
          kept.energy_forces(d["coords"], d["species"], d["box"]), f_atol=1e-3)
    x = d["coords"] + 0.01
    _same(fresh.energy_forces(x, d["species"], d["box"]),
          kept.energy_forces(x, d["species"], d["box"]), f_atol=1e-3)
