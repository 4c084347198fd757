"""Deterministic mode (nnp_set_deterministic): repeated calls give bitwise
identical energies, forces and virials, and agree with the normal mode and the
FP64 oracle.

In the normal mode the order of atoms inside a cell and of AEV rows inside a
species segment follows atomic counters, and forces, energies and virials are
summed with floating-point atomics, so repeated calls differ in the last bits.
The deterministic mode sorts the atoms and rows and sums every contribution in a
fixed order; a change between repeated calls in this mode would be a race.
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


def outputs(pot, systems, virial=True):
    outs = pot.energy_forces_batch([to_cuda(s) for s in systems], virial=virial)
    return [(o["energy"].cpu().numpy().copy(), o["forces"].cpu().numpy().copy(),
             o["virial"].cpu().numpy().copy() if virial else None) for o in outs]


def same_bits(a, b):
    for (e1, f1, v1), (e0, f0, v0) in zip(a, b):
        assert np.array_equal(e1.view(np.uint64), e0.view(np.uint64))
        assert np.array_equal(f1.view(np.uint32), f0.view(np.uint32))
        if v1 is not None:
            assert np.array_equal(v1.view(np.uint64), v0.view(np.uint64))


CASES = [
    ("ani4", "fp32_split", lambda: [synth.water_box(300, 20.5, 7, seed=41)] +
     list(synth.workload("molecules64")[0][:6])),
    ("ani7", "fp32_split", lambda: [synth.solvated_solute(300, 200, 22.0, seed=17)]),
    ("ani7", "fp32_simt", lambda: [synth.solvated_solute(300, 200, 22.0, seed=17)]),
    ("ani7x8", "bf16", lambda: [synth.solvated_solute(150, 60, 18.0, seed=6)]),
]


@pytest.mark.parametrize("kind,precision,make", CASES)
def test_deterministic_calls_repeat_bitwise(torch_cuda, kind, precision, make):
    """Three calls in deterministic mode (the second a graph replay, the third
    after a call of another batch) are bitwise equal; they agree with the normal
    mode to its own tolerance and with the FP64 oracle.  The 7-species solvated
    box has solute centres with more than 48 angular neighbours, so the
    CTA-per-centre force kernel is covered too."""
    from paper_2207_14276_gb300 import Potential
    spec, w = model_for(kind)
    systems = make()
    pot = Potential(spec, w, precision=precision)
    normal = outputs(pot, systems)
    pot.set_deterministic(True)
    first = outputs(pot, systems)
    second = outputs(pot, systems)
    outputs(pot, list(synth.workload("molecules64")[0][:3]) if kind == "ani4" else
            [synth.solvated_solute(100, 30, 16.0, seed=9)])
    third = outputs(pot, systems)
    same_bits(second, first)
    same_bits(third, first)
    orc = oracle.Model(spec, w)
    bf16 = precision == "bf16"
    for s, (e1, f1, v1), (e0, f0, v0) in zip(systems, first, normal):
        f_rms = float(np.sqrt(np.mean(f0.astype(np.float64) ** 2))) + 1e-9
        rms, _ = force_errors(f1, f0)
        assert rms <= (2e-2 if bf16 else 1e-5) * f_rms
        ref = orc.energy_forces(s.coords, s.species, s.box)
        scale = float(np.abs(ref["atom_energies"]).sum())
        assert abs(float(e1[0]) - ref["energy"]) <= (2e-3 * scale + 1e-4 if bf16 else 1e-3)
        rms, _ = force_errors(f1, ref["forces"])
        assert rms <= (2e-2 if bf16 else 1e-4) * float(np.sqrt(np.mean(ref["forces"] ** 2))) + 1e-7
        if s.box is not None:
            np.testing.assert_allclose(v1.reshape(3, 3), ref["virial"],
                                       atol=(2e-2 if bf16 else 5e-4) * np.abs(ref["virial"]).max() + 1e-6)


def test_deterministic_trajectory_with_persistent_lists(torch_cuda):
    """A short trajectory with skin lists, run twice from the same start on
    fresh handles in deterministic mode: every step bitwise equal."""
    from paper_2207_14276_gb300 import Potential
    spec, w = model_for("ani4")
    s = synth.water_box(300, 20.5, 7, seed=41)
    runs = []
    for _ in range(2):
        pot = Potential(spec, w, precision="fp32_split")
        pot.set_skin(1.0)
        pot.set_deterministic(True)
        rng = np.random.Generator(np.random.PCG64(3))
        x = s.coords.copy()
        steps = []
        for _ in range(4):
            x = (x + rng.normal(0.0, 0.02, x.shape)).astype(np.float32)
            steps.append(outputs(pot, [synth.System(s.name, x, s.species, s.box, s.mask)])[0])
        runs.append(steps)
    for a, b in zip(runs[0], runs[1]):
        same_bits([a], [b])
