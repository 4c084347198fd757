"""BF16 tensor-core network path (tcgen05, FP32 accumulation) against the FP64 oracle.

The networks run with BF16 operands (AEV, weights, activations, CELU'
factors and back-propagated deltas rounded to 8 significant bits) and FP32
accumulation; AEVs, their backward and the energy sum stay FP32/FP64.  The
bar is the stated BF16 target: force RMS error <= 5e-3 kcal/mol/A.  BF16
keeps 2^-9 relative precision per operand, so each atomic energy is off by up
to about 2e-3 of its size; the rounding of shared quantities (weights, similar
AEVs) biases all atoms of one species alike, so the errors add linearly and the
energy bound is 2e-3 * sum_i |E_i|.
"""
import numpy as np
import pytest

import oracle
import synth
from tests._common import force_errors, model_for, to_cuda

pytestmark = pytest.mark.gpu

F_RMS_BF16 = 5e-3


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def run(kind, s, precision):
    from paper_2207_14276_gb300 import Potential
    spec, w = model_for(kind)
    pot = Potential(spec, w, precision=precision)
    d = to_cuda(s)
    outs = pot.energy_forces_batch([d], atom_energies=True)
    return (float(outs[0]["energy"].cpu()[0]), outs[0]["forces"].cpu().numpy(),
            outs[0]["atom_energies"].cpu().numpy(), spec, w)


def energy_bound(ae_ref, n):
    # 2^-9-level relative error per atom, systematic across atoms: linear sum
    return 2e-3 * float(np.abs(ae_ref).sum()) + 1e-4


@pytest.mark.parametrize("kind,system", [
    ("ani4", lambda: synth.workload("water9000")[0][0]),
    ("ani4", lambda: synth.workload("gas24")[0][0]),
    ("ani7", lambda: synth.solvated_solute(400, 120, 24.0, seed=5)),
    ("ani7x8", lambda: synth.solvated_solute(150, 60, 18.0, seed=6)),
])
def test_bf16_matches_oracle(torch_cuda, kind, system):
    s = system()
    E, F, ae, spec, w = run(kind, s, "bf16")
    ref = oracle.Model(spec, w).energy_forces(s.coords, s.species, s.box, s.mask)
    rms, mx = force_errors(F, ref["forces"])
    f_rms = float(np.sqrt(np.mean(ref["forces"] ** 2)))
    print(f"{kind} n={s.n_atoms}: |dE|={abs(E - ref['energy']):.3e} force RMS err={rms:.3e} "
          f"(rel {rms / f_rms:.2e}) max={mx:.3e}")
    assert rms <= F_RMS_BF16
    assert rms <= 2e-2 * f_rms
    assert abs(E - ref["energy"]) <= energy_bound(ref["atom_energies"], s.n_atoms)
    np.testing.assert_allclose(ae, ref["atom_energies"],
                               atol=2e-2 * float(np.abs(ref["atom_energies"]).max()) + 1e-5)


def test_bf16_close_to_fp32_path(torch_cuda):
    s = synth.water_box(500, 24.0, 8, seed=51)
    E16, F16, _, _, _ = run("ani4", s, "bf16")
    E32, F32, _, _, _ = run("ani4", s, "fp32")
    rms, _ = force_errors(F16, F32)
    assert rms <= 2e-2 * float(np.sqrt(np.mean(F32.astype(np.float64) ** 2)))


def test_bf16_batch_alone_equals_in_mix(torch_cuda):
    from paper_2207_14276_gb300 import Potential
    spec, w = model_for("ani4")
    pot = Potential(spec, w, precision="bf16")
    mols, _, _ = synth.workload("molecules64")
    outs = pot.energy_forces_batch([to_cuda(m) for m in mols])
    for k in (0, 31, 63):
        d = to_cuda(mols[k])
        E, F = pot.energy_forces(d["coords"], d["species"])
        # identical BF16 arithmetic per row; only FP32 atomic order differs
        assert float(E.cpu()[0]) == pytest.approx(float(outs[k]["energy"].cpu()[0]), abs=1e-4)
        np.testing.assert_allclose(F.cpu().numpy(), outs[k]["forces"].cpu().numpy(), atol=1e-4)
