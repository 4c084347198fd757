"""Multiple-time-step driver around the potential (paper Eq. 7; the MM terms of
the hybrid energy belong to the host engine and are left out).

With no inner forces one outer step is a velocity-Verlet step, so the ML
region's total energy (potential + kinetic) must be conserved to O(dt^2); the
atoms outside the mask must not move; and the persistent lists must be rebuilt
only occasionally along the trajectory.
"""
import numpy as np
import pytest

import synth
from tests._common import model_for, to_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def _driver(s, kind="ani4", **kw):
    from paper_2207_14276_gb300 import Potential
    from paper_2207_14276_gb300.respa import RespaDriver
    spec, w = model_for(kind)
    pot = Potential(spec, w)
    d = to_cuda(s)
    x = d["coords"].clone()
    drv = RespaDriver(pot, x, d["species"], spec.atomic_numbers, box=d["box"], mask=d["mask"], **kw)
    return drv, pot, x


def test_energy_conservation_gas_molecule(torch_cuda):
    systems, _, _ = synth.workload("molecules64")
    drv, pot, _ = _driver(systems[7], dt_outer=0.1, n_inner=2, temperature=300.0, seed=1)
    etot = []
    for _ in range(200):
        drv.step()
        ep, ek = drv.energies()
        etot.append(ep + ek)
    etot = np.array(etot)
    # velocity Verlet on a smooth surface: no secular drift, fluctuations small
    # against the kinetic energy of the molecule
    _, ek = drv.energies()
    assert np.abs(etot - etot[0]).max() < 0.02 * max(ek, 1.0), (np.ptp(etot), ek)
    # the trajectory uses few list builds
    builds, calls = pot.list_stats()
    assert calls >= 200 and builds < calls // 4


def test_masked_solute_moves_and_solvent_stays(torch_cuda):
    torch = torch_cuda
    s = synth.solvated_solute(800, 30, 30.0, seed=9, name="hybrid", mask_solute=True)
    drv, pot, x = _driver(s, kind="ani7", dt_outer=0.5, n_inner=4, temperature=300.0, seed=2)
    x0 = x.clone()
    for _ in range(20):
        drv.step()
    m = torch.from_numpy(s.mask).cuda().bool()
    moved = (x - x0).norm(dim=1)
    assert float(moved[~m].max()) == 0.0
    assert float(moved[m].mean()) > 1e-3
    # forces act only on the ML region
    assert float(drv.F[~m].abs().max()) == 0.0
