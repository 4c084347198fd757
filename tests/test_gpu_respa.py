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


def _fp64_velocity_verlet(orc, s, x0, v0, masses, dt, steps, mask=None):
    """Reference trajectory: velocity Verlet in FP64 on the oracle's forces of the
    ML region (the outer step of the multiple-time-step scheme with no inner
    forces: half kick, drift by dt, new forces, half kick)."""
    acc = 4.184e-4                     # 1 kcal/mol/A per g/mol in A/fs^2
    x = x0.astype(np.float64).copy()
    v = v0.astype(np.float64).copy()
    mv = np.ones(len(x), bool) if mask is None else mask.astype(bool)
    inv_m = (acc / masses)[:, None]
    F = orc.energy_forces(x, s.species, s.box, mask)["forces"]
    out = []
    for _ in range(steps):
        v[mv] += 0.5 * dt * F[mv] * inv_m[mv]
        x[mv] += dt * v[mv]
        r = orc.energy_forces(x, s.species, s.box, mask)
        F = r["forces"]
        v[mv] += 0.5 * dt * F[mv] * inv_m[mv]
        ke = 0.5 * float(np.sum((v[mv] ** 2).sum(1) * masses[mv])) / acc
        out.append((x.copy(), r["energy"], ke))
    return out


@pytest.mark.parametrize("case", ["gas", "masked"])
def test_trajectory_matches_fp64_velocity_verlet_on_oracle_forces(torch_cuda, case):
    """Ten outer steps of the driver (no inner forces: velocity Verlet) against the
    same integrator in FP64 on the oracle's forces, from the same start: positions
    within 2e-4 A, ML potential energy within 1e-3 kcal/mol and kinetic energy
    within 1e-4 relative at every step (FP32 positions and forces; no chaotic
    growth over ten steps)."""
    import oracle
    from paper_2207_14276_gb300.respa import MASSES
    if case == "gas":
        s = synth.workload("molecules64")[0][12]
        kind, dt, n_inner = "ani4", 0.5, 2
    else:
        s = synth.solvated_solute(300, 24, 22.0, seed=19, name="hybrid", mask_solute=True)
        kind, dt, n_inner = "ani7", 0.5, 4
    drv, pot, x = _driver(s, kind=kind, dt_outer=dt, n_inner=n_inner, temperature=300.0,
                          seed=5, skin=0.5)
    spec, w = model_for(kind)
    orc = oracle.Model(spec, w)
    masses = np.array([MASSES[int(z)] for z in np.asarray(spec.atomic_numbers)[s.species]])
    ref = _fp64_velocity_verlet(orc, s, x.cpu().numpy(), drv.v.cpu().numpy(), masses, dt, 10,
                                s.mask)
    for k in range(10):
        drv.step()
        ep, ek = drv.energies()
        xr, er, kr = ref[k]
        dx = float(np.abs(x.cpu().numpy().astype(np.float64) - xr).max())
        assert dx <= 2e-4, (k, dx)
        assert abs(ep - er) <= 1e-3, (k, ep, er)
        assert abs(ek - kr) <= 1e-4 * kr + 1e-6, (k, ek, kr)
