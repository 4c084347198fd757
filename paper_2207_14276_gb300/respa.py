"""Multiple-time-step (RESPA) driver around the potential (paper Eq. 7).

The hybrid energy is V = V_MM(all) + V_ML(P) - V_MM(P).  The paper integrates
it with a multiple-time-step scheme in which the ML correction is a slow force
applied every outer step.  This driver is that outer loop for the ML part only:
every outer step it evaluates the potential on the masked region P (persistent
neighbour lists with a skin keep the search off most steps) and applies the
force as a half kick on either side of `n_inner` inner steps.  The inner (fast)
forces of the MM engine are left out.  A caller may supply them as a callback
returning a force tensor, or None.  Kicks and drifts run in `nnp_integrate`.

Units: A, fs, kcal/mol, g/mol.
"""
from __future__ import annotations

import numpy as np
import torch

from ._lib import check, lib
from .potential import _ptr, _stream_ptr

# masses by atomic number (g/mol)
MASSES = {1: 1.008, 6: 12.011, 7: 14.007, 8: 15.999, 9: 18.998, 16: 32.06, 17: 35.45}
BOLTZMANN = 0.0019872041   # kcal/mol/K


def integrate(coords, velocities, forces, inv_masses, mask, dt_kick, dt_drift, kinetic=None,
              stream=None):
    """v += dt_kick a(F); x += dt_drift v on the masked atoms (device tensors, in place)."""
    check(lib().nnp_integrate(coords.shape[0], _ptr(coords), _ptr(velocities), _ptr(forces),
                              _ptr(inv_masses), _ptr(mask), float(dt_kick), float(dt_drift),
                              _ptr(kinetic), _stream_ptr(stream)))


class RespaDriver:
    """Outer-step loop for the ML region of a hybrid system.

    potential: a Potential; coords (cuda float32 [n, 3]) are updated in place;
    species: cuda uint8 [n]; atomic_numbers: the model's species order;
    mask: cuda uint8 [n] (the ML region P) or None for all atoms;
    dt_outer: outer time step in fs; n_inner: inner steps per outer step;
    skin: Verlet skin of the potential's neighbour lists (0 disables)."""

    def __init__(self, potential, coords, species, atomic_numbers, box=None, mask=None,
                 dt_outer=1.0, n_inner=1, skin=0.5, temperature=0.0, seed=0,
                 inner_forces=None):
        self.pot = potential
        self.x = coords
        self.sp = species
        self.box = box
        self.mask = mask
        self.dt = float(dt_outer)
        self.n_inner = int(n_inner)
        self.inner_forces = inner_forces
        dev = coords.device
        z = np.asarray(atomic_numbers)[species.cpu().numpy()]
        m = np.array([MASSES[int(a)] for a in z], dtype=np.float32)
        self.inv_m = torch.from_numpy(1.0 / m).to(dev)
        rng = np.random.default_rng(seed)
        # Maxwell-Boltzmann: sigma_v = sqrt(kT / m); 1 kcal/mol per g/mol = 4.184e-4 A^2/fs^2
        v = rng.normal(size=(len(m), 3)) * np.sqrt(BOLTZMANN * temperature * 4.184e-4 / m[:, None])
        self.v = torch.from_numpy(v.astype(np.float32)).to(dev)
        if mask is not None:
            self.v[mask == 0] = 0.0
        self.E = torch.zeros(1, dtype=torch.float64, device=dev)
        self.F = torch.zeros((len(m), 3), dtype=torch.float32, device=dev)
        self.ke = torch.zeros(1, dtype=torch.float64, device=dev)
        self.pot.set_skin(skin)
        self._forces()

    def _forces(self):
        self.pot.energy_forces_into(self.x, self.sp, self.box, self.mask, self.E, self.F)

    def step(self):
        """One outer step: half kick (ML), inner steps, new ML forces, half kick."""
        h = 0.5 * self.dt
        integrate(self.x, self.v, self.F, self.inv_m, self.mask, h, 0.0)
        dt_in = self.dt / self.n_inner
        for _ in range(self.n_inner):
            if self.inner_forces is not None:
                f = self.inner_forces(self.x)
                integrate(self.x, self.v, f, self.inv_m, self.mask, 0.5 * dt_in, dt_in)
                f = self.inner_forces(self.x)
                integrate(self.x, self.v, f, self.inv_m, self.mask, 0.5 * dt_in, 0.0)
            else:
                integrate(self.x, self.v, None, self.inv_m, self.mask, 0.0, dt_in)
        self._forces()
        integrate(self.x, self.v, self.F, self.inv_m, self.mask, h, 0.0, self.ke)

    def energies(self):
        """(potential energy of the ML region, kinetic energy of its atoms) in kcal/mol."""
        return float(self.E.cpu()[0]), float(self.ke.cpu()[0])
