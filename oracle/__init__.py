"""FP64 CPU oracle (test infrastructure).

Plain double-precision restatement of the paper's neural-network potential
(Eqs. 2-5 and the hybrid mask of Eq. 7) used to check the CUDA library.  Only
the tests, ``__graft_entry__.smoke()`` and the benchmark's ``cpu_baseline`` leg
may import this package.  It shares no code with the CUDA path; both receive
the same seeded inputs from ``synth``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with the host C++ compiler (portable flags only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        d, i, i64 = ctypes.c_double, ctypes.c_int, ctypes.c_int64
        lib.oracle_model_new.restype = P
        lib.oracle_model_new.argtypes = [i, d, d, i, P, d, d, d, i, P, i, P, d, i, i, P, P, P, d]
        lib.oracle_model_free.argtypes = [P]
        lib.oracle_aev_dim.restype = i
        lib.oracle_aev_dim.argtypes = [P]
        lib.oracle_n_weights.restype = i64
        lib.oracle_n_weights.argtypes = [P]
        for f in (lib.oracle_neighbours_brute, lib.oracle_neighbours_cells):
            f.restype = i64
            f.argtypes = [i, P, P, P, d, i64, P]
        lib.oracle_energy_forces.restype = d
        lib.oracle_energy_forces.argtypes = [P, i, P, P, P, P, P, P, P, P, P, P]
        lib.oracle_force_matching.restype = d
        lib.oracle_force_matching.argtypes = [P, i, P, P, P, P, P, P, P, P]
        lib.oracle_energy_forces_centres.restype = d
        lib.oracle_energy_forces_centres.argtypes = [P, i, P, P, P, P, i, P, P]
        lib.oracle_sample.restype = None
        lib.oracle_sample.argtypes = [P, i, P, P, P, P, i, P, P, P, P]
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _u8(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.uint8)


class Model:
    """An FP64 copy of a model: AEV hyper-parameters + flat weights (synth layout)."""

    def __init__(self, spec, weights, shift=None):
        lib = _load()
        p = spec.aev
        self.spec = spec
        self.n_species = p.n_species
        self._keep = [np.asarray(p.shf_r, np.float64), np.asarray(p.shf_a, np.float64),
                      np.asarray(p.shf_z, np.float64),
                      np.asarray(spec.widths, np.int32),
                      np.ascontiguousarray(weights, dtype=np.float64),
                      None if shift is None else np.asarray(shift, np.float64)]
        shf_r, shf_a, shf_z, widths, w, sh = self._keep
        self._h = lib.oracle_model_new(
            p.n_species, p.rc_r, p.eta_r, len(shf_r), _ptr(shf_r), p.rc_a, p.eta_a, p.zeta,
            len(shf_a), _ptr(shf_a), len(shf_z), _ptr(shf_z), p.cos_scale, spec.n_ensemble,
            len(spec.widths) - 1, _ptr(widths), _ptr(w), _ptr(sh), spec.celu_alpha)
        self.D = lib.oracle_aev_dim(self._h)
        self.n_weights = lib.oracle_n_weights(self._h)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.oracle_model_free(self._h)
            self._h = None

    def energy_forces(self, coords, species, box=None, mask=None, want_aev=False,
                      want_dEdG=False, want_dEdW=False):
        """Returns dict: energy, forces [n,3], virial [3,3], atom_energies [n] and
        optionally aev [n,D], dEdG [n,D], dEdW (flat)."""
        x = _f64(coords)
        n = x.shape[0]
        F = np.zeros((n, 3))
        V = np.zeros((3, 3))
        ae = np.zeros(n)
        aev = np.zeros((n, self.D)) if want_aev else None
        dG = np.zeros((n, self.D)) if want_dEdG else None
        dW = np.zeros(self.n_weights) if want_dEdW else None
        E = _load().oracle_energy_forces(self._h, n, _ptr(x), _ptr(_u8(species)),
                                         _ptr(_f64(box)), _ptr(_u8(mask)), _ptr(F), _ptr(V),
                                         _ptr(ae), _ptr(aev), _ptr(dG), _ptr(dW))
        out = dict(energy=E, forces=F, virial=V, atom_energies=ae)
        if want_aev:
            out["aev"] = aev
        if want_dEdG:
            out["dEdG"] = dG
        if want_dEdW:
            out["dEdW"] = dW
        return out

    def force_matching(self, coords, species, v, box=None, mask=None):
        """v = dL/dF [n,3].  Returns (energy, forces, dL/dcoords, dL/dweights)."""
        x = _f64(coords)
        n = x.shape[0]
        vv = _f64(v, (n, 3))
        F = np.zeros((n, 3))
        gx = np.zeros((n, 3))
        gw = np.zeros(self.n_weights)
        E = _load().oracle_force_matching(self._h, n, _ptr(x), _ptr(_u8(species)),
                                          _ptr(_f64(box)), _ptr(_u8(mask)), _ptr(vv),
                                          _ptr(F), _ptr(gx), _ptr(gw))
        return E, F, gx, gw

    def energy_forces_centres(self, coords, species, centres, box=None, mask=None):
        """Energy of the listed centres and the forces of their terms (a bounded sample
        of the full evaluation with the same work per centre)."""
        x = _f64(coords)
        n = x.shape[0]
        c = np.ascontiguousarray(centres, dtype=np.int32)
        F = np.zeros((n, 3))
        E = _load().oracle_energy_forces_centres(self._h, n, _ptr(x), _ptr(_u8(species)),
                                                 _ptr(_f64(box)), _ptr(_u8(mask)), c.shape[0],
                                                 _ptr(c), _ptr(F))
        return E, F

    def sample(self, coords, species, idx, box=None, mask=None, want_aev=False):
        """Per-atom energies, forces and (optionally) AEV rows of the atoms in idx."""
        x = _f64(coords)
        n = x.shape[0]
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        k = idx.shape[0]
        ae = np.zeros(k)
        F = np.zeros((k, 3))
        aev = np.zeros((k, self.D)) if want_aev else None
        _load().oracle_sample(self._h, n, _ptr(x), _ptr(_u8(species)), _ptr(_f64(box)),
                              _ptr(_u8(mask)), k, _ptr(idx), _ptr(ae), _ptr(F), _ptr(aev))
        return dict(atom_energies=ae, forces=F, aev=aev)


def neighbours(coords, rc, box=None, mask=None, method="brute"):
    """Directed neighbour pairs (i, j), i != j, R_ij <= rc, as an int32 [m, 2] array."""
    lib = _load()
    x = _f64(coords)
    n = x.shape[0]
    f = lib.oracle_neighbours_brute if method == "brute" else lib.oracle_neighbours_cells
    cnt = f(n, _ptr(x), _ptr(_f64(box)), _ptr(_u8(mask)), rc, 0, None)
    out = np.zeros((max(cnt, 1), 2), dtype=np.int32)
    cnt2 = f(n, _ptr(x), _ptr(_f64(box)), _ptr(_u8(mask)), rc, cnt, _ptr(out))
    assert cnt2 == cnt
    return out[:cnt]
