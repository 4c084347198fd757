"""Python binding of the C ABI (argument marshalling only).

Every step of the energy/force evaluation runs in libnnp's CUDA kernels; torch
only allocates device memory and supplies the CUDA stream.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import check, lib


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Potential:
    """ANI-style neural-network potential on one GPU.

    spec: an object with ``aev`` (n_species, rc_r, eta_r, shf_r, rc_a, eta_a, zeta,
    shf_a, shf_z, cos_scale), ``widths``, ``n_ensemble``, ``celu_alpha`` and
    ``atomic_numbers``; weights: flat float32 vector (layout of include/nnp.h).
    precision: "fp32" (FP32-accurate: network layers on the tensor cores with
    split BF16 operands, the same as "fp32_split"), "fp32_simt" (network layers
    on the FP32 FMA pipes), or "bf16" (tensor-core layers on BF16 operands).
    """

    def __init__(self, spec, weights, precision="fp32", shift=None, hbm_budget=0, _clone_of=None):
        L = lib()
        self.spec = spec
        self.precision = precision
        h = ctypes.c_void_p()
        if _clone_of is not None:
            check(L.nnp_clone(_clone_of._h, ctypes.byref(h)))
        else:
            p = spec.aev
            sp = _lib.SpeciesT()
            sp.n_species = p.n_species
            for k, z in enumerate(spec.atomic_numbers):
                sp.atomic_numbers[k] = z
            ap = _lib.AevParamsT()
            ap.rc_r, ap.eta_r, ap.n_shf_r = p.rc_r, p.eta_r, len(p.shf_r)
            for k, v in enumerate(p.shf_r):
                ap.shf_r[k] = v
            ap.rc_a, ap.eta_a, ap.zeta, ap.n_shf_a = p.rc_a, p.eta_a, p.zeta, len(p.shf_a)
            for k, v in enumerate(p.shf_a):
                ap.shf_a[k] = v
            ap.n_shf_z = len(p.shf_z)
            for k, v in enumerate(p.shf_z):
                ap.shf_z[k] = v
            ap.cos_scale = p.cos_scale
            widths = (ctypes.c_int * len(spec.widths))(*spec.widths)
            w = np.ascontiguousarray(weights, dtype=np.float32)
            shift_arr = None if shift is None else np.ascontiguousarray(shift, dtype=np.float64)
            wt = _lib.WeightsT()
            wt.n_ensemble = spec.n_ensemble
            wt.n_layers = len(spec.widths) - 1
            wt.widths = widths
            wt.params = w.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
            wt.species_shift = (None if shift_arr is None
                                else shift_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
            wt.celu_alpha = spec.celu_alpha
            if precision not in _lib.PRECISIONS:
                raise ValueError(f"precision must be one of {sorted(_lib.PRECISIONS)}")
            prec = _lib.PRECISIONS[precision]
            check(L.nnp_create(ctypes.byref(sp), ctypes.byref(ap), ctypes.byref(wt), prec,
                               hbm_budget, ctypes.byref(h)))
        self._h = h
        self.D = L.nnp_aev_dim(h)

    def clone(self):
        """Second handle on the same device weights with its own work arena."""
        return Potential(self.spec, None, self.precision, _clone_of=self)

    def close(self):
        if getattr(self, "_h", None):
            lib().nnp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ calls
    def reserve(self, max_atoms, max_systems=1, max_neighbors_radial=0, max_neighbors_angular=0):
        check(lib().nnp_reserve(self._h, int(max_atoms), int(max_systems),
                                int(max_neighbors_radial), int(max_neighbors_angular)))

    def sync_status(self, stream=None):
        return lib().nnp_sync_status(self._h, _stream_ptr(stream))

    def set_fused_chain(self, enable):
        """Tensor-core paths: run L2, L3, B3 and B2 as one fused kernel (default)
        or as four layer GEMMs."""
        check(lib().nnp_set_fused_chain(self._h, 1 if enable else 0))

    def set_deterministic(self, enable):
        """Bitwise repeatable energies, forces and virials (sorted atom order,
        fixed-order sums of per-contribution slots); slower, more memory."""
        check(lib().nnp_set_deterministic(self._h, 1 if enable else 0))

    def set_sparse_rows(self, enable):
        """Tensor-core paths: write and multiply only the live 64-column slices of
        the AEV rows (default on; the result is the same)."""
        check(lib().nnp_set_sparse_rows(self._h, 1 if enable else 0))

    def tile_masks(self, max_tiles=1 << 20, stream=None):
        """Live 64-column slice masks of the last call's 128-row AEV tiles (numpy
        uint32; empty when the last call wrote whole rows)."""
        out = np.zeros(max_tiles, dtype=np.uint32)
        n = ctypes.c_int()
        check(lib().nnp_debug_tile_masks(self._h, _stream_ptr(stream),
                                         out.ctypes.data_as(ctypes.c_void_p), max_tiles,
                                         ctypes.byref(n)))
        return out[:n.value]

    def set_fused_aev_l1(self, enable):
        """BF16 one-network models: compute the AEV on chip and feed it to the first
        layer in the same kernel (the AEV never goes to HBM)."""
        check(lib().nnp_set_fused_aev_l1(self._h, 1 if enable else 0))

    def network_path(self):
        """'fp32_split', 'fp32_simt' or 'bf16': the path this handle's networks run."""
        code = lib().nnp_network_path(self._h)
        return {v: k for k, v in _lib.PRECISIONS.items()}[code]

    def launch_count(self):
        return lib().nnp_last_launch_count(self._h)

    def set_skin(self, skin):
        """Keep neighbour lists between calls, rebuilt once an atom has moved more
        than skin/2 A since the last build (0 disables)."""
        check(lib().nnp_set_skin(self._h, float(skin)))

    def list_stats(self, stream=None):
        """(list builds, calls made with a skin) since the skin was set."""
        b, c = ctypes.c_int64(), ctypes.c_int64()
        check(lib().nnp_list_stats(self._h, _stream_ptr(stream), ctypes.byref(b), ctypes.byref(c)))
        return b.value, c.value

    def energy_forces_into(self, coords, species, box, mask, energy, forces, virial=None,
                           stream=None):
        """Asynchronous call on preallocated device tensors (no synchronisation)."""
        n = coords.shape[0]
        box_arr = None
        if box is not None:
            box_arr = (ctypes.c_double * 3)(*[float(x) for x in box])
        check(lib().nnp_energy_forces(self._h, n, _ptr(coords), _ptr(species), box_arr,
                                      _ptr(mask), _ptr(energy), _ptr(forces), _ptr(virial),
                                      _stream_ptr(stream)))

    def energy_forces(self, coords, species, box=None, mask=None, virial=False, stream=None,
                      check_status=True):
        """coords: cuda float32 [n,3]; species: cuda uint8 [n]; box: 3 floats or None;
        mask: cuda uint8 [n] or None.  Returns (energy float64 [1], forces [n,3][, virial])."""
        dev = coords.device
        n = coords.shape[0]
        E = torch.empty(1, dtype=torch.float64, device=dev)
        F = torch.empty((n, 3), dtype=torch.float32, device=dev)
        V = torch.empty(9, dtype=torch.float64, device=dev) if virial else None
        for attempt in range(2):
            self.energy_forces_into(coords, species, box, mask, E, F, V, stream)
            if not check_status:
                break
            rc = self.sync_status(stream)
            if rc == _lib.NNP_ERR_CAPACITY and attempt == 0:
                continue
            check(rc)
            break
        return (E, F, V.view(3, 3)) if virial else (E, F)

    def energy_forces_batch(self, systems, stream=None, check_status=True, atom_energies=False,
                            virial=False, outputs=None, forces=True):
        """systems: list of dicts with coords, species, optional box and mask (cuda tensors).
        Returns a list of dicts with energy [1], forces [n,3] (and virial / atom energies)."""
        L = lib()
        n_sys = len(systems)
        arr = (_lib.SystemT * max(n_sys, 1))()
        outs = outputs
        if outs is None:
            outs = []
            for s in systems:
                dev = s["coords"].device
                n = s["coords"].shape[0]
                o = {"energy": torch.empty(1, dtype=torch.float64, device=dev)}
                if forces:
                    o["forces"] = torch.empty((n, 3), dtype=torch.float32, device=dev)
                if virial:
                    o["virial"] = torch.empty(9, dtype=torch.float64, device=dev)
                if atom_energies:
                    o["atom_energies"] = torch.empty(n, dtype=torch.float32, device=dev)
                outs.append(o)
        for k, (s, o) in enumerate(zip(systems, outs)):
            d = arr[k]
            d.n_atoms = s["coords"].shape[0]
            d.coords = s["coords"].data_ptr()
            d.species = s["species"].data_ptr()
            d.mask = s["mask"].data_ptr() if s.get("mask") is not None else None
            box = s.get("box")
            d.periodic = 1 if box is not None else 0
            if box is not None:
                for c in range(3):
                    d.box[c] = float(box[c])
            d.energy = o["energy"].data_ptr()
            d.forces = o["forces"].data_ptr() if "forces" in o else None
            d.virial = o["virial"].data_ptr() if "virial" in o else None
            d.atom_energies = o["atom_energies"].data_ptr() if "atom_energies" in o else None
        for attempt in range(2):
            check(L.nnp_energy_forces_batch(self._h, n_sys, arr, _stream_ptr(stream)))
            if not check_status:
                break
            rc = self.sync_status(stream)
            if rc == _lib.NNP_ERR_CAPACITY and attempt == 0:
                continue
            check(rc)
            break
        return outs

    def energy_forces_host(self, coords, species, box=None, mask=None, virial=False):
        """Host numpy arrays in and out; copies and synchronisation inside the library."""
        x = np.ascontiguousarray(coords, dtype=np.float32)
        sp = np.ascontiguousarray(species, dtype=np.uint8)
        m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        return self.energy_forces_host_into(x, sp, box, m, virial)

    def energy_forces_host_into(self, x, sp, box, m, virial=False, out_forces=None):
        n = x.shape[0]
        E = np.zeros(1, dtype=np.float64)
        F = out_forces if out_forces is not None else np.empty((n, 3), dtype=np.float32)
        V = np.zeros(9, dtype=np.float64) if virial else None
        box_arr = None if box is None else (ctypes.c_double * 3)(*[float(b) for b in box])
        vp = lambda a: None if a is None else a.ctypes.data   # plain address
        check(lib().nnp_energy_forces_host(self._h, n, vp(x), vp(sp), box_arr, vp(m), vp(E),
                                           vp(F), vp(V)))
        return (E[0], F, V.reshape(3, 3)) if virial else (E[0], F)

    @property
    def n_weights(self):
        return lib().nnp_n_weights(self._h)

    def force_vjp_batch(self, systems, dL_dE, dL_dF, stream=None):
        """Vector-Jacobian product of (E, F) for a batch (FP32 handles).
        systems: list of dicts (coords, species, box, mask) of cuda tensors; dL_dE: per-system
        floats; dL_dF: list of cuda float32 [n,3].  Returns (energies [n_sys] float64,
        forces list, dL/dcoords list, dL/dweights flat float32)."""
        n_sys = len(systems)
        arr = (_lib.VjpSystemT * n_sys)()
        dev = systems[0]["coords"].device
        E = torch.empty(n_sys, dtype=torch.float64, device=dev)
        Fs, Gs, keep = [], [], []
        for k, s in enumerate(systems):
            n = s["coords"].shape[0]
            F = torch.empty((n, 3), dtype=torch.float32, device=dev)
            G = torch.empty((n, 3), dtype=torch.float32, device=dev)
            v = dL_dF[k].contiguous().float()
            keep.append(v)
            d = arr[k]
            d.sys.n_atoms = n
            d.sys.coords = s["coords"].data_ptr()
            d.sys.species = s["species"].data_ptr()
            d.sys.mask = s["mask"].data_ptr() if s.get("mask") is not None else None
            box = s.get("box")
            d.sys.periodic = 1 if box is not None else 0
            if box is not None:
                for c in range(3):
                    d.sys.box[c] = float(box[c])
            d.sys.energy = E.data_ptr() + 8 * k
            d.sys.forces = F.data_ptr()
            d.dL_dE = float(dL_dE[k])
            d.dL_dF = v.data_ptr()
            d.dL_dcoords = G.data_ptr()
            Fs.append(F)
            Gs.append(G)
        W = torch.empty(self.n_weights, dtype=torch.float32, device=dev)
        for attempt in range(2):
            check(lib().nnp_force_vjp_batch(self._h, n_sys, arr, _ptr(W), _stream_ptr(stream)))
            rc = self.sync_status(stream)
            if rc == _lib.NNP_ERR_CAPACITY and attempt == 0:
                continue
            check(rc)
            break
        return E, Fs, Gs, W

    def profile(self, enable=True):
        check(lib().nnp_profile(self._h, 1 if enable else 0))

    def profile_read(self, reset=True):
        """{stage: (total_ms, n_event_pairs)} of the calls recorded since the last reset."""
        L = lib()
        ms = (ctypes.c_double * 32)()
        calls = (ctypes.c_longlong * 32)()
        n = ctypes.c_int()
        check(L.nnp_profile_read(self._h, 1 if reset else 0, ms, calls, 32, ctypes.byref(n)))
        return {L.nnp_profile_stage_name(i).decode(): (ms[i], calls[i]) for i in range(n.value)}

    # ------------------------------------------------------------------ diagnostics
    def debug_rows(self, which, n_atoms, device="cuda"):
        """AEV (which=0) or dE/dG (which=1) rows of the last call, input atom order."""
        out = torch.zeros((n_atoms, self.D), dtype=torch.float32, device=device)
        check(lib().nnp_debug_rows(self._h, which, _ptr(out), _stream_ptr(None)))
        torch.cuda.synchronize()
        return out

    def debug_neighbors(self, n_atoms, angular=False, cap=512, device="cuda"):
        out = torch.full((n_atoms, cap), -1, dtype=torch.int32, device=device)
        check(lib().nnp_debug_neighbors(self._h, 1 if angular else 0, cap, _ptr(out),
                                        _stream_ptr(None)))
        torch.cuda.synchronize()
        return out
