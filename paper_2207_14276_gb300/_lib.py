"""ctypes view of libnnp.so (declarations mirror include/nnp.h).

The shared library is built in-tree by ``paper_2207_14276_gb300.build``.  There
is no fallback: if the library is missing or cannot be loaded, every entry
point raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# NNP_DEBUG_BOUNDS=1 in the environment selects the bounds-checked build
DEBUG_BOUNDS = os.environ.get("NNP_DEBUG_BOUNDS", "0") not in ("", "0")
LIB_PATH = os.path.join(HERE, "libnnp_debug.so" if DEBUG_BOUNDS else "libnnp.so")

NNP_OK = 0
NNP_ERR_ARG = 1
NNP_ERR_SPECIES = 2
NNP_ERR_BOX_TOO_SMALL = 3
NNP_ERR_NONFINITE = 4
NNP_ERR_CAPACITY = 5
NNP_ERR_OOM = 6
NNP_ERR_CUDA = 7
NNP_ERR_TIMEOUT = 8
NNP_PENDING = 9
NNP_ERR_UNSUPPORTED = 10
NNP_ERR_BOUNDS = 11
NNP_BUILD_BOUNDS_CHECKS = 1
NNP_FP32 = 0
NNP_BF16_MLP = 1
NNP_FP32_SPLIT = 2
NNP_FP32_SIMT = 3
PRECISIONS = {"fp32": NNP_FP32, "bf16": NNP_BF16_MLP, "fp32_split": NNP_FP32_SPLIT,
              "fp32_simt": NNP_FP32_SIMT}

STATUS_NAMES = {
    0: "NNP_OK", 1: "NNP_ERR_ARG", 2: "NNP_ERR_SPECIES", 3: "NNP_ERR_BOX_TOO_SMALL",
    4: "NNP_ERR_NONFINITE", 5: "NNP_ERR_CAPACITY", 6: "NNP_ERR_OOM", 7: "NNP_ERR_CUDA",
    8: "NNP_ERR_TIMEOUT", 9: "NNP_PENDING", 10: "NNP_ERR_UNSUPPORTED", 11: "NNP_ERR_BOUNDS",
}

# every symbol include/nnp.h declares (checked by the CPU test-suite)
EXPORTS = (
    "nnp_create", "nnp_clone", "nnp_destroy", "nnp_reserve", "nnp_energy_forces",
    "nnp_energy_forces_batch", "nnp_energy_forces_host", "nnp_sync_status", "nnp_aev_dim",
    "nnp_last_launch_count", "nnp_last_error", "nnp_debug_rows", "nnp_debug_neighbors",
    "nnp_profile", "nnp_profile_read", "nnp_profile_stage_name", "nnp_energy_forces_noalloc",
    "nnp_server_create", "nnp_server_destroy", "nnp_server_register", "nnp_server_submit",
    "nnp_server_poll", "nnp_server_stats", "nnp_force_vjp_batch", "nnp_force_vjp",
    "nnp_n_weights", "nnp_debug_wait_probe", "nnp_set_skin", "nnp_list_stats",
    "nnp_integrate", "nnp_noalloc_max_atoms", "nnp_debug_cell_grid", "nnp_network_path",
    "nnp_set_fused_chain", "nnp_set_fused_aev_l1", "nnp_set_sparse_rows",
    "nnp_debug_tile_masks", "nnp_build_flags", "nnp_debug_check_index", "nnp_set_deterministic",
)


class NNPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class SpeciesT(ctypes.Structure):
    _fields_ = [("n_species", ctypes.c_int), ("atomic_numbers", ctypes.c_int * 8)]


class AevParamsT(ctypes.Structure):
    _fields_ = [("rc_r", ctypes.c_float), ("eta_r", ctypes.c_float), ("n_shf_r", ctypes.c_int),
                ("shf_r", ctypes.c_float * 32), ("rc_a", ctypes.c_float),
                ("eta_a", ctypes.c_float), ("zeta", ctypes.c_float), ("n_shf_a", ctypes.c_int),
                ("shf_a", ctypes.c_float * 16), ("n_shf_z", ctypes.c_int),
                ("shf_z", ctypes.c_float * 16), ("cos_scale", ctypes.c_float)]


class WeightsT(ctypes.Structure):
    _fields_ = [("n_ensemble", ctypes.c_int), ("n_layers", ctypes.c_int),
                ("widths", ctypes.POINTER(ctypes.c_int)), ("params", ctypes.POINTER(ctypes.c_float)),
                ("species_shift", ctypes.POINTER(ctypes.c_double)), ("celu_alpha", ctypes.c_float)]


class SystemT(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int64), ("coords", ctypes.c_void_p),
                ("species", ctypes.c_void_p), ("mask", ctypes.c_void_p),
                ("box", ctypes.c_double * 3), ("periodic", ctypes.c_int),
                ("energy", ctypes.c_void_p), ("forces", ctypes.c_void_p),
                ("virial", ctypes.c_void_p), ("atom_energies", ctypes.c_void_p)]


class VjpSystemT(ctypes.Structure):
    _fields_ = [("sys", SystemT), ("dL_dE", ctypes.c_double), ("dL_dF", ctypes.c_void_p),
                ("dL_dcoords", ctypes.c_void_p)]


class RequestT(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int64), ("coords", ctypes.c_void_p),
                ("species", ctypes.c_void_p), ("mask", ctypes.c_void_p),
                ("box", ctypes.c_double * 3), ("periodic", ctypes.c_int),
                ("resident_id", ctypes.c_int), ("energy", ctypes.c_void_p),
                ("forces", ctypes.c_void_p)]


_lib = None


def lib():
    """Load libnnp.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libnnp.so not found at {LIB_PATH}: run paper_2207_14276_gb300.build")
    L = ctypes.CDLL(LIB_PATH)
    P, i, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
    L.nnp_create.argtypes = [ctypes.POINTER(SpeciesT), ctypes.POINTER(AevParamsT),
                             ctypes.POINTER(WeightsT), i, sz, ctypes.POINTER(P)]
    L.nnp_clone.argtypes = [P, ctypes.POINTER(P)]
    L.nnp_destroy.argtypes = [P]
    L.nnp_destroy.restype = None
    L.nnp_reserve.argtypes = [P, i64, i, i, i]
    L.nnp_energy_forces.argtypes = [P, i64, P, P, P, P, P, P, P, P]
    L.nnp_energy_forces_batch.argtypes = [P, i, ctypes.POINTER(SystemT), P]
    L.nnp_energy_forces_host.argtypes = [P, i64, P, P, P, P, P, P, P]
    L.nnp_sync_status.argtypes = [P, P]
    L.nnp_aev_dim.argtypes = [P]
    L.nnp_build_flags.argtypes = []
    L.nnp_debug_check_index.argtypes = [i, i64, i64, ctypes.POINTER(i)]
    L.nnp_network_path.argtypes = [P]
    L.nnp_set_fused_chain.argtypes = [P, i]
    L.nnp_set_fused_aev_l1.argtypes = [P, i]
    L.nnp_set_sparse_rows.argtypes = [P, i]
    L.nnp_set_deterministic.argtypes = [P, i]
    L.nnp_debug_tile_masks.argtypes = [P, P, P, i, ctypes.POINTER(i)]
    L.nnp_last_launch_count.argtypes = [P]
    L.nnp_last_error.restype = ctypes.c_char_p
    L.nnp_last_error.argtypes = []
    L.nnp_debug_rows.argtypes = [P, i, P, P]
    L.nnp_debug_neighbors.argtypes = [P, i, i, P, P]
    L.nnp_energy_forces_noalloc.argtypes = [P, i64, P, P, P, P, P, P, P, P]
    L.nnp_noalloc_max_atoms.argtypes = [P, ctypes.POINTER(i64)]
    L.nnp_debug_cell_grid.argtypes = [P, ctypes.c_float, i64, P, ctypes.POINTER(i64)]
    L.nnp_server_create.argtypes = [P, i, i64, i, ctypes.POINTER(P)]
    L.nnp_server_destroy.argtypes = [P]
    L.nnp_server_destroy.restype = None
    L.nnp_server_register.argtypes = [P, i64, P, P, P, P, ctypes.POINTER(ctypes.c_int)]
    L.nnp_server_submit.argtypes = [P, ctypes.POINTER(RequestT), ctypes.POINTER(ctypes.c_uint64)]
    L.nnp_server_poll.argtypes = [P, ctypes.c_uint64, i, ctypes.POINTER(ctypes.c_double)]
    L.nnp_server_stats.argtypes = [P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
    L.nnp_force_vjp_batch.argtypes = [P, i, ctypes.POINTER(VjpSystemT), P, P]
    L.nnp_force_vjp.argtypes = [P, i64, P, P, P, P, ctypes.c_double, P, P, P, P, P, P]
    L.nnp_n_weights.argtypes = [P]
    L.nnp_n_weights.restype = i64
    L.nnp_debug_wait_probe.argtypes = [P, ctypes.c_uint, P]
    L.nnp_set_skin.argtypes = [P, ctypes.c_float]
    L.nnp_list_stats.argtypes = [P, P, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.nnp_integrate.argtypes = [i64, P, P, P, P, P, ctypes.c_float, ctypes.c_float, P, P]
    L.nnp_profile.argtypes = [P, i]
    L.nnp_profile_read.argtypes = [P, i, P, P, i, P]
    L.nnp_profile_stage_name.restype = ctypes.c_char_p
    L.nnp_profile_stage_name.argtypes = [i]
    _lib = L
    return L


def check(code):
    if code != NNP_OK:
        raise NNPError(code, lib().nnp_last_error().decode())
    return code
