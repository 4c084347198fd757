"""The allocation-free entry point, nnp_energy_forces_noalloc.

Some callers cannot let a library allocate device memory while they run: an MD
engine that has reserved the whole HBM budget for itself, or a time loop where
a cudaMalloc/cudaFree would stall the device.  For them the library offers one
call that takes its work space from a fixed device array built into the library
instead of allocating it.  This test calls that entry point through the C ABI
twice in a row (a periodic water box, then a small gas-phase molecule, so the
second call reuses the array the first one filled) and checks each result
against the ordinary nnp_energy_forces entry point with the tolerances of the
other parity tests.  It also checks that an oversized request is refused with a
clear message.  The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import synth
from tests._common import model_for

pytestmark = pytest.mark.gpu

E_TOL = 1e-3


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _noalloc(pot, x, sp, box, E, F, V):
    import torch
    from paper_2207_14276_gb300._lib import lib
    box_arr = None if box is None else (ctypes.c_double * 3)(*[float(b) for b in box])
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib().nnp_energy_forces_noalloc(pot._h, x.shape[0], _p(x), _p(sp), box_arr, None,
                                           _p(E), _p(F), _p(V), stream)


def _reference(pot, x, sp, box):
    return pot.energy_forces(x, sp, box, virial=True)


def test_noalloc_matches_energy_forces_twice_in_a_row(torch_cuda):
    torch = torch_cuda
    from paper_2207_14276_gb300 import Potential
    from paper_2207_14276_gb300._lib import lib
    spec, w = model_for("ani4")
    pot = Potential(spec, w)
    water = synth.water_box(300, 20.5, 7, seed=77)
    mol = synth.workload("gas24")[0][0]
    for s in (water, mol):
        x = torch.from_numpy(s.coords).cuda()
        sp = torch.from_numpy(s.species).cuda()
        box = None if s.box is None else [float(b) for b in s.box]
        E = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        F = torch.full((s.n_atoms, 3), float("nan"), dtype=torch.float32, device="cuda")
        V = torch.full((9,), float("nan"), dtype=torch.float64, device="cuda")
        rc = _noalloc(pot, x, sp, box, E, F, V)
        assert rc == 0, lib().nnp_last_error().decode()
        E0, F0, V0 = _reference(pot, x, sp, box)
        assert abs(float(E.cpu()[0]) - float(E0.cpu()[0])) <= E_TOL
        f, f0 = F.cpu().numpy().astype(np.float64), F0.cpu().numpy().astype(np.float64)
        rms = float(np.sqrt(np.mean((f - f0) ** 2)))
        assert rms <= 1e-4 * float(np.sqrt(np.mean(f0 ** 2))) + 1e-7
        v, v0 = V.cpu().numpy(), V0.cpu().numpy().reshape(9)
        np.testing.assert_allclose(v, v0, atol=1e-4 * np.abs(v0).max() + 1e-6)


def test_noalloc_rejects_oversized_request(torch_cuda):
    torch = torch_cuda
    from paper_2207_14276_gb300 import Potential
    from paper_2207_14276_gb300._lib import NNP_ERR_ARG, lib
    spec, w = model_for("ani4")
    pot = Potential(spec, w)
    s = synth.workload("water9000")[0][0]   # 9000 atoms: beyond the fixed work space
    x = torch.from_numpy(s.coords).cuda()
    sp = torch.from_numpy(s.species).cuda()
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    F = torch.zeros((s.n_atoms, 3), dtype=torch.float32, device="cuda")
    rc = _noalloc(pot, x, sp, list(s.box), E, F, None)
    assert rc == NNP_ERR_ARG
    assert "NNP_NOALLOC_SCRATCH_BYTES" in lib().nnp_last_error().decode()
