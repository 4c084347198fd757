"""The allocation-free entry point, nnp_energy_forces_noalloc.

Some callers cannot let a library allocate device memory while they run: an MD
engine that has reserved the whole HBM budget for itself, or a time loop where
a cudaMalloc/cudaFree would stall the device.  For them the library offers one
call that takes its work space from a fixed device array built into the library
instead of allocating it.  This test calls that entry point through the C ABI
twice in a row (a periodic water box, then a small gas-phase molecule, so the
second call reuses the array the first one filled) and checks each result
against the ordinary nnp_energy_forces entry point with the tolerances of the
other parity tests, and against the FP64 oracle.  It also checks the call's
refusals: a request beyond the array (the limit nnp_noalloc_max_atoms reports is
accepted, one atom more is not), an atom with more neighbours than the fixed
lists hold, and a BF16 handle.  The file is named so that pytest collects it
last.
"""
import ctypes

import numpy as np
import pytest

import oracle
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
    orc = oracle.Model(spec, w)
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
        # and against the FP64 oracle (the FP32 bar of the parity tests)
        ref = orc.energy_forces(s.coords, s.species, s.box)
        assert abs(float(E.cpu()[0]) - ref["energy"]) <= E_TOL
        d = f - ref["forces"]
        assert float(np.sqrt(np.mean(d * d))) <= 1e-4 * float(np.sqrt(np.mean(ref["forces"] ** 2))) + 1e-7


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


def test_noalloc_limit_is_the_reported_one(torch_cuda):
    """nnp_noalloc_max_atoms gives the largest accepted atom count: a cluster of
    exactly that many atoms (cut from a water box, non-periodic) runs, one more is
    refused with NNP_ERR_ARG before any work."""
    torch = torch_cuda
    from paper_2207_14276_gb300 import Potential
    from paper_2207_14276_gb300._lib import NNP_ERR_ARG, lib
    spec, w = model_for("ani4")
    pot = Potential(spec, w)
    lim = ctypes.c_int64()
    assert lib().nnp_noalloc_max_atoms(pot._h, ctypes.byref(lim)) == 0
    n = lim.value
    assert 6000 < n < 8000                 # about 6,900 for this network
    s = synth.workload("water9000")[0][0]
    assert n + 1 <= s.n_atoms
    for k, want in ((n, 0), (n + 1, NNP_ERR_ARG)):
        x = torch.from_numpy(np.ascontiguousarray(s.coords[:k])).cuda()
        sp = torch.from_numpy(np.ascontiguousarray(s.species[:k])).cuda()
        E = torch.zeros(1, dtype=torch.float64, device="cuda")
        F = torch.zeros((k, 3), dtype=torch.float32, device="cuda")
        rc = _noalloc(pot, x, sp, None, E, F, None)
        assert rc == want, (k, rc, lib().nnp_last_error().decode())


def test_noalloc_refuses_overfull_lists_and_bf16(torch_cuda):
    """A box at about eleven times liquid density fits the array but gives atoms
    more than 96 angular (and 256 radial) neighbours: NNP_ERR_CAPACITY with a
    message naming the fixed lists.  A BF16 handle: NNP_ERR_UNSUPPORTED."""
    torch = torch_cuda
    from paper_2207_14276_gb300 import Potential
    from paper_2207_14276_gb300._lib import NNP_ERR_CAPACITY, NNP_ERR_UNSUPPORTED, lib
    spec, w = model_for("ani4")
    pot = Potential(spec, w)
    s = synth.water_box(1000, 14.0, 10, seed=23)
    x = torch.from_numpy(s.coords).cuda()
    sp = torch.from_numpy(s.species).cuda()
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    F = torch.zeros((s.n_atoms, 3), dtype=torch.float32, device="cuda")
    rc = _noalloc(pot, x, sp, None, E, F, None)
    assert rc == NNP_ERR_CAPACITY
    assert "neighbours" in lib().nnp_last_error().decode()
    pb = Potential(spec, w, precision="bf16")
    rc = _noalloc(pb, x[:24], sp[:24], None, E, F, None)
    assert rc == NNP_ERR_UNSUPPORTED
