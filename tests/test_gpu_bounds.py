"""The bounds-checked build (libnnp_debug.so, NNP_DEBUG_BOUNDS=1) on the GPU.

Its kernels check the indexes of the neighbour lists, packed positions, AEV
rows, force targets, triplet slots and GEMM output rows before they use them
(compute-sanitizer is not available, so this build stands in for a memory
checker).  Run in a child process, since the build is chosen when the package
loads: every workload shape of the other tests (gas batches, periodic water,
dense solute centres on the CTA-per-centre backward, the 7-species ensemble on
the split and BF16 tensor-core paths, persistent lists, the allocation-free
entry point) must finish without a failed check and agree with the FP64 oracle.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import torch
import oracle, synth
from paper_2207_14276_gb300 import Potential, _lib
from tests._common import force_errors, model_for, to_cuda

assert _lib.LIB_PATH.endswith("libnnp_debug.so"), _lib.LIB_PATH
assert _lib.lib().nnp_build_flags() == _lib.NNP_BUILD_BOUNDS_CHECKS

def agree(outs, systems, orc, bf16=False):
    for o, s in zip(outs, systems):
        ref = orc.energy_forces(s.coords, s.species, s.box, s.mask)
        e = float(o["energy"].cpu()[0])
        rms, _ = force_errors(o["forces"].cpu().numpy(), ref["forces"])
        f_rms = float(np.sqrt(np.mean(ref["forces"] ** 2)))
        e_tol = 2e-3 * float(np.abs(ref["atom_energies"]).sum()) + 1e-4 if bf16 else 1e-3
        assert abs(e - ref["energy"]) <= e_tol, (s.name, e, ref["energy"])
        assert rms <= (2e-2 if bf16 else 1e-4) * f_rms + 1e-6, (s.name, rms, f_rms)

cases = [
    ("ani4", "fp32_simt", [synth.water_box(300, 20.5, 7, seed=41)] +
     list(synth.workload("molecules64")[0][:8])),
    ("ani4", "fp32_split", [synth.water_box(500, 24.0, 8, seed=51)]),
    ("ani7", "fp32_split", [synth.solvated_solute(300, 200, 22.0, seed=17)]),
    ("ani7", "fp32_simt", [synth.solvated_solute(300, 200, 22.0, seed=17)]),
    ("ani7x8", "bf16", [synth.solvated_solute(150, 60, 18.0, seed=6)]),
    ("ani7x8", "fp32_split", [synth.solvated_solute(150, 60, 18.0, seed=6)]),
]
for kind, prec, systems in cases:
    spec, w = model_for(kind)
    pot = Potential(spec, w, precision=prec)
    orc = oracle.Model(spec, w)
    for rep in range(2):   # the second call replays a captured graph
        outs = pot.energy_forces_batch([to_cuda(s) for s in systems], virial=True)
        agree(outs, systems, orc, bf16=(prec == "bf16"))
    print(kind, prec, "ok", flush=True)

# persistent lists with a skin along a short trajectory
spec, w = model_for("ani4")
pot = Potential(spec, w, precision="fp32_simt")
pot.set_skin(1.0)
orc = oracle.Model(spec, w)
s = synth.water_box(300, 20.5, 7, seed=41)
rng = np.random.Generator(np.random.PCG64(3))
x = s.coords.copy()
for step in range(4):
    x = (x + rng.normal(0.0, 0.02, x.shape)).astype(np.float32)
    s2 = synth.System(s.name, x, s.species, s.box, s.mask)
    agree(pot.energy_forces_batch([to_cuda(s2)]), [s2], orc)
print("skin ok", flush=True)

# the allocation-free entry point
import ctypes
pot = Potential(spec, w, precision="fp32_simt")
d = to_cuda(s)
E = torch.zeros(1, dtype=torch.float64, device="cuda")
F = torch.zeros((s.n_atoms, 3), dtype=torch.float32, device="cuda")
ptr = lambda t: ctypes.c_void_p(t.data_ptr())
box = (ctypes.c_double * 3)(*[float(b) for b in s.box])
stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
rc = _lib.lib().nnp_energy_forces_noalloc(pot._h, s.n_atoms, ptr(d["coords"]), ptr(d["species"]),
                                          box, None, ptr(E), ptr(F), None, stream)
assert rc == 0, _lib.lib().nnp_last_error().decode()
torch.cuda.synchronize()
ref = orc.energy_forces(s.coords, s.species, s.box)
assert abs(float(E.cpu()[0]) - ref["energy"]) <= 1e-3
rms, _ = force_errors(F.cpu().numpy(), ref["forces"])
assert rms <= 1e-4 * float(np.sqrt(np.mean(ref["forces"] ** 2))) + 1e-6
print("noalloc ok", flush=True)
"""


def test_bounds_checked_build_runs_every_path_clean():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    env = dict(os.environ, NNP_DEBUG_BOUNDS="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    print(r.stdout[-3000:], r.stderr[-3000:])
    assert r.returncode == 0
    assert "noalloc ok" in r.stdout
