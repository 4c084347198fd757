"""Force-matching gradients (the double backward) against the FP64 oracle and
finite differences.

Workload: 64 random 4-species molecules of 20-60 atoms, F_target ~ N(0, 1
kcal/mol/A), loss L = sum (F - F_target)^2, gradients w.r.t. every network
weight and every coordinate through torch.autograd with the library's
hand-written backward.  FP32 bound: the gradients are sums of many FP32 products
(relative rounding ~1e-6 per term), so elements must agree with the FP64 oracle
within 1e-3 of the gradient's largest magnitude and within 1e-3 relative in
norm.  Central differences (h = 1e-4 A for coordinates, scaled for weights) of
the FP32 loss carry ~1e-7/h relative noise, so they are checked to 2%.
"""
import numpy as np
import pytest

import oracle
import synth
from tests._common import model_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def _norm_close(a, b, rel=1e-3):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    assert np.linalg.norm(a - b) <= rel * np.linalg.norm(b) + 1e-12
    np.testing.assert_allclose(a, b, atol=rel * np.abs(b).max() + 1e-12)


@pytest.mark.parametrize("precision", ["fp32", "fp32_simt"])
def test_force_matching_batch_matches_oracle(torch_cuda, precision):
    # an "fp32" handle runs its energy calls on the tensor cores (split operands)
    # and the VJP's networks in FP32; a "fp32_simt" handle both in FP32; both must
    # give the oracle's gradients
    torch = torch_cuda
    from paper_2207_14276_gb300 import Potential
    from paper_2207_14276_gb300.autograd import NNPBatchFunction
    spec, w = model_for("ani4")
    pot = Potential(spec, w, precision=precision)
    mols, _, _ = synth.workload("molecules64")
    rng = np.random.Generator(np.random.PCG64(4))
    targets = [rng.normal(0.0, 1.0, size=(m.n_atoms, 3)) for m in mols]
    sizes = [m.n_atoms for m in mols]
    x = torch.from_numpy(np.concatenate([m.coords for m in mols])).cuda().requires_grad_(True)
    sp = torch.from_numpy(np.concatenate([m.species for m in mols])).cuda()
    wt = torch.from_numpy(w).cuda().requires_grad_(True)
    Ft = torch.from_numpy(np.concatenate(targets)).float().cuda()
    E, F = NNPBatchFunction.apply(x, wt, pot, sp, sizes)
    loss = ((F - Ft) ** 2).sum()
    loss.backward()
    gx = x.grad.cpu().numpy()
    gw = wt.grad.cpu().numpy()
    orc = oracle.Model(spec, w)
    gw_ref = np.zeros(w.size)
    gx_ref = []
    for m, t in zip(mols, targets):
        Fm = orc.energy_forces(m.coords, m.species)["forces"]
        _, _, gxm, gwm = orc.force_matching(m.coords, m.species, 2 * (Fm - t))
        gw_ref += gwm
        gx_ref.append(gxm)
    gx_ref = np.concatenate(gx_ref)
    _norm_close(gx, gx_ref)
    _norm_close(gw, gw_ref)


def test_energy_and_force_gradients_periodic(torch_cuda):
    """dL/dE != 0 and a periodic box: L = 0.5 E + sum v.F with fixed v."""
    torch = torch_cuda
    from paper_2207_14276_gb300 import Potential
    from paper_2207_14276_gb300.autograd import NNPFunction
    spec, w = model_for("ani4")
    pot = Potential(spec, w)
    s = synth.water_box(100, 14.5, 5, seed=61)
    rng = np.random.Generator(np.random.PCG64(5))
    v = rng.normal(size=(s.n_atoms, 3))
    x = torch.from_numpy(s.coords).cuda().requires_grad_(True)
    wt = torch.from_numpy(w).cuda().requires_grad_(True)
    E, F = NNPFunction.apply(x, wt, pot, torch.from_numpy(s.species).cuda(), list(s.box))
    loss = 0.5 * E.sum() + (F * torch.from_numpy(v).float().cuda()).sum()
    loss.backward()
    orc = oracle.Model(spec, w)
    r = orc.energy_forces(s.coords, s.species, s.box, want_dEdW=True)
    _, _, gx, gwv = orc.force_matching(s.coords, s.species, v, s.box)
    _norm_close(x.grad.cpu().numpy(), gx - 0.5 * r["forces"])
    _norm_close(wt.grad.cpu().numpy(), gwv + 0.5 * r["dEdW"])


def test_force_matching_central_differences(torch_cuda):
    torch = torch_cuda
    from paper_2207_14276_gb300 import Potential
    spec, w = model_for("ani4")
    mols, _, _ = synth.workload("molecules64")
    mols = mols[:6]
    rng = np.random.Generator(np.random.PCG64(6))
    targets = [rng.normal(0.0, 1.0, size=(m.n_atoms, 3)) for m in mols]

    def loss_and_grads(wv, coords_list, grads=False):
        # FP32 FMA networks: central differences need a loss that is smooth at
        # FP32 resolution (split BF16 operands would round the perturbed weight)
        pot = Potential(spec, wv, precision="fp32_simt")
        systems = [{"coords": torch.from_numpy(c.astype(np.float32)).cuda(),
                    "species": torch.from_numpy(m.species).cuda()} for c, m in zip(coords_list, mols)]
        outs = pot.energy_forces_batch(systems)
        F = [o["forces"].double().cpu().numpy() for o in outs]
        L = sum(float(((f - t) ** 2).sum()) for f, t in zip(F, targets))
        if not grads:
            return L
        v = [torch.from_numpy(2 * (f - t)).float().cuda() for f, t in zip(F, targets)]
        _, _, G, W = pot.force_vjp_batch(systems, [0.0] * len(mols), v)
        return L, [g.cpu().numpy() for g in G], W.cpu().numpy()

    coords = [m.coords.astype(np.float64) for m in mols]
    L0, gx, gw = loss_and_grads(w, coords, grads=True)
    # coordinates with the largest gradients
    flat = np.concatenate([g.ravel() for g in gx])
    for idx in np.argsort(-np.abs(flat))[:6]:
        mi = np.searchsorted(np.cumsum([g.size for g in gx]), idx, side="right")
        off = idx - sum(g.size for g in gx[:mi])
        a, c = divmod(off, 3)
        h = 1e-3
        cp = [x.copy() for x in coords]; cp[mi][a, c] += h
        cm = [x.copy() for x in coords]; cm[mi][a, c] -= h
        fd = (loss_and_grads(w, cp) - loss_and_grads(w, cm)) / (2 * h)
        assert fd == pytest.approx(flat[idx], rel=2e-2)
    # weights with the largest gradients
    for k in np.argsort(-np.abs(gw))[:6]:
        h = 1e-3 * max(abs(float(w[k])), 1e-2)
        wp = w.copy(); wp[k] += h
        wm = w.copy(); wm[k] -= h
        fd = (loss_and_grads(wp, coords) - loss_and_grads(wm, coords)) / (2 * h)
        assert fd == pytest.approx(gw[k], rel=2e-2)


def test_vjp_against_fp64_central_differences(torch_cuda):
    """The library's force-matching gradient against central differences (h = 1e-4,
    the step the differentiation workload specifies) of the same loss evaluated
    by the FP64 oracle's energy and forces -- an FD reference independent of the
    oracle's dual-number gradient and free of FP32 noise.  Every coordinate of
    one molecule and 40 weights (the 16 largest gradients and 24 drawn at
    random): within 1e-3 of the largest gradient of each kind."""
    torch = torch_cuda
    from paper_2207_14276_gb300 import Potential
    from paper_2207_14276_gb300.autograd import NNPBatchFunction
    spec, w = model_for("ani4")
    orc = oracle.Model(spec, w)
    mols, _, _ = synth.workload("molecules64")
    mols = mols[:4]
    rng = np.random.Generator(np.random.PCG64(8))
    targets = [rng.normal(0.0, 1.0, size=(m.n_atoms, 3)) for m in mols]
    sizes = [m.n_atoms for m in mols]
    pot = Potential(spec, w)
    x = torch.from_numpy(np.concatenate([m.coords for m in mols])).cuda().requires_grad_(True)
    sp = torch.from_numpy(np.concatenate([m.species for m in mols])).cuda()
    wt = torch.from_numpy(w).cuda().requires_grad_(True)
    Ft = torch.from_numpy(np.concatenate(targets)).float().cuda()
    E, F = NNPBatchFunction.apply(x, wt, pot, sp, sizes)
    ((F - Ft) ** 2).sum().backward()
    gx = x.grad.double().cpu().numpy()
    gw = wt.grad.double().cpu().numpy()

    def loss(model, coords):
        return sum(float(((model.energy_forces(c, m.species)["forces"] - t) ** 2).sum())
                   for c, m, t in zip(coords, mols, targets))

    h = 1e-4
    base = [m.coords.astype(np.float64) for m in mols]
    fdx = []
    for mi in (0,):
        for a in range(mols[mi].n_atoms):
            for c in range(3):
                cp = [b.copy() for b in base]; cp[mi][a, c] += h
                cm = [b.copy() for b in base]; cm[mi][a, c] -= h
                fdx.append((loss(orc, cp) - loss(orc, cm)) / (2 * h))
    n0 = mols[0].n_atoms
    np.testing.assert_allclose(gx[:n0].reshape(-1), np.array(fdx), atol=1e-3 * np.abs(fdx).max())
    ks = np.concatenate([np.argsort(-np.abs(gw))[:16], rng.choice(w.size, 24, replace=False)])
    fdw = []
    for k in ks:
        wp = w.astype(np.float64).copy(); wp[k] += h
        wm = w.astype(np.float64).copy(); wm[k] -= h
        fdw.append((loss(oracle.Model(spec, wp), base) - loss(oracle.Model(spec, wm), base)) / (2 * h))
    np.testing.assert_allclose(gw[ks], np.array(fdw), atol=1e-3 * np.abs(gw).max())
