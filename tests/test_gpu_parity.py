"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (FP32 path): energy within 1e-3 kcal/mol and force RMS error within
1e-3 kcal/mol/A of the oracle (the stated FP32 bar), plus relative bounds that
FP32 arithmetic meets with margin: force RMS error <= 1e-4 of the force RMS and
AEV elements within 2e-5 relative (+1e-6 absolute).  Neighbour lists are
compared as sets (index work: exact), except for pairs within 1e-4 A of the
cutoff where FP32 and FP64 may legitimately decide differently (such pairs
contribute exactly zero: f_c(Rc) = f_c'(Rc) = 0, Eq. 3).
"""
import numpy as np
import pytest

import oracle
import synth
from tests._common import force_errors, model_for, to_cuda

pytestmark = pytest.mark.gpu

E_TOL = 1e-3
F_RMS_TOL = 1e-3


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def make(kind, precision="fp32", cos_scale=1.0):
    from paper_2207_14276_gb300 import Potential
    spec, w = model_for(kind, cos_scale=cos_scale)
    return Potential(spec, w, precision=precision), oracle.Model(spec, w)


def check_system(pot, orc, s, rel_f=1e-4, aev=True):
    d = to_cuda(s)
    E, F = pot.energy_forces(d["coords"], d["species"], d["box"], d["mask"])
    ref = orc.energy_forces(s.coords, s.species, s.box, s.mask, want_aev=aev)
    E = float(E.cpu()[0])
    F = F.cpu().numpy()
    assert abs(E - ref["energy"]) <= E_TOL, (E, ref["energy"])
    rms, mx = force_errors(F, ref["forces"])
    f_rms = float(np.sqrt(np.mean(ref["forces"] ** 2)))
    assert rms <= F_RMS_TOL
    assert rms <= rel_f * f_rms + 1e-7, (rms, f_rms)
    if s.mask is not None:
        assert np.all(F[s.mask == 0] == 0.0)
    if aev:
        G = pot.debug_rows(0, s.n_atoms).cpu().numpy()
        Gr = ref["aev"]
        sel = np.ones(s.n_atoms, bool) if s.mask is None else s.mask == 1
        np.testing.assert_allclose(G[sel], Gr[sel], rtol=2e-5, atol=1e-6)
    return E, F, ref


def neighbour_sets(pot, s, angular):
    nb = pot.debug_neighbors(s.n_atoms, angular=angular).cpu().numpy()
    pairs = set()
    for i in range(s.n_atoms):
        if s.mask is not None and not s.mask[i]:
            continue
        for j in nb[i]:
            if j < 0:
                break
            pairs.add((i, int(j)))
    return pairs


def near_cutoff(s, pairs, rc, tol=1e-4):
    x = s.coords.astype(np.float64)
    out = set()
    for i, j in pairs:
        d = x[j] - x[i]
        if s.box is not None:
            d -= s.box * np.round(d / s.box)
        if abs(np.linalg.norm(d) - rc) < tol:
            out.add((i, j))
    return out


def compare_neighbours(pot, s, spec):
    for angular, rc in ((False, spec.aev.rc_r), (True, spec.aev.rc_a)):
        got = neighbour_sets(pot, s, angular)
        ref = set(map(tuple, oracle.neighbours(s.coords, rc, s.box, s.mask).tolist()))
        diff = got ^ ref
        assert diff == near_cutoff(s, diff, rc), sorted(diff)[:10]


def test_gas24_energy_forces_aev_neighbours(torch_cuda):
    pot, orc = make("ani4")
    systems, _, _ = synth.workload("gas24")
    s = systems[0]
    check_system(pot, orc, s)
    compare_neighbours(pot, s, pot.spec)
    # dE/dG (the network gradient) elementwise, on the AEV blocks (16 radial or
    # 32 angular features) of each row that hold a nonzero element: the entries
    # the forces read (with sparse rows the library computes no others; dE/dG
    # of an all-zero block multiplies dG/dr = 0)
    r = orc.energy_forces(s.coords, s.species, want_aev=True, want_dEdG=True)
    ref, G = r["dEdG"], r["aev"]
    g = pot.debug_rows(1, s.n_atoms).cpu().numpy()
    S = pot.spec.aev.n_species
    edges = [16 * k for k in range(S + 1)] + [16 * S + 32 * q for q in range(1, S * (S + 1) // 2 + 1)]
    live = np.zeros_like(G, dtype=bool)
    for a, b in zip(edges[:-1], edges[1:]):
        live[:, a:b] = np.any(G[:, a:b] != 0.0, axis=1)[:, None]
    assert live.any(axis=1).all()
    np.testing.assert_allclose(g[live], ref[live], rtol=1e-4, atol=1e-7)


def test_dense_box_neighbourhood_beyond_the_stage(torch_cuda):
    # three times liquid density: the 27-cell neighbourhood of every home cell
    # (about 3000 atoms) exceeds the shared-memory candidate stage of the
    # neighbour kernel, so every centre takes the per-centre global-memory search
    pot, orc = make("ani4")
    s = synth.water_box(1000, 18.0, 10, seed=21)
    check_system(pot, orc, s, rel_f=3e-4, aev=False)
    compare_neighbours(pot, s, pot.spec)


@pytest.mark.parametrize("n_mol,edge,n_side", [(1000, 21.5, 10), (600, 16.0, 9)])
def test_octant_candidate_lists_at_high_density(torch_cuda, n_mol, edge, n_side):
    # about 1,270 candidates per home cell at three times liquid density (4 cells
    # per edge): every centre scans its octant's list of ~350 candidates; 1,800
    # atoms in a 16 A box (3 cells per edge, the whole box is every home cell's
    # neighbourhood): most octant lists exceed their 512 entries and those
    # centres scan all candidates.  Either way the lists equal the oracle's.
    pot, orc = make("ani4")
    s = synth.water_box(n_mol, edge, n_side, seed=23)
    check_system(pot, orc, s, rel_f=3e-4, aev=False)
    compare_neighbours(pot, s, pot.spec)


@pytest.mark.parametrize("precision", ["fp32", "fp32_simt"])
def test_water9000_fp32(torch_cuda, precision):
    # "fp32": tensor-core layers on split BF16 operands (three products per
    # term); "fp32_simt": the fused FP32 FMA kernel of this one-network model
    pot, orc = make("ani4", precision=precision)
    systems, _, _ = synth.workload("water9000")
    s = systems[0]
    E, F, ref = check_system(pot, orc, s)
    compare_neighbours(pot, s, pot.spec)
    assert np.abs(F.astype(np.float64).sum(0)).max() < 1e-3


def test_cos_scale_variant(torch_cuda):
    pot, orc = make("ani4", cos_scale=0.95)
    s = synth.water_box(300, 20.5, 7, seed=41)
    check_system(pot, orc, s)


@pytest.mark.parametrize("precision", ["fp32", "fp32_simt"])
def test_seven_species_solute(torch_cuda, precision):
    pot, orc = make("ani7", precision=precision)
    s = synth.solvated_solute(400, 120, 24.0, seed=5)
    check_system(pot, orc, s)


@pytest.mark.parametrize("precision", ["fp32", "fp32_simt"])
def test_ensemble_of_eight(torch_cuda, precision):
    # "fp32" takes the split tensor-core path; "fp32_simt" the six FP32 FMA GEMMs
    pot, orc = make("ani7x8", precision=precision)
    s = synth.solvated_solute(150, 60, 18.0, seed=6)
    check_system(pot, orc, s)


def test_hybrid_mask(torch_cuda):
    # Eq. 7: only the solute is in the ML region; waters get zero force
    pot, orc = make("ani7")
    s = synth.solvated_solute(600, 50, 27.0, seed=7, mask_solute=True)
    E, F, ref = check_system(pot, orc, s)
    np.testing.assert_array_equal(F[s.mask == 0], 0.0)
    compare_neighbours(pot, s, pot.spec)


def test_batch_of_molecules_matches_oracle_and_single_calls(torch_cuda):
    pot, orc = make("ani4")
    mols, _, _ = synth.workload("molecules64")
    outs = pot.energy_forces_batch([to_cuda(m) for m in mols])
    for m, o in zip(mols, outs):
        ref = orc.energy_forces(m.coords, m.species)
        assert abs(float(o["energy"].cpu()[0]) - ref["energy"]) <= E_TOL
        rms, _ = force_errors(o["forces"].cpu().numpy(), ref["forces"])
        assert rms <= 1e-4 * np.sqrt(np.mean(ref["forces"] ** 2)) + 1e-7
    # the same molecule alone gives the same result as inside the batch
    for k in (0, 17, 63):
        d = to_cuda(mols[k])
        E, F = pot.energy_forces(d["coords"], d["species"])
        assert float(E.cpu()[0]) == pytest.approx(float(outs[k]["energy"].cpu()[0]), abs=1e-5)
        np.testing.assert_allclose(F.cpu().numpy(), outs[k]["forces"].cpu().numpy(), atol=1e-5)


def test_mixed_batch_periodic_and_gas(torch_cuda):
    pot, orc = make("ani4")
    a = synth.water_box(200, 18.0, 6, seed=8)
    b = synth.workload("gas24")[0][0]
    c = synth.water_box(100, 15.0, 5, seed=9)
    outs = pot.energy_forces_batch([to_cuda(a), to_cuda(b), to_cuda(c)], virial=True)
    for s, o in zip((a, b, c), outs):
        ref = orc.energy_forces(s.coords, s.species, s.box)
        assert abs(float(o["energy"].cpu()[0]) - ref["energy"]) <= E_TOL
        rms, _ = force_errors(o["forces"].cpu().numpy(), ref["forces"])
        assert rms <= 1e-4 * np.sqrt(np.mean(ref["forces"] ** 2)) + 1e-7
        np.testing.assert_allclose(o["virial"].cpu().numpy().reshape(3, 3), ref["virial"],
                                   atol=1e-4 * np.abs(ref["virial"]).max() + 1e-6)


def test_unwrapped_periodic_coordinates(torch_cuda):
    pot, orc = make("ani4")
    s = synth.water_box(200, 18.0, 6, seed=10)
    shifted = synth.System("shift", (s.coords + np.float32(18.0)).astype(np.float32), s.species, s.box)
    d0, d1 = to_cuda(s), to_cuda(shifted)
    E0, F0 = pot.energy_forces(d0["coords"], d0["species"], d0["box"])
    E1, F1 = pot.energy_forces(d1["coords"], d1["species"], d1["box"])
    assert float(E0.cpu()[0]) == pytest.approx(float(E1.cpu()[0]), abs=1e-4)
    np.testing.assert_allclose(F0.cpu().numpy(), F1.cpu().numpy(), atol=1e-4)


def test_edge_cases(torch_cuda):
    import torch
    pot, orc = make("ani4")
    # empty system
    E, F = pot.energy_forces(torch.zeros((0, 3), device="cuda"),
                             torch.zeros(0, dtype=torch.uint8, device="cuda"))
    assert float(E.cpu()[0]) == 0.0 and F.shape == (0, 3)
    # a single isolated atom: E = network of a zero AEV, zero force
    x = np.array([[1.0, 2.0, 3.0]], np.float32)
    sp = np.array([2], np.uint8)
    E, F = pot.energy_forces(torch.from_numpy(x).cuda(), torch.from_numpy(sp).cuda())
    ref = orc.energy_forces(x, sp)
    assert float(E.cpu()[0]) == pytest.approx(ref["energy"], abs=1e-5)
    assert np.all(F.cpu().numpy() == 0.0)
    # all atoms masked out: zero energy and forces
    s = synth.water_box(50, 12.0, 4, seed=11)
    d = to_cuda(s)
    E, F = pot.energy_forces(d["coords"], d["species"], d["box"],
                             torch.zeros(s.n_atoms, dtype=torch.uint8, device="cuda"))
    assert float(E.cpu()[0]) == 0.0 and torch.count_nonzero(F).item() == 0
    # two atoms just inside / outside the cutoff
    for dist in (5.19, 5.21):
        x = np.array([[0, 0, 0], [dist, 0, 0]], np.float32)
        sp = np.array([0, 3], np.uint8)
        E, F = pot.energy_forces(torch.from_numpy(x).cuda(), torch.from_numpy(sp).cuda())
        ref = orc.energy_forces(x, sp)
        assert float(E.cpu()[0]) == pytest.approx(ref["energy"], abs=1e-6)
        np.testing.assert_allclose(F.cpu().numpy(), ref["forces"], atol=1e-7)


def test_errors_are_reported(torch_cuda):
    import torch
    from paper_2207_14276_gb300 import NNPError
    pot, _ = make("ani4")
    s = synth.water_box(50, 12.0, 4, seed=12)
    d = to_cuda(s)
    with pytest.raises(NNPError, match="BOX_TOO_SMALL"):
        pot.energy_forces(d["coords"], d["species"], [10.0, 12.0, 12.0])
    bad = d["species"].clone()
    bad[3] = 9
    with pytest.raises(NNPError, match="SPECIES"):
        pot.energy_forces(d["coords"], bad, d["box"])
    x = d["coords"].clone()
    x[5, 1] = float("nan")
    with pytest.raises(NNPError, match="NONFINITE"):
        pot.energy_forces(x, d["species"], d["box"])
    # the handle stays usable after the errors
    E, F = pot.energy_forces(d["coords"], d["species"], d["box"])
    assert torch.isfinite(F).all()


def test_capacity_overflow_grows_and_retries(torch_cuda):
    pot, orc = make("ani4")
    pot.reserve(4000, 1, 32, 32)   # too small for liquid water (~60 radial neighbours)
    s = synth.water_box(300, 20.5, 7, seed=13)
    check_system(pot, orc, s, aev=False)


def test_host_entry_point(torch_cuda):
    pot, orc = make("ani4")
    # lists too small for liquid water: the first call overflows and the entry
    # point repeats it with grown lists before it returns
    pot.reserve(400, 1, 32, 32)
    s = synth.water_box(300, 20.5, 7, seed=14)
    E, F = pot.energy_forces_host(s.coords, s.species, s.box)
    ref = orc.energy_forces(s.coords, s.species, s.box)
    assert abs(E - ref["energy"]) <= E_TOL
    f_rms = np.sqrt(np.mean(ref["forces"] ** 2))
    assert force_errors(F, ref["forces"])[0] <= 1e-4 * f_rms
    # repeated calls (the second one a graph replay), with the virial
    for _ in range(3):
        E2, F2, V2 = pot.energy_forces_host(s.coords, s.species, s.box, virial=True)
        assert abs(E2 - ref["energy"]) <= E_TOL
        assert force_errors(F2, ref["forces"])[0] <= 1e-4 * f_rms
        # the virial sums r_e x dE/dr_e over every pair term: on the default path
        # (split BF16 operands, about 2^-16 relative each) the diagonal, a sum of
        # terms of both signs, carries ~1e-4 of its size
        np.testing.assert_allclose(V2, ref["virial"], atol=5e-4 * np.abs(ref["virial"]).max() + 1e-6)
    # an out-of-range species is reported, and the handle keeps working
    bad = s.species.copy()
    bad[5] = 9
    with pytest.raises(RuntimeError):
        pot.energy_forces_host(s.coords, bad, s.box)
    E3, _ = pot.energy_forces_host(s.coords, s.species, s.box)
    assert abs(E3 - ref["energy"]) <= E_TOL


@pytest.mark.parametrize("precision", ["fp32", "fp32_simt"])
def test_solvated100k_sampled(torch_cuda, precision):
    """Full-size 100k-atom, 7-species, 8-network system: sampled atoms against the
    oracle (per-atom energies, AEV rows and forces computed one by one), plus
    properties that hold at any size (net force ~ 0)."""
    import torch
    pot, orc = make("ani7x8", precision=precision)
    s = synth.workload("solvated100k")[0][0]
    d = to_cuda(s)
    outs = pot.energy_forces_batch([d], atom_energies=True)
    E = float(outs[0]["energy"].cpu()[0])
    F = outs[0]["forces"].cpu().numpy()
    ae = outs[0]["atom_energies"].cpu().numpy()
    assert E == pytest.approx(ae.astype(np.float64).sum(), rel=1e-6)
    rng = np.random.Generator(np.random.PCG64(0))
    idx = np.concatenate([np.arange(0, 1000, 97), rng.choice(s.n_atoms, 24, replace=False)])
    ref = orc.sample(s.coords, s.species, idx, s.box, want_aev=True)
    np.testing.assert_allclose(ae[idx], ref["atom_energies"], rtol=1e-4, atol=1e-5)
    rms, _ = force_errors(F[idx], ref["forces"])
    assert rms <= 1e-4 * np.sqrt(np.mean(ref["forces"] ** 2)) + 1e-6
    G = pot.debug_rows(0, s.n_atoms)[torch.from_numpy(idx).cuda()].cpu().numpy()
    np.testing.assert_allclose(G, ref["aev"], rtol=2e-5, atol=1e-6)
    assert np.abs(F.astype(np.float64).sum(0)).max() < 1e-2


def test_bounded_wait_times_out_and_context_survives(torch_cuda):
    """A device wait on a barrier that nothing completes gives up after its limit,
    the host reads NNP_ERR_TIMEOUT from the status word, and the next call works."""
    import ctypes
    import torch
    from paper_2207_14276_gb300 import _lib
    pot, orc = make("ani4")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert _lib.lib().nnp_debug_wait_probe(pot._h, 1 << 16, stream) == 0
    assert pot.sync_status() == _lib.NNP_ERR_TIMEOUT
    assert pot.sync_status() == 0          # the status word was cleared by the read
    s = synth.workload("gas24")[0][0]
    check_system(pot, orc, s, aev=False)


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp32_simt"])
def test_energy_only_matches_full_evaluation(torch_cuda, precision):
    """Energy-only re-evaluation (no forces requested: backward kernels skipped)
    returns the energies of the full evaluation (same forward arithmetic)."""
    pot, orc = make("ani4", precision=precision)
    mols, _, _ = synth.workload("molecules64")
    systems = [to_cuda(m) for m in mols[:20]] + [to_cuda(synth.water_box(200, 18.0, 6, seed=15))]
    full = pot.energy_forces_batch(systems)
    eonly = pot.energy_forces_batch(systems, forces=False)
    for a, b in zip(full, eonly):
        e0, e1 = float(a["energy"].cpu()[0]), float(b["energy"].cpu()[0])
        assert e1 == pytest.approx(e0, rel=1e-6, abs=1e-6)
        assert "forces" not in b
    # and the energy-only energies against the FP64 oracle: the FP32 bar for the
    # FP32 paths, the BF16 bound of tests/test_gpu_bf16.py for BF16 networks
    for m, b in zip(list(mols[:20]) + [synth.water_box(200, 18.0, 6, seed=15)], eonly):
        ref = orc.energy_forces(m.coords, m.species, m.box)
        e1 = float(b["energy"].cpu()[0])
        if precision == "bf16":
            assert abs(e1 - ref["energy"]) <= 2e-3 * np.abs(ref["atom_energies"]).sum() + 1e-4
        else:
            assert abs(e1 - ref["energy"]) <= E_TOL, (e1, ref["energy"])


def test_golden_closed_form_aev_values(torch_cuda):
    # the kernels' AEV (FP32) against the hand-derived values of Eqs. 3-5 in
    # tests/golden/aev_closed_forms.txt, not only against the oracle
    torch = torch_cuda
    from paper_2207_14276_gb300 import Potential
    from tests._golden import closed_form_cases
    for c in closed_form_cases():
        pot = Potential(c["spec"], synth.make_weights(c["spec"], 7))
        x = torch.tensor(c["coords"], dtype=torch.float32, device="cuda")
        sp = torch.tensor(c["species"], device="cuda")
        pot.energy_forces(x, sp)
        G = pot.debug_rows(0, len(c["species"])).cpu().numpy().astype(np.float64)
        for i, f, v in c["expect"]:
            assert abs(G[i, f] - v) <= 2e-5 * abs(v) + 1e-6, (c["name"], i, f, G[i, f], v)
        for i, a, b in c["zero"]:
            assert np.all(np.abs(G[i, a:b + 1]) <= 1e-6), (c["name"], i, a, b)
        pot.close()


@pytest.mark.parametrize("kind,max_na", [("ani4", 32), ("ani4", 64), ("ani4", 128),
                                         ("ani7", 32), ("ani7", 64)])
def test_angular_accumulator_copies(torch_cuda, kind, max_na):
    # the force kernel keeps 4, 2 or 1 copies of its angular accumulators,
    # depending on the angular list capacity and the species-pair count; every
    # choice must give the oracle's forces
    pot, orc = make(kind)
    pot.reserve(1000, 1, 128, max_na)
    s = synth.water_box(300, 20.5, 7, seed=41)
    check_system(pot, orc, s, aev=False)


def test_centres_with_more_live_blocks_than_staged(torch_cuda):
    # a dense 7-species cluster: most centres see neighbours of every species, so
    # more than 16 of the 28 angular blocks have triplets and the force kernel
    # stages their dE/dG in two groups
    pot, orc = make("ani7")
    rng = np.random.Generator(np.random.PCG64(43))
    sp = (np.arange(120) % 7).astype(np.uint8)
    rng.shuffle(sp)
    s = synth.gas_molecule(rng, 120, sp, density=0.15)
    d = s.coords.astype(np.float64)
    r = np.linalg.norm(d[:, None, :] - d[None, :, :], axis=-1)
    live = []
    for i in range(s.n_atoms):
        nb = np.nonzero((r[i] <= 3.5) & (np.arange(s.n_atoms) != i))[0]
        present = np.bincount(sp[nb], minlength=7) > 0
        k = int(present.sum())
        pairs = k * (k - 1) // 2 + int(sum(np.bincount(sp[nb], minlength=7) >= 2))
        live.append(pairs)
    assert max(live) > 16
    check_system(pot, orc, s)


@pytest.mark.parametrize("precision", ["fp32_split", "fp32_simt"])
def test_dense_centres_take_the_cta_per_centre_backward(torch_cuda, precision):
    """A compact branched solute in water: its core atoms have more than 48
    angular neighbours (thousands of triplets each), so the warp-per-centre force
    kernel hands them to the CTA-per-centre one, while the waters stay on the
    warp kernel.  Energy, forces and virial of the mix against the oracle."""
    pot, orc = make("ani7", precision=precision)
    s = synth.solvated_solute(300, 200, 22.0, seed=17)
    x = s.coords.astype(np.float64)
    d = x[:, None, :] - x[None, :, :]
    d -= s.box * np.round(d / s.box)
    n_a = ((np.linalg.norm(d, axis=-1) <= 3.5).sum(1) - 1)
    assert (n_a > 48).sum() >= 5 and (n_a <= 48).sum() > 500
    check_system(pot, orc, s, aev=False)
    out = pot.energy_forces_batch([to_cuda(s)], virial=True)[0]
    ref = orc.energy_forces(s.coords, s.species, s.box)
    np.testing.assert_allclose(out["virial"].cpu().numpy().reshape(3, 3), ref["virial"],
                               atol=1e-4 * np.abs(ref["virial"]).max() + 1e-6)


@pytest.mark.parametrize("kind", ["ani4", "ani7x8"])
def test_split_path_batch_of_small_molecules(torch_cuda, kind):
    """The split tensor-core path on a batch of 20-60-atom molecules: few 128-row
    tiles, so the layers take narrow N tiles and two CTAs per SM where the stages
    allow; every molecule's energy and forces against the oracle."""
    pot, orc = make(kind, precision="fp32_split")
    mols, _, _ = synth.workload("molecules64")
    if kind == "ani7x8":
        rng = np.random.Generator(np.random.PCG64(5))
        mols = [synth.gas_molecule(rng, int(n), synth.systems._species_exact(
            synth.systems.SOLUTE_FRACTIONS, int(n), rng)) for n in rng.integers(20, 61, 12)]
    outs = pot.energy_forces_batch([to_cuda(m) for m in mols])
    for m, o in zip(mols, outs):
        ref = orc.energy_forces(m.coords, m.species)
        assert abs(float(o["energy"].cpu()[0]) - ref["energy"]) <= E_TOL
        rms, _ = force_errors(o["forces"].cpu().numpy(), ref["forces"])
        assert rms <= 1e-4 * np.sqrt(np.mean(ref["forces"] ** 2)) + 1e-7


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("kind", ["ani4", "ani7x8"])
def test_sparse_rows_equal_dense_rows(torch_cuda, precision, kind):
    """AEV rows written only in their live slices, the first layer over the tile's
    live K slices and the last backward layer over its live N tiles, against
    whole rows, on a batch mixing water-like tiles (few live slices) with solute
    and gas tiles (many).  The skipped products are exact zeros, but the tensor
    cores' FP32 accumulation does not add an all-zero slice as an exact no-op,
    so the two differ in the last bits of the first layer: by the FP32 bar on
    the split path (energy 1e-5 relative, forces 1e-4 of their RMS), and by
    BF16 rounding flips downstream on the BF16 path (1e-3 of sum_i |E_i|, 2e-3
    of the force RMS).  The AEV rows read back equal the oracle's."""
    torch = torch_cuda
    pot, orc = make(kind, precision=precision)
    if kind == "ani4":
        systems = [synth.water_box(300, 20.5, 7, seed=41)] + list(synth.workload("molecules64")[0][:5])
    else:
        systems = [synth.solvated_solute(300, 60, 22.0, seed=6)]
    d = [to_cuda(s) for s in systems]
    res = {}
    for sparse in (False, True):
        pot.set_sparse_rows(sparse)
        outs = pot.energy_forces_batch(d, atom_energies=True)
        res[sparse] = [(float(o["energy"].cpu()[0]), o["forces"].cpu().numpy().astype(np.float64),
                        o["atom_energies"].cpu().numpy().astype(np.float64)) for o in outs]
    for (e1, f1, _), (e0, f0, a0) in zip(res[True], res[False]):
        f_rms = float(np.sqrt(np.mean(f0 ** 2))) + 1e-12
        d_rms = float(np.sqrt(np.mean((f1 - f0) ** 2)))
        if precision == "fp32":
            assert abs(e1 - e0) <= 1e-5 * (abs(e0) + 1.0)
            assert d_rms <= 1e-4 * f_rms
        else:
            assert abs(e1 - e0) <= 1e-3 * float(np.abs(a0).sum()) + 1e-6
            assert d_rms <= 2e-3 * f_rms
    # the AEV rows of the last system, sparse, against the oracle
    s = systems[-1]
    pot.energy_forces_batch([d[-1]])
    G = pot.debug_rows(0, s.n_atoms).cpu().numpy()
    Gr = orc.energy_forces(s.coords, s.species, s.box, want_aev=True)["aev"]
    tol = 2e-5 if precision == "fp32" else 5e-3
    np.testing.assert_allclose(G, Gr, rtol=tol, atol=1e-6)


@pytest.mark.parametrize("precision", ["fp32_split", "bf16"])
def test_batch_of_more_systems_than_one_parameter_chunk(torch_cuda, precision):
    """150 molecules in one call: the descriptors travel as kernel parameters in
    chunks of 64 systems, so the front end runs three init and prep launches and
    the later kernels index systems across chunks.  Every molecule's energy and
    forces against the oracle, plus a periodic box in the last chunk."""
    pot, orc = make("ani7", precision=precision)
    rng = np.random.Generator(np.random.PCG64(77))
    mols = [synth.gas_molecule(rng, int(n), synth.systems._species_exact(
        synth.systems.SOLUTE_FRACTIONS, int(n), rng)) for n in rng.integers(8, 33, 149)]
    mols.append(synth.water_box(100, 14.5, 5, seed=3))
    outs = pot.energy_forces_batch([to_cuda(m) for m in mols], atom_energies=True)
    bf16 = precision == "bf16"
    for m, o in zip(mols, outs):
        ref = orc.energy_forces(m.coords, m.species, m.box)
        scale = float(np.abs(ref["atom_energies"]).sum())
        assert abs(float(o["energy"].cpu()[0]) - ref["energy"]) <= (2e-3 * scale + 1e-4 if bf16 else E_TOL)
        rms, _ = force_errors(o["forces"].cpu().numpy(), ref["forces"])
        f_rms = float(np.sqrt(np.mean(ref["forces"] ** 2)))
        assert rms <= (2e-2 if bf16 else 1e-4) * f_rms + 1e-7
