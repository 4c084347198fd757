"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

* closed-form special values of Eqs. 3-5 (cutoff at half radius, Gaussian at
  its centre or half height, angular factor at theta = theta_s), which fix the
  block indices, the 2^(1-zeta) prefactor, the unordered-pair reading and the
  averaged-distance Gaussian;
* a library special case: the per-species network equals a numpy FP64 chain
  x @ W.T + b with CELU (the paper's feed-forward networks, Eq. 2);
* invariants: translation / rotation / same-species permutation, zero net force
  and torque, extensivity, an isolated atom, the hybrid mask (Eq. 7);
* finite differences of the energy (forces, virial, weight gradients) and of
  the force-matching loss (its gradient w.r.t. weights and coordinates);
* brute-force O(N^2) neighbour pairs against an independent linked-cell list.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.filterwarnings("ignore")


def small_model(kind="ani4", seed=1, cos_scale=1.0, shift=None):
    spec = synth.model_spec(kind)
    if cos_scale != 1.0:
        spec = dataclasses.replace(spec, aev=dataclasses.replace(spec.aev, cos_scale=cos_scale))
    return spec, oracle.Model(spec, synth.make_weights(spec, seed), shift=shift)


def custom_model(S=2, rc_r=5.2, eta_r=16.0, shf_r=(0.0, 2.6), rc_a=4.0, eta_a=8.0,
                 zeta=32.0, shf_a=(2.0,), shf_z=(math.pi / 2,), widths_h=(4,)):
    p = synth.AevParams(S, rc_r, eta_r, tuple(shf_r), rc_a, eta_a, zeta, tuple(shf_a),
                        tuple(shf_z))
    D = synth.aev_dim(p)
    spec = synth.ModelSpec(p, (D,) + tuple(widths_h) + (1,), 1, 0.1, tuple(range(1, S + 1)))
    return spec, oracle.Model(spec, synth.make_weights(spec, 7))


def molecule(seed, n=20, S=4, edge=None):
    rng = np.random.Generator(np.random.PCG64(seed))
    sp = rng.integers(0, S, size=n).astype(np.uint8)
    density = 0.024 if edge is None else n / edge ** 3
    return synth.gas_molecule(rng, n, sp, density=density)


def rot(seed):
    q = np.random.Generator(np.random.PCG64(seed)).normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


# ------------------------------------------------------------------ Eqs. 3-4 special values
def test_two_atom_radial_special_values():
    # shells at 0 and 2.6 = Rc/2; a partner at 2.6 A sits on the second shell where
    # exp(0) = 1 and the cosine cutoff is exactly 1/2 (Eq. 3 at R = Rc/2).
    spec, m = custom_model(S=2, rc_a=1.0)
    xyz = np.array([[0.0, 0.0, 0.0], [2.6, 0.0, 0.0]])
    r = m.energy_forces(xyz, np.array([0, 1]), want_aev=True)
    G = r["aev"]
    nr = 2
    # atom 0 (species 0) sees one neighbour of species 1: block 1 only
    assert G[0, 1 * nr + 1] == pytest.approx(0.5, abs=1e-15)
    assert G[0, 0] == 0.0 and G[0, 1] == 0.0
    # shell at 0: exp(-16*2.6^2) * 1/2
    assert G[0, 1 * nr + 0] == pytest.approx(0.5 * math.exp(-16 * 2.6 ** 2), rel=1e-12)
    # atom 1 (species 1) sees species 0: block 0
    assert G[1, 0 * nr + 1] == pytest.approx(0.5, abs=1e-15)
    assert G[1, 1 * nr + 1] == 0.0
    # no angular terms with a single neighbour
    assert np.all(G[:, 2 * nr:] == 0.0)


def test_radial_gaussian_half_height_and_cutoff_edge():
    eta = 16.0
    x = math.sqrt(math.log(2.0) / eta)  # exp(-eta x^2) = 1/2
    spec, m = custom_model(S=1, shf_r=(2.6 - x,), rc_a=1.0)
    r = m.energy_forces(np.array([[0, 0, 0], [2.6, 0, 0]], float), np.array([0, 0]), want_aev=True)
    assert r["aev"][0, 0] == pytest.approx(0.25, rel=1e-12)  # 1/2 * f_c(Rc/2)
    # exactly at the cutoff and beyond it the pair contributes nothing (Eq. 3)
    for d in (5.2, 5.3):
        r = m.energy_forces(np.array([[0, 0, 0], [d, 0, 0]], float), np.array([0, 0]), want_aev=True)
        assert abs(r["aev"][0, 0]) < 1e-30


def _triplet(Rj, Rk, theta):
    return np.array([[0.0, 0.0, 0.0], [Rj, 0.0, 0.0],
                     [Rk * math.cos(theta), Rk * math.sin(theta), 0.0]])


def test_angular_special_values():
    # Rc_a = 4: f_c(4/3) = 3/4, f_c(8/3) = 1/4.  Shell centre 2 = (4/3 + 8/3)/2 so the
    # Gaussian of the averaged distance is exp(0) = 1.  theta = theta_s = pi/2 makes
    # (1 + cos 0)^zeta 2^(1-zeta) = 2.  One unordered pair: G = 2 * 3/4 * 1/4.
    spec, m = custom_model(S=3, rc_r=4.5, rc_a=4.0, shf_a=(2.0,), shf_z=(math.pi / 2,))
    xyz = _triplet(4.0 / 3.0, 8.0 / 3.0, math.pi / 2)
    sp = np.array([0, 1, 2])
    G = m.energy_forces(xyz, sp, want_aev=True)["aev"]
    nr = 2
    base = 3 * nr
    # centre 0 (species 0) sees the unordered pair {1, 2}: block p(1,2) = 3 + 1 = 4
    blocks = G[0, base:]
    assert blocks[4] == pytest.approx(0.375, rel=1e-12)
    assert np.count_nonzero(blocks) == 1
    # swapping the neighbour species gives the same block (unordered pair)
    G2 = m.energy_forces(xyz, np.array([0, 2, 1]), want_aev=True)["aev"]
    assert G2[0, base + 4] == pytest.approx(0.375, rel=1e-12)


def test_angular_half_height_and_angle_factor():
    # Gaussian of the averaged distance at half height, theta - theta_s = pi/2:
    # (1 + cos(pi/2))^zeta 2^(1-zeta) = 2^(1-zeta).
    eta = 8.0
    x = math.sqrt(math.log(2.0) / eta)
    zeta = 4.0
    spec, m = custom_model(S=1, rc_r=4.5, rc_a=4.0, eta_a=eta, zeta=zeta, shf_a=(2.0 - x,),
                           shf_z=(0.0,))
    G = m.energy_forces(_triplet(4.0 / 3.0, 8.0 / 3.0, math.pi / 2), np.array([0, 0, 0]),
                        want_aev=True)["aev"]
    assert G[0, 2] == pytest.approx(0.5 * 0.1875 * 2.0 ** (1 - zeta), rel=1e-12)
    # theta = pi with theta_s = 0: (1 + cos pi) = 0 -> term vanishes
    G = m.energy_forces(_triplet(4.0 / 3.0, 8.0 / 3.0, math.pi), np.array([0, 0, 0]),
                        want_aev=True)["aev"]
    assert abs(G[0, 2]) < 1e-30


def test_aev_layout_dimensions():
    for kind, D in (("ani4", 384), ("ani7", 1008)):
        spec, m = small_model(kind)
        assert m.D == D == spec.widths[0]


# ------------------------------------------------------------------ networks (Eq. 2)
def _numpy_net(spec, w, s, e, G):
    widths = spec.widths
    S = spec.aev.n_species
    L = len(widths) - 1
    per = [widths[l + 1] * widths[l] + widths[l + 1] for l in range(L)]
    ofs = (e * S + s) * sum(per)
    h = G
    for l in range(L):
        W = w[ofs:ofs + widths[l + 1] * widths[l]].reshape(widths[l + 1], widths[l])
        b = w[ofs + widths[l + 1] * widths[l]:ofs + per[l]]
        ofs += per[l]
        z = h @ W.T + b
        h = z if l == L - 1 else np.where(z > 0, z, spec.celu_alpha * np.expm1(z / spec.celu_alpha))
    return h[..., 0]


@pytest.mark.parametrize("kind", ["ani4", "ani7x8"])
def test_network_matches_numpy_chain(kind):
    spec = synth.model_spec(kind)
    w = synth.make_weights(spec, 3).astype(np.float64)
    shift = np.linspace(-1.0, 1.0, spec.aev.n_species)
    m = oracle.Model(spec, w, shift=shift)
    s = molecule(11, n=14, S=spec.aev.n_species)
    r = m.energy_forces(s.coords, s.species, want_aev=True)
    ref = np.zeros(s.n_atoms)
    for e in range(spec.n_ensemble):
        for i in range(s.n_atoms):
            ref[i] += _numpy_net(spec, w, int(s.species[i]), e, r["aev"][i]) / spec.n_ensemble
    ref += shift[s.species]
    np.testing.assert_allclose(r["atom_energies"], ref, rtol=1e-12, atol=1e-12)
    assert r["energy"] == pytest.approx(ref.sum(), rel=1e-12)


def test_isolated_atom_is_network_of_zero():
    spec = synth.model_spec("ani4")
    w = synth.make_weights(spec, 1).astype(np.float64)
    shift = np.array([0.1, 0.2, 0.3, 0.4])
    m = oracle.Model(spec, w, shift=shift)
    xyz = np.array([[0, 0, 0], [1.2, 0, 0], [30.0, 0, 0]])
    sp = np.array([1, 0, 3])
    r = m.energy_forces(xyz, sp)
    far = _numpy_net(spec, w, 3, 0, np.zeros(384)) + 0.4
    assert r["atom_energies"][2] == pytest.approx(far, rel=1e-13)
    assert np.all(r["forces"][2] == 0.0)


# ------------------------------------------------------------------ invariants
@pytest.mark.parametrize("cos_scale", [1.0, 0.95])
def test_translation_rotation_permutation(cos_scale):
    spec, m = small_model(cos_scale=cos_scale)
    s = molecule(5, n=22)
    base = m.energy_forces(s.coords, s.species)
    x = s.coords.astype(np.float64)
    e_t = m.energy_forces(x + np.array([3.1, -2.2, 7.5]), s.species)["energy"]
    R = rot(9)
    r_rot = m.energy_forces(x @ R.T, s.species)
    perm = np.arange(s.n_atoms)
    for sp in range(4):  # permute atoms within each species
        idx = np.flatnonzero(s.species == sp)
        perm[idx] = np.random.Generator(np.random.PCG64(sp)).permutation(idx)
    r_perm = m.energy_forces(x[perm], s.species[perm])
    E = base["energy"]
    for e in (e_t, r_rot["energy"], r_perm["energy"]):
        assert e == pytest.approx(E, rel=1e-10, abs=1e-12)
    # forces rotate with the frame and follow the permutation
    np.testing.assert_allclose(r_rot["forces"], base["forces"] @ R.T, atol=1e-10)
    np.testing.assert_allclose(r_perm["forces"], base["forces"][perm], atol=1e-12)


def test_net_force_and_torque_vanish():
    spec, m = small_model()
    s = molecule(6, n=25)
    r = m.energy_forces(s.coords, s.species)
    F = r["forces"]
    assert np.abs(F.sum(0)).max() < 1e-12
    torque = np.cross(s.coords.astype(np.float64), F).sum(0)
    assert np.abs(torque).max() < 1e-11
    # non-periodic virial sum_a r_a (x) F_a equals the edge-form virial
    np.testing.assert_allclose(r["virial"], s.coords.astype(np.float64).T @ F, atol=1e-11)


@pytest.mark.parametrize("cos_scale", [1.0, 0.95])
def test_forces_match_central_differences(cos_scale):
    spec, m = small_model(cos_scale=cos_scale)
    s = molecule(7, n=18)
    x = s.coords.astype(np.float64)
    F = m.energy_forces(x, s.species)["forces"]
    h = 1e-4
    fd = np.zeros_like(F)
    for a in range(s.n_atoms):
        for c in range(3):
            xp = x.copy(); xp[a, c] += h
            xm = x.copy(); xm[a, c] -= h
            fd[a, c] = -(m.energy_forces(xp, s.species)["energy"]
                         - m.energy_forces(xm, s.species)["energy"]) / (2 * h)
    scale = np.abs(F).max()
    np.testing.assert_allclose(fd, F, atol=1e-7 * max(scale, 1.0) + 1e-9)
    assert np.abs(fd - F).max() < 1e-6 * scale


def test_periodic_forces_fd_and_translation():
    sys = synth.water_box(48, 11.0, 4, seed=21)
    spec, m = small_model()
    x = sys.coords.astype(np.float64)
    r = m.energy_forces(x, sys.species, box=sys.box)
    assert np.abs(r["forces"].sum(0)).max() < 1e-11
    # translation across the periodic boundary (wrapped or not) leaves E unchanged
    sh = np.mod(x + np.array([5.3, -7.1, 2.2]), 11.0)
    assert m.energy_forces(sh, sys.species, box=sys.box)["energy"] == pytest.approx(r["energy"], rel=1e-11)
    assert m.energy_forces(x + 11.0, sys.species, box=sys.box)["energy"] == pytest.approx(r["energy"], rel=1e-11)
    h = 1e-4
    rng = np.random.Generator(np.random.PCG64(3))
    for a in rng.choice(sys.n_atoms, 12, replace=False):
        for c in range(3):
            xp = x.copy(); xp[a, c] += h
            xm = x.copy(); xm[a, c] -= h
            fd = -(m.energy_forces(xp, sys.species, box=sys.box)["energy"]
                   - m.energy_forces(xm, sys.species, box=sys.box)["energy"]) / (2 * h)
            assert fd == pytest.approx(r["forces"][a, c], abs=1e-8)


def test_virial_matches_strain_derivative():
    sys = synth.water_box(48, 11.0, 4, seed=22)
    spec, m = small_model()
    x = sys.coords.astype(np.float64)
    W = m.energy_forces(x, sys.species, box=sys.box)["virial"]
    h = 1e-5
    for a in range(3):
        for b in range(3):
            def energy(eps):
                Eps = np.eye(3)
                Eps[a, b] += eps
                box = sys.box.copy()
                if a == b:
                    box[a] *= (1 + eps)
                    return m.energy_forces(x @ Eps.T, sys.species, box=box)["energy"]
                return None
            if a == b:
                dE = (energy(h) - energy(-h)) / (2 * h)
                assert -dE == pytest.approx(W[a, b], rel=1e-6, abs=1e-9)
    # off-diagonal: non-periodic molecule under a shear of all coordinates
    s = molecule(8, n=16)
    xm = s.coords.astype(np.float64)
    Wm = m.energy_forces(xm, s.species)["virial"]
    for a in range(3):
        for b in range(3):
            Ep = np.eye(3); Ep[a, b] += h
            Em = np.eye(3); Em[a, b] -= h
            dE = (m.energy_forces(xm @ Ep.T, s.species)["energy"]
                  - m.energy_forces(xm @ Em.T, s.species)["energy"]) / (2 * h)
            assert -dE == pytest.approx(Wm[a, b], rel=1e-6, abs=1e-9)


def test_extensivity_two_distant_copies():
    spec, m = small_model()
    s = molecule(9, n=15)
    x = s.coords.astype(np.float64)
    E1 = m.energy_forces(x, s.species)["energy"]
    x2 = np.concatenate([x, x + np.array([60.0, 0, 0])])
    sp2 = np.concatenate([s.species, s.species])
    r2 = m.energy_forces(x2, sp2)
    assert r2["energy"] == pytest.approx(2 * E1, rel=1e-12)


def test_mask_equals_removing_unmasked_atoms():
    # Eq. 7: the ML region P alone enters V_ML(P); atoms outside P are neither
    # centres nor neighbours and carry zero force.
    spec, m = small_model()
    s = molecule(10, n=30, edge=9.0)
    mask = np.zeros(30, np.uint8)
    mask[::3] = 1
    mask[1] = 1
    r = m.energy_forces(s.coords, s.species, mask=mask)
    sub = m.energy_forces(s.coords[mask == 1], s.species[mask == 1])
    assert r["energy"] == pytest.approx(sub["energy"], rel=1e-13)
    np.testing.assert_array_equal(r["forces"][mask == 0], 0.0)
    np.testing.assert_allclose(r["forces"][mask == 1], sub["forces"], atol=1e-14)


# ------------------------------------------------------------------ neighbour lists
@pytest.mark.parametrize("case", ["gas", "water", "masked", "tiny_box"])
def test_brute_force_pairs_equal_cell_list(case):
    mask = None
    box = None
    if case == "gas":
        s = molecule(12, n=200, edge=14.0)
        x = s.coords
    elif case == "water":
        s = synth.water_box(400, 23.0, 8, seed=4)
        x, box = s.coords, s.box
    elif case == "masked":
        s = synth.water_box(400, 23.0, 8, seed=5)
        x, box = s.coords, s.box
        mask = (np.arange(s.n_atoms) % 4 != 0).astype(np.uint8)
    else:  # 2 cells per dimension: every neighbour cell is visited once
        s = synth.water_box(40, 10.5, 4, seed=6)
        x, box = s.coords, s.box
    a = oracle.neighbours(x, 5.2, box, mask, "brute")
    b = oracle.neighbours(x, 5.2, box, mask, "cells")
    sa = set(map(tuple, a.tolist()))
    sb = set(map(tuple, b.tolist()))
    assert len(sa) == len(a) and sa == sb
    # symmetric: (i, j) present iff (j, i) present
    assert sa == {(j, i) for i, j in sa}
    if mask is not None:
        assert all(mask[i] and mask[j] for i, j in sa)


# ------------------------------------------------------------------ gradients w.r.t. weights
def test_energy_weight_gradient_matches_fd():
    spec, m = small_model()
    w0 = synth.make_weights(spec, 1).astype(np.float64)
    s = molecule(13, n=12)
    g = m.energy_forces(s.coords, s.species, want_dEdW=True)["dEdW"]
    rng = np.random.Generator(np.random.PCG64(0))
    idx = np.concatenate([rng.choice(w0.size, 40, replace=False), np.flatnonzero(g)[-20:]])
    h = 1e-5
    for k in idx:
        wp = w0.copy(); wp[k] += h
        wm = w0.copy(); wm[k] -= h
        Ep = oracle.Model(spec, wp).energy_forces(s.coords, s.species)["energy"]
        Em = oracle.Model(spec, wm).energy_forces(s.coords, s.species)["energy"]
        assert (Ep - Em) / (2 * h) == pytest.approx(g[k], rel=1e-6, abs=1e-9)


def _fm_loss(model, x, sp, Ft):
    F = model.energy_forces(x, sp)["forces"]
    return float(np.sum((F - Ft) ** 2))


def test_force_matching_gradient_matches_fd():
    spec, m = small_model()
    w0 = synth.make_weights(spec, 1).astype(np.float64)
    s = molecule(14, n=10)
    x = s.coords.astype(np.float64)
    rng = np.random.Generator(np.random.PCG64(4))
    Ft = rng.normal(0.0, 1.0, size=(s.n_atoms, 3)) * 0.05
    F = m.energy_forces(x, s.species)["forces"]
    v = 2 * (F - Ft)
    E, F2, gx, gw = m.force_matching(x, s.species, v)
    np.testing.assert_allclose(F2, F, atol=1e-14)
    h = 1e-4
    for a in range(s.n_atoms):
        for c in range(3):
            xp = x.copy(); xp[a, c] += h
            xm = x.copy(); xm[a, c] -= h
            fd = (_fm_loss(m, xp, s.species, Ft) - _fm_loss(m, xm, s.species, Ft)) / (2 * h)
            assert fd == pytest.approx(gx[a, c], rel=2e-5, abs=1e-9)
    # weights: the whole output layer of two species plus a sample of the rest
    widths = spec.widths
    per = sum(widths[l + 1] * widths[l] + widths[l + 1] for l in range(4))
    last = per - (widths[4] * widths[3] + widths[4])
    idx = list(range(last, per)) + list(range(per + last, 2 * per))
    idx += list(rng.choice(w0.size, 60, replace=False))
    idx += list(np.argsort(-np.abs(gw))[:20])
    for k in idx:
        wp = w0.copy(); wp[k] += h
        wm = w0.copy(); wm[k] -= h
        fd = (_fm_loss(oracle.Model(spec, wp), x, s.species, Ft)
              - _fm_loss(oracle.Model(spec, wm), x, s.species, Ft)) / (2 * h)
        assert fd == pytest.approx(gw[k], rel=1e-5, abs=1e-10)


def test_sample_matches_full_evaluation():
    sys = synth.water_box(300, 20.5, 7, seed=31)
    spec, m = small_model()
    full = m.energy_forces(sys.coords, sys.species, box=sys.box, want_aev=True)
    idx = np.array([0, 5, 17, 250, 899])
    smp = m.sample(sys.coords, sys.species, idx, box=sys.box, want_aev=True)
    np.testing.assert_allclose(smp["atom_energies"], full["atom_energies"][idx], rtol=1e-12)
    np.testing.assert_allclose(smp["forces"], full["forces"][idx], atol=1e-13)
    np.testing.assert_allclose(smp["aev"], full["aev"][idx], atol=1e-13)


# ------------------------------------------------------------------ golden fixtures
def test_golden_closed_form_aev_values():
    # hand-derived values of Eqs. 3-5 at special geometries (tests/golden/aev_closed_forms.txt)
    from tests._golden import closed_form_cases
    cases = closed_form_cases()
    assert len(cases) == 4
    for c in cases:
        m = oracle.Model(c["spec"], synth.make_weights(c["spec"], 7))
        G = m.energy_forces(c["coords"], c["species"], want_aev=True)["aev"]
        for i, f, v in c["expect"]:
            assert G[i, f] == pytest.approx(v, rel=1e-12, abs=1e-15), (c["name"], i, f)
        for i, a, b in c["zero"]:
            assert np.all(np.abs(G[i, a:b + 1]) <= 1e-15), (c["name"], i, a, b)


def test_golden_paper_constants():
    # the cutoff radius and the sub-AEV counts the paper prints (tests/golden/paper_constants.txt)
    from tests._golden import paper_constants
    k = paper_constants()
    (rc,), = k["rc_r"]
    for kind in ("ani4", "ani7", "ani7x8"):
        assert synth.model_spec(kind).aev.rc_r == rc
    for N, n_rad, n_ang in k["sub_aevs"]:
        spec, m = small_model("ani4" if N == 4 else "ani7")
        p = spec.aev
        assert p.n_species == N
        assert m.D == n_rad * len(p.shf_r) + n_ang * len(p.shf_a) * len(p.shf_z)
