"""Host-side logic on CPU: the synthetic inputs match the recipe the benchmarks
and parity tests are quoted on, and the benchmark's work and traffic accounting
gives the figures its roofline fractions are built from."""
import hashlib
import math

import numpy as np
import pytest

import bench
import synth
from synth.systems import H, O

AVOGADRO = 6.02214076e23
WATER_G_PER_MOL = 2 * 1.008 + 15.999


def _min_image(d, box):
    return d - box * np.round(d / box)


def test_water9000_recipe():
    # 3000 rigid waters (O-H 0.96 A, H-O-H 104.5 deg) in a periodic 44.77 A cube:
    # 1 g/cm^3
    (s,), kind, _ = synth.workload("water9000")
    assert kind == "ani4" and s.n_atoms == 9000
    assert np.allclose(s.box, 44.77)
    x = s.coords.astype(np.float64).reshape(3000, 3, 3)
    assert np.all(s.species.reshape(3000, 3) == [O, H, H])
    oh1 = _min_image(x[:, 1] - x[:, 0], s.box)
    oh2 = _min_image(x[:, 2] - x[:, 0], s.box)
    r1, r2 = np.linalg.norm(oh1, axis=1), np.linalg.norm(oh2, axis=1)
    assert np.allclose(r1, 0.96, atol=2e-5) and np.allclose(r2, 0.96, atol=2e-5)
    ang = np.degrees(np.arccos(np.sum(oh1 * oh2, axis=1) / (r1 * r2)))
    assert np.allclose(ang, 104.5, atol=1e-2)
    density = 3000 * WATER_G_PER_MOL / AVOGADRO / (44.77e-8) ** 3
    assert density == pytest.approx(1.0, abs=0.01)
    # coordinates wrapped into the box, as the kernels' cell binning expects
    assert s.coords.min() >= 0.0 and s.coords.max() < 44.77


def test_gas24_and_molecules_recipes():
    (g,), kind, _ = synth.workload("gas24")
    assert kind == "ani4" and g.box is None
    assert np.bincount(g.species, minlength=4).tolist() == [12, 7, 3, 2]   # H C N O
    d = np.linalg.norm(g.coords[:, None].astype(np.float64) - g.coords[None], axis=-1)
    assert d[np.triu_indices(24, 1)].min() >= 0.9 - 1e-6
    mols, kind, _ = synth.workload("molecules64")
    assert kind == "ani4" and len(mols) == 64
    assert all(20 <= m.n_atoms <= 60 for m in mols)


@pytest.mark.parametrize("name,n_atoms,edge,n_solute", [("solvated20k", 20051, 58.4, 50),
                                                        ("solvated100k", 100000, 99.9, 1000)])
def test_solvated_recipes(name, n_atoms, edge, n_solute):
    (s,), kind, _ = synth.workload(name)
    assert kind == "ani7x8" and s.n_atoms == n_atoms and np.allclose(s.box, edge)
    sol = s.coords[:n_solute].astype(np.float64)
    oxy = s.coords[n_solute::3].astype(np.float64)
    assert np.all(s.species[n_solute::3] == O)
    # every water oxygen sits on a lattice site farther than 2.5 A from the
    # solute, moved by at most 0.25 A per coordinate
    near = np.inf
    for c in range(0, oxy.shape[0], 8192):
        d = _min_image(oxy[c:c + 8192, None, :] - sol[None, :, :], s.box)
        near = min(near, np.sqrt(np.min(np.sum(d * d, axis=2))))
    assert near > 2.5 - 0.25 * math.sqrt(3)
    # solute composition (C 35, H 45, N 7, O 8, S 2, F 1.5, Cl 1.5 %) and no
    # solute pair closer than 1 A
    counts = np.bincount(s.species[:n_solute], minlength=7) / n_solute
    frac = synth.systems.SOLUTE_FRACTIONS
    for z, f in frac.items():
        assert counts[z] == pytest.approx(f, abs=1.0 / n_solute + 1e-9)
    d = _min_image(sol[:, None, :] - sol[None, :, :], s.box)
    r = np.sqrt(np.sum(d * d, axis=2))
    assert r[np.triu_indices(n_solute, 1)].min() >= 1.0 - 1e-5


def test_stage_work_figures():
    spec = synth.model_spec("ani4")
    # the fused network kernel: 2 FLOP per weight per row forward (with the
    # output layer) and backward to the input (without it): 2 x (94,304 + 94,208)
    # = 377,024 FLOP per atom for 384-160-128-96-1, 3.39e9 per 9000-atom launch
    flops, unit, bound = bench.stage_work("mlp", spec, (59.4, 17.0), 9000, "fp32")
    assert (unit, bound) == ("FLOP", "alu")
    assert flops == 9000 * 377024 == pytest.approx(3.393e9, rel=1e-3)
    # AEV kernels: 16 shells x 5 (forward) / 8 (backward) FLOP per radial pair,
    # 200 / 330 FLOP per unordered angular pair
    na = 17.0
    tri = na * (na - 1) / 2
    assert bench.stage_work("aev_fwd", spec, (59.4, na), 1, "fp32")[0] == pytest.approx(
        59.4 * 80 + tri * 200)
    assert bench.stage_work("aev_bwd", spec, (59.4, na), 1, "fp32")[0] == pytest.approx(
        59.4 * 128 + tri * 330)
    # neighbour search bytes: coordinates, list entries and the header per atom
    assert bench.stage_work("neighbors", spec, (59.4, na), 1, "fp32") == (
        16 + 4 * (59.4 + na) + 32, "B", "hbm")
    # tensor-core layer GEMMs of the 8-network model: 2 K N per row
    s8 = synth.model_spec("ani7x8")
    assert bench.stage_work("mlp_l1", s8, (0, 0), 10, "bf16") == (2.0 * 10 * 1008 * 8 * 256, "FLOP",
                                                                 "tensor")
    assert bench.stage_work("mlp_b2", s8, (0, 0), 10, "bf16")[0] == 2.0 * 10 * 192 * 256 * 8
    assert bench.stage_work("finalize", spec, (0, 0), 10, "fp32") is None


def test_fp32_alu_peak():
    # 152 SMs x 128 FP32 lanes x 2 FLOP x 2070 MHz
    assert bench.fp32_alu_peak_tflops(2070) == pytest.approx(80.54784)


def test_recorded_traffic_follows_the_kernel_source(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2207_14276_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = csrc / "mlp_fused.cu"
    src.write_text("kernel v1\n")
    sha = hashlib.sha256(b"kernel v1\n").hexdigest()[:16]
    (tmp_path / "profiles" / "dram_traffic.txt").write_text(
        "# stage workload bytes sha summary\n"
        f"mlp water9000 15467264 {sha} profiles/x.md\n")
    monkeypatch.setattr(bench, "__file__", str(tmp_path / "bench.py"))
    assert bench.recorded_traffic("mlp", "water9000") == 15467264
    assert bench.recorded_traffic("mlp", "solvated100k") is None
    assert bench.recorded_traffic("finalize", "water9000") is None
    # a changed kernel source invalidates the record
    src.write_text("kernel v2\n")
    assert bench.recorded_traffic("mlp", "water9000") is None
    # a record of the current source is found after older records of the stage
    sha2 = hashlib.sha256(b"kernel v2\n").hexdigest()[:16]
    with open(tmp_path / "profiles" / "dram_traffic.txt", "a") as f:
        f.write(f"mlp water9000 12345 {sha2} profiles/y.md (a note)\n")
    assert bench.recorded_traffic("mlp", "water9000") == 12345


def test_oracle_baselines_run_on_the_host():
    # the bench's CPU baseline legs: the single-thread sample and one spawned
    # oracle process per host core
    n, times = bench.oracle_sample_rate("gas24", 10, 2, seed=3)
    assert n == 10 and len(times) == 2 and all(t > 0 for t in times)
    rate, cores = bench.oracle_all_cores("gas24", 5)
    assert cores >= 1 and rate > 0


def test_cell_grid_never_exceeds_the_arena_capacity():
    """The cell grid of one system (linked cells of edge >= the cutoff) holds at
    most 2 n + 27 cells, the per-system capacity the work arena is sized for, and
    every cell is at least the cutoff wide -- also for extents that would
    overflow a plain product of the per-dimension counts (huge, non-finite or
    degenerate bounding boxes).  Host computation of the same function the
    kernels use, through the C ABI (no device call)."""
    import ctypes
    from paper_2207_14276_gb300 import _lib
    L = _lib.lib()
    rng = np.random.Generator(np.random.PCG64(7))
    cases = [((99.9, 99.9, 99.9), 100000), ((44.77,) * 3, 9000), ((10.0, 10.0, 10.0), 24),
             ((1e30, 1e30, 1e30), 10), ((3e38, 1.0, 5e9), 2), ((float("inf"), 1.0, 1.0), 5),
             ((float("nan"), 30.0, 30.0), 50), ((1e-3, 1e-3, 1e-3), 1), ((1e7, 1e7, 1e7), 0),
             ((2.1e9, 2.1e9, 2.1e9), 1 << 30)]
    for _ in range(300):
        n = int(rng.integers(0, 200000))
        cases.append((tuple(float(10.0 ** rng.uniform(-3, 12)) for _ in range(3)), n))
    nc = (ctypes.c_int * 3)()
    cells = ctypes.c_int64()
    for ln, n in cases:
        arr = (ctypes.c_float * 3)(*ln)
        assert L.nnp_debug_cell_grid(arr, ctypes.c_float(5.2), n, nc, ctypes.byref(cells)) == 0
        cap = 2 * n + 27
        got = [nc[0], nc[1], nc[2]]
        assert all(c >= 1 for c in got)
        assert cells.value == got[0] * got[1] * got[2] <= cap, (ln, n, got)
        for c, l in zip(got, np.float32(ln)):
            if c > 1:   # every cell at least the cutoff wide
                assert np.float32(l) / np.float32(c) >= np.float32(5.2) * (1 - 1e-6), (ln, got)
    # a grid that fits is not reshaped: floor(L / rc) cells per dimension
    arr = (ctypes.c_float * 3)(99.9, 99.9, 99.9)
    L.nnp_debug_cell_grid(arr, ctypes.c_float(5.2), 100000, nc, ctypes.byref(cells))
    assert [nc[0], nc[1], nc[2]] == [19, 19, 19]
    assert L.nnp_debug_cell_grid(arr, ctypes.c_float(0.0), 10, nc, ctypes.byref(cells)) != 0


def test_gemm_bytes_and_binding_ceiling():
    """Compulsory bytes of the layer GEMMs, and the roofline entry picks the
    ceiling that binds: B2 on the split path moves 2.25 GB per 100k atoms, more
    time at 6.78 TB/s than its 78.6 GFLOP at a third of 1.89 PFLOP/s."""
    import bench
    s8 = bench.synth.model_spec("ani7x8")
    n = 100000
    b2 = bench.gemm_bytes("mlp_b2", s8, n, "fp32_split")
    assert b2 == pytest.approx(n * (8 * 192 * 4 + 2 * 8 * 256 * 4))
    assert bench.gemm_bytes("mlp_b2", s8, n, "bf16") == pytest.approx(b2 / 2)
    assert bench.gemm_bytes("mlp_b1", s8, n, "fp32_split", (1.0, 0.5)) == pytest.approx(
        n * (8 * 256 * 4 + 1008 * 0.5 * 4))
    assert bench.gemm_bytes("aev_bwd", s8, n, "fp32_split") is None
    peaks = {"hbm_gbs": 6780.0, "bf16_tflops": 1888.8}
    r = bench.roofline({"mlp_b2": (0.5, 1)}, s8, (60.0, 17.0), n, "fp32_split", peaks, "measured",
                       "solvated100k")
    assert r["bound"] == "hbm" and r["kernel"] == "mlp_b2"
    assert r["achieved"] == pytest.approx(b2 / 0.5e-3 / 1e9)
    assert set(r["ceilings"]) == {"tensor", "hbm"}
    assert r["ceilings"]["tensor"]["frac"] < r["frac"]

