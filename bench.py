#!/usr/bin/env python3
"""Throughput and latency of the neural-network-potential energy+force evaluation.

One step = one energy+force evaluation of the whole workload through the C ABI
(cell list -> AEVs -> per-species networks -> analytic forces), inputs resident
in HBM.  Default workload: 'solvated100k' (a 1000-atom solute in 33,000 waters,
100,000 atoms, periodic 99.9 A box, 7-species 1008-dim AEV, an ensemble of 8
networks 1008-256-192-160-1) at FP32 accuracy, the largest single-GPU
configuration; the BF16-network path on the same workload is measured beside
it, and both are compared with the FP64 oracle on a seeded sample of atoms.

  python bench.py [--gpus N --steps K --warmup W] [--workload solvated100k]
                  [--precision fp32|fp32_split|fp32_simt|bf16] [--impl ours|reference]

Under torchrun (N > 1) every rank evaluates its own replica of the workload on
its own GPU (independent replicas, no data-path collective); the time is the
maximum over ranks.  Rank 0 prints one JSON line.

--impl reference times the FP64 CPU oracle (the slow, obviously-correct
restatement of the paper's equations) on the host cores, on a bounded sample of
the same workload's centres per step; under torchrun only rank 0 runs it.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "NN-potential energy+force atom-evals/s at 1 GB300; p50/p99 request latency"
UNIT = "atom-evals/s"
L2_FLUSH_BYTES = 512 << 20   # > 129 MB L2

WORKLOAD_DESC = {
    "water9000": "water9000: 3000 rigid waters (O-H 0.96 A, 104.5 deg) on a jittered lattice, "
                 "9000 atoms, periodic cubic box 44.77 A (1 g/cm^3); 4-species 384-dim AEV "
                 "(16 radial shells Rc 5.2 A, 4x8 angular terms Rc 3.5 A); per-species networks "
                 "384-160-128-96-1 CELU; energy+forces per call",
    "solvated100k": "solvated100k: 1000-atom branched solute in 33,000 waters, 100,000 atoms, "
                    "periodic 99.9 A box; 7-species 1008-dim AEV; 8 networks 1008-256-192-160-1",
    "gas24": "gas24: one 24-atom molecule (H12 C7 N3 O2), non-periodic",
    "water99k": "water99k: 33,000 rigid waters (99,000 atoms) on a jittered 33^3 lattice, "
                "periodic cubic box 99.6 A (1 g/cm^3); 4-species 384-dim AEV; networks "
                "384-160-128-96-1",
    "solvated20k": "solvated20k: 50-atom solute in 6,667 waters, ~20,000 atoms, periodic 58.4 A "
                   "box; 7-species 1008-dim AEV; 8 networks 1008-256-192-160-1",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="solvated100k")
    ap.add_argument("--precision", default="fp32",
                    choices=["fp32", "fp32_split", "fp32_simt", "bf16"])
    ap.add_argument("--fused-chain", action="store_true",
                    help="tensor-core paths: run L2, L3, B3, B2 as the fused per-network "
                         "kernel instead of four layer GEMMs")
    ap.add_argument("--fused-aev-l1", action="store_true",
                    help="BF16 one-network models: AEV computed on chip and fed to the first "
                         "layer in one kernel")
    ap.add_argument("--no-bf16-beside", action="store_true",
                    help="skip the BF16-network measurement beside an FP32 headline")
    ap.add_argument("--no-force-matching", action="store_true",
                    help="skip the force-matching (double backward) measurement")
    ap.add_argument("--oracle-atoms", type=int, default=24,
                    help="seeded sample of atoms whose energies and forces are compared "
                         "with the FP64 oracle (0 to skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--serving-rates", default="1000,2000,5000,10000,20000,50000,1e9",
                    help="Poisson request rates (req/s) of the serving stream (1e8 or more: "
                         "the whole stream at once, the sustained capacity); an empty "
                         "string skips the serving section")
    ap.add_argument("--serving-precision", default="fp32", choices=["fp32", "bf16"],
                    help="network path of the batched server (fp32 by default: one run of "
                         "the BF16 server raised an illegal-address fault whose cause is "
                         "not known, so it runs only when asked for)")
    ap.add_argument("--serving-requests", type=int, default=2000)
    ap.add_argument("--md-steps", type=int, default=100,
                    help="MD-like trajectory steps for the persistent-list (skin) measurement; 0 to skip")
    return ap.parse_args()


# ------------------------------------------------------------------ peaks and roofline
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


SMS = 152
FP32_LANES_PER_SM = 128


def fp32_alu_peak_tflops(sm_mhz):
    """FP32 FMA pipe: 152 SMs x 128 lanes x 2 FLOP per clock."""
    return SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


STAGE_SOURCE = {"mlp": "mlp_fused.cu", "aev_bwd": "aev.cu", "aev_fwd": "aev.cu",
                "neighbors": "nl.cu", "mlp_l1": "mlp_tc.cu", "mlp_l2": "mlp_tc.cu",
                "mlp_l3": "mlp_tc.cu", "mlp_b3": "mlp_tc.cu", "mlp_b2": "mlp_tc.cu",
                "mlp_b1": "mlp_tc.cu", "mlp_chain": "mlp_chain.cu", "aev_l1": "aev.cu"}


def recorded_traffic(stage, workload):
    """DRAM bytes per launch of a stage's kernel from the committed ncu summary, or
    None if there is none for this workload or the kernel source changed since."""
    import hashlib
    here = os.path.dirname(os.path.abspath(__file__))
    src = STAGE_SOURCE.get(stage)
    path = os.path.join(here, "profiles", "dram_traffic.txt")
    if src is None or not os.path.exists(path):
        return None
    with open(os.path.join(here, "paper_2207_14276_gb300", "csrc", src), "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()[:16]
    for line in open(path):
        f = line.split()
        if (len(f) >= 4 and not line.startswith("#") and f[0] == stage and f[1] == workload
                and f[3] == sha):
            return int(f[2])
    return None


# N tile width of the last backward layer by network path (csrc/mlp_tc.cu: on
# the split path 128 wherever the AEV width is a multiple of 128); the layer
# computes the tiles with a live slice
def b1_n_tile(path, Dp):
    return 128 if path == "fp32_split" and Dp % 128 == 0 else 256


def sparse_fractions(masks, Dp, n_tile=256):
    """(fraction of the AEV's 64-column K slices the first layer processes, fraction
    of the last backward layer's N columns it computes) from the tile masks:
    every live slice of a tile, and every n_tile-column block with one."""
    if masks is None or len(masks) == 0:
        return 1.0, 1.0
    n_sl = (Dp + 63) // 64
    k = float(np.mean([bin(int(m) & ((1 << n_sl) - 1)).count("1") for m in masks])) / n_sl
    per = n_tile // 64
    blocks = [(int(m) >> b) & ((1 << per) - 1) for m in masks for b in range(0, n_sl, per)]
    nfrac = float(np.mean([1.0 if x else 0.0 for x in blocks]))
    return k, nfrac


def stage_work(stage, spec, counts, n_atoms, path, sparse=(1.0, 1.0)):
    """Algorithmic work of one launch of a stage: (amount, unit, bound).

    counts: mean radial neighbours n_r and angular neighbours n_a per atom.
    Bytes are compulsory DRAM traffic; FLOPs count the arithmetic the equations
    require: per radial pair 16 shells x 5 FLOP forward / 8 backward (Gaussian,
    cutoff and their derivatives), per angular (j, k) pair 200 forward / 330
    backward (4 Gaussians, 8 factors (1 + cos(theta - theta_z))^32, the 32-term
    contraction and, backward, the derivatives and two edge gradients), and
    2 K N per row for a network layer.  path: the network path of the handle
    ('fp32_simt', 'fp32_split' or 'bf16'); a split-path layer issues three BF16
    tensor products per term of its 2 K N, so its bound is the BF16 peak / 3.
    sparse: the fractions of the first layer's K and the last backward layer's N
    that sparse AEV rows leave (the rest multiplies exact zeros or yields
    columns nothing reads)."""
    D = spec.widths[0]
    E = spec.n_ensemble
    h1, h2, h3 = spec.widths[1:4]
    nr, na = counts
    tri = na * (na - 1) / 2.0
    if stage == "aev_fwd":
        flops = n_atoms * (nr * 16 * 5 + tri * 200)
        return flops, "FLOP", "alu"
    if stage == "aev_bwd":
        flops = n_atoms * (nr * 16 * 8 + tri * 330)
        return flops, "FLOP", "alu"
    if stage == "neighbors":
        return n_atoms * (16 + 4 * (nr + na) + 32), "B", "hbm"
    if stage == "mlp":   # the fused FP32 chain: three layers, output dot, backward to G
        fwd = D * h1 + h1 * h2 + h2 * h3 + h3
        bwd = h3 * h2 + h2 * h1 + h1 * D
        return 2.0 * n_atoms * E * (fwd + bwd), "FLOP", "alu"
    if stage == "aev_l1":   # the AEV forward and the first layer in one kernel (BF16)
        return n_atoms * (nr * 16 * 5 + tri * 200) + 2.0 * n_atoms * D * h1, "FLOP", "alu"
    if stage == "mlp_chain":   # L2, L3, B3, B2 of every member, one fused kernel
        bound = {"bf16": "tensor", "fp32_split": "tensor_split"}.get(path, "alu")
        return 2.0 * n_atoms * E * (2 * h1 * h2 + 2 * h2 * h3), "FLOP", bound
    gemm = {"mlp_l1": (D, E * h1), "mlp_l2": (h1, h2 * E), "mlp_l3": (h2, h3 * E),
            "mlp_b3": (h3, h2 * E), "mlp_b2": (h2, h1 * E), "mlp_b1": (E * h1, D)}
    if stage in gemm:
        k, n = gemm[stage]
        if stage == "mlp_l1":
            k = k * sparse[0]
        if stage == "mlp_b1":
            n = n * sparse[1]
        bound = {"bf16": "tensor", "fp32_split": "tensor_split"}.get(path, "alu")
        return 2.0 * n_atoms * k * n, "FLOP", bound
    return None


def gemm_bytes(stage, spec, n_atoms, path, sparse=(1.0, 1.0)):
    """Compulsory DRAM bytes of one launch of a tensor-core layer: its activation
    input A, the stored activation it multiplies by CELU' (B3, B2), and its
    output, each once (the weights stay in L2).  Stored values take 4 bytes on
    the split path (high and low BF16 parts) and 2 on the BF16 path; the first
    layer reads the live K fraction of the AEV rows, the last writes FP32 dE/dG
    over the live N fraction.  None for other stages."""
    if path not in ("fp32_split", "bf16"):
        return None
    D = spec.widths[0]
    E = spec.n_ensemble
    h1, h2, h3 = spec.widths[1:4]
    v = 4 if path == "fp32_split" else 2
    n = float(n_atoms)
    per_row = {"mlp_l1": D * sparse[0] * v + E * h1 * v,
               "mlp_l2": E * h1 * v + E * h2 * v,
               "mlp_l3": E * h2 * v + E * h3 * v + E * 4,
               "mlp_b3": E * h3 * v + 2 * E * h2 * v,
               "mlp_b2": E * h2 * v + 2 * E * h1 * v,
               "mlp_b1": E * h1 * v + D * sparse[1] * 4}
    return n * per_row[stage] if stage in per_row else None


def roofline(stages, spec, counts, n_eval, path, peaks, peak_src, workload, sparse=(1.0, 1.0)):
    """Roofline entry of the dominant stage (largest time over the profiled pass).

    A tensor-core layer has two ceilings, its FLOPs at the tensor peak and its
    compulsory bytes at the HBM peak; the entry reports the one that binds (the
    longer of the two times) and lists both under "ceilings"."""
    live = [k for k in stages if stages[k][1] > 0]
    if not live:
        return None
    dom = max(live, key=lambda k: stages[k][0])
    dom_ms = stages[dom][0] / stages[dom][1]
    work = stage_work(dom, spec, counts, n_eval, path, sparse)
    if work is None:
        return None
    amount, unit, bound = work
    if unit == "B":
        achieved = amount / (dom_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": float(peaks["hbm_gbs"]),
                "unit": "GB/s", "peak_source": f"{peak_src} (hbm_gbs)"}
    elif bound in ("tensor", "tensor_split"):
        achieved = amount / (dom_ms / 1e3) / 1e12
        peak = float(peaks["bf16_tflops"])
        src = f"{peak_src} (bf16_tflops, burst)"
        if bound == "tensor_split":
            # three BF16 products per FP32-accurate term: the rate this algorithm
            # can reach is a third of the BF16 peak
            peak /= 3.0
            src += " / 3: split operands, three BF16 tensor products per term"
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "peak_source": src}
    else:
        achieved = amount / (dom_ms / 1e3) / 1e12
        peak = fp32_alu_peak_tflops(float(peaks.get("sm_max_mhz", 2070.0)))
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 FLOP x max SM clock "
                               "(the measured-peaks file has no FP32 figure)"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    nbytes = gemm_bytes(dom, spec, n_eval, path, sparse) if roof["bound"] == "tensor" else None
    if nbytes is not None:
        bw = float(peaks["hbm_gbs"])
        hbm = {"bound": "hbm", "achieved": nbytes / (dom_ms / 1e3) / 1e9, "peak": bw, "unit": "GB/s",
               "peak_source": f"{peak_src} (hbm_gbs)", "work_per_launch": nbytes}
        hbm["frac"] = hbm["achieved"] / bw
        ten = {k: roof[k] for k in ("bound", "achieved", "peak", "unit", "peak_source", "frac")}
        ten["work_per_launch"] = amount
        roof["ceilings"] = {"tensor": ten, "hbm": hbm}
        if hbm["frac"] > ten["frac"]:   # the bytes take longer than the FLOPs at their peaks
            roof.update({k: hbm[k] for k in ("bound", "achieved", "peak", "unit", "peak_source", "frac")})
            amount, unit = nbytes, "B"
    roof["traffic"] = recorded_traffic(dom, workload)
    roof.update({"kernel": dom, "launch_ms": dom_ms, "work_per_launch": amount,
                 "work_unit": unit, "network_path": path,
                 "timing": "CUDA events around the kernel on its launching stream, "
                           "second pass of the same K steps"})
    return roof


def oracle_errors(outs, ref, idx):
    """Errors of one evaluation against the FP64 oracle on the sampled atoms idx."""
    ae = outs["atom_energies"].double().cpu().numpy()[idx]
    F = outs["forces"].double().cpu().numpy()[idx]
    dF = F - ref["forces"]
    return {"atom_energy_abs_err_max_kcal_mol": float(np.abs(ae - ref["atom_energies"]).max()),
            "atom_energy_sum_abs_err_kcal_mol": float(abs(ae.sum() - ref["atom_energies"].sum())),
            "force_err_rms_kcal_mol_A": float(np.sqrt(np.mean(dF * dF))),
            "force_err_max_kcal_mol_A": float(np.abs(dF).max()),
            "force_rms_kcal_mol_A": float(np.sqrt(np.mean(ref["forces"] ** 2)))}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """SM clock and clock-event reasons sampled during the timed region.

    Reads NVML directly (read-only queries, ~1 ms period) so that short timed
    regions still get samples; falls back to `nvidia-smi -lms 100`."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid, index):
        self.samples = []       # (time, sm_mhz, max_mhz, reasons_bitmask)
        self.stop_flag = threading.Event()
        self.nvml = None
        self.proc = None
        try:
            import ctypes
            L = ctypes.CDLL("libnvidia-ml.so.1")
            if L.nvmlInit_v2() == 0:
                h = ctypes.c_void_p()
                ok = -1
                if uuid:
                    ok = L.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(h))
                if ok != 0:
                    ok = L.nvmlDeviceGetHandleByIndex_v2(int(index), ctypes.byref(h))
                if ok == 0:
                    self.nvml, self.h, self.ct = L, h, ctypes
        except OSError:
            self.nvml = None

    def _poll_nvml(self):
        ct, L, h = self.ct, self.nvml, self.h
        mhz, mx, rs = ct.c_uint(), ct.c_uint(), ct.c_ulonglong()
        get_r = getattr(L, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            L.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self.stop_flag.is_set():
            L.nvmlDeviceGetClockInfo(h, 1, ct.byref(mhz))
            L.nvmlDeviceGetMaxClockInfo(h, 1, ct.byref(mx))
            get_r(h, ct.byref(rs))
            self.samples.append((time.time(), mhz.value, mx.value, rs.value))
            time.sleep(0.001)

    def _read_smi(self):
        for line in self.proc.stdout:
            f = [x.strip() for x in line.split(",")]
            try:
                bits = 0
                for bit, v in zip((0x8, 0x40, 0x20, 0x4), f[5:9]):
                    if v.lower() == "active":
                        bits |= bit
                self.samples.append((time.time(), float(f[1]), float(f[2]), bits))
            except (ValueError, IndexError):
                pass

    def start(self):
        if self.nvml is not None:
            self.t = threading.Thread(target=self._poll_nvml, daemon=True)
            self.t.start()
            return
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read_smi, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        self.stop_flag.set()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if getattr(self, "t", None) is not None:
            self.t.join(timeout=2)

    def summary(self, t0, t1):
        sel = [s for s in self.samples if t0 <= s[0] <= t1]
        if not sel:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        reasons = set()
        for s in sel:
            for bit, name in self.REASONS.items():
                if s[3] & bit:
                    reasons.add(name)
        return {"sm_mhz": statistics.median(s[1] for s in sel),
                "sm_max_mhz": max(s[2] for s in sel), "reasons": sorted(reasons),
                "samples": len(sel), "source": "nvml" if self.nvml is not None else "nvidia-smi"}


# ------------------------------------------------------------------ reference arm (oracle)
def oracle_sample_rate(workload, n_centres, reps, seed=0):
    import oracle
    systems, kind, wseed = synth.workload(workload)
    s = systems[0]
    spec = synth.model_spec(kind)
    m = oracle.Model(spec, synth.make_weights(spec, wseed))
    rng = np.random.Generator(np.random.PCG64(seed))
    times = []
    for _ in range(reps):
        c = rng.choice(s.n_ml, size=min(n_centres, s.n_ml), replace=False)
        t0 = time.perf_counter()
        m.energy_forces_centres(s.coords, s.species, c, s.box, s.mask)
        times.append(time.perf_counter() - t0)
    return len(c), times


_ORACLE = {}


def _oracle_init(workload):
    import oracle
    systems, kind, wseed = synth.workload(workload)
    spec = synth.model_spec(kind)
    _ORACLE["s"] = systems[0]
    _ORACLE["m"] = oracle.Model(spec, synth.make_weights(spec, wseed))


def _oracle_job(a):
    n_centres, seed = a
    s, m = _ORACLE["s"], _ORACLE["m"]
    rng = np.random.Generator(np.random.PCG64(seed))
    c = rng.choice(s.n_ml, size=min(n_centres, s.n_ml), replace=False)
    m.energy_forces_centres(s.coords, s.species, c, s.box, s.mask)
    return len(c)


def oracle_all_cores(workload, n_centres):
    """The oracle on every host core at once: one process per core (spawned, so
    that no worker inherits the CUDA context), each on its own sample of centres.
    Returns (centres per second, processes)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(cores, initializer=_oracle_init, initargs=(workload,)) as pool:
        pool.map(_oracle_job, [(20, 900 + k) for k in range(cores)])   # workers loaded
        t0 = time.perf_counter()
        done = pool.map(_oracle_job, [(n_centres, 1000 + k) for k in range(cores)])
        wall = time.perf_counter() - t0
    return sum(done) / wall, cores


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n_c = 500
    n, times = oracle_sample_rate(args.workload, n_c, args.warmup + args.steps)
    t = times[args.warmup:]
    value = n * len(t) / sum(t)
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(t) / len(t), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC.get(args.workload, args.workload),
                   "sample": f"{n} random centres per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{n} centres of {args.workload} per step, single thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))
    return 0


# ------------------------------------------------------------------ multi-rank aggregation
def max_over_ranks(x, dist=None, device=None):
    """Maximum of a float over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step, steps, local_ms, dist=None, device=None):
    """Whole-job throughput of independent replicas: every rank processes
    units_per_rank_step per step; the job takes as long as its slowest rank."""
    world = dist.get_world_size() if (dist is not None and dist.is_initialized()) else 1
    total_ms = max_over_ranks(local_ms, dist, device)
    return units_per_rank_step * steps * world / (total_ms / 1e3), total_ms


# ------------------------------------------------------------------ serving
def drive_stream(srv, reqs, rids):
    """Submit requests at their scheduled Poisson arrival times from this thread,
    poll completions from a second one.  Latency = completion - scheduled arrival
    (the lag of the submitting thread plus the server's submit-to-done time)."""
    n = len(reqs)
    tickets = [0] * n
    lag = [0.0] * n
    done = [None] * n

    def poller():
        for k in range(n):
            while tickets[k] == 0:
                time.sleep(0)
            done[k] = srv.poll(tickets[k])

    th = threading.Thread(target=poller)
    th.start()
    t0 = time.perf_counter() + 0.02
    t_sub = time.perf_counter()
    for k, r in enumerate(reqs):
        target = t0 + r.arrival_s
        while True:
            now = time.perf_counter()
            if now >= target:
                break
            if target - now > 2e-3:
                time.sleep(target - now - 1e-3)
        if r.system is not None:
            tk = srv.submit(r.system.coords, r.system.species)
        else:
            tk = srv.submit(r.solute_xyz, resident_id=rids[r.box_id])
        lag[k] = time.perf_counter() - target
        tickets[k] = tk
    t_sub = time.perf_counter() - max(t_sub, t0)
    th.join()
    lat = np.array([lag[k] + done[k][3] for k in range(n)])
    bad = sum(1 for d in done if d[0] != 0)
    makespan = max(reqs[k].arrival_s + lat[k] for k in range(n))
    atoms = sum(r.n_ml for r in reqs)
    out = {"p50_ms": 1e3 * float(np.percentile(lat, 50)),
           "p99_ms": 1e3 * float(np.percentile(lat, 99)),
           "atom_evals_per_s": atoms / makespan,
           "offered_atom_evals_per_s": atoms / max(reqs[-1].arrival_s, 1e-9),
           "submit_req_per_s": n / max(t_sub, 1e-9),
           "requests": n, "failed": bad}
    return out, done


def run_serving(rates, n_requests, precision="fp32", lanes=2, max_systems=256,
                max_atoms=262144, seed=3, oracle_sample=0):
    from paper_2207_14276_gb300 import Potential
    from paper_2207_14276_gb300.serving import Server
    spec = synth.model_spec("ani7")
    pot = Potential(spec, synth.make_weights(spec, 1), precision=precision)
    boxes = synth.resident_boxes()
    srv = Server(pot, n_lanes=lanes, max_batch_atoms=max_atoms, max_batch_systems=max_systems)
    rids = [srv.register(b.coords, b.species, b.box, b.mask) for b in boxes]
    # warm-up: every lane sees a full-size batch once
    drive_stream(srv, synth.request_stream(1e6, 64, seed=999, boxes=boxes), rids)
    out = {}
    errs = []
    for i, rate in enumerate(rates):
        # at least 0.4 s of arrivals per rate; a rate of 1e8 req/s or more submits
        # the whole stream at once and so measures the sustained capacity
        saturated = rate >= 1e8
        n_req = 5 * n_requests if saturated else max(n_requests, int(0.4 * rate))
        reqs = synth.request_stream(rate, n_req, seed=seed + i, boxes=boxes)
        b0, r0 = srv.stats()
        res, done = drive_stream(srv, reqs, rids)
        b1, r1 = srv.stats()
        res["mean_batch"] = (r1 - r0) / max(b1 - b0, 1)
        if saturated:
            del res["offered_atom_evals_per_s"]
        out["saturated" if saturated else str(int(rate))] = res
        if oracle_sample and i == len(rates) - 1:
            # the served results of the first gas-phase requests of the last
            # stream (the largest batches) against the FP64 oracle
            import oracle
            orc = oracle.Model(spec, synth.make_weights(spec, 1))
            for r, d in zip(reqs, done):
                if r.system is None or d[0] != 0:
                    continue
                ref = orc.energy_forces(r.system.coords, r.system.species)
                dF = np.asarray(d[2], np.float64).reshape(-1, 3) - ref["forces"]
                errs.append((abs(float(d[1]) - ref["energy"]), float(np.sqrt(np.mean(dF * dF))),
                             float(np.abs(dF).max())))
                if len(errs) >= oracle_sample:
                    break
    if errs:
        e = np.array(errs)
        out["errors_vs_oracle"] = {
            "sample": f"the first {len(errs)} gas-phase requests of the last stream "
                      f"({'saturated' if rates[-1] >= 1e8 else f'{int(rates[-1])} req/s'})",
            "energy_abs_err_max_kcal_mol": float(e[:, 0].max()),
            "force_err_rms_kcal_mol_A": float(np.sqrt(np.mean(e[:, 1] ** 2))),
            "force_err_max_kcal_mol_A": float(e[:, 2].max())}
    srv.close()
    return out


def force_matching_section(dev, stream, steps=20, warmup=3):
    """The differentiation workload: 64 molecules of 20-60 atoms (4-species model),
    loss sum((F - F_target)^2) with F_target ~ N(0, 1 kcal/mol/A) (PCG64(4)),
    gradients w.r.t. every weight and coordinate through the autograd wrapper
    whose backward is the library's force vector-Jacobian product.  Timed per
    forward + backward step with CUDA events; gradients compared once with the
    FP64 oracle's (dual-number) force-matching gradient."""
    import torch
    import oracle
    from paper_2207_14276_gb300 import Potential
    from paper_2207_14276_gb300.autograd import NNPBatchFunction
    spec = synth.model_spec("ani4")
    w = synth.make_weights(spec, 1)
    pot = Potential(spec, w)
    mols, _, _ = synth.workload("molecules64")
    rng = np.random.Generator(np.random.PCG64(4))
    targets = [rng.normal(0.0, 1.0, size=(m.n_atoms, 3)) for m in mols]
    sizes = [m.n_atoms for m in mols]
    x0 = torch.from_numpy(np.concatenate([m.coords for m in mols])).to(dev)
    sp = torch.from_numpy(np.concatenate([m.species for m in mols])).to(dev)
    Ft = torch.from_numpy(np.concatenate(targets)).float().to(dev)
    w0 = torch.from_numpy(w).to(dev)

    def step():
        x = x0.clone().requires_grad_(True)
        wt = w0.clone().requires_grad_(True)
        E, F = NNPBatchFunction.apply(x, wt, pot, sp, sizes)
        loss = ((F - Ft) ** 2).sum()
        loss.backward()
        return x.grad, wt.grad

    for _ in range(warmup):
        step()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(steps):
        gx, gw = step()
    ev[1].record(stream)
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / steps
    orc = oracle.Model(spec, w)
    gw_ref = np.zeros(w.size)
    gx_ref = []
    for m, t in zip(mols, targets):
        Fm = orc.energy_forces(m.coords, m.species)["forces"]
        _, _, gxm, gwm = orc.force_matching(m.coords, m.species, 2 * (Fm - t))
        gw_ref += gwm
        gx_ref.append(gxm)
    gx_ref = np.concatenate(gx_ref)

    def err(a, b):
        a = a.double().cpu().numpy().reshape(-1)
        b = b.reshape(-1)
        return {"max_abs_err_over_max_abs": float(np.abs(a - b).max() / np.abs(b).max()),
                "norm_rel_err": float(np.linalg.norm(a - b) / np.linalg.norm(b))}
    n_at = sum(sizes)
    return {"workload": "64 molecules of 20-60 atoms (H:C:N:O 12:7:3:2), 4-species model; loss "
                        "sum((F - F_target)^2), F_target ~ N(0, 1 kcal/mol/A); gradients w.r.t. "
                        "all weights and coordinates (forward + hand-written double backward)",
            "ms_per_step": ms, "value": n_at / (ms / 1e3), "unit": UNIT + " (forward + backward)",
            "errors_vs_oracle": {"dL_dcoords": err(gx, gx_ref), "dL_dweights": err(gw, gw_ref)}}


# ------------------------------------------------------------------ our arm
def md_trajectory(spec, w, precision, x0, sp, box, mask, n_eval, steps, skin, sigma, flush, dev):
    """Energy+force calls along a random-walk trajectory (each coordinate moves by
    N(0, sigma) A per step), every frame copied into one coordinate buffer as an
    integrator would update it.  Returns (ms per step incl. the copy, list builds)."""
    import torch
    from paper_2207_14276_gb300 import Potential
    pot = Potential(spec, w, precision=precision)
    pot.set_skin(skin)
    gen = torch.Generator(device=dev).manual_seed(11)
    frames = [x0]
    for _ in range(steps):
        frames.append(frames[-1] + sigma * torch.randn(x0.shape, device=dev, generator=gen))
    xb = x0.clone()
    E = torch.empty(1, dtype=torch.float64, device=dev)
    F = torch.empty((x0.shape[0], 3), dtype=torch.float32, device=dev)
    pot.energy_forces(xb, sp, box, mask)      # establishes capacities
    for _ in range(3):
        pot.energy_forces_into(xb, sp, box, mask, E, F)
    stream = torch.cuda.current_stream(dev)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    b0 = pot.list_stats()[0]
    for k in range(steps):
        flush.fill_(k & 0xff)
        starts[k].record(stream)
        xb.copy_(frames[k + 1])
        pot.energy_forces_into(xb, sp, box, mask, E, F)
        ends[k].record(stream)
    torch.cuda.synchronize()
    if pot.sync_status() != 0:
        raise RuntimeError("device status after the trajectory")
    ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends)) / steps
    return ms, pot.list_stats()[0] - b0


def run_ours(args):
    import torch
    from paper_2207_14276_gb300 import Potential

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    systems, kind, wseed = synth.workload(args.workload)
    spec = synth.model_spec(kind)
    w = synth.make_weights(spec, wseed)
    pot = Potential(spec, w, precision=args.precision)
    if args.fused_chain:
        pot.set_fused_chain(True)
    pot.set_fused_aev_l1(args.fused_aev_l1)
    s = systems[0]
    x = torch.from_numpy(s.coords).to(dev)
    sp = torch.from_numpy(s.species).to(dev)
    mask = None if s.mask is None else torch.from_numpy(s.mask).to(dev)
    box = None if s.box is None else [float(b) for b in s.box]
    n_eval = s.n_ml
    E = torch.empty(1, dtype=torch.float64, device=dev)
    F = torch.empty((s.n_atoms, 3), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    # first call establishes the neighbour capacity (grows and retries if needed)
    pot.energy_forces(x, sp, box, mask)
    for _ in range(args.warmup):
        pot.energy_forces_into(x, sp, box, mask, E, F)
    assert pot.sync_status() == 0
    launches_per_step = pot.launch_count()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    # neighbour statistics for the roofline accounting
    nb_r = pot.debug_neighbors(s.n_atoms, angular=False).ne(-1).sum(1).float()
    nb_a = pot.debug_neighbors(s.n_atoms, angular=True).ne(-1).sum(1).float()
    sel = torch.ones(s.n_atoms, dtype=torch.bool, device=dev) if mask is None else mask.bool()
    counts = (float(nb_r[sel].mean()), float(nb_a[sel].mean()))

    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)
    uuid = ("GPU-" + str(uuid)) if uuid is not None else None
    clocks = ClockSampler(uuid, local)
    clocks.start()
    time.sleep(0.3)
    def timed_steps(profile, p=pot):
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        p.profile_read(reset=True)
        p.profile(profile)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        t_a = time.time()
        for k in range(args.steps):
            flush.fill_(k & 0xff)        # evict the previous step's data from L2
            starts[k].record(stream)
            p.energy_forces_into(x, sp, box, mask, E, F)
            ends[k].record(stream)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        t_b = time.time()
        p.profile(False)
        rc = p.sync_status()
        if rc != 0:
            raise RuntimeError(f"device status {rc} after the timed region")
        return [a.elapsed_time(b) for a, b in zip(starts, ends)], t_a, t_b

    # timed region: K steps, no per-stage events
    step_ms, t0, t1 = timed_steps(False)
    clocks.stop()
    total_ms = sum(step_ms)
    # second pass over the same K steps with CUDA events around every stage on the
    # launching stream: per-kernel durations for the roofline
    prof_ms, _, _ = timed_steps(True)
    stages = pot.profile_read(reset=True)
    value, total_ms = whole_job_rate(n_eval, args.steps, total_ms, dist, dev)

    # roofline of the dominant kernel (largest stage time over the timed region)
    peaks, peak_src = measured_peaks()
    clk = clocks.summary(t0, t1)
    path = pot.network_path()
    Dp = (spec.widths[0] + 63) // 64 * 64
    sparse = sparse_fractions(pot.tile_masks() if path != "fp32_simt" else None, Dp, b1_n_tile(path, Dp))
    roof = roofline(stages, spec, counts, n_eval, path, peaks, peak_src, args.workload, sparse)

    # end to end through the host entry point (pinned host buffers, copies inside)
    e2e = None
    if args.e2e_steps > 0:
        hx = torch.from_numpy(s.coords).pin_memory().numpy()
        hs = torch.from_numpy(s.species).pin_memory().numpy()
        hm = None if s.mask is None else torch.from_numpy(s.mask).pin_memory().numpy()
        hF = torch.empty((s.n_atoms, 3), dtype=torch.float32).pin_memory().numpy()
        for _ in range(2):
            pot.energy_forces_host_into(hx, hs, s.box, hm, out_forces=hF)
        e2e_t = []
        for _ in range(args.e2e_steps):
            t_a = time.perf_counter()
            pot.energy_forces_host_into(hx, hs, s.box, hm, out_forces=hF)
            e2e_t.append(time.perf_counter() - t_a)
        h2d = s.n_atoms * 12 + s.n_atoms + (s.n_atoms if s.mask is not None else 0)
        e2e = {"value": n_eval * len(e2e_t) / sum(e2e_t), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 8 + s.n_atoms * 12,
               "p50_ms": 1e3 * float(np.percentile(e2e_t, 50)),
               "p99_ms": 1e3 * float(np.percentile(e2e_t, 99))}
        if dist is not None:
            # whole-job e2e rate: every rank's replica, limited by the slowest rank
            e2e["value"] = world * n_eval / max_over_ranks(n_eval / e2e["value"], dist, dev)

    # accuracy against the FP64 oracle on a seeded sample of (ML-region) atoms
    errors = None
    idx = None
    if args.oracle_atoms > 0 and rank == 0:
        import oracle
        rng = np.random.Generator(np.random.PCG64(11))
        ml = np.nonzero(s.mask)[0] if s.mask is not None else np.arange(s.n_atoms)
        idx = np.sort(rng.choice(ml, size=min(args.oracle_atoms, ml.size), replace=False))
        t_o = time.perf_counter()
        ref = oracle.Model(spec, w).sample(s.coords, s.species, idx, s.box, s.mask)
        t_o = time.perf_counter() - t_o
        d = {"coords": x, "species": sp, "box": box, "mask": mask}
        errors = {"sample": f"{idx.size} atoms of {args.workload} drawn with PCG64(11) among "
                            f"the ML-region atoms; oracle time {t_o:.1f} s",
                  path: oracle_errors(pot.energy_forces_batch([d], atom_energies=True)[0],
                                      ref, idx)}

    # the BF16-network path on the same workload, beside an FP32 headline
    beside = None
    if args.precision != "bf16" and not args.no_bf16_beside:
        pb = Potential(spec, w, precision="bf16")
        if args.fused_chain:
            pb.set_fused_chain(True)
        pb.energy_forces(x, sp, box, mask)
        for _ in range(args.warmup):
            pb.energy_forces_into(x, sp, box, mask, E, F)
        assert pb.sync_status() == 0
        b_ms, _, _ = timed_steps(False, pb)
        b_value, b_total = whole_job_rate(n_eval, args.steps, sum(b_ms), dist, dev)
        timed_steps(True, pb)
        b_stages = pb.profile_read(reset=True)
        beside = {"precision": "bf16", "value": b_value, "unit": UNIT,
                  "ms_per_step": b_total / args.steps,
                  "latency_ms": {"p50": float(np.percentile(b_ms, 50)),
                                 "p99": float(np.percentile(b_ms, 99))},
                  "roofline": roofline(b_stages, spec, counts, n_eval, "bf16", peaks, peak_src,
                                       args.workload, sparse_fractions(pb.tile_masks(), Dp, b1_n_tile("bf16", Dp))),
                  "stages_ms_per_step": {k: v[0] / max(v[1], 1) for k, v in b_stages.items()
                                         if v[1]}}
        if errors is not None:
            d = {"coords": x, "species": sp, "box": box, "mask": mask}
            errors["bf16"] = oracle_errors(pb.energy_forces_batch([d], atom_energies=True)[0],
                                           ref, idx)
            beside["errors_vs_oracle"] = errors["bf16"]
        pb.close()

    md = None
    if args.md_steps > 0 and rank == 0:
        sigma = 0.01
        t_rb, b_rb = md_trajectory(spec, w, args.precision, x, sp, box, mask, n_eval,
                                   args.md_steps, 0.0, sigma, flush, dev)
        md = {"workload": f"{args.workload} along a random-walk trajectory, every coordinate "
                          f"N(0, {sigma} A) per step, frame copied into the coordinate buffer "
                          "inside the timed step; L2 flushed between steps",
              "steps": args.md_steps,
              "lists_rebuilt_every_step": {"ms_per_step": t_rb, "value": n_eval / (t_rb / 1e3),
                                           "unit": UNIT}}
        for skin in (0.5, 1.0):
            t_sk, b_sk = md_trajectory(spec, w, args.precision, x, sp, box, mask, n_eval,
                                       args.md_steps, skin, sigma, flush, dev)
            md[f"skin_{skin}A"] = {"ms_per_step": t_sk, "value": n_eval / (t_sk / 1e3),
                                   "unit": UNIT, "list_builds": b_sk}

    # multiple-time-step driver: ML forces on a masked solute every outer step
    respa = None
    if args.md_steps > 0 and rank == 0:
        from paper_2207_14276_gb300.respa import RespaDriver
        hs = synth.resident_boxes(n_boxes=1)[0]
        hspec = synth.model_spec("ani7")
        hw = synth.make_weights(hspec, 1)
        hx = torch.from_numpy(hs.coords).to(dev)
        drv = RespaDriver(Potential(hspec, hw, precision=args.precision), hx,
                          torch.from_numpy(hs.species).to(dev), hspec.atomic_numbers,
                          box=[float(b) for b in hs.box], mask=torch.from_numpy(hs.mask).to(dev),
                          dt_outer=2.0, n_inner=4, skin=0.5, temperature=300.0, seed=3)
        for _ in range(5):
            drv.step()
        torch.cuda.synchronize()
        b0 = drv.pot.list_stats()[0]
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        for _ in range(args.md_steps):
            drv.step()
        ev[1].record(stream)
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / args.md_steps
        n_ml = int(hs.mask.sum())
        respa = {"workload": f"{n_ml}-atom solute (ML region, mask) in a {hs.n_atoms}-atom "
                             "solvated box, 7-species model; outer step 2 fs with 4 inner "
                             "drifts (MM forces left out), 0.5 A skin; 300 K start",
                 "outer_steps": args.md_steps, "ms_per_outer_step": ms,
                 "outer_steps_per_s": 1e3 / ms, "value": n_ml / (ms / 1e3), "unit": UNIT,
                 "list_builds": drv.pot.list_stats()[0] - b0}

    # energy-only re-evaluation of a batch of snapshots (reweighting, no forces)
    snap = None
    if args.md_steps > 0 and rank == 0:
        n_frames = 16 if s.n_atoms <= 20000 else 4
        gen = torch.Generator(device=dev).manual_seed(12)
        frames = [{"coords": x + 0.05 * torch.randn(x.shape, device=dev, generator=gen),
                   "species": sp, "box": box, "mask": mask} for _ in range(n_frames)]
        snap = {"workload": f"{n_frames} snapshots of {args.workload} (coordinates "
                            "perturbed by N(0, 0.05 A)) as one batch call; L2 flushed between calls"}
        for name, want_f in (("energy_only", False), ("energy_forces", True)):
            pb = Potential(spec, w, precision=args.precision)
            outs = pb.energy_forces_batch(frames, forces=want_f)
            for _ in range(3):
                outs = pb.energy_forces_batch(frames, forces=want_f, check_status=False,
                                              outputs=outs)
            reps = 10
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
            for k in range(reps):
                flush.fill_(k & 0xff)
                ev[2 * k].record(stream)
                outs = pb.energy_forces_batch(frames, forces=want_f, check_status=False,
                                              outputs=outs)
                ev[2 * k + 1].record(stream)
            torch.cuda.synchronize()
            if pb.sync_status() != 0:
                raise RuntimeError("device status after the snapshot batch")
            ms = sum(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(reps)) / reps
            snap[name] = {"ms_per_batch": ms, "value": n_frames * n_eval / (ms / 1e3), "unit": UNIT}

    fmatch = None
    if not args.no_force_matching and rank == 0:
        fmatch = force_matching_section(dev, stream)

    serving = None
    if args.serving_rates and rank == 0:
        rates = [float(r) for r in args.serving_rates.split(",") if r]
        serving = {
            "workload": "request stream: 70% gas-phase molecules of 10-120 atoms, 30% new "
                        "solute coordinates (30-80 atoms) for one of 8 resident ~20k-atom "
                        "solvated boxes (mask = solute); 7-species 1008-dim AEV, networks "
                        "1008-256-192-160-1; Poisson arrivals; latency from scheduled arrival"}
        # the serving runs come last among the GPU sections: a failure there is
        # recorded in its entry and leaves the measurements above intact
        for key, fn in ((f"batched_{args.serving_precision}",
                         lambda: run_serving(rates, args.serving_requests, args.serving_precision,
                                             lanes=2, oracle_sample=100)),
                        ("one_system_per_launch_fp32",
                         lambda: run_serving([r for r in rates if r <= 5000] + [1e9],
                                             args.serving_requests, "fp32",
                                             lanes=1, max_systems=1))):
            try:
                serving[key] = fn()
            except Exception as e:   # noqa: BLE001 - reported in the JSON line
                serving[key] = {"error": f"{type(e).__name__}: {e}"}
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        # about 10 s of single-thread oracle work: a 100-centre probe sizes the sample
        n_p, t_p = oracle_sample_rate(args.workload, 100, 1, seed=2)
        n_s = int(min(20000, max(200, n_p / t_p[0] * 10.0 / 4)))
        n_c, times = oracle_sample_rate(args.workload, n_s, 4, seed=1)
        cpu = {"value": n_c * len(times) / sum(times), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{len(times)} x {n_c} random centres of {args.workload} "
                         f"(energy + forces of their terms), FP64, single thread, "
                         f"{sum(times):.1f} s"}
        try:
            rate, cores = oracle_all_cores(args.workload, n_c)
            cpu["all_cores"] = {"value": rate, "unit": UNIT, "cores": cores,
                                "sample": f"{cores} processes x {n_c} random centres of "
                                          f"{args.workload}, one process per host core"}
        except Exception as e:   # noqa: BLE001 - the single-thread figure stands alone
            cpu["all_cores"] = {"error": f"{type(e).__name__}: {e}"}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16-mlp/f32" if path == "bf16" else "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC.get(args.workload, args.workload),
                   "atoms_per_step": n_eval, "systems_per_step": 1,
                   "parallelism": f"replicas x{world}",
                   "l2": "flushed between steps (512 MB write)", "precision": args.precision,
                   "network_path": {"fp32_split": "tensor cores, FP32 operands split into "
                                                  "two BF16 parts, three products per term, "
                                                  "FP32 accumulation",
                                    "fp32_simt": "FP32 FMA pipes",
                                    "bf16": "tensor cores, BF16 operands, FP32 "
                                            "accumulation"}[path]},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                       "p99": float(np.percentile(step_ms, 99))},
        "roofline": roof,
        "errors_vs_oracle": errors,
        "bf16_beside": beside,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk,
        "gpu_launches": launches_per_step * args.steps,
        "stages_ms_per_step": {k: v[0] / max(v[1], 1) for k, v in stages.items() if v[1]},
        "stage_pass_ms_per_step": sum(prof_ms) / len(prof_ms),
        "neighbours_per_atom": {"radial": counts[0], "angular": counts[1]},
        "sparse_aev_rows": {"first_layer_k_fraction": sparse[0],
                            "last_layer_n_fraction": sparse[1]},
        "serving": serving,
        "persistent_lists": md,
        "snapshot_batch": snap,
        "respa_driver": respa,
        "force_matching": fmatch,
    }
    print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
