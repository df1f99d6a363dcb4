#!/usr/bin/env python
"""Throughput of NNP energy + force evaluation on GB300, in atom-evals/s.

One step = one energy + force evaluation of a whole batch (neighbour lists,
features, the 8-network ensemble forward and reverse, the featurizer's reverse
pass to coordinates), i.e. every stage of the path.  Default workload: 512
molecules with 20-120 atoms (H .45, C .35, N .08, O .08, F/S/Cl .04), random
Xavier-normal ANI-2x-architecture weights, network products in BF16 on the
tensor cores (three split-operand products per forward layer, the form that
meets the stated per-molecule energy bound; FP16 is timed alongside),
replayed as one CUDA graph per step.  An atom-eval is one atom's share of E
and F for the full ensemble.

Also reported in the same line: the same batch with FP32 networks (batched,
graph) and with single-product 16-bit networks; the plain FP32 unbatched GPU
path on a sample of the same molecules (one molecule per call, direct
launches); the per-molecule errors of every precision against the FP64 oracle
over the whole batch; the end-to-end number through the host-buffer entry
point; per-stage times with their rooflines; the 4096-molecule workload with
its 1500-atom periodic pocket and its device memory; the 60-atom molecule over
1000 perturbed steps; the NNP-MM coupling term; and the FP64 CPU oracle on all
host cores and on one.

Usage: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2201_08110_gb300 import workloads as W  # noqa: E402

METRIC = "NNP energy+force atom-evals/s vs plain FP32 path on 1 GB300 at stated error"
UNIT = "atom-evals/s"
L2_BYTES = 129 * 1024 * 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16", "fp16"],
                    help="arithmetic of the networks' matrix products (16-bit: three split-operand "
                         "products per forward layer unless --single-pass)")
    ap.add_argument("--single-pass", action="store_true",
                    help="16-bit networks with one product per forward layer (faster; misses the "
                         "per-molecule relative energy bound where atomic energies cancel)")
    ap.add_argument("--alt-precision", default="fp16", choices=["none", "fp32", "bf16", "fp16"],
                    help="a second precision timed the same way and reported alongside")
    ap.add_argument("--workload", type=int, default=3, choices=[2, 3, 5],
                    help="3: the 512-molecule batch (default, headline, with every other "
                         "measurement in the same line); 2: one 60-atom molecule over perturbed "
                         "coordinates; 5: 4096 molecules of 30-250 atoms plus a 1500-atom "
                         "periodic pocket")
    ap.add_argument("--w2-fast", action="store_true",
                    help="workload 2 on the --precision tensor-core path with graph replay "
                         "instead of the plain FP32 path")
    ap.add_argument("--molecules", type=int, default=512)
    ap.add_argument("--unbatched-sample", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-coupling", action="store_true",
                    help="skip the NNP-MM coupling term's measurement")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline only: skip the FP32 / single-pass batches, the error report, "
                         "workloads 2 and 5 and the MD loop")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default schedule instead of nnp_autotune's choice")
    ap.add_argument("--schedule", default=None,
                    help="pin the schedule instead of autotuning: featurizer warps, reverse "
                         "warps, reverse centres per item, first-layer N tile, shared "
                         "accumulators (comma-separated, as autotune reports them)")
    return ap.parse_args()


# ---------------------------------------------------------------- helpers ----

def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def rank_batch(n_mols: int, rank: int):
    """Workload 3's batch on rank 0; other ranks draw their own molecules of the
    same distribution (weak scaling: per-rank work is fixed)."""
    b, w, M = W.config3(n_mols)
    if rank == 0:
        return b, w, M
    sizes = np.random.Generator(np.random.PCG64(W.workload_seed(3) + 100 + rank)).integers(
        20, 121, size=n_mols)
    return W.batch(W.workload_seed(3) + 7919 * rank, sizes), w, M


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


class Clocks:
    """nvidia-smi sampling during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, n in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(n)
        loaded = [s for s in sm if s > 0.5 * (max(mx) if mx else 1)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d["hbm_gbs"], d["bf16_tflops"], d.get("bf16_tflops_sustained"), "measured", d.get("sm_max_mhz", 2070.0)
    return 6800.0, 1900.0, 1700.0, "fallback", 2070.0




# Algorithmic work per stage: operations (or bytes) per unit of work, times the units.
HID = W.HIDDEN
# FP32 operations of the featurizer per directed radial pair / unordered
# angular pair of neighbours (exp2 and log2 counted as one operation each).
FLOP_RADIAL_FWD, FLOP_ANGULAR_FWD = 100.0, 142.0
FLOP_RADIAL_REV, FLOP_ANGULAR_REV = 137.0, 300.0
FLOP_DISTANCE = 8.0  # one neighbour-search distance test
N_FEATURES = 1008


def stage_work(Z, M: int, n_pairs: float, n_triples: float, n_tests: float, prec: str,
               split: bool):
    """{stage: (bound, algorithmic work, work executed, hbm bytes)}.

    Tensor stages: FLOPs of the method's matrix products from the element
    counts (first-layer K = the 1008 real features); "executed" counts the
    products the kernels issue (three per forward product with split operands;
    the split path's reverse kernel also recomputes its single-product forward).
    Featurizer stages: FP32 operations from the pair / triple counts, and the
    bytes the method must move per atom: the feature row as stored (FP32, or
    16-bit hi and lo halves) and its position (featurizer), dE/dG in FP32, the
    position and the FP64 force (reverse pass)."""
    zs = list(W.ELEMENTS_Z)
    cnt = [int(np.sum(Z == z)) for z in zs]
    n = float(sum(cnt))
    l1 = l2 = l3 = out = 0.0
    for e, k in enumerate(cnt):
        h1, h2, h3 = HID[e]
        l1 += 2.0 * k * M * h1 * N_FEATURES
        l2 += 2.0 * k * M * h1 * h2
        l3 += 2.0 * k * M * h2 * h3
        out += 2.0 * k * M * h3
    f = 3.0 if split else 1.0
    feat_bytes = {"fp32": 4.0, "bf16": 2.0, "fp16": 2.0}[prec] * (2.0 if split else 1.0)
    work = {
        "neighbors": ("alu", n_tests * FLOP_DISTANCE, None, None),
        "features": ("alu", n_pairs * FLOP_RADIAL_FWD + n_triples * FLOP_ANGULAR_FWD, None,
                     n * (N_FEATURES * feat_bytes + 16.0)),
        "l1_fwd": ("tensor", l1, f * l1, None),
        "l1_rev": ("tensor", l1, l1, None),
        "adjoint": ("alu", n_pairs * FLOP_RADIAL_REV + n_triples * FLOP_ANGULAR_REV, None,
                    n * (N_FEATURES * 4.0 + 16.0 + 24.0)),
    }
    if prec == "fp32":
        work.update({"l2_fwd": ("tensor", l2, l2, None), "l3_fwd": ("tensor", l3 + out, l3 + out, None),
                     "l3_rev": ("tensor", l3, l3, None), "l2_rev": ("tensor", l2, l2, None)})
    elif split:
        # the tail: layers 2 and 3 forward (three products each) with the
        # output layer, and both hidden layers reverse
        work["tail"] = ("tensor", 2 * l2 + 2 * l3 + out, 4 * l2 + 4 * l3 + out, None)
    else:
        # the fused tail: both hidden layers forward, the output layer and both reverse
        work["tail"] = ("tensor", 2 * l2 + 2 * l3 + out, 2 * l2 + 2 * l3 + out, None)
    return work


def shown_stages(stages: dict, prec: str) -> dict:
    """Stage times under the names of the kernels that ran (nnp_compute_timed's
    slots: the fused tail in l2_fwd)."""
    if prec == "fp32":
        return dict(stages)
    out = {k: v for k, v in stages.items() if k not in ("l2_fwd", "l3_fwd", "l3_rev", "l2_rev")}
    out["tail"] = stages["l2_fwd"]
    return out


def rooflines_of(shown: dict, work: dict, tensor_path: bool, hbm: float, bf16: float,
                 peak_kind: str, fp32_peak: float) -> dict:
    out = {}
    for k, ms in shown.items():
        if k not in work or ms <= 0:
            continue
        bound, amount, executed, nbytes = work[k]
        if bound == "tensor" and tensor_path:
            peak, unit, note = bf16, "TFLOP/s", f"{peak_kind} dense bf16 (fp16 equal rate)"
        else:
            bound = "alu"
            peak, unit, note = fp32_peak, "TFLOP/s", "derived FP32 FMA peak: 152 SMs x 128 lanes x 2 x max SM clock"
        achieved = amount / (ms * 1e-3) / 1e12
        r = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
             "frac": achieved / peak, "work": amount, "ms": ms, "peak_note": note}
        if executed is not None and executed != amount:
            r["executed_work"] = executed
            r["executed_frac"] = executed / (ms * 1e-3) / 1e12 / peak
        if nbytes is not None:
            gbs = nbytes / (ms * 1e-3) / 1e9
            r["hbm"] = {"bytes": nbytes, "achieved_gbs": gbs, "peak_gbs": hbm,
                        "frac": gbs / hbm, "peak_note": f"{peak_kind} copy bandwidth"}
        out[k] = r
    return out


# The kernel behind each stage of the tensor-core path: the first layer's
# pair kernel runs two launches a step (its forward and its reverse
# product); on the FP32 path every stage is its own launch.
KERNEL_STAGES = {"k_gemm_tc2": ("l1_fwd", "l1_rev"), "k_mlp_tail": ("tail",), "k_aev": ("features",),
                 "k_aev_adjoint": ("adjoint",), "k_neighbors_mol": ("neighbors",)}
KERNEL_SRC = {"k_gemm_tc2": "mlp_tc.cu", "k_mlp_tail": "mlp_tail_tc.cu", "k_aev": "aev.cu",
              "k_aev_adjoint": "aev.cu", "k_neighbors_mol": "aev.cu"}


def dominant_kernel(rooflines: dict, tensor_path: bool, n_atoms: int) -> dict:
    """The roofline of the kernel with the most time per step: its work and
    time per launch averaged over its launches (achieved = algorithmic work
    per launch / average launch duration), the ncu DRAM traffic per launch
    when the kernel's source still matches the capture, else null."""
    if tensor_path:
        groups = {k: [s for s in st if s in rooflines] for k, st in KERNEL_STAGES.items()}
    else:
        groups = {s: [s] for s in rooflines}
    groups = {k: st for k, st in groups.items() if st}
    name = max(groups, key=lambda k: sum(rooflines[s]["ms"] for s in groups[k]))
    st = groups[name]
    n = len(st)
    r0 = rooflines[st[0]]
    ms = sum(rooflines[s]["ms"] for s in st) / n
    work = sum(rooflines[s]["work"] for s in st) / n
    executed = sum(rooflines[s].get("executed_work", rooflines[s]["work"]) for s in st) / n
    achieved = work / (ms * 1e-3) / 1e12
    roof = {"bound": r0["bound"], "achieved": achieved, "peak": r0["peak"], "unit": r0["unit"],
            "frac": achieved / r0["peak"], "work": work, "ms": ms, "peak_note": r0["peak_note"],
            "kernel": name if tensor_path else None, "stages": st, "launches_per_step": n}
    if executed != work:
        roof["executed_work"] = executed
        roof["executed_frac"] = executed / (ms * 1e-3) / 1e12 / r0["peak"]
    src = KERNEL_SRC.get(name) if tensor_path else "mlp_simt.cu"
    tr = [NCU_TRAFFIC.get((s, src_hash(src))) if src else None for s in st]
    roof["traffic"] = None if any(t is None for t in tr) else sum(tr) / n * n_atoms
    return roof


def src_hash(*names):
    h = hashlib.sha256()
    for n in names:
        h.update(open(os.path.join(ROOT, "paper_2201_08110_gb300", "csrc", n), "rb").read())
    return h.hexdigest()[:12]


# ncu dram__bytes_read.sum + dram__bytes_write.sum per launch of the dominant
# kernel, keyed by the kernel's source hash at capture time, in bytes per atom;
# scaled to the bench workload by atoms.  A kernel changed since its capture
# finds no entry and reports null.
NCU_TRAFFIC = {
    # ncu --set full, 512-molecule batch, split BF16 step (first launches of each kernel)
    ("features", "9212797d998e"): 2849.1,
    ("adjoint", "9212797d998e"): 4585.2,  # main launch (the overflow launch moves ~1 KB)
    ("l1_fwd", "4baba2fdbf12"): 12062.0,  # first layer forward, CTA pairs
    ("l1_rev", "4baba2fdbf12"): 7299.3,   # the same kernel's second launch, first-layer reverse
    ("tail", "2a9bf57dcfbd"): 11042.4,    # layers 2 and 3 forward and reverse
}


# ------------------------------------------------------------ the oracle ----

def oracle_refs(b, w, M, nthreads: int = 0, model: str = "ani2x"):
    """Per-molecule oracle results (energy, forces, atomic energies) from one
    call over the whole batch, and the call's wall time."""
    import oracle
    t0 = time.perf_counter()
    r = oracle.compute(b.Z, b.pos, b.mol_off, w, M, box=b.box, atom_energies=True, nthreads=nthreads,
                       model=model)
    dt = time.perf_counter() - t0
    refs = {}
    for m in range(b.n_mols):
        a0, a1 = int(b.mol_off[m]), int(b.mol_off[m + 1])
        refs[m] = (float(r["energy"][m]), r["forces"][a0:a1], r["atom_energies"][a0:a1])
    return refs, dt


def oracle_single_thread(b, w, M, target_s: float = 3.0):
    """The oracle on one host thread over the batch's first molecules, until
    target_s has passed: (atom-evals/s, sample)."""
    import oracle
    t0 = time.perf_counter()
    atoms = mols = 0
    while time.perf_counter() - t0 < target_s and mols < b.n_mols:
        sub = b.molecule(mols)
        oracle.compute(sub.Z, sub.pos, sub.mol_off, w, M, nthreads=1)
        atoms += sub.n_atoms
        mols += 1
    dt = time.perf_counter() - t0
    return atoms / dt, f"first {mols} molecules ({atoms} atoms) of the batch, one thread, {dt:.1f} s"


# Energy rule per molecule (the parity tests' rule): |dE| / |E_ref|, or
# |dE| / S (S = sum_i |E_i,ref|) for molecules flagged near zero, |E_ref| < kappa S.
ERROR_RULE = {"fp32": (1e-5, 0.1, "max"), "bf16": (2e-3, 1e-3, "rms"), "fp16": (2e-3, 1e-3, "rms")}


def error_stats(E, F, b, refs, prec: str) -> dict:
    tol, kappa_used, ftype = ERROR_RULE[prec]  # single-product modes: the same rule, reported
    a5, gross, fmax, frms, flagged, fails = [], [], [], [], 0, 0
    for m in range(b.n_mols):
        a0, a1 = int(b.mol_off[m]), int(b.mol_off[m + 1])
        if a1 == a0:
            continue
        e_ref, f_ref, ea = refs[m]
        s = float(np.abs(ea).sum())
        de = abs(float(E[m]) - e_ref)
        flag = abs(e_ref) < kappa_used * s
        flagged += int(flag)
        err = de / (s if flag else abs(e_ref))
        a5.append(err)
        gross.append(de / s)
        fails += int(err > tol)
        rms = float(np.sqrt(np.mean(f_ref ** 2)))
        d = F[a0:a1] - f_ref
        fmax.append(float(np.abs(d).max()) / rms)
        frms.append(float(np.sqrt(np.mean(d ** 2))) / rms)
    return {"molecules": len(a5), "energy_rule": f"|dE|/|E| <= {tol:g} (|dE|/S for |E| < {kappa_used:g} S)",
            "flagged": flagged, "failing": fails,
            "worst_rel_energy": max(a5), "median_rel_energy": float(np.median(a5)),
            "worst_dE_over_S": max(gross), "worst_max_force_over_rms": max(fmax),
            "worst_rms_force_over_rms": max(frms),
            "force_rule": ("max |dF| <= 1e-4 RMS(F)" if ftype == "max" else "RMS(dF) <= 1e-2 RMS(F)"),
            "force_failing": int(sum(x > 1e-4 for x in fmax) if ftype == "max" else sum(x > 1e-2 for x in frms))}


# FP32 arithmetic of one NNP-MM pair of the coupling term (FMA = 2 FLOP):
# displacement 3, r^2 5, 1/sqrt 1, r^-2 1, combination 2, (sigma/r)^6 4,
# Coulomb 2, energy 4, -dV/dr / r 6, the two force updates 12.
FLOP_COUPLING_PAIR = 40


def measure_coupling(steps: int, flush, stream, fp32_peak: float, with_oracle: bool):
    """The NNP-MM coupling term (Eq. 4) of the 60-atom workload-2 molecule in
    60,000 water-like MM atoms: CUDA-event time per call with the L2 flushed
    between calls, pair throughput, roofline, and the FP64 oracle's time for
    the same call on the host cores."""
    import torch
    from paper_2201_08110_gb300 import nnp
    b, env = W.coupling_config()
    dev = lambda a: torch.tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")
    ins = [dev(b.pos), dev(env.nnp_q), dev(env.nnp_sigma), dev(env.nnp_eps), dev(env.mm_pos),
           dev(env.mm_q), dev(env.mm_sigma), dev(env.mm_eps)]
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    fn = torch.zeros(b.n_atoms, 3, dtype=torch.float64, device="cuda")
    fm = torch.zeros(env.n_mm, 3, dtype=torch.float64, device="cuda")
    call = lambda: nnp.mm_coupling(*ins, W.COULOMB_KCAL, energy=e, nnp_forces=fn, mm_forces=fm,
                                   stream=stream)
    for _ in range(3):
        call()
    torch.cuda.synchronize()
    t_ms = []
    for _ in range(steps):
        flush.zero_()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        call()
        s1.record(stream)
        s1.synchronize()
        t_ms.append(s0.elapsed_time(s1))
    ms = statistics.median(t_ms)
    pairs = b.n_atoms * env.n_mm
    achieved = FLOP_COUPLING_PAIR * pairs / (ms * 1e-3) / 1e12
    out = {"workload": f"{b.n_atoms}-atom molecule (workload 2) in {env.n_mm} water-like MM atoms",
           "n_nnp": b.n_atoms, "n_mm": env.n_mm, "ms_per_call": ms,
           "pairs_per_s": pairs / (ms * 1e-3), "calls": steps,
           "l2": "flushed between calls, outside the timed events",
           "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                        "frac": achieved / fp32_peak, "work": FLOP_COUPLING_PAIR * pairs,
                        "peak_note": "derived FP32 FMA peak: 152 SMs x 128 lanes x 2 x max SM clock"}}
    # the fixed cost of one call: the same call on fewer MM atoms (a line fit
    # of time against pairs gives the intercept) and a one-element kernel
    # timed the same way (the floor of any single launch on this stream)
    def timed(fn, n=steps):
        t = []
        for _ in range(n):
            flush.zero_()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            fn()
            a1.record(stream)
            a1.synchronize()
            t.append(a0.elapsed_time(a1))
        return statistics.median(t)
    sizes = [n for n in (2000, 6000, 20000) if n < env.n_mm] + [env.n_mm]
    per_size = {}
    for n in sizes[:-1]:
        sub = [ins[0], ins[1], ins[2], ins[3], ins[4][:n].contiguous(), ins[5][:n].contiguous(),
               ins[6][:n].contiguous(), ins[7][:n].contiguous()]
        fm_n = torch.zeros(n, 3, dtype=torch.float64, device="cuda")
        f = lambda: nnp.mm_coupling(*sub, W.COULOMB_KCAL, energy=e, nnp_forces=fn, mm_forces=fm_n,
                                    stream=stream)
        for _ in range(3):
            f()
        per_size[n] = timed(f)
    per_size[env.n_mm] = ms
    x = np.array([b.n_atoms * n for n in per_size], dtype=np.float64)
    y = np.array(list(per_size.values()), dtype=np.float64)
    slope, intercept = np.polyfit(x, y, 1)
    one = torch.zeros(1, dtype=torch.float32, device="cuda")
    floor_ms = timed(lambda: one.zero_())
    out["fixed_cost"] = {
        "ms_by_mm_atoms": {str(k): v for k, v in per_size.items()},
        "fit_intercept_ms": float(intercept), "fit_ms_per_mpair": float(slope * 1e6),
        "one_element_kernel_ms": floor_ms,
        "note": "intercept of a line through the call times at the MM sizes shown: the part of a "
                "call that does not grow with the pairs; one_element_kernel_ms: a 1-float fill "
                "timed the same way (events around one launch, L2 flushed before), the floor of "
                "any launch on this stream"}
    if with_oracle:
        import oracle
        t0 = time.perf_counter()
        oracle.coupling(b.pos, env.nnp_q, env.nnp_sigma, env.nnp_eps, env.mm_pos, env.mm_q,
                        env.mm_sigma, env.mm_eps, W.COULOMB_KCAL)
        out["cpu_oracle_ms"] = 1e3 * (time.perf_counter() - t0)
    return out


# ------------------------------------------------------- the reference arm ----

def run_reference(args):
    """The oracle (FP64 C, OpenMP over molecules) timed on the host cores."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    b, w, M = W.config3(args.molecules)
    cores = os.cpu_count() or 1
    per_step_mols = min(max(cores, 16), b.n_mols)
    sub = slice(0, per_step_mols)
    a1 = int(b.mol_off[per_step_mols])
    Z, pos, off = b.Z[:a1], b.pos[:a1], b.mol_off[:per_step_mols + 1]
    for _ in range(max(0, min(args.warmup, 1))):
        oracle.compute(Z, pos, off, w, M, nthreads=cores)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.compute(Z, pos, off, w, M, nthreads=cores)
        ts.append(time.perf_counter() - t0)
    ms = 1e3 * sum(ts) / len(ts)
    value = a1 / (ms / 1e3)
    sample = f"{per_step_mols} molecules ({a1} atoms) of workload 3 per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            # the same workload as the kernel arm's line (its config keys), timed on a
            # bounded sample of its molecules
            "config": {"workload": f"{args.molecules} molecules, 20-120 atoms, 8-network ensemble "
                                   f"(workload 3 batch; {args.precision} networks as workload 4)",
                       "n_molecules": b.n_mols, "n_atoms_per_rank": b.n_atoms, "n_models": M,
                       "precision": "fp64 (the oracle)", "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    del sub
    return 0


def max_over_ranks(x: float, dist) -> float:
    """The maximum of a per-rank number (the timing rule: max over ranks)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, dist) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())




# ------------------------------------------------------- measurement parts ----

def timed_steps(model, pos, E, F, steps: int, flush, stream):
    """Sum of per-step CUDA-event times (ms); the L2 flush between steps is
    outside the events."""
    import torch
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        starts[k].record(stream)
        model.compute(pos, E, F)
        ends[k].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in zip(starts, ends))


def make_model(nnp, b, w, M, prec, single, pos, E, F, args, schedules, key, model="ani2x"):
    """A graph-replay handle for the batch, tuned (or pinned) and warmed up."""
    import torch
    m = nnp.NNP(b.Z, w, M, mol_off=b.mol_off, precision=prec, single_pass=single, box=b.box,
                use_graph=True, model=model)
    if args.schedule:
        vals = [int(v) for v in args.schedule.split(",")]
        schedules[key] = dict(zip(nnp.NNP.SCHEDULE_KEYS, vals))
        m.set_schedule(schedules[key])
    elif not args.no_autotune:
        schedules[key] = m.autotune(pos)
    for _ in range(max(3, args.warmup)):
        m.compute(pos, E, F)
    torch.cuda.synchronize()
    m.status()
    return m


def workload5_measurement(nnp, prec, steps: int, warmup: int, flush, stream):
    """4096 molecules (30-250 atoms, log-uniform) plus the 1500-atom periodic
    pocket, BF16 networks, features kept only for the forward pass
    (recompute_aev): ms per step, atom-evals/s and the device memory of the two
    handles (free memory before and after creating them)."""
    import torch
    batch, pocket, w, M = W.config5()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    hb = nnp.NNP(batch.Z, w, M, mol_off=batch.mol_off, precision=prec, use_graph=True,
                 recompute_aev=True)
    hp = nnp.NNP(pocket.Z, w, M, precision=prec, box=pocket.box, use_graph=True, recompute_aev=True)
    pb = torch.tensor(batch.pos, device="cuda")
    pp = torch.tensor(pocket.pos, device="cuda")
    Eb = torch.empty(batch.n_mols, dtype=torch.float64, device="cuda")
    Fb = torch.empty(batch.n_atoms, 3, dtype=torch.float64, device="cuda")
    Ep = torch.empty(1, dtype=torch.float64, device="cuda")
    Fp = torch.empty(pocket.n_atoms, 3, dtype=torch.float64, device="cuda")
    schedules = {"batch": hb.autotune(pb), "pocket": hp.autotune(pp)}
    for _ in range(max(3, warmup)):
        hb.compute(pb, Eb, Fb)
        hp.compute(pp, Ep, Fp)
    torch.cuda.synchronize()
    hb.status()
    hp.status()
    footprint = free0 - torch.cuda.mem_get_info()[0]
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        starts[k].record(stream)
        hb.compute(pb, Eb, Fb)
        hp.compute(pp, Ep, Fp)
        ends[k].record(stream)
    torch.cuda.synchronize()
    hb.status()
    hp.status()
    ms = sum(a.elapsed_time(b2) for a, b2 in zip(starts, ends)) / steps
    n = batch.n_atoms + pocket.n_atoms
    stages_b = hb.compute_timed(pb, Eb, Fb)
    stages_p = hp.compute_timed(pp, Ep, Fp)
    out = {"workload": "4096 molecules, 30-250 atoms (log-uniform), plus a 1500-atom periodic pocket "
                       "(24.7 A cube, cell list); 8 networks; features kept only for the forward "
                       "pass (recompute_aev)",
           "precision": prec, "n_atoms": n, "steps": steps, "ms_per_step": ms,
           "value": n / (ms * 1e-3), "unit": UNIT,
           "device_bytes": int(footprint),
           "device_bytes_note": "device memory taken by the two handles and their outputs "
                                "(free memory before and after), which is the peak: a step "
                                "allocates nothing",
           "stages_ms_batch": stages_b, "stages_ms_pocket": stages_p, "schedules": schedules,
           "gpu_launches_per_step": hb.kernels_per_step(True) + hp.kernels_per_step(True)}
    hb.close()
    hp.close()
    return out


def ani1x_measurement(nnp, args, flush, stream, with_oracle: bool):
    """The ANI-1x model (Sec. 3, "Extensibility with other NNPs") on a batch of
    the 512-molecule batch's sizes with H, C, N, O molecules, 8 networks: the
    timed step in the headline arithmetic and in FP32, each with its
    per-molecule errors against the oracle's ANI-1x model."""
    import torch
    b, w, M = W.config3_ani1x()
    refs = dt = None
    if with_oracle:
        refs, dt = oracle_refs(b, w, M, model="ani1x")
    pos = torch.tensor(b.pos, device="cuda")
    E = torch.empty(b.n_mols, dtype=torch.float64, device="cuda")
    F = torch.empty(b.n_atoms, 3, dtype=torch.float64, device="cuda")
    out = {"workload": f"{b.n_mols} H/C/N/O molecules, 20-120 atoms, 8-network ANI-1x ensemble "
                       "(384 features; widths 144 and 112 padded to 160 and 128 with zero weights)",
           "n_atoms": b.n_atoms, "unit": UNIT}
    if dt is not None:
        out["oracle_all_cores"] = {"value": b.n_atoms / dt, "unit": UNIT, "cores": os.cpu_count() or 1}
    schedules = {}
    for prec in dict.fromkeys((args.precision, "fp32")):
        m = make_model(nnp, b, w, M, prec, False, pos, E, F, args, schedules, prec, model="ani1x")
        t = timed_steps(m, pos, E, F, args.steps, flush, stream)
        r = {"ms_per_step": t / args.steps, "value": b.n_atoms * args.steps / (t / 1e3),
             "stages_ms": m.compute_timed(pos, E, F), "schedule": schedules.get(prec)}
        if refs is not None:
            m.compute(pos, E, F)
            torch.cuda.synchronize()
            m.status()
            r["errors"] = error_stats(E.cpu().numpy(), F.cpu().numpy(), b, refs, prec)
        m.close()
        out[prec] = r
    return out


def workload2_measurement(nnp, prec, steps: int, warmup: int):
    """One 60-atom molecule, 8 networks, new coordinates every step (independent
    N(0, 0.01^2) A perturbations, drawn beforehand and resident on the device):
    the plain FP32 path with direct launches, and the 16-bit tensor-core path
    replayed as one CUDA graph per step (the single-ligand MD case the paper
    times)."""
    import torch
    b, w, M = W.config2()
    g = W.rng(W.workload_seed(2) + 50)
    P = torch.tensor(np.stack([W.perturb(g, b.pos) for _ in range(steps + warmup)]), device="cuda")
    out = {"workload": "one 60-atom molecule (H27 C21 N5 O4 F S Cl), 8 networks, new coordinates "
                       "each step (N(0, 0.01^2) A perturbations)", "steps": steps}
    for key, p, graph in (("plain_fp32", "fp32", False), ("tensor_graph", prec, True)):
        model = nnp.NNP(b.Z, w, M, precision=p, use_graph=graph)
        pos = torch.empty(b.n_atoms, 3, dtype=torch.float32, device="cuda")
        E = torch.empty(1, dtype=torch.float64, device="cuda")
        F = torch.empty(b.n_atoms, 3, dtype=torch.float64, device="cuda")
        for k in range(warmup):
            pos.copy_(P[k])
            model.compute(pos, E, F)
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        for k in range(steps):
            pos.copy_(P[warmup + k])
            model.compute(pos, E, F)
        s1.record()
        torch.cuda.synchronize()
        model.status()
        ms = s0.elapsed_time(s1) / steps
        out[key] = {"precision": p, "graph": graph, "ms_per_step": ms,
                    "value": b.n_atoms / (ms * 1e-3), "unit": UNIT,
                    "gpu_launches_per_step": model.kernels_per_step(True)}
        model.close()
    return out


def md_measurement(nnp, prec, steps: int, warmup: int):
    """The replica MD loop (Langevin BAOAB, normal draws resident on the
    device) of the 60-atom workload-2 molecule in its 60,000-atom water-like
    environment (the coupling term with the MM atoms held), 1 and 8 replicas,
    with the coupling term after the NNP term on one stream and on a second
    stream beside it: ms and steps per second (each run also evaluates the
    forces once at its starting positions), and the time the concurrent
    stream saves."""
    import torch
    b, env = W.coupling_config()
    _, w, M = W.config2()
    mass = {1: 1.008, 6: 12.011, 7: 14.007, 8: 15.999, 9: 18.998, 16: 32.06, 17: 35.45}
    dev = lambda a: torch.tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")
    out = {"workload": "the 60-atom molecule of workload 2 in 60,000 fixed water-like MM atoms "
                       "(coupling term of Eq. 4), Langevin BAOAB, one CUDA graph replay per step",
           "precision": prec, "steps": steps}
    for R in (1, 8):
        Z = np.tile(b.Z, R)
        pos = np.tile(b.pos, (R, 1))
        off = np.arange(R + 1, dtype=np.int32) * b.n_atoms
        model = nnp.NNP(Z, w, M, mol_off=off, precision=prec)

        class Env:
            pass
        e = Env()
        e.nnp_q, e.nnp_sigma, e.nnp_eps = dev(np.tile(env.nnp_q, R)), dev(np.tile(env.nnp_sigma, R)), \
            dev(np.tile(env.nnp_eps, R))
        e.mm_pos, e.mm_q, e.mm_sigma, e.mm_eps = dev(env.mm_pos), dev(env.mm_q), dev(env.mm_sigma), \
            dev(env.mm_eps)
        masses = np.array([mass[int(z)] for z in Z])
        noise = torch.randn(steps, R * b.n_atoms, 3, dtype=torch.float64, device="cuda")
        r = {"replicas": R, "atoms": R * b.n_atoms}
        for conc in (False, True):
            md = nnp.MD(model, masses, 0.5, integrator="baoab", gamma=0.01, kT=0.6, env=e,
                        coulomb_k=W.COULOMB_KCAL, concurrent=conc)
            x0 = torch.tensor(pos.astype(np.float64), device="cuda")
            x, v = x0.clone(), torch.zeros_like(x0)
            md.run(x, v, steps, noise=noise)  # captures the step graph for these buffers
            torch.cuda.synchronize()
            x.copy_(x0)
            v.zero_()
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record()
            md.run(x, v, steps, noise=noise)
            s1.record()
            torch.cuda.synchronize()
            model.status()
            ms = s0.elapsed_time(s1) / steps
            r["concurrent" if conc else "serial"] = {"ms_per_step": ms, "steps_per_s": 1e3 / ms}
            md.close()
        r["overlap_saved_ms_per_step"] = r["serial"]["ms_per_step"] - r["concurrent"]["ms_per_step"]
        out[f"replicas_{R}"] = r
        model.close()
    return out


# ------------------------------------------------------------------ arms ----

def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2201_08110_gb300 import build, nnp
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()

    b, w, M = rank_batch(args.molecules, rank)
    single = bool(args.single_pass) and args.precision != "fp32"
    extras = rank == 0 and world == 1 and not args.no_extras
    # the FP64 oracle over the whole batch first (no CUDA work in flight; it uses
    # its own threads): the CPU baseline on all host cores and the reference
    # values of the error report
    cpu = refs = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        refs, dt = oracle_refs(b, w, M)
        cores = os.cpu_count() or 1
        cpu = {"value": b.n_atoms / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"all {b.n_mols} molecules ({b.n_atoms} atoms) of the batch, {dt:.1f} s",
               "cpu_model": cpu_model()}
        rate1, sample1 = oracle_single_thread(b, w, M)
        cpu["single_thread"] = {"value": rate1, "unit": UNIT, "cores": 1, "sample": sample1}

    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    pos = torch.tensor(b.pos, device="cuda")
    E = torch.empty(b.n_mols, dtype=torch.float64, device="cuda")
    F = torch.empty(b.n_atoms, 3, dtype=torch.float64, device="cuda")
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    schedules = {}

    model = make_model(nnp, b, w, M, args.precision, single, pos, E, F, args, schedules, "headline")
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    clk.start()
    total_ms = timed_steps(model, pos, E, F, args.steps, flush, stream)
    clocks = clk.stop()
    model.status()
    if dist is not None:
        dist.barrier()
    total_ms = max_over_ranks(total_ms, dist)
    atoms_all = sum_over_ranks(b.n_atoms, dist)
    ms_per_step = total_ms / args.steps
    value = atoms_all * args.steps / (total_ms / 1e3)

    def other(prec, one_product, key):
        m2 = make_model(nnp, b, w, M, prec, one_product, pos, E, F, args, schedules, key)
        t = max_over_ranks(timed_steps(m2, pos, E, F, args.steps, flush, stream), dist)
        return m2, {"precision": prec, "single_pass": one_product,
                    "value": atoms_all * args.steps / (t / 1e3), "unit": UNIT,
                    "ms_per_step": t / args.steps}

    alt = None
    if args.alt_precision not in ("none", args.precision):
        m2, alt = other(args.alt_precision, single and args.alt_precision != "fp32", "alt")
        if extras and refs is not None:
            m2.compute(pos, E, F)
            torch.cuda.synchronize()
            alt["errors"] = error_stats(E.cpu().numpy(), F.cpu().numpy(), b, refs, args.alt_precision)
        m2.close()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    # ---- errors of the timed configuration against the oracle, every molecule ----
    errors = None
    if refs is not None:
        model.compute(pos, E, F)
        torch.cuda.synchronize()
        model.status()
        errors = error_stats(E.cpu().numpy(), F.cpu().numpy(), b, refs, args.precision)

    # ---- per-stage times, algorithmic work and rooflines ----
    split = args.precision != "fp32" and not single
    stage_runs = [model.compute_timed(pos, E, F) for _ in range(5)]
    stages = {k: statistics.median(r[k] for r in stage_runs) for k in stage_runs[0]}
    cr, _ = model.neighbors(0)
    ca, _ = model.neighbors(1)
    cr = cr.cpu().numpy().astype(np.float64)
    ca = ca.cpu().numpy().astype(np.float64)
    sizes = np.diff(b.mol_off).astype(np.float64)
    work = stage_work(b.Z, M, float(cr.sum()), float((ca * (ca - 1) / 2).sum()),
                      float((sizes * (sizes - 1)).sum()), args.precision, split)
    hbm, bf16, bf16_sus, peak_kind, sm_max = peaks()
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12  # FP32 lanes x 2 x max SM clock, TFLOP/s
    tensor_path = args.precision != "fp32"
    shown = shown_stages(stages, args.precision)
    rooflines = rooflines_of(shown, work, tensor_path, hbm, bf16, peak_kind, fp32_peak)
    roof = dominant_kernel(rooflines, tensor_path, b.n_atoms)
    total_stage = max(sum(shown.values()), 1e-12)
    stage_share = {k: v / total_stage for k, v in shown.items()}

    # ---- end to end through the host-buffer entry point (pinned buffers) ----
    hpos = torch.from_numpy(b.pos.copy()).pin_memory()
    hE = torch.empty(b.n_mols, dtype=torch.float64).pin_memory()
    hF = torch.empty(b.n_atoms, 3, dtype=torch.float64).pin_memory()
    lib = nnp.load_library()
    for _ in range(2):
        lib.nnp_compute_host(model._h, hpos.data_ptr(), hE.data_ptr(), hF.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rc = lib.nnp_compute_host(model._h, hpos.data_ptr(), hE.data_ptr(), hF.data_ptr(),
                                  stream.cuda_stream)
        assert rc == 0
    e2e_s = time.perf_counter() - t0
    e2e = {"value": b.n_atoms * args.steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(hpos.numel() * 4),
           "d2h_bytes_per_step": int(hE.numel() * 8 + hF.numel() * 8)}
    launches = model.kernels_per_step(True)
    model.close()

    # ---- the same batch in the other arithmetics: FP32 networks (batched,
    # graph) and single-product 16-bit networks, each with its errors ----
    others = {}
    if extras:
        for key, prec, one in (("fp32_batched", "fp32", False), ("bf16_single_pass", "bf16", True),
                               ("fp16_single_pass", "fp16", True)):
            if prec == args.precision and one == single:
                continue
            m2, r = other(prec, one, key)
            if refs is not None:
                m2.compute(pos, E, F)
                torch.cuda.synchronize()
                r["errors"] = error_stats(E.cpu().numpy(), F.cpu().numpy(), b, refs, prec)
            m2.close()
            others[key] = r

    # ---- the plain FP32 unbatched path on a sample of the same molecules ----
    unb = None
    if args.unbatched_sample > 0:
        ids = np.random.Generator(np.random.PCG64(17)).choice(
            b.n_mols, min(args.unbatched_sample, b.n_mols), replace=False)
        tot_ms, tot_atoms = 0.0, 0
        for m in ids:
            sub = b.molecule(int(m))
            h1 = nnp.NNP(sub.Z, w, M, precision="fp32", use_graph=False)
            p1 = torch.tensor(sub.pos, device="cuda")
            e1 = torch.empty(1, dtype=torch.float64, device="cuda")
            f1 = torch.empty(sub.n_atoms, 3, dtype=torch.float64, device="cuda")
            for _ in range(3):
                h1.compute(p1, e1, f1)
            torch.cuda.synchronize()
            reps = 10
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            for _ in range(reps):
                h1.compute(p1, e1, f1)
            s1.record(stream)
            torch.cuda.synchronize()
            tot_ms += s0.elapsed_time(s1) / reps
            tot_atoms += sub.n_atoms
            h1.close()
        unb = {"value": tot_atoms / (tot_ms / 1e3), "unit": UNIT,
               "sample": f"{len(ids)} molecules of the batch, one per call, FP32 networks, "
                         "direct launches", "ms_per_molecule": tot_ms / len(ids)}

    mode = ("single-product" if single else "three split-operand products per forward layer") \
        if args.precision != "fp32" else "SIMT FP32"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": f"{args.molecules} molecules, 20-120 atoms, 8-network ensemble "
                                   f"(workload 3 batch with {args.precision} networks, {mode}: "
                                   "workload 4)",
                       "n_molecules": b.n_mols, "n_atoms_per_rank": b.n_atoms, "n_models": M,
                       "precision": args.precision, "forward_products": mode, "graph": True,
                       "schedule": schedules.get("headline", "default"),
                       "l2": "flushed (256 MB write) between timed steps, outside the timed events",
                       "parallelism": f"replicas x{world}, no collective on the data path"},
            "roofline": roof, "rooflines": rooflines, "stages_ms": shown, "stage_share": stage_share,
            "e2e": e2e, "gpu_launches": launches * args.steps, "clocks": clocks}
    if errors is not None:
        line["errors"] = errors
    if alt is not None:
        line["alt_precision"] = alt
    line.update(others)
    if unb is not None:
        line["fp32_unbatched"] = unb
        line["speedup_vs_fp32_unbatched"] = value / world / unb["value"]
        if "fp32_batched" in others:
            line["speedup_fp32_batched_vs_unbatched"] = others["fp32_batched"]["value"] / unb["value"]
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if extras:
        for key, fn in (("workload5", lambda: workload5_measurement(nnp, args.precision, 5, 3, flush, stream)),
                        ("workload2", lambda: workload2_measurement(nnp, args.precision, 1000, 10)),
                        ("md", lambda: md_measurement(nnp, args.precision, 200, 10)),
                        ("ani1x", lambda: ani1x_measurement(nnp, args, flush, stream,
                                                            not args.no_cpu_baseline))):
            try:
                line[key] = fn()
            except Exception as exc:  # reported in the line; the measurements above stand
                line[key] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
    if not args.no_coupling:
        try:
            line["coupling"] = measure_coupling(max(args.steps, 10), flush, stream, fp32_peak,
                                                rank == 0 and world == 1 and not args.no_cpu_baseline)
        except Exception as exc:  # reported in the line; the step's measurement above stands
            line["coupling"] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_workload2(args):
    """Workload 2 alone: one 60-atom molecule over perturbed coordinates."""
    import torch
    from paper_2201_08110_gb300 import build, nnp
    build.build()
    torch.cuda.set_device(0)
    r = workload2_measurement(nnp, args.precision, args.steps, args.warmup)
    key = "tensor_graph" if args.w2_fast else "plain_fp32"
    b, _, _ = W.config2()
    line = {"metric": METRIC, "value": r[key]["value"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r[key]["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": r[key]["precision"], "data": "synthetic",
            "config": {"workload": r["workload"] + (", tensor-core networks, one CUDA graph replay "
                                                    "per step" if args.w2_fast else
                                                    ", plain FP32 path, direct launches")},
            "gpu_launches": r[key]["gpu_launches_per_step"] * args.steps, "workload2": r}
    print(json.dumps(line), flush=True)
    return 0


def run_workload5(args):
    """Workload 5 alone: 4096 molecules plus the 1500-atom periodic pocket."""
    import torch
    from paper_2201_08110_gb300 import build, nnp
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    clk = Clocks(0)
    clk.start()
    r = workload5_measurement(nnp, args.precision, args.steps, args.warmup, flush, stream)
    clocks = clk.stop()
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": r["workload"], "n_atoms": r["n_atoms"], "precision": args.precision,
                       "graph": True},
            "device_bytes": r["device_bytes"], "gpu_launches": r["gpu_launches_per_step"] * args.steps,
            "clocks": clocks, "workload5": r}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == 2:
        return run_workload2(args)
    if args.workload == 5:
        return run_workload5(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
