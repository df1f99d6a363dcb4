#!/usr/bin/env python
"""Throughput of NNP energy + force evaluation on GB300, in atom-evals/s.

One step = one energy + force evaluation of a whole batch (neighbour lists,
features, the 8-network ensemble forward and reverse, the featurizer's reverse
pass to coordinates), i.e. every stage of the path.  Default workload: 512
molecules with 20-120 atoms (H .45, C .35, N .08, O .08, F/S/Cl .04), random
Xavier-normal ANI-2x-architecture weights, network products in FP16 (the
16-bit format that meets the stated error bounds; BF16 is timed alongside),
replayed as one CUDA graph per step.  An atom-eval is one atom's share of E
and F for the full ensemble.

Also reported: the plain FP32 unbatched GPU path on a sample of the same
molecules (one molecule per call, direct launches), the end-to-end number
through the host-buffer entry point, per-stage times with the roofline of the
dominant stage, and the FP64 CPU oracle on the host cores.

Usage: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
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
    ap.add_argument("--precision", default="fp16", choices=["fp32", "bf16", "fp16"],
                    help="arithmetic of the networks' matrix products (FP16 meets the stated "
                         "2e-3 energy / 1e-2 force bounds; single-pass BF16 does not on every "
                         "molecule: its weight rounding errors add coherently)")
    ap.add_argument("--alt-precision", default="bf16", choices=["none", "fp32", "bf16", "fp16"],
                    help="a second precision timed the same way and reported alongside")
    ap.add_argument("--workload", type=int, default=3, choices=[2, 3, 5],
                    help="3: the 512-molecule batch (default, headline); 2: one 60-atom "
                         "molecule on the plain FP32 path over perturbed coordinates; 5: 4096 "
                         "molecules of 30-250 atoms plus a 1500-atom periodic pocket")
    ap.add_argument("--w2-fast", action="store_true",
                    help="workload 2 on the --precision tensor-core path with graph replay "
                         "instead of the plain FP32 path")
    ap.add_argument("--molecules", type=int, default=512)
    ap.add_argument("--unbatched-sample", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-coupling", action="store_true",
                    help="skip the NNP-MM coupling term's measurement")
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


# Algorithmic work per stage: operations per unit of work, times the units.
HID = W.HIDDEN
# FP32 operations of the featurizer per directed radial pair / unordered
# angular pair of neighbours (exp2 and log2 counted as one operation each).
FLOP_RADIAL_FWD, FLOP_ANGULAR_FWD = 100.0, 142.0
FLOP_RADIAL_REV, FLOP_ANGULAR_REV = 137.0, 300.0
FLOP_DISTANCE = 8.0  # one neighbour-search distance test


def stage_work(Z, M: int, n_pairs: float, n_triples: float, n_tests: float):
    """{stage: (bound, algorithmic work)}: FLOPs of the matrix products from the
    element counts (first-layer K = the 1008 real features), FP32 operations
    of the featurizer from the pair / triple counts."""
    zs = list(W.ELEMENTS_Z)
    cnt = [int(np.sum(Z == z)) for z in zs]
    l1 = l2 = l3 = out = 0.0
    for e, n in enumerate(cnt):
        h1, h2, h3 = HID[e]
        l1 += 2.0 * n * M * h1 * 1008
        l2 += 2.0 * n * M * h1 * h2
        l3 += 2.0 * n * M * h2 * h3
        out += 2.0 * n * M * h3
    return {
        "neighbors": ("alu", n_tests * FLOP_DISTANCE),
        "features": ("alu", n_pairs * FLOP_RADIAL_FWD + n_triples * FLOP_ANGULAR_FWD),
        "l1_fwd": ("tensor", l1),
        # on the tensor-core path the l2_fwd stage is the fused tail: both
        # hidden layers forward, the output layer and both hidden layers reverse
        "tail": ("tensor", 2 * l2 + 2 * l3 + out),
        "l2_fwd": ("tensor", l2), "l3_fwd": ("tensor", l3 + out), "l3_rev": ("tensor", l3),
        "l2_rev": ("tensor", l2),
        "l1_rev": ("tensor", l1),
        "adjoint": ("alu", n_pairs * FLOP_RADIAL_REV + n_triples * FLOP_ANGULAR_REV),
    }


def src_hash(*names):
    h = hashlib.sha256()
    for n in names:
        h.update(open(os.path.join(ROOT, "paper_2201_08110_gb300", "csrc", n), "rb").read())
    return h.hexdigest()[:12]


# ncu dram__bytes_read.sum + dram__bytes_write.sum per launch of the dominant
# kernel, keyed by the kernel's source hash at capture time, in bytes per atom;
# scaled to the bench workload by atoms.
NCU_TRAFFIC = {
    ("adjoint", "1dd06ca99192"): 4604.8,  # ncu --set full, 512-molecule batch, FP16
    ("features", "1dd06ca99192"): 807.2,  # ncu --set full, 512-molecule batch, FP16
    ("tail", "b875ce9262f5"): 6404.4,  # ncu --set full, 512-molecule batch, FP16
}


def cpu_oracle_rate(b, w, M, target_s: float = 12.0):
    """The FP64 oracle as it stands, on all host cores, over a bounded sample
    of the batch's molecules (atom-evals/s, sample description, cores)."""
    import oracle
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    n_done = 0
    atoms = 0
    m = 0
    chunk = max(1, cores)
    while time.perf_counter() - t0 < target_s and m < b.n_mols:
        hi = min(b.n_mols, m + chunk)
        sub_off = b.mol_off[m:hi + 1] - b.mol_off[m]
        a0, a1 = int(b.mol_off[m]), int(b.mol_off[hi])
        oracle.compute(b.Z[a0:a1], b.pos[a0:a1], sub_off, w, M, nthreads=cores)
        atoms += a1 - a0
        n_done += hi - m
        m = hi
    dt = time.perf_counter() - t0
    return atoms / dt, f"first {n_done} molecules ({atoms} atoms) of the batch, {dt:.1f} s", cores


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
    if with_oracle:
        import oracle
        t0 = time.perf_counter()
        oracle.coupling(b.pos, env.nnp_q, env.nnp_sigma, env.nnp_eps, env.mm_pos, env.mm_q,
                        env.mm_sigma, env.mm_eps, W.COULOMB_KCAL)
        out["cpu_oracle_ms"] = 1e3 * (time.perf_counter() - t0)
    return out


# ------------------------------------------------------------------ arms ----

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
    # CPU baseline first (no CUDA work in flight; the oracle uses its own threads)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        rate, sample, cores = cpu_oracle_rate(b, w, M)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    pos = torch.tensor(b.pos, device="cuda")
    E = torch.empty(b.n_mols, dtype=torch.float64, device="cuda")
    F = torch.empty(b.n_atoms, 3, dtype=torch.float64, device="cuda")
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    schedules = {}

    def make(prec):
        m = nnp.NNP(b.Z, w, M, mol_off=b.mol_off, precision=prec, use_graph=True)
        if args.schedule:
            vals = [int(v) for v in args.schedule.split(",")]
            schedules[prec] = dict(zip(nnp.NNP.SCHEDULE_KEYS, vals))
            m.set_schedule(schedules[prec])
        elif not args.no_autotune:
            schedules[prec] = m.autotune(pos)
        for _ in range(max(3, args.warmup)):
            m.compute(pos, E, F)
        torch.cuda.synchronize()
        m.status()
        return m

    model = make(args.precision)
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

    alt = None
    if args.alt_precision not in ("none", args.precision):
        m2 = make(args.alt_precision)
        alt_ms = max_over_ranks(timed_steps(m2, pos, E, F, args.steps, flush, stream), dist)
        alt = {"precision": args.alt_precision, "value": atoms_all * args.steps / (alt_ms / 1e3),
               "unit": UNIT, "ms_per_step": alt_ms / args.steps}
        m2.close()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    # ---- per-stage times, algorithmic work and rooflines ----
    stage_runs = [model.compute_timed(pos, E, F) for _ in range(5)]
    stages = {k: statistics.median(r[k] for r in stage_runs) for k in stage_runs[0]}
    cr, _ = model.neighbors(0)
    ca, _ = model.neighbors(1)
    cr = cr.cpu().numpy().astype(np.float64)
    ca = ca.cpu().numpy().astype(np.float64)
    sizes = np.diff(b.mol_off).astype(np.float64)
    work = stage_work(b.Z, M, float(cr.sum()), float((ca * (ca - 1) / 2).sum()),
                      float((sizes * (sizes - 1)).sum()))
    hbm, bf16, bf16_sus, peak_kind, sm_max = peaks()
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12  # FP32 lanes x 2 x max SM clock, TFLOP/s
    tensor_path = args.precision != "fp32"
    shown = dict(stages)
    if tensor_path:  # the fused tail runs in the l2_fwd slot
        shown = {k: v for k, v in stages.items() if k not in ("l2_fwd", "l3_fwd", "l3_rev", "l2_rev")}
        shown["tail"] = stages["l2_fwd"]
    rooflines = {}
    for k, ms in shown.items():
        if k not in work or ms <= 0:
            continue
        bound, amount = work[k]
        if bound == "tensor" and tensor_path:
            peak, unit, note = bf16, "TFLOP/s", f"{peak_kind} dense bf16 (fp16 equal rate)"
        else:
            bound = "alu"
            peak, unit, note = fp32_peak, "TFLOP/s", "derived FP32 FMA peak: 152 SMs x 128 lanes x 2 x max SM clock"
        achieved = amount / (ms * 1e-3) / 1e12
        rooflines[k] = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                        "frac": achieved / peak, "work": amount, "ms": ms, "peak_note": note}
    dom = max(rooflines, key=lambda k: rooflines[k]["ms"])
    kernel_src = {"features": "aev.cu", "adjoint": "aev.cu", "neighbors": "aev.cu",
                  "tail": "mlp_tail_tc.cu"}.get(dom, "mlp_tc.cu" if tensor_path else "mlp_simt.cu")
    tr = NCU_TRAFFIC.get((dom, src_hash(kernel_src)))
    roof = dict(rooflines[dom])
    roof.update({"stage": dom, "traffic": None if tr is None else tr * b.n_atoms})
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

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": f"{args.molecules} molecules, 20-120 atoms, 8-network ensemble "
                                   f"(workload 3 batch; {args.precision} networks as workload 4)",
                       "n_molecules": b.n_mols, "n_atoms_per_rank": b.n_atoms, "n_models": M,
                       "precision": args.precision, "graph": True,
                       "schedule": schedules.get(args.precision, "default"),
                       "l2": "flushed (256 MB write) between timed steps, outside the timed events",
                       "parallelism": f"replicas x{world}, no collective on the data path"},
            "roofline": roof, "rooflines": rooflines, "stages_ms": shown, "stage_share": stage_share,
            "e2e": e2e, "gpu_launches": model.kernels_per_step(True) * args.steps,
            "clocks": clocks}
    if alt is not None:
        line["alt_precision"] = alt
    if unb is not None:
        line["fp32_unbatched"] = unb
        line["speedup_vs_fp32_unbatched"] = value / world / unb["value"]
    if cpu is not None:
        line["cpu_baseline"] = cpu
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
    """One 60-atom molecule, 8 networks, new coordinates every step (independent
    N(0, 0.01^2) A perturbations): the plain FP32 path with direct launches,
    or with --w2-fast the tensor-core path replayed as one CUDA graph (the
    single-ligand MD case the paper times)."""
    import torch
    from paper_2201_08110_gb300 import build, nnp
    build.build()
    b, w, M = W.config2()
    steps = args.steps
    g = W.rng(W.workload_seed(2) + 50)
    P = torch.tensor(np.stack([W.perturb(g, b.pos) for _ in range(steps + args.warmup)]),
                     device="cuda")
    prec = args.precision if args.w2_fast else "fp32"
    model = nnp.NNP(b.Z, w, M, precision=prec, use_graph=bool(args.w2_fast))
    pos = torch.empty(b.n_atoms, 3, dtype=torch.float32, device="cuda")
    E = torch.empty(1, dtype=torch.float64, device="cuda")
    F = torch.empty(b.n_atoms, 3, dtype=torch.float64, device="cuda")
    for k in range(args.warmup):
        pos.copy_(P[k])
        model.compute(pos, E, F)
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record()
    for k in range(steps):
        pos.copy_(P[args.warmup + k])
        model.compute(pos, E, F)
    s1.record()
    torch.cuda.synchronize()
    model.status()
    ms = s0.elapsed_time(s1)
    line = {"metric": METRIC, "value": b.n_atoms * steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": steps, "warmup": args.warmup, "ms_per_step": ms / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": prec,
            "data": "synthetic",
            "config": {"workload": "one 60-atom molecule (H27 C21 N5 O4 F S Cl), 8 networks, "
                                   + ("tensor-core networks, one CUDA graph replay per step"
                                      if args.w2_fast else "plain FP32 path, direct launches")
                                   + ", new coordinates each step"},
            "gpu_launches": model.kernels_per_step(True) * steps}
    print(json.dumps(line), flush=True)
    return 0


def run_workload5(args):
    """4096 molecules (30-250 atoms, log-uniform) plus one 1500-atom periodic
    pocket; one step evaluates both; reports the handles' device memory."""
    import torch
    from paper_2201_08110_gb300 import build, nnp
    build.build()
    batch, pocket, w, M = W.config5()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    free0 = torch.cuda.mem_get_info()[0]
    hb = nnp.NNP(batch.Z, w, M, mol_off=batch.mol_off, precision=args.precision, use_graph=True)
    hp = nnp.NNP(pocket.Z, w, M, precision=args.precision, box=pocket.box, use_graph=True)
    torch.cuda.synchronize()
    footprint = free0 - torch.cuda.mem_get_info()[0]
    pb = torch.tensor(batch.pos, device="cuda")
    pp = torch.tensor(pocket.pos, device="cuda")
    Eb = torch.empty(batch.n_mols, dtype=torch.float64, device="cuda")
    Fb = torch.empty(batch.n_atoms, 3, dtype=torch.float64, device="cuda")
    Ep = torch.empty(1, dtype=torch.float64, device="cuda")
    Fp = torch.empty(pocket.n_atoms, 3, dtype=torch.float64, device="cuda")
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(max(3, args.warmup)):
        hb.compute(pb, Eb, Fb)
        hp.compute(pp, Ep, Fp)
    torch.cuda.synchronize()
    hb.status()
    hp.status()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clk = Clocks(0)
    clk.start()
    for k in range(args.steps):
        flush.zero_()
        starts[k].record(stream)
        hb.compute(pb, Eb, Fb)
        hp.compute(pp, Ep, Fp)
        ends[k].record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    hb.status()
    hp.status()
    ms = sum(a.elapsed_time(b2) for a, b2 in zip(starts, ends))
    n = batch.n_atoms + pocket.n_atoms
    stages_b = hb.compute_timed(pb, Eb, Fb)
    stages_p = hp.compute_timed(pp, Ep, Fp)
    line = {"metric": METRIC, "value": n * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.precision, "data": "synthetic",
            "config": {"workload": "4096 molecules, 30-250 atoms (log-uniform), plus a 1500-atom "
                                   "periodic pocket (24.7 A cube); 8 networks",
                       "n_atoms": n, "precision": args.precision, "graph": True},
            "device_bytes": int(footprint), "stages_ms_batch": stages_b,
            "stages_ms_pocket": stages_p,
            "gpu_launches": (hb.kernels_per_step(True) + hp.kernels_per_step(True)) * args.steps,
            "clocks": clocks}
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
