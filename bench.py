#!/usr/bin/env python
"""Throughput benchmark of the batched RGF conductance path on one GB300 (or N).

Workload (default): the W = 30 nm armchair ribbon, N = 245 dimer lines
(M = 490 orbitals per unit cell), L = 4000 cells (1.7 um), Anderson disorder
U[-0.25, 0.25] eV (seed 1), 69 energies: 64 uniform in [-0.5, 0.5] eV plus
E in {0, +-1 meV, +-5 meV}; eta = 1e-8 eV in device and leads.  One step is one
rgf_conductance call over all 69 chains: lead decimation, the slice recursion
and the trace.  The unit is one unit-cell slice step of one chain
(slice-inversions/s, M = 490); chains that report an error status do no sweep
work and are not counted.

Arms:
  default           mixed precision path with the dense contractions on the
                    tcgen05 tensor cores (RGF_MIXED_TC), device-resident inputs;
                    also the FP64 path once on the same ribbon for |dT|.
  --precision mixed the double-float path on the FP32 pipes alone (RGF_MIXED).
  --impl reference  the CPU oracle on a bounded sample of the same workload.
Under torchrun the job holds one disorder realisation per rank (seed + rank)
at every energy, and its chain list is sharded over the ranks by the
library's longest-processing-time partition (paper_1107_5300_gb300.shard): no
collective on the data path, one gather of T to rank 0 after the timed
region ("weak" scaling: the work per GPU is fixed as ranks are added).

Other workloads: --workload batched_uneven_chains (2048 uneven chains;
--cells caps L), agnr101_L500_grad (dT/d eps), agnr1001_L2000 (the 123 nm
ribbon, N = 1001; --cells and --energies take a bounded sample).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

import workloads  # noqa: E402


def kernel_sources_digest(csrc: Path | None = None) -> str:
    """SHA-256 over the sources the sweep kernels are compiled from (rgf_sweep.cu,
    rgf_batch.cu and every header; file names and bytes, in name order): the
    DRAM counters of a capture hold only for the sources they were taken on."""
    import hashlib
    csrc = csrc or ROOT / "paper_1107_5300_gb300" / "csrc"
    h = hashlib.sha256()
    for p in sorted({csrc / "rgf_sweep.cu", csrc / "rgf_batch.cu", *csrc.glob("*.cuh"), *csrc.glob("*.h")}):
        h.update(p.name.encode() + b"\0" + p.read_bytes())
    return h.hexdigest()


METRIC = "RGF slice-inversions/s (M=490, batched energies)"
UNIT = "slice-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="tc", choices=["tc", "mixed", "fp64", "fp64tc"])
    ap.add_argument("--workload", default="agnr245_L4000_anderson")
    ap.add_argument("--cells", type=int, default=0, help="override L (profiling runs)")
    ap.add_argument("--energies", type=int, default=0, help="use only the first n energies")
    ap.add_argument("--no-check", action="store_true", help="skip the FP64 comparison run")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-cells", type=int, default=60)
    ap.add_argument("--chains", type=int, default=0,
                    help="batched_uneven_chains: number of chains (default 2048)")
    ap.add_argument("--grad", action="store_true",
                    help="time rgf_conductance_grad on the workload (its gradient energies)")
    ap.add_argument("--schedule", default="phased", choices=["persistent", "phased"],
                    help="phased: three launches per step (default); persistent: the batch kernel "
                         "with its device work queue")
    ap.add_argument("--no-graph", action="store_true",
                    help="each step through rgf_conductance_dev instead of a prepared CUDA-graph "
                         "batch")
    ap.add_argument("--domains", type=int, default=2,
                    help="domains per chain (default 2; 0: automatic, more than 2 for few long chains)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="default schedule instead of the autotuner's choice for the width")
    ap.add_argument("--check-chains", type=int, default=0,
                    help="batched_uneven_chains: compare only the first n chains with binary64")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def flops_per_cell(N: int) -> float:
    """Algorithmic real flops of one unit-cell step in the column slicing.

    Per column of K orbitals: the inverse (K^3 complex multiply-adds) and the
    corner-strip product (KL x K x K); 8 real flops per complex multiply-add.
    """
    KL, KR = (N + 1) // 2, N // 2
    f = 0.0
    for K in (KL, KL, KR, KR):
        f += 8.0 * K ** 3 + 8.0 * KL * K * K
    return f


def pair_step_flops_per_cell(N: int) -> float:
    """Real flops one half sweep executes per unit cell with pair steps: one
    inverse (K^3 complex multiply-adds) and one strip product (KL x K x K) for
    each of the pairs c0-c1 (K = KL) and c2-c3 (K = KR); O(K^2) terms left out."""
    KL, KR = (N + 1) // 2, N // 2
    return 8.0 * KL ** 3 + 8.0 * KL ** 3 + 8.0 * KR ** 3 + 8.0 * KL * KR * KR


def cell_slicing_flops_per_step(N: int) -> float:
    """Algorithmic real flops of one slice step when the slice is the whole unit
    cell (M = 2N orbitals): an LU of the M x M slice matrix (8/3 M^3), the solve
    for the floor(N/2) columns the next step needs (8 M^2 floor(N/2)) and the
    corner-strip product (8 ceil(N/2)^2 floor(N/2)).  Reported beside the
    column recursion's own count (flops_per_cell), which is lower."""
    M, KL, KR = 2 * N, (N + 1) // 2, N // 2
    return 8.0 / 3.0 * M ** 3 + 8.0 * M * M * KR + 8.0 * KL * KL * KR


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(self.idx)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        try:
            rows = [r.split(",") for r in Path(self.f.name).read_text().strip().splitlines() if r.strip()]
        except Exception:
            rows = []
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if len(r) > 5 + i and "Active" in r[5 + i] and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        try:
            return json.loads(p.read_text()), "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def cpu_oracle_sample(N, L_s, E, W, seed, rem_p=0.0, edge_seed=0):
    """Times the CPU oracle (as it stands) on one energy x L_s cells."""
    from oracle import rgf as orgf
    eps = workloads.anderson_onsite(N, L_s, W, seed)
    rem = workloads.edge_removed(N, L_s, rem_p, edge_seed) if rem_p > 0 else None
    t0 = time.perf_counter()
    orgf.transmission(N, L_s, E, 1e-8, 1e-8, -2.7, eps, rem)
    return time.perf_counter() - t0


def cpu_baseline(N, cells, W, seed):
    """The oracle as it stands on 1 energy x `cells` cells of the workload, with
    all BLAS threads and with one (a child process started with the BLAS
    thread count set to 1 in its environment)."""
    dt = cpu_oracle_sample(N, cells, 0.3, W, seed)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = (f"import sys; sys.path.insert(0, {str(ROOT)!r}); import bench; "
            f"print(bench.cpu_oracle_sample({N}, {cells}, 0.3, {W}, {seed}))")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       cwd=str(ROOT))
    dt1 = float(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else float("nan")
    sample = f"1 energy (E=0.3 eV) x {cells} cells of N={N}, whole path (decimation + recursion + trace)"
    return {"value": cells / dt, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
            "sample": sample,
            "single_thread": {"value": cells / dt1, "unit": UNIT, "cores": 1, "kind": "oracle",
                              "sample": sample}}


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        return max((i.get("num_threads", 1) for i in info), default=os.cpu_count())
    except Exception:
        return os.cpu_count()


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = workloads.WORKLOADS[args.workload]
    N = w["N"]
    L_s = args.cpu_cells
    E = 0.3
    times = []
    for i in range(args.warmup + args.steps):
        dt = cpu_oracle_sample(N, L_s, E, w["W"], w["seed"])
        if i >= args.warmup:
            times.append(dt)
    t = sum(times)
    value = args.steps * L_s / t
    cores = blas_threads()
    sample = f"1 energy (E=0.3 eV) x {L_s} cells of N={N}, whole path (decimation + recursion + trace)"
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": args.workload, "N": N, "L": w["L"], "sample_cells": L_s},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_uneven(args):
    """The uneven batch: independent chains with N ~ U{51..401}, L ~ U{100..2000},
    E ~ U[-1, 1] eV, Anderson U[-0.1, 0.1] eV and edge roughness p = 0.05 (seed 3),
    all in one call; --cells caps L (a sample of the workload)."""
    import torch
    from paper_1107_5300_gb300 import rgf
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    prec = {"mixed": rgf.RGF_MIXED, "tc": rgf.RGF_MIXED_TC, "fp64": rgf.RGF_FP64,
            "fp64tc": rgf.RGF_FP64_TC}[args.precision]
    chains = workloads.batched_uneven_chains(args.chains or 2048, seed=3)
    ribs, Es, cells, Ns = [], [], [], []
    for ch in chains:
        L = min(ch["L"], args.cells) if args.cells else ch["L"]
        ribs.append(rgf.Ribbon(ch["N"], L, -2.7, W=ch["W"], seed=ch["seed"], edge_p=ch["edge_p"],
                               edge_seed=ch["edge_seed"]))
        Es.append(ch["E"]); cells.append(L); Ns.append(ch["N"])
    Es, cells, Ns = np.array(Es), np.array(cells), np.array(Ns)
    n = len(ribs)
    stream = torch.cuda.Stream()
    Ed = torch.tensor(Es, dtype=torch.float64, device="cuda")
    Td = torch.empty(n, dtype=torch.float64, device="cuda")
    Sd = torch.empty(n, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    # autotuned schedule per column size (eight widths spanning N in [51, 401]),
    # then the batch as one prepared CUDA graph (persistent kernel per engine)
    rgf.set_schedule(rgf.RGF_SCHED_PHASED if args.schedule == "phased" else rgf.RGF_SCHED_PERSISTENT)
    tuned = None
    if not args.no_autotune:
        t0 = time.perf_counter()
        widths = [51, 101, 151, 201, 251, 301, 351, 401]
        table, _ = rgf.autotune(prec, widths, cells=4, reps=2)
        tuned = {"table": table, "tuning_s": round(time.perf_counter() - t0, 2)}
    groups = 1
    if prec in (rgf.RGF_MIXED_TC, rgf.RGF_FP64_TC):
        eng = {rgf.tune_lookup(prec, int(N))["engine"] for N in Ns}
        groups = len(eng)
    rgf.profile_enable(True)
    use_graph = not args.no_graph
    if use_graph:
        batch = rgf.Batch(ribs, Ed.data_ptr(), n, Td.data_ptr(), Sd.data_ptr(), 1e-8, 1e-8, prec)

        def step():
            batch.launch(stream.cuda_stream)
    else:
        def step():
            rgf.conductance_dev(ribs, Ed.data_ptr(), n, Td.data_ptr(), Sd.data_ptr(), 1e-8, 1e-8,
                                prec, stream.cuda_stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    stream.synchronize()
    ms, ms_sweep = [], []
    sampler = ClockSampler(local)
    with sampler:
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                step()
                e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            ms_sweep.append(rgf.profile_read_phases()[2])
    rgf.profile_enable(False)
    status = Sd.cpu().numpy()
    T = Td.cpu().numpy()
    ok = status == 0
    units = float(cells[ok].sum())
    t = sum(ms) / 1e3
    parity = None
    if not args.no_check and prec != rgf.RGF_FP64:
        nc = args.check_chains or n
        T64, s64 = rgf.conductance(ribs[:nc], Es[:nc], 1e-8, 1e-8, rgf.RGF_FP64, check=False)
        both = ok[:nc] & (s64 == 0)
        parity = {"max_abs_dT_vs_fp64": float(np.abs(T[:nc] - T64)[both].max()) if both.any() else None,
                  "chains_compared": int(both.sum()),
                  "status_mismatch": int((status[:nc] != s64).sum()), "tolerance": 1e-6}
    fl = sum(cell_slicing_flops_per_step(int(N)) * float(L) for N, L, o in zip(Ns, cells, ok) if o)
    achieved = fl / (statistics.mean(ms_sweep) / 1e3) / 1e12
    peaks, src = measured_peaks()
    if prec != rgf.RGF_FP64:
        bound, peak = "tensor", float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")))
        peak_src = f"bf16_tflops_sustained of MEASURED_PEAKS.json ({src})"
    else:
        bound, peak, peak_src = "alu", 1.25, "nominal GB300 FP64 rate (no measured figure)"
    clocks = sampler.summary()
    out = {"metric": "RGF slice-inversions/s (uneven batch, M in [102, 802])", "value": units * args.steps / t,
           "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64" if prec in (rgf.RGF_FP64, rgf.RGF_FP64_TC) else "f32x2", "data": "synthetic",
           "config": {"workload": "batched_uneven_chains", "chains": n, "chains_ok": int(ok.sum()),
                      "cells_cap": args.cells or None, "cells_total": int(cells.sum()),
                      "precision": args.precision, "l2": "flushed (256 MB write) between steps",
                      "schedule": args.schedule + (" (CUDA graph)" if use_graph else ""),
                      "launch_groups": groups, "tuning": tuned},
           "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"],
                      "reasons": clocks["reasons"]},
           "gpu_launches": (2 + groups * (1 if args.schedule == "persistent" else 3)) * args.steps,
           "roofline": {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                        "frac": achieved / peak, "traffic": None,
                        "kernel": ("batch_kernel (end columns, half sweeps and joins)"
                                   if args.schedule == "persistent" else "half_kernel (the half sweeps alone)"),
                        "flops_note": "F_alg(M = 2N) per unit-cell slice step of each chain",
                        "peak_source": peak_src},
           "parity": parity,
           "status_counts": {rgf.STATUS_NAMES[s]: int((status == s).sum()) for s in set(status.tolist())}}
    print(json.dumps(out), flush=True)


def run_grad(args):
    """dT/d eps for every on-site energy (rgf_conductance_grad, host buffers): the
    N = 101, L = 500 ribbon, Anderson +-0.15 eV, 128 energies in [-0.8, 0.8] eV,
    checkpoints every 23 cells.  One step = one call over all energies; the unit
    is one unit-cell step of one chain (right-to-left sweep, segment recompute
    and left-to-right sweep of the two-sided gradient)."""
    import torch
    from paper_1107_5300_gb300 import rgf
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    prec = {"mixed": rgf.RGF_MIXED, "tc": rgf.RGF_MIXED_TC, "fp64": rgf.RGF_FP64,
            "fp64tc": rgf.RGF_FP64_TC}[args.precision]
    w = workloads.WORKLOADS[args.workload]
    N, L = w["N"], (args.cells or w["L"])
    eps = workloads.anderson_onsite(N, L, w["W"], w["seed"])
    rem = workloads.edge_removed(N, L, w["edge_p"], w["edge_seed"]) if w["edge_p"] > 0 else None
    Es = w["energies"]()
    if "grad_idx" in w:
        Es = Es[w["grad_idx"]]
    if args.energies:
        Es = Es[: args.energies]
    rib = rgf.Ribbon(N, L, -2.7, onsite=eps, removed=rem)
    ribs = [rib] * len(Es)
    for _ in range(args.warmup):
        rgf.conductance_grad(ribs, Es, 1e-8, 1e-8, prec, ckpt_stride=w.get("ckpt_stride", 0),
                             check=False)
    torch.cuda.synchronize()
    ts = []
    sampler = ClockSampler(local)
    with sampler:
        for _ in range(args.steps):
            t0 = time.perf_counter()
            T, g, st = rgf.conductance_grad(ribs, Es, 1e-8, 1e-8, prec,
                                            ckpt_stride=w.get("ckpt_stride", 0), check=False)
            ts.append(time.perf_counter() - t0)
    ok = st == 0
    t = sum(ts)
    parity = None
    if not args.no_check and prec != rgf.RGF_FP64:
        T64, g64, s64 = rgf.conductance_grad(ribs, Es, 1e-8, 1e-8, rgf.RGF_FP64,
                                             ckpt_stride=w.get("ckpt_stride", 0), check=False)
        both = ok & (s64 == 0)
        scale = np.abs(g64).max(axis=(1, 2))
        rel = np.abs(g - g64).max(axis=(1, 2)) / np.where(scale > 0, scale, 1.0)
        far = both & (np.abs(Es) >= 0.1)
        near = both & (np.abs(Es) < 0.1)
        # energies near the charge-neutrality point (where the half systems'
        # poles make the gradient ill-conditioned) reported apart
        parity = {"max_rel_dgrad_vs_fp64_absE_ge_0.1": float(rel[far].max()) if far.any() else None,
                  "median_rel_dgrad_vs_fp64": float(np.median(rel[both])) if both.any() else None,
                  "max_rel_dgrad_vs_fp64_absE_lt_0.1": float(rel[near].max()) if near.any() else None,
                  "max_abs_dT_vs_fp64": float(np.abs(T - T64)[both].max()) if both.any() else None,
                  "chains_compared": int(both.sum()), "chains_absE_lt_0.1": int(near.sum())}
    clocks = sampler.summary()
    out = {"metric": f"RGF two-sided gradient slice-steps/s (dT/d eps, N={N}, batched energies)",
           "value": float(ok.sum()) * L * args.steps / t, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if prec in (rgf.RGF_FP64, rgf.RGF_FP64_TC) else "f32x2", "data": "synthetic",
           "config": {"workload": args.workload, "N": N, "L": L, "energies": int(len(Es)),
                      "ckpt_stride": w.get("ckpt_stride", 0), "precision": args.precision,
                      "timing": "host wall clock around the host-buffer call"},
           "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"],
                      "reasons": clocks["reasons"]},
           "parity": parity,
           "status_counts": {rgf.STATUS_NAMES[s]: int((st == s).sum()) for s in set(st.tolist())}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batched_uneven_chains":
        run_uneven(args)
        return
    if args.workload == "agnr101_L500_grad" or args.grad:
        run_grad(args)
        return
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1107_5300_gb300 import rgf, shard

    prec = {"mixed": rgf.RGF_MIXED, "tc": rgf.RGF_MIXED_TC, "fp64": rgf.RGF_FP64,
            "fp64tc": rgf.RGF_FP64_TC}[args.precision]
    w = workloads.WORKLOADS[args.workload]
    N, L = w["N"], (args.cells or w["L"])
    Es_all = w["energies"]()
    if args.energies:
        Es_all = Es_all[: args.energies]
    # The job: one disorder realisation (seed + r) per rank, every energy of the
    # grid; the chain list is sharded over the ranks longest-processing-time
    # first (shard.lpt_partition), so each rank evaluates its share with no
    # exchange on the data path and one gather brings T to rank 0.
    job = [dict(N=N, L=L, seed=w["seed"] + r, E=float(e), idx=(r, i))
           for r in range(world) for i, e in enumerate(Es_all)]
    mine = [job[i] for i in shard.lpt_partition([shard.chain_cost(N, L)] * len(job), world)[rank]]
    seeds = sorted({c["seed"] for c in mine})
    arrays = {sd: (workloads.anderson_onsite(N, L, w["W"], sd),
                   workloads.edge_removed(N, L, w["edge_p"], w["edge_seed"] + sd - w["seed"])
                   if w["edge_p"] > 0 else None) for sd in seeds}
    ribbons = {sd: rgf.Ribbon(N, L, -2.7, onsite=arrays[sd][0], removed=arrays[sd][1]) for sd in seeds}
    ribs = [ribbons[c["seed"]] for c in mine]
    Es = np.array([c["E"] for c in mine])
    n = Es.size
    stream = torch.cuda.Stream()
    Ed = torch.tensor(Es, dtype=torch.float64, device="cuda")
    Td = torch.empty(n, dtype=torch.float64, device="cuda")
    Sd = torch.empty(n, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    # The schedule: the autotuner's choice for this width (untimed, before the
    # warm-up), then either one prepared CUDA graph per step (energy fill,
    # lead decimation, work-queue reset, persistent batch kernel) or the same
    # launches through rgf_conductance_dev.
    rgf.set_schedule(rgf.RGF_SCHED_PHASED if args.schedule == "phased" else rgf.RGF_SCHED_PERSISTENT)
    rgf.set_domains(args.domains)
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    ndom = args.domains if args.domains >= 2 else rgf.auto_domains(n, 4 * L, nsm)
    ndom = max(2, min(ndom, 2 * L))
    tuned = None
    if not args.no_autotune:
        t0 = time.perf_counter()
        table, tms = rgf.autotune(prec, [N], cells=8 if N <= 300 else 2, reps=2)
        tuned = {"entry": table[0], "candidates_half_ms": [round(float(x), 3) for x in tms[0]],
                 "candidates": "engine (tensor, pipes) x panel (16, 8, 4) x pairs (1, 0)",
                 "tuning_s": round(time.perf_counter() - t0, 2)}
    rgf.profile_enable(True)
    use_graph = not args.no_graph
    if use_graph:
        batch = rgf.Batch(ribs, Ed.data_ptr(), n, Td.data_ptr(), Sd.data_ptr(), 1e-8, 1e-8, prec)

        def step():
            batch.launch(stream.cuda_stream)
    else:
        def step():
            rgf.conductance_dev(ribs, Ed.data_ptr(), n, Td.data_ptr(), Sd.data_ptr(), 1e-8, 1e-8,
                                prec, stream.cuda_stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        stream.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    peaks, peaks_src = measured_peaks()
    ms_steps, phases = [], []
    sampler = ClockSampler(local)
    with sampler:
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)          # evict L2 (129 MB) between timed steps
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                step()
                e1.record(stream)
            e1.synchronize()
            ms_steps.append(e0.elapsed_time(e1))
            phases.append(rgf.profile_read_phases())
    torch.cuda.synchronize()
    rgf.profile_enable(False)
    if dist:
        dist.barrier()
    status = Sd.cpu().numpy()
    T = Td.cpu().numpy()
    ok = status == 0
    units_local = float(ok.sum()) * L
    t_local = sum(ms_steps) / 1e3
    if dist:
        tt = torch.tensor([t_local, units_local], dtype=torch.float64, device="cuda")
        tmax = tt.clone(); dist.all_reduce(tmax[:1], op=dist.ReduceOp.MAX)
        usum = tt.clone(); dist.all_reduce(usum[1:], op=dist.ReduceOp.SUM)
        t_job, units = float(tmax[0]), float(usum[1])
        gathered = [None] * world if rank == 0 else None
        dist.gather_object(([c["idx"] for c in mine], T, status), gathered, dst=0)
    else:
        t_job, units = t_local, units_local
        gathered = [([c["idx"] for c in mine], T, status)]
    value = units * args.steps / t_job

    # Parity of this arm against the FP64 GPU path on the same chains (untimed).
    parity = None
    if not args.no_check and prec != rgf.RGF_FP64:
        # binary64 reference on the same chains, untimed (three launches)
        T64, s64 = rgf.conductance(ribs, Es, 1e-8, 1e-8, rgf.RGF_FP64, check=False)
        both = ok & (s64 == 0)
        d = np.abs(T - T64)
        low = both & (np.abs(Es) <= 5e-3)
        parity = {"max_abs_dT_vs_fp64": float(d[both].max()) if both.any() else None,
                  "max_abs_dT_low_energy": float(d[low].max()) if low.any() else None,
                  "abs_dT_at_E0": (float(d[both & (Es == 0.0)].max())
                                   if (both & (Es == 0.0)).any() else None),
                  "chains_compared": int(both.sum()),
                  "status_mismatch": int((status != s64).sum()),
                  "tolerance": 1e-6}

    # End to end through the host-buffer ABI: ribbon upload + energies in, T out.
    e2e = None
    if not args.no_e2e:
        e2e_steps = min(args.steps, 2)
        h2d = d2h = 0
        okn = 0
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            rs = {sd: rgf.Ribbon(N, L, -2.7, onsite=arrays[sd][0], removed=arrays[sd][1])
                  for sd in seeds}
            Th, sh = rgf.conductance([rs[c["seed"]] for c in mine], Es, 1e-8, 1e-8, prec, check=False)
            for r in rs.values():
                r.close()
            okn += int((sh == 0).sum())
        te = time.perf_counter() - t0
        for sd in seeds:
            h2d += arrays[sd][0].nbytes + (arrays[sd][1].nbytes if arrays[sd][1] is not None else 0)
        h2d += Es.nbytes
        d2h = Th.nbytes + sh.nbytes
        if dist:
            tt = torch.tensor([te, okn * L], dtype=torch.float64, device="cuda")
            tm = tt.clone(); dist.all_reduce(tm[:1], op=dist.ReduceOp.MAX)
            us = tt.clone(); dist.all_reduce(us[1:], op=dist.ReduceOp.SUM)
            te, e2e_units = float(tm[0]), float(us[1])
        else:
            e2e_units = okn * L
        e2e = {"value": e2e_units / te, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    # Roofline of the dominant kernel (the persistent batch kernel, or the half
    # sweeps of the phased schedule): algorithmic flops of the slice steps it
    # processes (the unit-cell count F_alg(M)) over its CUDA-event duration,
    # against the measured sustained bf16 tensor peak.
    ph = np.array(phases)                       # [steps, 4]: lead, prep, half, merge
    half_s = float(ph[:, 2].mean()) / 1e3
    if ndom > 2:                                # the joins are part of the recursion's work
        half_s = float((ph[:, 2] + ph[:, 3]).mean()) / 1e3
    steps_ok = float(ok.sum()) * L
    F_alg = cell_slicing_flops_per_step(N)
    achieved = F_alg * steps_ok / half_s / 1e12
    smax = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = 152 * 128 * smax * 1e6 * 8.0 / 54.0 / 1e12
    if prec == rgf.RGF_FP64:
        # binary64 runs on the FP64 pipe: its bound is the executed binary64
        # flop rate (pair steps), not the unit-cell count
        achieved = pair_step_flops_per_cell(N) * steps_ok / half_s / 1e12
        bound, peak, peak_src = "alu", 1.25, ("nominal GB300 FP64 rate (no measured figure); achieved "
                                              "at the executed pair-step count")
    else:
        bound, peak = "tensor", float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")))
        peak_src = f"bf16_tflops_sustained of MEASURED_PEAKS.json ({peaks_src})"
    kernel_tag = ("domain" if ndom > 2 else
                  "batch" if args.schedule == "persistent" else "half")
    traffic_file = ROOT / "profiles" / "traffic.json"
    traffic, traffic_note = None, "no DRAM counters recorded for this kernel and workload"
    if traffic_file.exists():
        try:
            rec = json.loads(traffic_file.read_text())
            traffic = rec.get(f"{kernel_tag}_{args.precision}_{args.workload}")
            if traffic is not None:
                traffic = float(traffic) * (L / float(rec.get("_cells", L)))
            if traffic is not None and rec.get("_sources_sha256") != kernel_sources_digest():
                traffic = None
                traffic_note = "DRAM counters were taken on other kernel sources; not reported"
        except Exception:
            traffic = None
    algo_bytes = float(ok.sum()) * L * 2 * N * 8     # the on-site energies each slice step reads
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic,
            **({} if traffic is not None else {"traffic_note": traffic_note}),
            "kernel": f"{kernel_tag}_kernel" + {0: "<double>", 1: "<df32>", 2: "<df32,tc>", 3: "<double,tc>"}[prec],
            "flops_per_step": F_alg,
            "flops_note": "F_alg(M) = 8/3 M^3 + 8 M^2 floor(N/2) + 8 ceil(N/2)^2 floor(N/2) per unit-cell "
                          "slice step (M = 2N); achieved = F_alg x slice steps / time of the kernel "
                          "(persistent: end columns, half sweeps and joins in one kernel)",
            "peak_source": peak_src,
            "algorithmic_bytes_per_launch": algo_bytes,
            "executed_flops_per_step": pair_step_flops_per_cell(N),
            "achieved_at_executed_count": pair_step_flops_per_cell(N) * steps_ok / half_s / 1e12,
            "column_slicing_flops_per_step": flops_per_cell(N),
            "achieved_at_column_slicing_count": flops_per_cell(N) * steps_ok / half_s / 1e12,
            "alu_peak_double_float": alu_peak,
            "frac_of_alu_peak_at_column_slicing_count": flops_per_cell(N) * steps_ok / half_s / 1e12 / alu_peak,
            "ms_kernel": float(ph[:, 2].mean()), "ms_lead": float(ph[:, 0].mean()),
            "ms_prep": float(ph[:, 1].mean()), "ms_merge": float(ph[:, 3].mean()),
            "phases_note": ("persistent: ms_kernel = the batch kernel (end columns, half sweeps, joins), "
                            "ms_prep = the work-queue reset, ms_merge = 0"
                            if kernel_tag == "batch" else
                            "domains: achieved over ms_kernel (every domain of every chain) + "
                            "ms_merge (the joins and the trace)"
                            if kernel_tag == "domain" else
                            "phased: ms_kernel = the half-sweep launch")}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(N, args.cpu_cells, w["W"], w["seed"])

    clocks = sampler.summary()
    # our kernels per step: energy fill, lead decimation, then the batch kernel
    # (persistent) or preparation, half sweeps and join (phased); one width,
    # so one launch group
    launches_per_step = 2 + (1 if args.schedule == "persistent" and ndom == 2 else 3)
    if rank == 0:
        T_all = np.full(len(job), np.nan)
        for idx, Tr, _ in gathered:
            for (r, i), t in zip(idx, Tr):
                T_all[r * len(Es_all) + i] = t
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": t_job * 1e3 / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "f64" if prec in (rgf.RGF_FP64, rgf.RGF_FP64_TC) else "f32x2", "data": "synthetic",
               "config": {"workload": args.workload, "N": N, "M": 2 * N, "L": L,
                          "energies": int(len(Es_all)), "chains_per_rank": int(n),
                          "chains_ok": int(ok.sum()), "W_eV": w["W"], "eta_eV": 1e-8,
                          "precision": args.precision, "l2": "flushed (256 MB write) between steps",
                          "parallelism": f"chains sharded over {world} rank(s) (LPT), one disorder "
                                         "realisation per rank",
                          "schedule": (args.schedule if ndom == 2 else "phased") +
                                      (" (CUDA graph)" if use_graph else ""),
                          "domains_per_chain": ndom,
                          "tuning": tuned},
               "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"],
                          "reasons": clocks["reasons"]},
               "e2e": e2e, "gpu_launches": launches_per_step * args.steps, "roofline": roof,
               "cpu_baseline": cpu, "parity": parity,
               "T_gathered_finite": int(np.isfinite(T_all).sum()),
               "status_counts": {rgf.STATUS_NAMES[s]: int((status == s).sum()) for s in set(status.tolist())}}
        print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
