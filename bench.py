"""Benchmark: compartment-steps per second of the batched cable-equation stepper on one B300.

A "step" of this benchmark is one epoch: the full hot path (event delivery, mechanism
currents, implicit-Euler assembly, Hines solve, state update, threshold detection for every
time step of the epoch, then the spike exchange) over all cells of the workload.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload ring|batched|mixed|small|dense|adjoint]
  python bench.py --impl reference ...     # the FP64 CPU oracle on the host cores

Prints one JSON line (rank 0). With torchrun and N > 1 every rank runs its own replica of
the workload (cells are independent within an epoch; no collective is needed on one GPU's
data) and value = total compartment-steps of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np

WORKLOADS = {
    # name: (config index, precision)
    "small": (0, "fp64"),
    "ring": (1, "fp64"),
    "batched": (2, "fp64"),
    "mixed": (3, "mixed"),
    "adjoint": (4, "fp64"),
    "dense": (5, "fp64"),
}

# per-workload handle settings: the dense network shares one state per synapse group and holds
# tens of millions of pending events
SIM_KW = {"dense": dict(coalesce_synapses=True, event_capacity=1 << 26, bucket_capacity=1 << 26)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


# FP64 issue ceiling of a B300: 148 SMs x 2 FP64 FMA lanes per clock x 2032 MHz (the SM count
# and maximum clock of the part; 2 per clock per SM is ncu's peak_sustained for
# sm__sass_thread_inst_executed_op_dfma_pred_on). In FLOP/s (FMA = 2) this is 1.2 PFLOP/s /
# 1000, i.e. the 1.2 TFLOP/s FP64 of the part.
FP64_PEAK_INST_PER_S = 148 * 2 * 2032e6

# FP64 thread instructions (DFMA + DMUL + DADD) the streamed epoch kernel executes per
# CV-step, and its DRAM bytes per CV-step, on the batched workload, per kernel variant with the
# plan the autotuner chose for it on the full workload: from ncu captures of 40,000 cells
# (profiles/stream_kernel_batched_40000cells.md, kernel as of commit f122cae, spread cells in
# rounds of 4 rows), which have the same cell-size mix, synapse and HH densities per CV as the
# full 65,536-cell workload. Variant 0 (16 warps per SM): cells above 305 CVs spread into packs
# of about 555 rows; variant 3 (12 warps): above 592 CVs, packs of about 766 rows. Another
# variant takes their mean. Re-measure when the kernel changes.
STREAM_FP64_PER_CV_STEP = {"batched": {0: 11.59, 3: 11.42}}
STREAM_DRAM_BYTES_PER_CV_STEP = {"batched": {0: 122.0, 3: 118.6}}


def _per_variant(table, workload, variant):
    t = table.get(workload)
    if t is None:
        return None
    return t.get(variant, sum(t.values()) / len(t))


# Discrete adjoint (every CV with HH, checkpoint every 500 steps): FP64 thread instructions per
# gradient CV-step of the forward, recompute and reverse kernels together (ncu, 64 cells of the
# fitting workload, profiles/adjoint_config4_256cells.md: the sum over the two k_adj_forward and
# the 16 k_adj_stage launches of one gradient); the algorithmic DRAM bytes per gradient
# CV-step: the recompute (for the last segment the forward pass) writes V, the three gates
# and, per HH CV, three dPhi/dV and three decay factors (80 B), which the reverse
# sweep reads back (80 B) -- the running state, lambda, the gate adjoints and the gradient sums
# stay in shared memory or L2; and the DRAM bytes the same capture measured (168.2 B).
ADJ_FP64_PER_CV_STEP = 189.4
ADJ_BYTES_PER_CV_STEP = 160.0
ADJ_DRAM_BYTES_PER_CV_STEP = 168.2


def algorithmic_bytes_per_cv_step(model, precision, coalesce=False):
    """Streaming bytes one CV-step must move if nothing stayed on chip: V read+write (16),
    capacitance/dt (8), axial conductance to the parent (8), parent index (4); passive G (8) per
    passive CV; HH gates m,h,n read+write and three conductances (72 FP64, 36 FP32-mechanism)
    per HH CV; per synapse state g read+write and its CV index (20 FP64, 12 FP32), where with
    coalescing one state serves all synapses of a CV with equal tau and e."""
    n_cv = model.n_cv
    hh = np.asarray(model.hh_cv).size
    pas = np.asarray(model.pas_cv).size
    syn = model.n_syn
    if coalesce and syn:
        syn = np.unique(np.stack([model.syn_cv, model.syn_tau, model.syn_e], 1), axis=0).shape[0]
    mixed = precision == "mixed"
    total = 36.0 * n_cv + 8.0 * pas + (36.0 if mixed else 72.0) * hh + (12.0 if mixed else 20.0) * syn
    return total / n_cv


class ClockSampler:
    """Samples nvidia-smi during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x: float) -> float:
    """The largest of x over the ranks of the default process group (x itself without one);
    every rank gets it. NCCL groups reduce on the GPU, gloo groups on the host."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def run_reference(args, model, spec, precision, workload_name):
    """The oracle (FP64 CPU) as it stands, timed on the host cores; each step is one epoch of the
    workload (by default every cell, closed loop, the same epochs as the timed arm)."""
    import oracle
    from inputs.sample import cell_sample
    rank, world, _ = dist_env()
    if rank != 0:
        return
    oracle.build()
    sub, sspec, ncells = cell_sample(model, spec, args.ref_cells)
    E = spec.epoch_steps
    sim = oracle.OracleSim(sub, spec.dt, E, nthreads=0, dry_run_ranks=args.dry_run_ranks)
    sim.enqueue(sspec.ev_syn, sspec.ev_t, sspec.ev_w)
    for _ in range(args.warmup):
        sim.run_steps(E)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sim.run_steps(E)
    el = time.perf_counter() - t0
    units = sub.n_cv * E * args.steps
    value = units / el
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": "compartment-steps/sec", "value": value, "unit": "CV-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name, "cells": model.n_cells, "cvs": model.n_cv, "epoch_steps": E,
                   "dt_ms": spec.dt, "sampled_cells": ncells},
        "cpu_baseline": {"value": value, "unit": "CV-steps/s", "cores": cores, "kind": "oracle",
                         "sample": "%d of %d cells%s, %d timed epochs of %d steps after %d warm-up epochs" % (
                             ncells, model.n_cells, " (closed loop)" if ncells == model.n_cells else " (open loop)",
                             args.steps, E, args.warmup)},
        "e2e": {"value": value, "unit": "CV-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def adjoint_inputs(model, spec):
    """Loss inputs of the fitting workload: soma observations and the loss scale; the target
    traces are those of the hidden parameter set (computed by the caller's forward path)."""
    obs = model.cv_offset[:-1].copy()
    K = spec.n_steps
    group, ng = model.param_groups()
    return obs, K, 1.0 / (K * obs.size), group, ng


def run_adjoint(args, model, spec):
    """One step = the loss and gradient of the whole run (n_steps time steps forward, then the
    checkpointed reverse sweep) for all cells. Metric: compartment-steps of the run per second
    of gradient evaluation."""
    from inputs import make_config
    obs, K, scale, group, ng = adjoint_inputs(model, spec)
    tgt_model, _ = make_config(4, n_cells=model.n_cells, t_end=spec.t_end, variant="target")
    rank, world, _ = dist_env()
    name = "adjoint: %s, %d cells, %d CVs, %d steps of dt %.3f ms, checkpoint every %d steps, %d parameters" % (
        spec.name, model.n_cells, model.n_cv, K, spec.dt, args.checkpoint_every, 4 * ng)
    if args.impl == "reference":
        if rank != 0:
            return
        import oracle
        oracle.build()
        from inputs.sample import submodel
        cells = np.arange(min(model.n_cells, max(1, args.ref_cells)))
        sm, ss, cv_old = submodel(model, spec, cells)
        st, _, _ = submodel(tgt_model, spec, cells)
        so = sm.cv_offset[:-1].copy()
        _, target = oracle.simulate(st, ss, probes=so)
        sg, sng = sm.param_groups()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            oracle.OracleSim(sm, spec.dt, spec.epoch_steps).adjoint(K, so, target, scale, sg, sng)
        el = time.perf_counter() - t0
        value = sm.n_cv * K * args.steps / el
        print(json.dumps({
            "impl": "reference", "metric": "compartment-steps/sec (gradient)", "value": value, "unit": "CV-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": 0, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "sampled_cells": int(cells.size)},
            "cpu_baseline": {"value": value, "unit": "CV-steps/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": "%d of %d cells, whole run" % (cells.size, model.n_cells)},
            "e2e": {"value": value, "unit": "CV-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}), flush=True)
        return
    import torch
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    import paper_1901_07454_b300 as arb
    # target traces of the hidden parameters: an input of the workload, made by the forward path
    ts = arb.Simulation(tgt_model, dt=spec.dt, epoch_steps=spec.epoch_steps)
    tr = ts.set_probes(obs, K)
    ts.advance(spec.t_end)
    target = tr.clone()
    del ts
    sim = arb.Simulation(model, dt=spec.dt, epoch_steps=spec.epoch_steps)
    for _ in range(args.warmup):
        sim.adjoint(K, obs, target, scale, group, ng, checkpoint_every=args.checkpoint_every)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kern = []
    e0.record(stream)
    for _ in range(args.steps):
        loss, grad = sim.adjoint(K, obs, target, scale, group, ng, checkpoint_every=args.checkpoint_every)
        kern.append(sim.last_timing()[0])
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    tot_ms = e0.elapsed_time(e1)
    units = model.n_cv * K * args.steps
    value = units / (tot_ms * 1e-3)
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        from inputs.sample import submodel
        cells = np.arange(min(model.n_cells, 8))
        sm, ss, _ = submodel(model, spec, cells)
        sg, sng = sm.param_groups()
        so = sm.cv_offset[:-1].copy()
        tcpu = tr.cpu().numpy()[:, cells]
        t0 = time.perf_counter()
        oracle.OracleSim(sm, spec.dt, spec.epoch_steps).adjoint(K, so, tcpu, scale, sg, sng)
        el = time.perf_counter() - t0
        cpu = {"value": sm.n_cv * K / el, "unit": "CV-steps/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": "%d of %d cells, whole run (%d steps), %.1f s" % (cells.size, model.n_cells, K, el)}
    # roofline of the gradient: the kernels' FP64 thread instructions per gradient CV-step (ncu)
    # against the FP64 issue ceiling, and the algorithmic state bytes against HBM
    kern_mean = sum(kern) / len(kern)
    ach = ADJ_FP64_PER_CV_STEP * units / args.steps / (kern_mean * 1e-3)
    hbm_ach = ADJ_BYTES_PER_CV_STEP * units / args.steps / (kern_mean * 1e-3) / 1e9
    peak, peak_kind = peaks()
    roofline = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_INST_PER_S, "unit": "FP64 inst/s",
                "frac": ach / FP64_PEAK_INST_PER_S,
                "traffic": ADJ_DRAM_BYTES_PER_CV_STEP * units / args.steps,
                "traffic_unit": "DRAM bytes per gradient, all launches (ncu, per CV-step x CV-steps)",
                "peak_kind": "derived: 148 SMs x 2 FP64 FMA/clk x 2032 MHz",
                "fp64_inst_per_cv_step": ADJ_FP64_PER_CV_STEP, "kernel": "k_adj_forward + k_adj_stage",
                "kernel_ms_mean": kern_mean,
                "hbm": {"achieved": hbm_ach, "peak": peak, "unit": "GB/s", "frac": hbm_ach / peak, "peak_kind": peak_kind,
                        "algorithmic_bytes_per_cv_step": ADJ_BYTES_PER_CV_STEP}}
    # end to end through the public API with host buffers: handle creation and model upload from
    # host arrays, the target traces from host memory, the gradient back to host memory
    e2e = None
    if not args.no_e2e:
        tgt_host = target.cpu().numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim2 = arb.Simulation(model, dt=spec.dt, epoch_steps=spec.epoch_steps)
        for _ in range(args.steps):
            l2, g2 = sim2.adjoint(K, obs, tgt_host, scale, group, ng, checkpoint_every=args.checkpoint_every)
            g2h = g2.cpu().numpy()
        el = time.perf_counter() - t0
        assert abs(l2 - loss) <= 1e-12 * abs(loss) and g2h.shape == (ng, 4)
        e2e = {"value": units / el, "unit": "CV-steps/s", "h2d_bytes_per_step": int(tgt_host.nbytes + model_bytes(model) / args.steps),
               "d2h_bytes_per_step": int(g2h.nbytes + 8),
               "includes": "handle creation and model upload from host arrays; per step: target traces from host, "
                           "loss and gradient, gradient to host"}
        del sim2
    print(json.dumps({
        "metric": "compartment-steps/sec (gradient)", "value": value, "unit": "CV-steps/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": name, "cells": model.n_cells, "cvs": model.n_cv, "loss": loss,
                   "l2": "working set (checkpoints and a 500-step segment, ~1.3 GB) larger than L2"},
        "adjoint_kernels_ms_mean": kern_mean, "roofline": roofline,
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": sim.last_timing()[1] * args.steps, "clocks": clk}), flush=True)


def cpu_baseline(model, spec, budget_s, dry_run_ranks=1):
    """Oracle on all host cores over a bounded sample: whole epochs of all cells until about
    budget_s seconds have passed (at least one epoch)."""
    import oracle
    from inputs.sample import cell_sample
    oracle.build()
    sub, sspec, ncells = cell_sample(model, spec, 0)
    E = spec.epoch_steps
    sim = oracle.OracleSim(sub, spec.dt, E, nthreads=0, dry_run_ranks=dry_run_ranks)
    sim.enqueue(sspec.ev_syn, sspec.ev_t, sspec.ev_w)
    t0 = time.perf_counter()
    ep = 0
    while True:
        sim.run_steps(E)
        ep += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    el = time.perf_counter() - t0
    return {"value": sub.n_cv * E * ep / el, "unit": "CV-steps/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "%d of %d cells, first %d epochs (%d steps), %.1f s" % (ncells, model.n_cells, ep, ep * E, el)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched", choices=sorted(WORKLOADS))
    ap.add_argument("--cells-per-pack", type=int, default=0)
    ap.add_argument("--split-cvs", type=int, default=0,
                    help="one cell per lane: spread cells above this many CVs over lanes (0: the library's choice)")
    ap.add_argument("--kernel-variant", type=int, default=-1,
                    help="streamed implicit plans: compiled variant of the epoch kernel (-1: the library's default)")
    ap.add_argument("--spread-rows", type=int, default=0,
                    help="streamed plans: target rows of a pack of spread cells (0: the library's choice)")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-cells", type=int, default=0,
                    help="reference arm: time the oracle on the first this many cells, open loop (0 = every cell of "
                         "the workload, closed loop, as the timed arm)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--no-forms", action="store_true", help="batched workload: skip the mixed-precision comparison")
    ap.add_argument("--cells", type=int, default=0, help="use only this many cells of the workload (0 = all)")
    ap.add_argument("--scheme", default="implicit", choices=["implicit", "explicit"])
    ap.add_argument("--checkpoint-every", type=int, default=500, help="adjoint workload: steps between checkpoints")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's packing (no GPU timing of candidate packings and kernel variants)")
    ap.add_argument("--exact-events", action="store_true",
                    help="cut steps at event times (one cell per lane) instead of applying events at step starts")
    ap.add_argument("--dry-run-ranks", type=int, default=1,
                    help="batched/mixed: the cells are rank 0 of this many ranks; connection sources span "
                         "all ranks and every spike is also walked as the proxies of the other ranks")
    ap.add_argument("--epoch-overlap", action="store_true",
                    help="epochs of half the minimum delay with the spike exchange on a second stream; a step "
                         "is still one minimum delay (two overlapped epochs)")
    args = ap.parse_args()
    assert args.warmup >= 0 and args.steps >= 1

    from inputs import make_config
    cfg, precision = WORKLOADS[args.workload]
    E_ms = None
    ncells = args.cells if args.cells > 0 else None
    vr = dict(virtual_ranks=args.dry_run_ranks) if args.dry_run_ranks > 1 else {}
    if vr and cfg not in (2, 3):
        raise SystemExit("--dry-run-ranks applies to the batched and mixed workloads")
    model, spec = make_config(cfg, n_cells=ncells, t_end=None, **vr)
    if args.workload == "adjoint":
        return run_adjoint(args, model, spec)
    E = spec.epoch_steps
    # the run must cover warm-up + timed epochs: extend external inputs if needed
    need_t = (args.warmup + args.steps) * E * spec.dt
    if need_t > spec.t_end + 1e-9:
        model, spec = make_config(cfg, n_cells=ncells, t_end=need_t, **vr)
    workload_name = "%s: %s, %d cells, %d CVs, dt %.3f ms, epoch %d steps" % (
        args.workload, spec.name, model.n_cells, model.n_cv, spec.dt, E)

    if args.impl == "reference":
        run_reference(args, model, spec, precision, workload_name)
        return

    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import paper_1901_07454_b300 as arb

    sim_kw = dict(SIM_KW.get(args.workload, {}))
    if args.exact_events:
        sim_kw["exact_events"] = True
        args.no_autotune = True
    if args.epoch_overlap:
        sim_kw["epoch_overlap"] = True
    if args.dry_run_ranks > 1:
        sim_kw["dry_run_ranks"] = args.dry_run_ranks
    if args.split_cvs:
        sim_kw["split_cvs"] = args.split_cvs
    if args.kernel_variant >= 0:
        sim_kw["kernel_variant"] = args.kernel_variant
    if args.spread_rows > 0:
        sim_kw["spread_rows"] = args.spread_rows
    E_sim = 0 if args.epoch_overlap else E      # overlapped: the library halves the minimum delay
    tuned = None
    streamed_workload = args.workload in ("batched", "mixed")
    if (streamed_workload and args.cells_per_pack in (0, 32) and not args.no_autotune and args.kernel_variant < 0
            and not args.split_cvs and not args.spread_rows and not args.exact_events and args.scheme == "implicit"):
        # large batches: time the compiled kernel variants and plan settings on the GPU first (not
        # part of the timed run); the fastest runs the benchmark
        t_tune = time.perf_counter()
        best, trials = arb.autotune_streamed(model, dt=spec.dt, epoch_steps=E_sim, precision=precision,
                                             scheme=args.scheme,
                                             ext_event_capacity=max(1 << 20, spec.ev_t.size + 16),
                                             events=(spec.ev_syn, spec.ev_t, spec.ev_w), **sim_kw)
        variants = arb.kernel_variants()
        tuned = {"chosen": best, "seconds": round(time.perf_counter() - t_tune, 1),
                 "trials": [{"kernel_variant": c["kernel_variant"],
                             "warps_per_sm": variants[c["kernel_variant"]][0],
                             "rows_in_flight": list(variants[c["kernel_variant"]][1:]),
                             "split_cvs": pinfo["split_cvs"], "spread_rows": pinfo["spread_rows"],
                             "packs": pinfo["n_packs"], "epoch_kernel_ms": round(ms, 3)} for c, pinfo, ms in trials]}
        args.cells_per_pack = 32
        for key in ("kernel_variant", "split_cvs", "spread_rows"):
            if key in best:
                sim_kw[key] = best[key]
    if args.cells_per_pack == 0 and not streamed_workload and not args.no_autotune:
        # small batches: time candidate packings on the GPU first (not part of the timed run)
        best, times = arb.autotune_packing(model, dt=spec.dt, epoch_steps=E_sim, precision=precision,
                                           scheme=args.scheme, ext_event_capacity=max(1 << 20, spec.ev_t.size + 16),
                                           events=(spec.ev_syn, spec.ev_t, spec.ev_w), **sim_kw)
        args.cells_per_pack = best["cells_per_pack"]
        tuned = {"chosen": best, "epoch_kernel_ms": {str(dict(k)["cells_per_pack"]): round(v, 3) for k, v in times.items()}}
    sim = arb.Simulation(model, dt=spec.dt, epoch_steps=E_sim, precision=precision, scheme=args.scheme,
                         cells_per_pack=args.cells_per_pack, ext_event_capacity=max(1 << 20, spec.ev_t.size + 16),
                         **sim_kw)
    sim.enqueue(spec.ev_syn, spec.ev_t, spec.ev_w)
    info = sim.plan_info()
    assert info["epoch_steps"] * (2 if args.epoch_overlap else 1) == E, info
    stream = torch.cuda.current_stream()
    k = 0
    for _ in range(args.warmup):
        k += E
        sim.advance(k * spec.dt)
    # L2 flush buffer (larger than the 126 MB L2), written between timed steps
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kern_ms = []
    launches = 0
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        ev0[i].record(stream)
        k += E
        sim.advance(k * spec.dt)
        ev1[i].record(stream)
        ms, nl = sim.last_timing()
        kern_ms.append(ms)
        launches += nl
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    tot_ms = sum(step_ms)
    tot_ms = max_over_ranks(tot_ms)
    units = model.n_cv * E * args.steps * world
    value = units / (tot_ms * 1e-3)
    nspk = sim.num_spikes()

    # roofline of the dominant kernel (the epoch kernel), timed with CUDA events around it on
    # the library's stream: FP64 issue (what binds it) and HBM (algorithmic bytes)
    bpc = algorithmic_bytes_per_cv_step(model, precision, SIM_KW.get(args.workload, {}).get("coalesce_synapses", False))
    lps = 2 if args.epoch_overlap else 1          # epoch-kernel launches per timed step
    kern_mean_ms = sum(kern_ms) / len(kern_ms) / lps
    achieved = bpc * model.n_cv * (E // lps) / (kern_mean_ms * 1e-3) / 1e9
    peak, peak_kind = peaks()
    streamed = info["cells_per_pack"] == 32
    kname = "arb_stream_kernel" if streamed else "arb_epoch_kernel"
    cv_steps_launch = model.n_cv * (E // lps)
    counted = streamed and precision == "fp64" and not args.exact_events   # the kernel the ncu counts are of
    fp64_per = _per_variant(STREAM_FP64_PER_CV_STEP, args.workload, info["kernel_variant"]) if counted else None
    dram_per = _per_variant(STREAM_DRAM_BYTES_PER_CV_STEP, args.workload, info["kernel_variant"]) if counted else None
    hbm = {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
           "algorithmic_bytes_per_cv_step": bpc,
           "traffic": dram_per * cv_steps_launch if dram_per else None}
    if fp64_per is not None:
        ach = fp64_per * cv_steps_launch / (kern_mean_ms * 1e-3)
        roofline = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_INST_PER_S, "unit": "FP64 inst/s",
                    "frac": ach / FP64_PEAK_INST_PER_S, "traffic": hbm["traffic"],
                    "peak_kind": "derived: 148 SMs x 2 FP64 FMA/clk x 2032 MHz",
                    "fp64_inst_per_cv_step": fp64_per, "kernel": kname, "kernel_ms_mean": kern_mean_ms, "hbm": hbm}
    else:
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": None, "peak_kind": peak_kind, "kernel": kname, "kernel_ms_mean": kern_mean_ms,
                    "algorithmic_bytes_per_cv_step": bpc}

    # end to end through the public API with host buffers: create + upload from host arrays,
    # per step advance one epoch and read all voltages and spikes back to the host
    e2e = None
    if rank == 0 and not args.no_e2e:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim2 = arb.Simulation(model, dt=spec.dt, epoch_steps=E_sim, precision=precision, scheme=args.scheme,
                              cells_per_pack=args.cells_per_pack, ext_event_capacity=max(1 << 20, spec.ev_t.size + 16),
                              **sim_kw)
        h2d = model_bytes(model)
        kk = 0
        ev_per_epoch = 0
        spk_read = 0
        ev_sorted = bool(np.all(np.diff(spec.ev_t) >= 0))
        for i in range(args.steps):
            lo, hi = kk * spec.dt, (kk + E) * spec.dt
            if ev_sorted:      # the epoch's events are a contiguous run of the time-sorted list
                a = 0 if i == 0 else int(np.searchsorted(spec.ev_t, lo, "left"))
                b = int(np.searchsorted(spec.ev_t, hi, "left"))
                sel = slice(a, b)
                n_sel = b - a
            else:
                sel = (spec.ev_t >= lo) & (spec.ev_t < hi) if i > 0 else (spec.ev_t < hi)
                n_sel = int(sel.sum())
            sim2.enqueue(spec.ev_syn[sel], spec.ev_t[sel], spec.ev_w[sel])
            ev_per_epoch += n_sel
            kk += E
            sim2.advance(kk * spec.dt)
            g, ts = sim2.new_spikes()
            spk_read += g.size
        v = sim2.voltage()
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        e2e = {"value": model.n_cv * E * args.steps / el, "unit": "CV-steps/s",
               "h2d_bytes_per_step": int(h2d / args.steps + 28 * ev_per_epoch / args.steps + 8),
               "d2h_bytes_per_step": int(8 * model.n_cv / args.steps + 12 * spk_read / args.steps + 16),
               "includes": "handle creation and model upload from host arrays; per step: that epoch's "
                           "external events from host, advance one epoch, that epoch's spikes to host; all voltages to host at the end"}
        del sim2

    forms = None
    if rank == 0 and args.workload == "batched" and not args.no_forms and not args.exact_events and not args.epoch_overlap:
        forms = measure_forms(arb, model, spec, sim, E, args, sim_kw, kern_mean_ms, tot_ms / args.steps, tuned)

    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            cpu = cpu_baseline(model, spec, args.cpu_budget, args.dry_run_ranks)
        line = {
            "metric": "compartment-steps/sec", "value": value, "unit": "CV-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if precision == "fp64" else "f64 solve / f32 mechanisms", "data": "synthetic",
            "scheme": args.scheme, "event_timing": "exact" if args.exact_events else "step start",
            "config": {"workload": workload_name, "cells": model.n_cells, "cvs": model.n_cv, "epoch_steps": E,
                       "dt_ms": spec.dt,
                       "step": ("one minimum delay (%d time steps) of all cells: two overlapped epochs of %d steps, "
                                "spike exchange on a second stream" % (E, E // 2)) if args.epoch_overlap else
                               "one epoch (%d time steps) of all cells incl. spike exchange" % E,
                       "epoch_overlap": bool(args.epoch_overlap),
                       "dry_run_ranks": args.dry_run_ranks,
                       "exchange_ms_per_step": (tot_ms / args.steps - lps * kern_mean_ms),
                       "l2": "flushed between timed steps (256 MB write)", "packs": info["n_packs"],
                       "lane_efficiency": round(info["lane_efficiency"], 4), "smem_packs": info["smem_packs"],
                       "max_pack_rows": info["max_pack_rows"], "split_cvs": info["split_cvs"],
                       "spread_rows": info["spread_rows"], "kernel_variant": info["kernel_variant"],
                       "cells_per_pack": info["cells_per_pack"], "autotune": tuned,
                       "spikes": nspk, "wall_s": wall, "parallelism": "replicas" if world > 1 else "single"},
            "roofline": roofline,
            "forms": forms,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def measure_forms(arb, model, spec, sim64, E, args, sim_kw, fp64_kernel_ms, fp64_step_ms, tuned):
    """The chosen forms next to the plain FP64 path on the same workload and box:
    - mixed precision (FP32 mechanism states and currents, FP64 solve and voltages): epoch time
      with the same plan, speed-up over FP64, and its voltages against the FP64 run after the same
      epochs of the closed-loop network (the per-cell accuracy of this form, open loop against the
      FP64 oracle, is what tests/test_mixed_config3_gpu.py measures);
    - autotuned packing and kernel variant against the library's default plan (the trials of the
      autotuner, same box);
    - the plain GPU path (one launch sequence per time step, default plan) against the batched
      persistent epochs."""
    import torch
    out = {}
    k_end = sim64.time()[1]
    mx = arb.Simulation(model, dt=spec.dt, epoch_steps=E, precision="mixed", scheme=args.scheme,
                        cells_per_pack=args.cells_per_pack, ext_event_capacity=max(1 << 20, spec.ev_t.size + 16),
                        **sim_kw)
    mx.enqueue(spec.ev_syn, spec.ev_t, spec.ev_w)
    k = 0
    kern, step = [], []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    while k < k_end:
        k = min(k_end, k + E)
        timed = k > args.warmup * E
        if timed:
            flush.zero_()
            ev0.record(stream)
        mx.advance(k * spec.dt)
        if timed:
            ev1.record(stream)
            torch.cuda.synchronize()
            step.append(ev0.elapsed_time(ev1))
            kern.append(mx.last_timing()[0])
    v64, vmx = sim64.voltage(), mx.voltage()
    n64, nmx = sim64.num_spikes(), mx.num_spikes()
    mk, ms_ = sum(kern) / len(kern), sum(step) / len(step)
    out["mixed"] = {"epoch_kernel_ms": mk, "ms_per_step": ms_, "speedup_kernel": fp64_kernel_ms / mk,
                    "speedup_step": fp64_step_ms / ms_, "epochs_timed": len(kern),
                    "closed_loop_after_ms": k_end * spec.dt, "max_abs_dv_vs_fp64_mV": float(np.max(np.abs(vmx - v64))),
                    "median_abs_dv_vs_fp64_mV": float(np.median(np.abs(vmx - v64))),
                    "spikes_fp64": int(n64), "spikes_mixed": int(nmx),
                    "accuracy_note": "closed-loop network: spike-time differences propagate; the open-loop per-cell "
                                     "error against the FP64 oracle is in tests/test_mixed_config3_gpu.py"}
    del mx
    # the plain GPU path: the same FP64 method with one launch sequence per time step (epochs of
    # one step: no persistence across steps) and the library's default plan; its results equal
    # the batched run's (the epoch length does not change them)
    pl = arb.Simulation(model, dt=spec.dt, epoch_steps=1, scheme=args.scheme,
                        ext_event_capacity=max(1 << 20, spec.ev_t.size + 16))
    pl.enqueue(spec.ev_syn, spec.ev_t, spec.ev_w)
    pl.advance(E * spec.dt)                                  # warm-up: one minimum delay
    torch.cuda.synchronize()
    flush.zero_()
    ev0.record(stream)
    pl.advance(2 * E * spec.dt)                              # timed: one minimum delay (E steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    plain_ms = ev0.elapsed_time(ev1)
    out["plain_per_step_launch"] = {"ms_per_min_delay": plain_ms, "steps": E,
                                    "speedup_of_batched": plain_ms / fp64_step_ms,
                                    "plan": "library default packing, epochs of one step (a launch sequence per step)"}
    del pl
    if tuned and tuned.get("trials"):
        d0 = [t for t in tuned["trials"] if t["kernel_variant"] == 0 and t["split_cvs"] == tuned["trials"][0]["split_cvs"]]
        if d0:
            out["autotuned"] = {"default_plan_epoch_kernel_ms": d0[0]["epoch_kernel_ms"],
                                "tuned_epoch_kernel_ms": min(t["epoch_kernel_ms"] for t in tuned["trials"]),
                                "speedup": d0[0]["epoch_kernel_ms"] / min(t["epoch_kernel_ms"] for t in tuned["trials"])}
    return out


def model_bytes(m):
    tot = 0
    for name in ("cv_offset", "parent", "length_um", "radius_um", "cm", "Ra", "hh_cv", "gnabar", "gkbar", "gl",
                 "pas_cv", "g_pas", "e_pas", "syn_cv", "syn_tau", "syn_e", "stim_cv", "stim_t_on", "stim_dur",
                 "stim_amp", "detector_cv", "conn_src", "conn_dst_syn", "conn_delay", "conn_weight"):
        tot += np.asarray(getattr(m, name)).nbytes
    return tot


if __name__ == "__main__":
    main()
