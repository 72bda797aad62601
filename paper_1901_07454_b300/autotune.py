"""Packing autotuner: times candidate packings of a model on the GPU and returns the fastest.

The library's default packing comes from a static cost model. Here each candidate (a dict of
Simulation settings: cells_per_pack; for streamed plans also the kernel variant, which fixes the
warps per SM and the rows each warp keeps in flight, the split threshold and the rows of a pack
of spread cells) is planned and bound like a normal handle, runs warm-up and timed epochs from
the model's initial state with the workload's first external events, and the epoch kernel's
device time (arb_last_timing) decides. Only handles are created and advanced: every step runs in
the library's kernels.
"""
from __future__ import annotations

import numpy as np

from ._lib import kernel_variants
from .sim import Simulation


def _time(model, dt, epoch_steps, cand, events, warmup, epochs, kw):
    args = dict(kw)
    args.update(cand)
    sim = Simulation(model, dt=dt, epoch_steps=epoch_steps, **args)
    if events is not None:
        sim.enqueue(*events)
    info = sim.plan_info()
    E = info["epoch_steps"]
    k = 0
    for _ in range(warmup):
        k += E
        sim.advance(k * dt)
    ms = []
    for _ in range(epochs):
        k += E
        sim.advance(k * dt)
        ms.append(sim.last_timing()[0])
    del sim
    return float(np.mean(ms)), info


def autotune_packing(model, dt=0.025, epoch_steps=0, candidates=None, events=None, warmup=1, epochs=2, **kw):
    """Returns (best settings dict, {settings key: mean epoch-kernel ms}). candidates: list of
    dicts of Simulation keyword arguments (default: cells_per_pack 16, 8, 4, 2 and the
    streamed plan); events: optional (syn, t, w) external events; kw: other Simulation
    arguments shared by all candidates (precision, scheme, capacities, ...)."""
    if candidates is None:
        candidates = [dict(cells_per_pack=k) for k in (16, 8, 4, 2)] + [dict(cells_per_pack=32)]
    times = {}
    best, best_ms = None, np.inf
    for cand in candidates:
        ms, _ = _time(model, dt, epoch_steps, cand, events, warmup, epochs, kw)
        key = tuple(sorted(cand.items()))
        times[key] = ms
        if ms < best_ms:
            best, best_ms = dict(cand), ms
    return best, times


def autotune_streamed(model, dt=0.025, epoch_steps=0, events=None, warmup=1, epochs=2, refine=3, **kw):
    """Streamed plans (one cell per lane, large cells spread over lanes): first every compiled
    kernel variant with the plan its cost model chooses, then, for the `refine` fastest, the
    split threshold at 0.27, 0.4, 0.55 and 0.75 of the chosen one and the spread packs' rows at 0.96 and
    1.06 of the chosen ones. Returns (best settings dict, [(settings, plan summary, epoch-kernel
    ms)])."""
    trials = []

    def run(cand):
        ms, info = _time(model, dt, epoch_steps, cand, events, warmup, epochs, kw)
        trials.append((dict(cand), {k: info[k] for k in ("split_cvs", "spread_rows", "n_packs", "max_pack_rows")}, ms))
        return ms, info

    first = []
    for v in range(len(kernel_variants())):
        ms, info = run(dict(cells_per_pack=32, kernel_variant=v))
        first.append((ms, v, info))
    first.sort(key=lambda x: x[0])
    for ms, v, info in first[:refine]:
        s, r = info["split_cvs"], info["spread_rows"]
        if s <= 0 or r <= 0:
            continue
        for cand in (dict(split_cvs=int(0.27 * s), spread_rows=r), dict(split_cvs=int(0.4 * s), spread_rows=r),
                     dict(split_cvs=int(0.55 * s), spread_rows=r),
                     dict(split_cvs=int(0.75 * s), spread_rows=r), dict(split_cvs=s, spread_rows=int(0.96 * r)),
                     dict(split_cvs=s, spread_rows=int(1.06 * r))):
            run(dict(cells_per_pack=32, kernel_variant=v, **cand))
    best = min(trials, key=lambda x: x[2])
    return best[0], trials
