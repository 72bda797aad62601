"""Packing autotuner: times candidate packings of a model on the GPU and returns the fastest.

The library's default packing comes from a static cost model. Here each candidate
(cells_per_pack, and for the streamed plan the split threshold) is planned and bound like a
normal handle, runs warm-up and timed epochs from the model's initial state with the
workload's first external events, and the epoch kernel's device time (arb_last_timing)
decides. Only handles are created and advanced: every step runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np

from .sim import Simulation


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
        args = dict(kw)
        args.update(cand)
        sim = Simulation(model, dt=dt, epoch_steps=epoch_steps, **args)
        if events is not None:
            sim.enqueue(*events)
        E = sim.plan_info()["epoch_steps"]
        k = 0
        for _ in range(warmup):
            k += E
            sim.advance(k * dt)
        ms = []
        for _ in range(epochs):
            k += E
            sim.advance(k * dt)
            ms.append(sim.last_timing()[0])
        key = tuple(sorted(cand.items()))
        times[key] = float(np.mean(ms))
        if times[key] < best_ms:
            best, best_ms = dict(cand), times[key]
        del sim
    return best, times
