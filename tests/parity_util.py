"""Runs one model on the CUDA library and on the oracle with the same seeded inputs."""
import numpy as np

import oracle


def rel_err(v_gpu, v_orc):
    """max |V_gpu - V_oracle| / max(|V_oracle|, 1 mV), over all entries compared."""
    v_gpu = np.asarray(v_gpu)
    v_orc = np.asarray(v_orc)
    return float(np.max(np.abs(v_gpu - v_orc) / np.maximum(np.abs(v_orc), 1.0))) if v_orc.size else 0.0


def run_gpu(model, spec, n_steps=None, probes=None, advance_every=None, **kw):
    import paper_1901_07454_b300 as arb
    steps = spec.n_steps if n_steps is None else int(n_steps)
    sim = arb.Simulation(model, dt=spec.dt, epoch_steps=spec.epoch_steps, **kw)
    sim.enqueue(spec.ev_syn, spec.ev_t, spec.ev_w)
    trace = sim.set_probes(probes, steps) if probes is not None else None
    if advance_every:
        k = 0
        while k < steps:
            k = min(steps, k + advance_every)
            sim.advance(k * spec.dt)
    else:
        sim.advance(steps * spec.dt)
    out = dict(V=sim.voltage(), spikes=sim.spikes(), sim=sim)
    if trace is not None:
        out["trace"] = trace.cpu().numpy()
    return out


def run_oracle(model, spec, n_steps=None, probes=None, nthreads=0, scheme="implicit", exact=False):
    steps = spec.n_steps if n_steps is None else int(n_steps)
    sim, trace = oracle.simulate(model, spec, nthreads=nthreads, probes=probes, n_steps=steps,
                                 explicit=(scheme == "explicit"), exact_events=exact)
    return dict(V=sim.voltage(), spikes=sim.spikes(), trace=trace, sim=sim)


def compare_spikes(a, b, t_tol=1e-6):
    ga, ta = a
    gb, tb = b
    assert len(ta) == len(tb), (len(ta), len(tb))
    # order by (gid, t) on both sides: ties in time between cells are compared per cell
    oa = np.lexsort((ta, ga))
    ob = np.lexsort((tb, gb))
    assert np.array_equal(ga[oa], gb[ob])
    if len(ta):
        assert np.max(np.abs(ta[oa] - tb[ob])) <= t_tol, np.max(np.abs(ta[oa] - tb[ob]))


from inputs.sample import submodel  # noqa: E402,F401


def oracle_sensitivity(model, spec, probes, scheme="implicit", n_steps=None, rel=2.0 ** -52, absolute=False):
    """How far the oracle moves from itself when every initial voltage is perturbed by one ulp:
    max over the probe trace of |dV| / max(|V|, 1 mV). Through spike upstrokes this is the
    conditioning of the trajectory; two FP64 implementations that round differently at every
    step cannot agree better than a small multiple of it."""
    steps = spec.n_steps if n_steps is None else int(n_steps)
    a = oracle.OracleSim(model, spec.dt, spec.epoch_steps or 400, explicit=(scheme == "explicit"))
    b = oracle.OracleSim(model, spec.dt, spec.epoch_steps or 400, explicit=(scheme == "explicit"))
    for s in (a, b):
        s.enqueue(spec.ev_syn, spec.ev_t, spec.ev_w)
    st = b.get_state()
    st["V"] = st["V"] * (1.0 + rel)
    b.set_state(st)
    ta = a.set_probes(probes, steps)
    tb = b.set_probes(probes, steps)
    a.run_steps(steps)
    b.run_steps(steps)
    return float(np.max(np.abs(tb - ta))) if absolute else rel_err(tb, ta)


TRACE_FACTOR = 20.0


def trace_bar(tol, spread, factor=TRACE_FACTOR):
    """Comparison bar for step-by-step traces through spikes: the tolerance, or a small multiple
    of how far two equally valid FP64 oracle runs drift apart (oracle_spread) when that is
    larger -- the trajectory's own conditioning."""
    return max(tol, factor * spread)


def record(kind, **vals):
    """Prints the error a parity check reached (and appends it to the file named by
    ARB_PARITY_LOG, one JSON object per line), tagged with the running test."""
    import json
    import os
    line = {"test": os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0], "kind": kind}
    line.update({k: (float(v) if isinstance(v, (int, float, np.floating, np.integer)) else v) for k, v in vals.items()})
    print("PARITY " + json.dumps(line))
    path = os.environ.get("ARB_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(line) + "\n")


def check_end(v_gpu, v_orc, tol=1e-9, **tags):
    """End-of-run voltages: max relative error (as rel_err) within tol."""
    e = rel_err(v_gpu, v_orc)
    record("end", err=e, bar=tol, **tags)
    assert e <= tol, (e, tol)
    return e


def check_trace(tr_gpu, tr_orc, spread, tol=1e-9, **tags):
    """Step-by-step traces: within trace_bar(tol, spread)."""
    e = rel_err(tr_gpu, tr_orc)
    bar = trace_bar(tol, spread)
    record("trace", err=e, bar=bar, spread=spread, ratio=(e / spread if spread > 0 else 0.0), **tags)
    assert e <= bar, (e, bar, spread)
    return e


def renumbered(model):
    """The same cells with every cell's CVs renumbered in another valid Hines order (children
    visited in reverse during a depth-first walk). Returns (model, perm) with
    new_V[perm] == old-order V. The oracle run on it rounds differently at every step."""
    from inputs import Model
    off = model.cv_offset
    order = np.empty(model.n_cv, np.int64)      # new position -> old CV
    for c in range(model.n_cells):
        lo, hi = off[c], off[c + 1]
        n = hi - lo
        par = model.parent[lo:hi]
        kids = [[] for _ in range(n)]
        for i in range(1, n):
            kids[par[i]].append(i)
        out, stack = [], [0]
        while stack:
            v = stack.pop()
            out.append(v)
            stack.extend(kids[v])            # last child first
        order[lo:hi] = lo + np.array(out)
    new_of_old = np.empty(model.n_cv, np.int64)
    new_of_old[order] = np.arange(model.n_cv)
    cell = np.repeat(np.arange(model.n_cells), np.diff(off))
    old_par = model.parent[order]
    new_par = np.where(old_par >= 0, new_of_old[off[cell] + np.maximum(old_par, 0)] - off[cell], -1).astype(np.int32)
    m = Model(cv_offset=off, parent=new_par, length_um=model.length_um[order], radius_um=model.radius_um[order],
              cm=model.cm[order], Ra=model.Ra[order], branch_of_cv=model.branch_of_cv[order],
              hh_cv=new_of_old[model.hh_cv], gnabar=model.gnabar, gkbar=model.gkbar, gl=model.gl,
              pas_cv=new_of_old[model.pas_cv], g_pas=model.g_pas, e_pas=model.e_pas,
              syn_cv=new_of_old[model.syn_cv], syn_tau=model.syn_tau, syn_e=model.syn_e,
              stim_cv=new_of_old[model.stim_cv], stim_t_on=model.stim_t_on, stim_dur=model.stim_dur,
              stim_amp=model.stim_amp, detector_cv=new_of_old[model.detector_cv], threshold=model.threshold,
              conn_src=model.conn_src, conn_dst_syn=model.conn_dst_syn, conn_delay=model.conn_delay,
              conn_weight=model.conn_weight)
    return m, new_of_old


def oracle_spread(model, spec, probes, scheme="implicit", n_steps=None, exact=False):
    """Disagreement between two equally valid FP64 oracle runs that round differently at every
    step (original vs renumbered CVs): max over the probe trace of |dV| / max(|V|, 1 mV)."""
    a = run_oracle(model, spec, n_steps=n_steps, probes=probes, scheme=scheme, exact=exact)
    m2, new_of_old = renumbered(model)
    b = run_oracle(m2, spec, n_steps=n_steps, probes=new_of_old[np.asarray(probes)], scheme=scheme, exact=exact)
    return rel_err(b["trace"], a["trace"])
