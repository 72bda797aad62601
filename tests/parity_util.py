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


def run_oracle(model, spec, n_steps=None, probes=None, nthreads=0):
    steps = spec.n_steps if n_steps is None else int(n_steps)
    sim, trace = oracle.simulate(model, spec, nthreads=nthreads, probes=probes, n_steps=steps)
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
