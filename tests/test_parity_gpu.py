"""CUDA path vs the FP64 oracle on the same seeded inputs (needs a B300).

Bar (FP64 form): max |V_gpu - V_oracle| / max(|V_oracle|, 1 mV) <= 1e-9 over every
compared voltage, identical spike counts, spike times within 1e-6 ms.
Mixed form (FP32 mechanisms): |V_gpu - V_oracle| <= 1e-3 mV and identical spike counts.
"""
import numpy as np
import pytest

from inputs import Model, SimSpec, make_config, small_tree_model, uniform_cable_model
from parity_util import check_end, check_trace, compare_spikes, record, oracle_sensitivity, oracle_spread, rel_err, run_gpu, run_oracle, submodel, trace_bar

pytestmark = pytest.mark.gpu
TOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1901_07454_b300 import _build
    _build.build()
    import oracle
    oracle.build()


def _with_events(m, seed, rate_hz, t_end, w=0.02):
    rng = np.random.default_rng(seed)
    n = rng.poisson(rate_hz * 1e-3 * t_end * max(m.n_syn, 1))
    syn = rng.integers(0, max(m.n_syn, 1), n) if m.n_syn else np.zeros(0, np.int64)
    t = rng.uniform(0, t_end, syn.size)
    return syn, t, np.full(syn.size, w)


@pytest.mark.parametrize("scheme", ["implicit", "explicit"])
def test_uniform_cable_every_step(scheme):
    m = uniform_cable_model(50, 1000.0, 1.0)
    m.stim_cv, m.stim_t_on, m.stim_dur, m.stim_amp = np.array([0]), np.array([0.0]), np.array([30.0]), np.array([0.1])
    m.__post_init__()
    spec = SimSpec(dt=0.025, t_end=50.0, epoch_steps=100)
    probes = np.arange(m.n_cv)
    g = run_gpu(m, spec, probes=probes, scheme=scheme)
    o = run_oracle(m, spec, probes=probes, scheme=scheme)
    check_end(g["trace"], o["trace"])
    check_end(g["V"], o["V"])


# cells_per_pack 32 is the streamed plan: split 0 lets the library spread cells over lanes (here
# every cell, as the batch is far smaller than the GPU), -1 keeps one cell per lane, 40 puts the
# cells above 40 CVs together into one pack whose lanes they share
@pytest.mark.parametrize("kpp,scheme,split", [(32, "implicit", 0), (32, "implicit", -1), (32, "implicit", 40),
                                              (8, "implicit", 0), (3, "implicit", 0), (1, "implicit", 0),
                                              (32, "explicit", -1), (32, "explicit", 40), (8, "explicit", 0)])
def test_random_trees_every_cv_every_step(kpp, scheme, split):
    # ragged trees, HH soma, passive dendrites, synapses with events, clamps that make cells fire
    m = small_tree_model(11, n_cells=37, n_branches=9, cv_range=(1, 12), n_syn=4)
    m.stim_cv = m.cv_offset[:-1:3].copy()
    k = m.stim_cv.size
    m.stim_t_on, m.stim_dur, m.stim_amp = np.full(k, 2.0), np.full(k, 10.0), np.linspace(0.05, 1.0, k)
    m.__post_init__()
    syn, t, w = _with_events(m, 3, 40.0, 30.0)
    spec = SimSpec(dt=0.025, t_end=30.0, epoch_steps=40, ev_syn=syn, ev_t=t, ev_w=w)
    probes = np.arange(m.n_cv)
    g = run_gpu(m, spec, probes=probes, cells_per_pack=kpp, scheme=scheme, split_cvs=split)
    o = run_oracle(m, spec, probes=probes, scheme=scheme)
    check_end(g["V"], o["V"])
    check_trace(g["trace"], o["trace"], oracle_spread(m, spec, probes, scheme))
    compare_spikes(g["spikes"], o["spikes"])
    assert len(o["spikes"][1]) > 0


def test_every_kernel_variant_keeps_parity():
    # each compiled variant of the streamed implicit kernel (warps per SM, rows in flight) on
    # ragged trees, with cells one per lane and spread over lanes
    import paper_1901_07454_b300 as arb
    m = small_tree_model(11, n_cells=37, n_branches=9, cv_range=(1, 12), n_syn=4)
    m.stim_cv = m.cv_offset[:-1:3].copy()
    k = m.stim_cv.size
    m.stim_t_on, m.stim_dur, m.stim_amp = np.full(k, 2.0), np.full(k, 10.0), np.linspace(0.05, 1.0, k)
    m.__post_init__()
    syn, t, w = _with_events(m, 3, 40.0, 30.0)
    spec = SimSpec(dt=0.025, t_end=30.0, epoch_steps=40, ev_syn=syn, ev_t=t, ev_w=w)
    probes = np.arange(m.n_cv)
    o = run_oracle(m, spec, probes=probes)
    bar = trace_bar(TOL, oracle_spread(m, spec, probes))
    variants = arb.kernel_variants()
    assert len(variants) >= 4
    for v in range(len(variants)):
        for split in (-1, 40):
            g = run_gpu(m, spec, probes=probes, cells_per_pack=32, split_cvs=split, kernel_variant=v)
            e_end, e_tr = rel_err(g["V"], o["V"]), rel_err(g["trace"], o["trace"])
            print("variant %d %s split %d: end %.2e trace %.2e (bar %.2e)" % (v, variants[v], split, e_end, e_tr, bar))
            assert e_end <= TOL and e_tr <= bar, (v, split, e_end, e_tr)
            compare_spikes(g["spikes"], o["spikes"])


@pytest.mark.parametrize("scheme", ["implicit", "explicit"])
def test_config0_plain_small_full_run(scheme):
    m, spec = make_config(0)
    probes = np.arange(m.n_cv)
    g = run_gpu(m, spec, probes=probes, scheme=scheme)
    o = run_oracle(m, spec, probes=probes, scheme=scheme)
    check_end(g["V"], o["V"])
    check_trace(g["trace"], o["trace"], oracle_spread(m, spec, probes, scheme))
    compare_spikes(g["spikes"], o["spikes"])


def test_ring_closed_loop_spikes():
    m, spec = make_config(1, n_cells=48, t_end=150.0)
    g = run_gpu(m, spec, probes=m.detector_cv)
    o = run_oracle(m, spec, probes=m.detector_cv)
    compare_spikes(g["spikes"], o["spikes"])
    assert len(o["spikes"][1]) >= 27
    check_trace(g["trace"], o["trace"], oracle_spread(m, spec, m.detector_cv))
    check_end(g["V"], o["V"])


def test_ring_per_epoch_spike_export():
    # new_spikes() after each advance returns that epoch's spikes only (arb_read_spikes_from);
    # the pieces lie inside their epochs and concatenate to the oracle's sorted spike list
    import paper_1901_07454_b300 as arb
    m, spec = make_config(1, n_cells=48, t_end=150.0)
    sim = arb.Simulation(m, dt=spec.dt, epoch_steps=spec.epoch_steps)
    sim.enqueue(spec.ev_syn, spec.ev_t, spec.ev_w)
    E = spec.epoch_steps
    gs, ts = [], []
    k = 0
    while k < spec.n_steps:
        k0, k = k, min(spec.n_steps, k + E)
        sim.advance(k * spec.dt)
        g, t = sim.new_spikes()
        assert np.all(t >= k0 * spec.dt - 1e-12) and np.all(t <= k * spec.dt + 1e-12)
        gs.append(g)
        ts.append(t)
    assert sim.new_spikes()[0].size == 0
    ga, ta = np.concatenate(gs), np.concatenate(ts)
    gall, tall = sim.spikes()
    assert np.array_equal(ga, gall) and np.array_equal(ta, tall)
    o = run_oracle(m, spec)
    compare_spikes((ga, ta), o["spikes"])
    assert sim.spikes(first=10 ** 9)[0].size == 0


def test_ring_divergence_of_the_explicit_scheme_is_reported():
    # With the membrane current on the right-hand side (explicit in V), the tiny soma CV of
    # cell 12 receives several simultaneous events and the step becomes unstable at 65 ms.
    # The oracle runs into NaN there; the library stops with ARB_E_NONFINITE.
    import paper_1901_07454_b300 as arb
    m, spec = make_config(1, n_cells=48, t_end=70.0)
    o = run_oracle(m, spec, scheme="explicit")
    assert np.isnan(o["V"]).any()
    bad_cells = np.unique(np.searchsorted(m.cv_offset, np.nonzero(np.isnan(o["V"]))[0], "right") - 1)
    assert 12 in bad_cells
    sim = arb.Simulation(m, dt=spec.dt, epoch_steps=spec.epoch_steps, scheme="explicit")
    with pytest.raises(arb.ArbError) as ei:
        sim.advance(70.0)
    assert "NONFINITE" in str(ei.value)


def test_ring_full_size_short_window():
    # the 1024-cell ring at full size for 20 ms (4 epochs), every CV at the end
    m, spec = make_config(1, t_end=20.0)
    g = run_gpu(m, spec)
    o = run_oracle(m, spec)
    check_end(g["V"], o["V"])
    compare_spikes(g["spikes"], o["spikes"])


def test_batched_network_small_closed_loop():
    m, spec = make_config(2, n_cells=384, t_end=40.0)
    probes = m.detector_cv
    g = run_gpu(m, spec, probes=probes)
    o = run_oracle(m, spec, probes=probes)
    check_end(g["V"], o["V"])
    check_trace(g["trace"], o["trace"], oracle_spread(m, spec, probes))
    compare_spikes(g["spikes"], o["spikes"])


def test_batched_full_size_sampled_cells():
    # 65,536 cells in the launch configuration of the benchmark; in the first millisecond no
    # spike can arrive (minimum delay 1 ms), so sampled cells evolve as models of their own
    m, spec = make_config(2, t_end=1.0)
    g = run_gpu(m, spec)
    rng = np.random.default_rng(0)
    cells = np.sort(rng.choice(m.n_cells, 48, replace=False))
    cells = np.unique(np.concatenate([cells, np.argsort(np.diff(m.cv_offset))[-4:]]))  # the largest too
    sm, ss, cv_old = submodel(m, spec, cells)
    o = run_oracle(sm, ss)
    check_end(g["V"][cv_old], o["V"])


def test_mixed_full_size_sampled_cells():
    # the 65,536-cell mixed workload (FP32 mechanisms) in the benchmark's launch configuration;
    # sampled cells against the FP64 oracle, open loop over the first millisecond
    m, spec = make_config(3, t_end=1.0)
    g = run_gpu(m, spec, precision="mixed")
    rng = np.random.default_rng(1)
    cells = np.unique(np.concatenate([rng.choice(1024, 24, replace=False),
                                      np.argsort(np.diff(m.cv_offset))[-4:]]))
    sm, ss, cv_old = submodel(m, spec, cells)
    o = run_oracle(sm, ss)
    assert np.max(np.abs(g["V"][cv_old] - o["V"])) <= 1e-3


def test_epoch_length_and_advance_chunks_are_bitwise_neutral():
    m, spec = make_config(1, n_cells=24, t_end=40.0)
    a = run_gpu(m, spec)
    b = run_gpu(m, SimSpec(dt=spec.dt, t_end=spec.t_end, epoch_steps=100))
    c = run_gpu(m, spec, advance_every=37)
    d = run_gpu(m, spec)
    for x in (b, c, d):
        assert np.array_equal(a["V"], x["V"])
        assert np.array_equal(a["spikes"][0], x["spikes"][0]) and np.array_equal(a["spikes"][1], x["spikes"][1])


def test_mixed_precision_within_1e3_mV():
    m = small_tree_model(11, n_cells=37, n_branches=9, cv_range=(1, 12), n_syn=4)
    m.stim_cv = m.cv_offset[:-1:3].copy()
    k = m.stim_cv.size
    m.stim_t_on, m.stim_dur, m.stim_amp = np.full(k, 2.0), np.full(k, 10.0), np.linspace(0.05, 1.0, k)
    m.__post_init__()
    syn, t, w = _with_events(m, 3, 40.0, 30.0)
    spec = SimSpec(dt=0.025, t_end=30.0, epoch_steps=40, ev_syn=syn, ev_t=t, ev_w=w)
    o = run_oracle(m, spec, probes=np.arange(m.n_cv))
    # through spikes, an FP32-sized change (2^-24) of the state moves the FP64 oracle itself by
    # this much: the bar is 1e-3 mV or a small multiple of that, whichever is larger
    sens32 = oracle_sensitivity(m, spec, np.arange(m.n_cv), rel=2.0 ** -24, absolute=True)
    for kw in ({}, {"cells_per_pack": 32, "split_cvs": 40}):
        g = run_gpu(m, spec, probes=np.arange(m.n_cv), precision="mixed", **kw)
        assert len(g["spikes"][1]) == len(o["spikes"][1])
        compare_spikes(g["spikes"], o["spikes"], t_tol=1e-3)
        assert np.max(np.abs(g["V"] - o["V"])) <= 1e-3
        err = float(np.max(np.abs(g["trace"] - o["trace"])))
        end = float(np.max(np.abs(g["V"] - o["V"])))
        record("mixed_trace_mV", err=err, end_err=end, bar=max(1e-3, 20.0 * sens32), sensitivity_f32=sens32,
               plan=str(kw))
        assert err <= max(1e-3, 20.0 * sens32), (kw, err, sens32)


def test_state_roundtrip_continues_identically():
    m = small_tree_model(4, n_cells=10, n_branches=6, cv_range=(2, 8), n_syn=2)
    m.stim_cv, m.stim_t_on, m.stim_dur, m.stim_amp = np.array([0]), np.array([0.0]), np.array([50.0]), np.array([0.5])
    m.__post_init__()
    import paper_1901_07454_b300 as arb
    a = arb.Simulation(m, epoch_steps=40)
    a.advance(10.0)
    st = a.get_state()
    b = arb.Simulation(m, epoch_steps=40)
    b.set_state(st)
    assert np.array_equal(b.get_state()["V"], st["V"])
    # b starts at t = 0 from the saved state; the oracle does the same
    o = run_oracle(m, SimSpec(dt=0.025, t_end=0.0, epoch_steps=40))["sim"]
    o.set_state(st)
    o.run_steps(200)
    b.advance(5.0)
    check_end(b.voltage(), o.voltage())


def test_edge_cases_single_cv_star_and_long_chain():
    # single-CV cells, a 12-way star, and one 2500-CV chain whose tile does not fit in shared memory
    cells = []
    for i in range(5):
        cells.append(np.array([-1], np.int32))
    star = np.array([-1] + [0] * 12 + list(range(1, 13)), np.int32)
    cells.append(star)
    cells.append(np.arange(-1, 2499, dtype=np.int32))
    parent = np.concatenate(cells)
    off = np.concatenate([[0], np.cumsum([c.size for c in cells])])
    n = parent.size
    rng = np.random.default_rng(2)
    m = Model(cv_offset=off, parent=parent, length_um=rng.uniform(5, 30, n), radius_um=rng.uniform(0.3, 2, n),
              cm=np.ones(n), Ra=np.full(n, 100.0), branch_of_cv=np.zeros(n, np.int32),
              hh_cv=off[:-1], gnabar=np.full(len(cells), 0.12), gkbar=np.full(len(cells), 0.036),
              gl=np.full(len(cells), 3e-4),
              pas_cv=np.setdiff1d(np.arange(n), off[:-1]), g_pas=np.full(n - len(cells), 1e-4),
              e_pas=np.full(n - len(cells), -65.0),
              stim_cv=off[:-1], stim_t_on=np.zeros(len(cells)), stim_dur=np.full(len(cells), 5.0),
              stim_amp=np.linspace(0.01, 0.3, len(cells)))
    spec = SimSpec(dt=0.025, t_end=15.0, epoch_steps=64)
    for kpp, split in ((32, 0), (32, -1), (2, 0)):
        g = run_gpu(m, spec, probes=np.arange(n), cells_per_pack=kpp, split_cvs=split)
        o = run_oracle(m, spec, probes=np.arange(n))
        check_end(g["V"], o["V"])
        check_trace(g["trace"], o["trace"], oracle_spread(m, spec, np.arange(n)))
        compare_spikes(g["spikes"], o["spikes"])


def test_overflow_is_reported_without_fault():
    import paper_1901_07454_b300 as arb
    m, spec = make_config(1, n_cells=16, t_end=40.0)
    sim = arb.Simulation(m, epoch_steps=200, spike_capacity=2)
    with pytest.raises(arb.ArbError) as ei:
        sim.advance(40.0)
    assert "OVERFLOW" in str(ei.value)


def test_nonfinite_is_reported():
    import paper_1901_07454_b300 as arb
    m = uniform_cable_model(3, 30.0, 1.0, g_pas=0.5)          # dt*G/C = 12.5: explicit leak diverges
    sim = arb.Simulation(m, dt=0.025, epoch_steps=100, scheme="explicit")
    st = sim.get_state()
    st["V"][:] = -20.0
    sim.set_state(st)
    with pytest.raises(arb.ArbError) as ei:
        sim.advance(100.0)
    assert "NONFINITE" in str(ei.value)


@pytest.mark.parametrize("kpp", [0, 32])
def test_coalesced_synapses_match_the_oracle(kpp):
    # many synapses per CV (three time constants, two reversals): coalesced states must give the
    # per-synapse oracle's voltages, and the state read-back carries each group's summed g
    import paper_1901_07454_b300 as arb
    m = small_tree_model(13, n_cells=20, n_branches=6, cv_range=(2, 9), n_syn=60)
    rng = np.random.default_rng(9)
    m.syn_tau = rng.choice([1.0, 2.0, 5.0], m.n_syn)
    m.syn_e = rng.choice([0.0, -70.0], m.n_syn)
    m.stim_cv = m.cv_offset[:-1:2].copy()
    k = m.stim_cv.size
    m.stim_t_on, m.stim_dur, m.stim_amp = np.full(k, 1.0), np.full(k, 8.0), np.linspace(0.1, 0.8, k)
    m.__post_init__()
    syn, t, w = _with_events(m, 4, 60.0, 20.0, w=0.01)
    spec = SimSpec(dt=0.025, t_end=20.0, epoch_steps=40, ev_syn=syn, ev_t=t, ev_w=w)
    g = run_gpu(m, spec, probes=m.cv_offset[:-1], cells_per_pack=kpp, coalesce_synapses=True)
    o = run_oracle(m, spec, probes=m.cv_offset[:-1])
    check_end(g["V"], o["V"])
    compare_spikes(g["spikes"], o["spikes"])
    # g per (CV, tau, e) group, reported on the group's lowest-index synapse
    key = np.stack([m.syn_cv, m.syn_tau, m.syn_e], 1)
    _, first, unit = np.unique(key, axis=0, return_index=True, return_inverse=True)
    og = o["sim"].get_state()["g"]
    want = np.zeros(m.n_syn)
    np.add.at(want, first[unit.ravel()], og)
    got = g["sim"].get_state()["g"]
    assert np.max(np.abs(got - want)) <= 1e-12 * max(1.0, np.max(np.abs(want)))
    assert np.count_nonzero(got) <= first.size
    # setting a state sums each group: the same state read back
    st = g["sim"].get_state()
    g["sim"].set_state(st)
    assert np.array_equal(g["sim"].get_state()["g"], got)


def test_dense_network_closed_loop_small():
    # the dense workload at 128 cells x 1,000 synapses: synchronous 50 Hz firing, every spike
    # fans out to ~1,000 synapses with delays of 10-20 ms
    m, spec = make_config(5, n_cells=128, syn_per_cell=1000, t_end=60.0)
    probes = m.cv_offset[:-1]
    o = run_oracle(m, spec, probes=probes)
    for co in (True, False):
        g = run_gpu(m, spec, probes=probes, coalesce_synapses=co)
        compare_spikes(g["spikes"], o["spikes"])
        check_end(g["V"], o["V"])
        check_trace(g["trace"], o["trace"], oracle_spread(m, spec, probes))
    assert len(o["spikes"][1]) == 3 * m.n_cells


def test_dense_full_size_two_epochs():
    # 4,096 cells x 10,000 synapses (41M connections) in the benchmark's configuration: the
    # synchronous spikes of the first epoch deliver ~41M events into the second
    m, spec = make_config(5, t_end=20.0)
    g = run_gpu(m, spec, coalesce_synapses=True, event_capacity=1 << 26, bucket_capacity=1 << 26)
    o = run_oracle(m, spec)
    compare_spikes(g["spikes"], o["spikes"])
    check_end(g["V"], o["V"])


def test_autotuned_packing_is_timed_and_keeps_parity():
    import paper_1901_07454_b300 as arb
    m, spec = make_config(1, n_cells=96, t_end=10.0)
    best, times = arb.autotune_packing(m, dt=spec.dt, epoch_steps=spec.epoch_steps,
                                       candidates=[dict(cells_per_pack=k) for k in (8, 2, 32)], epochs=1)
    assert len(times) == 3 and all(t > 0 for t in times.values())
    assert best["cells_per_pack"] in (8, 2, 32)
    assert times[tuple(sorted(best.items()))] == min(times.values())
    g = run_gpu(m, spec, **best)
    o = run_oracle(m, spec)
    check_end(g["V"], o["V"])


def test_streamed_autotuner_times_every_variant_and_keeps_parity():
    # the large-batch tuner on a 2,048-cell slice of the batched workload: every kernel variant is
    # timed, the refinements too, and the chosen settings give the oracle's voltages on sampled
    # cells (open loop over the first millisecond, before any network event can arrive)
    import paper_1901_07454_b300 as arb
    m, spec = make_config(2, n_cells=2048, t_end=1.0)
    best, trials = arb.autotune_streamed(m, dt=spec.dt, epoch_steps=spec.epoch_steps, warmup=1, epochs=1,
                                         events=(spec.ev_syn, spec.ev_t, spec.ev_w))
    nv = len(arb.kernel_variants())
    assert {c["kernel_variant"] for c, _, _ in trials} == set(range(nv))
    assert len(trials) > nv and all(ms > 0 for _, _, ms in trials)
    assert best == min(trials, key=lambda x: x[2])[0]
    g = run_gpu(m, spec, **best)
    cells = np.unique(np.concatenate([np.arange(0, m.n_cells, 97), np.argsort(np.diff(m.cv_offset))[-3:]]))
    sm, ss, cv_old = submodel(m, spec, cells)
    o = run_oracle(sm, ss)
    err = rel_err(g["V"][cv_old], o["V"])
    print("tuned %s: max rel err %.2e on %d sampled cells" % (best, err, cells.size))
    assert err <= TOL

