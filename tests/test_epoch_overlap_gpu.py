"""Overlapped spike exchange (epochs of half the minimum delay, Sec. "Implementation"): while
epoch i integrates, a second stream walks the spikes of epoch i-1 and builds the delivery lists
of epoch i+1. The schedule changes no arithmetic, so the voltages and spikes must equal those of
the serial schedule with the same epoch length bit for bit, and the oracle within the FP64 bar.
"""
import numpy as np
import pytest

from inputs import make_config
from parity_util import check_end, compare_spikes, rel_err, run_oracle

pytestmark = pytest.mark.gpu
TOL = 1e-9


def _run(m, spec, overlap, epoch_steps=0, advance_every=None, chunked_events=False, **kw):
    import paper_1901_07454_b300 as arb
    sim = arb.Simulation(m, dt=spec.dt, epoch_steps=epoch_steps, epoch_overlap=overlap, **kw)
    E = sim.plan_info()["epoch_steps"]
    n = spec.n_steps
    step = advance_every or n
    order = np.argsort(spec.ev_t, kind="stable")
    k = 0
    if not chunked_events:
        sim.enqueue(spec.ev_syn, spec.ev_t, spec.ev_w)
    while k < n:
        k1 = min(n, k + step)
        if chunked_events:     # only the events of the coming interval, enqueued just before it
            sel = order[(spec.ev_t[order] >= k * spec.dt) & (spec.ev_t[order] < k1 * spec.dt)] if k else \
                order[spec.ev_t[order] < k1 * spec.dt]
            sim.enqueue(spec.ev_syn[sel], spec.ev_t[sel], spec.ev_w[sel])
        sim.advance(k1 * spec.dt)
        k = k1
    return dict(V=sim.voltage(), spikes=sim.spikes(), E=E, sim=sim)


def _same(a, b):
    assert np.array_equal(a["V"], b["V"])
    assert np.array_equal(a["spikes"][0], b["spikes"][0]) and np.array_equal(a["spikes"][1], b["spikes"][1])


def test_ring_overlapped_equals_serial_and_oracle():
    m, spec = make_config(1, n_cells=48, t_end=150.0)
    ovl = _run(m, spec, True)
    assert ovl["E"] == 100
    ser = _run(m, spec, False, epoch_steps=100)
    _same(ovl, ser)
    o = run_oracle(m, spec)
    compare_spikes(ovl["spikes"], o["spikes"])
    assert len(o["spikes"][1]) >= 27
    check_end(ovl["V"], o["V"])


def test_overlapped_across_uneven_advances_and_late_enqueues():
    # the batched workload's network at 256 cells (20-step overlapped epochs); advance calls of
    # 13 steps end inside epochs and the external events are enqueued interval by interval, so
    # the pipeline drains at every call and restarts from the pending pool
    m, spec = make_config(2, n_cells=256, t_end=40.0)
    a = _run(m, spec, True, advance_every=13, chunked_events=True)
    b = _run(m, spec, False, epoch_steps=20)
    _same(a, b)
    o = run_oracle(m, spec)
    compare_spikes(a["spikes"], o["spikes"])
    check_end(a["V"], o["V"])


@pytest.mark.parametrize("coalesce", [True, False])
def test_dense_overlapped_equals_serial_and_oracle(coalesce):
    # 128 cells x 1,000 synapses firing synchronously at 50 Hz; delays 10-20 ms, so 200-step
    # epochs overlapped against 200-step serial ones
    m, spec = make_config(5, n_cells=128, syn_per_cell=1000, t_end=60.0)
    ovl = _run(m, spec, True, coalesce_synapses=coalesce)
    assert ovl["E"] == 200
    ser = _run(m, spec, False, epoch_steps=200, coalesce_synapses=coalesce)
    _same(ovl, ser)
    o = run_oracle(m, spec)
    compare_spikes(ovl["spikes"], o["spikes"])
    check_end(ovl["V"], o["V"])
    assert len(o["spikes"][1]) == 3 * m.n_cells


@pytest.mark.parametrize("cells_per_pack", [32, 0])
def test_batched_overlapped_streamed_and_tiled(cells_per_pack):
    # the batched workload's random network (100 synapses per cell, delays 1-10 ms: 20-step
    # overlapped epochs) on the streamed kernel (one cell per lane) and the tile kernel
    m, spec = make_config(2, n_cells=256, t_end=40.0)
    ovl = _run(m, spec, True, cells_per_pack=cells_per_pack)
    assert ovl["E"] == 20
    ser = _run(m, spec, False, epoch_steps=20, cells_per_pack=cells_per_pack)
    _same(ovl, ser)
    o = run_oracle(m, spec)
    compare_spikes(ovl["spikes"], o["spikes"])
    check_end(ovl["V"], o["V"])
    assert len(o["spikes"][1]) > 0
