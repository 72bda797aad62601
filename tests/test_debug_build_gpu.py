"""The debug build (libarb_b300_debug.so: ARB_DEBUG) on the small parity cases: every index the
kernels read from an index array is range-checked on the device and every workspace region is
followed by guard words. The runs must end with a clean status, intact guard words and the
oracle's results; a guard word changed from the host and an out-of-range detector slot written
into the workspace must both be reported (the debug check replaces the bad index by 0 before it
is used, so nothing is read out of bounds)."""
import numpy as np
import pytest

from inputs import SimSpec, make_config, small_tree_model
from parity_util import check_end, compare_spikes, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1901_07454_b300 import _build
    _build.build(debug=True)
    import paper_1901_07454_b300 as arb
    assert arb.load(debug=True).arb_debug_build() == 1 and arb.load().arb_debug_build() == 0


def _run_debug(m, spec, **kw):
    import paper_1901_07454_b300 as arb
    sim = arb.Simulation(m, dt=spec.dt, epoch_steps=spec.epoch_steps, debug=True, **kw)
    sim.enqueue(spec.ev_syn, spec.ev_t, spec.ev_w)
    sim.advance(spec.n_steps * spec.dt)          # raises on a debug-check flag or a broken guard word
    sim.check_canaries()
    return sim


def _trees():
    m = small_tree_model(11, n_cells=37, n_branches=9, cv_range=(1, 12), n_syn=4)
    m.stim_cv = m.cv_offset[:-1:3].copy()
    k = m.stim_cv.size
    m.stim_t_on, m.stim_dur, m.stim_amp = np.full(k, 2.0), np.full(k, 10.0), np.linspace(0.05, 1.0, k)
    m.__post_init__()
    rng = np.random.default_rng(3)
    n = rng.poisson(40.0 * 1e-3 * 30.0 * m.n_syn)
    syn = rng.integers(0, m.n_syn, n)
    t = rng.uniform(0, 30.0, syn.size)
    return m, SimSpec(dt=0.025, t_end=30.0, epoch_steps=40, ev_syn=syn, ev_t=t, ev_w=np.full(syn.size, 0.02))


@pytest.mark.parametrize("kw", [dict(cells_per_pack=32, split_cvs=-1), dict(cells_per_pack=32, split_cvs=40),
                                dict(cells_per_pack=8), dict(cells_per_pack=32, split_cvs=40, precision="mixed"),
                                dict(cells_per_pack=32, split_cvs=-1, scheme="explicit")])
def test_debug_build_random_trees_clean(kw):
    m, spec = _trees()
    sim = _run_debug(m, spec, **kw)
    o = run_oracle(m, spec, scheme=kw.get("scheme", "implicit"))
    if kw.get("precision") == "mixed":
        assert np.max(np.abs(sim.voltage() - o["V"])) <= 1e-3
    else:
        check_end(sim.voltage(), o["V"])
        compare_spikes(sim.spikes(), o["spikes"])


def test_debug_build_ring_closed_loop_clean():
    m, spec = make_config(1, n_cells=48, t_end=60.0)
    sim = _run_debug(m, spec)
    o = run_oracle(m, spec)
    check_end(sim.voltage(), o["V"])
    compare_spikes(sim.spikes(), o["spikes"])


def test_debug_build_reports_a_broken_guard_word_and_a_bad_index():
    import torch
    import paper_1901_07454_b300 as arb
    m, spec = _trees()
    sim = _run_debug(m, SimSpec(dt=spec.dt, t_end=1.0, epoch_steps=40, ev_syn=spec.ev_syn, ev_t=spec.ev_t, ev_w=spec.ev_w),
                     cells_per_pack=32, split_cvs=-1)
    # a byte of the guard words after "V", changed from the host
    off, nb = sim.workspace_region("V")
    guard = ((off + nb + 255) // 256) * 256
    ws = sim._ws[sim._ws_shift:]
    saved = ws[guard].item()
    ws[guard] = (saved + 1) % 256
    torch.cuda.synchronize()
    with pytest.raises(arb.ArbError) as ei:
        sim.check_canaries()
    assert "'V'" in str(ei.value)
    ws[guard] = saved
    torch.cuda.synchronize()
    sim.check_canaries()
    # an out-of-range detector slot: reported after the next epoch, read as slot 0
    off, nb = sim.workspace_region("det_slot")
    slots = ws[off:off + nb].view(torch.int32)
    slots[0] = 1 << 30
    torch.cuda.synchronize()
    with pytest.raises(arb.ArbError) as ei:
        sim.advance(2.0)
    assert "debug check" in str(ei.value)
