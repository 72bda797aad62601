"""Exact event times (steps cut at the events inside them, Sec. "Model") on the GPU against the
oracle's exact mode (needs a B300). Same bars as the fixed-step parity tests."""
import math

import numpy as np
import pytest

from inputs import Model, SimSpec, make_config, small_tree_model
from parity_util import check_end, check_trace, compare_spikes, oracle_spread, rel_err, run_gpu, run_oracle, submodel, trace_bar

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


def test_single_synapse_events_inside_steps():
    n = 1
    m = Model(cv_offset=np.array([0, 1]), parent=np.array([-1], np.int32), length_um=np.array([20.0]),
              radius_um=np.array([5.0]), cm=np.array([1.0]), Ra=np.array([100.0]), branch_of_cv=np.zeros(1, np.int32),
              hh_cv=np.zeros(0, np.int64), gnabar=np.zeros(0), gkbar=np.zeros(0), gl=np.zeros(0),
              pas_cv=np.array([0]), g_pas=np.array([1e-4]), e_pas=np.array([-65.0]),
              syn_cv=np.array([0]), syn_tau=np.array([2.0]), syn_e=np.array([0.0]),
              detector_cv=np.array([0]))
    te = np.array([1.2345, 1.2405, 3.0, 7.00001])
    spec = SimSpec(dt=0.025, t_end=10.0, epoch_steps=400, ev_syn=np.zeros(te.size, np.int64), ev_t=te,
                   ev_w=np.full(te.size, 0.004))
    g = run_gpu(m, spec, probes=[0], exact_events=True)
    o = run_oracle(m, spec, probes=[0], exact=True)
    assert rel_err(g["trace"], o["trace"]) <= 1e-12
    f = run_oracle(m, spec, probes=[0])                      # fixed-step rule differs
    assert rel_err(f["trace"], o["trace"]) > 1e-6


def _trees():
    m = small_tree_model(11, n_cells=37, n_branches=9, cv_range=(1, 12), n_syn=4)
    m.stim_cv = m.cv_offset[:-1:3].copy()
    k = m.stim_cv.size
    m.stim_t_on, m.stim_dur, m.stim_amp = np.full(k, 2.0), np.full(k, 10.0), np.linspace(0.05, 1.0, k)
    m.__post_init__()
    rng = np.random.default_rng(3)
    nev = rng.poisson(40.0 * 1e-3 * 30.0 * m.n_syn)
    syn = rng.integers(0, m.n_syn, nev)
    t = rng.uniform(0, 30.0, nev)
    return m, SimSpec(dt=0.025, t_end=30.0, epoch_steps=40, ev_syn=syn, ev_t=t, ev_w=np.full(nev, 0.02))


def test_random_trees_every_cv_every_step():
    m, spec = _trees()
    probes = np.arange(m.n_cv)
    g = run_gpu(m, spec, probes=probes, exact_events=True)
    o = run_oracle(m, spec, probes=probes, exact=True)
    check_end(g["V"], o["V"])
    check_trace(g["trace"], o["trace"], oracle_spread(m, spec, probes, exact=True))
    compare_spikes(g["spikes"], o["spikes"])
    assert len(o["spikes"][1]) > 0
    assert g["sim"].plan_info()["cells_per_pack"] == 32 and g["sim"].plan_info()["split_cvs"] == -1


def test_network_closed_loop_exact_spike_times():
    # the batched network at 384 cells: spikes become events at exact times t_spike + delay
    m, spec = make_config(2, n_cells=384, t_end=30.0)
    probes = m.detector_cv
    g = run_gpu(m, spec, probes=probes, exact_events=True)
    o = run_oracle(m, spec, probes=probes, exact=True)
    compare_spikes(g["spikes"], o["spikes"])
    check_end(g["V"], o["V"])
    check_trace(g["trace"], o["trace"], oracle_spread(m, spec, probes, exact=True))
    assert len(o["spikes"][1]) > 0


def test_full_size_sampled_cells():
    # 65,536 cells with exact event times in the benchmark's configuration, first millisecond
    m, spec = make_config(2, t_end=1.0)
    g = run_gpu(m, spec, exact_events=True)
    rng = np.random.default_rng(0)
    cells = np.unique(np.concatenate([rng.choice(m.n_cells, 48, replace=False), np.argsort(np.diff(m.cv_offset))[-4:]]))
    sm, ss, cv_old = submodel(m, spec, cells)
    o = run_oracle(sm, ss, exact=True)
    check_end(g["V"][cv_old], o["V"])
