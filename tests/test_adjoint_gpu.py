"""GPU discrete adjoint (arb_adjoint) against the oracle's adjoint and against central
differences of the GPU forward step (needs a B300).

Bar: loss within 1e-10 and gradients within 1e-8 (relative to each parameter kind's largest
component) of the FP64 oracle adjoint; within 1e-4 of central differences.
"""
import numpy as np
import pytest

import oracle
from inputs import SimSpec, make_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1901_07454_b300 import _build
    _build.build()
    oracle.build()


def _case(n_cells=2, t_end=5.0, t_on=1.0):
    m, _ = make_config(4, n_cells=n_cells, t_end=t_end)
    m.stim_t_on = np.full(m.stim_cv.size, t_on)
    m.__post_init__()
    tgt, _ = make_config(4, n_cells=n_cells, t_end=t_end, variant="target")
    tgt.stim_t_on = np.full(tgt.stim_cv.size, t_on)
    tgt.__post_init__()
    spec = SimSpec(dt=0.025, t_end=t_end, epoch_steps=400)
    obs = m.cv_offset[:-1].copy()
    _, target = oracle.simulate(tgt, spec, probes=obs)
    return m, spec, obs, target


def _close(g, o, rel=1e-8):
    for p in range(4):
        err = np.max(np.abs(g[:, p] - o[:, p]))
        assert err <= rel * np.max(np.abs(o[:, p])), (p, err, np.max(np.abs(o[:, p])))


def test_adjoint_matches_oracle_for_every_checkpoint_spacing():
    import paper_1901_07454_b300 as arb
    m, spec, obs, target = _case()
    K = spec.n_steps
    scale = 1.0 / (K * obs.size)
    group, ng = m.param_groups()
    lo, go = oracle.OracleSim(m, spec.dt, spec.epoch_steps).adjoint(K, obs, target, scale, group, ng)
    sim = arb.Simulation(m, dt=spec.dt, epoch_steps=spec.epoch_steps)
    ref = None
    for ck in (64, 1, 7, 200, 500):          # ragged last segment, one step, one segment, longer than the run
        lg, gg = sim.adjoint(K, obs, target, scale, group, ng, checkpoint_every=ck)
        gg = gg.cpu().numpy()
        assert abs(lg - lo) <= 1e-10 * lo, (ck, lg, lo)
        _close(gg, go)
        if ref is None:
            ref = (lg, gg)
        else:                                # recomputation from checkpoints is exact
            assert lg == ref[0] and np.array_equal(gg, ref[1]), ck
    # the handle is unchanged: advancing it reproduces the adjoint's own forward loss
    tr = sim.set_probes(obs, K)
    sim.advance(spec.t_end)
    l_fwd = float(np.sum((tr.cpu().numpy() - target) ** 2)) * scale
    assert abs(l_fwd - lo) <= 1e-10 * lo


def test_adjoint_matches_central_differences_of_the_gpu_forward():
    import paper_1901_07454_b300 as arb
    m, spec, obs, target = _case()
    K = spec.n_steps
    scale = 1.0 / (K * obs.size)
    group, ng = m.param_groups()
    theta = m.group_params()
    _, g = arb.Simulation(m, dt=spec.dt).adjoint(K, obs, target, scale, group, ng, checkpoint_every=50)
    g = g.cpu().numpy()

    def loss(th):
        s = arb.Simulation(arb.spread_params(m, group, th), dt=spec.dt, epoch_steps=spec.epoch_steps)
        tr = s.set_probes(obs, K)
        s.advance(spec.t_end)
        return float(np.sum((tr.cpu().numpy() - target) ** 2)) * scale

    rng = np.random.default_rng(5)
    for gi, p in zip(rng.choice(ng, 10, replace=False), [0, 1, 2, 3, 0, 1, 2, 3, 3, 0]):
        h = 1e-6 * abs(theta[gi, p])
        tp, tm = theta.copy(), theta.copy()
        tp[gi, p] += h
        tm[gi, p] -= h
        fd = (loss(tp) - loss(tm)) / (2 * h)
        assert abs(g[gi, p] - fd) <= 1e-4 * abs(fd) + 1e-7 * np.max(np.abs(g[:, p])), (gi, p, g[gi, p], fd)


def test_autograd_function_and_a_descent_step():
    import torch
    import paper_1901_07454_b300 as arb
    m, spec, obs, target = _case()
    K = spec.n_steps
    scale = 1.0 / (K * obs.size)
    group, ng = m.param_groups()
    theta = torch.tensor(m.group_params(), dtype=torch.float64, requires_grad=True)
    L = arb.adjoint_loss(theta, m, group, obs, target, scale, K, spec.dt, 100)
    L.backward()
    _, g = arb.Simulation(m, dt=spec.dt).adjoint(K, obs, target, scale, group, ng, checkpoint_every=100)
    assert np.array_equal(theta.grad.numpy(), g.cpu().numpy())
    # a small step against the gradient lowers the loss
    with torch.no_grad():
        step = 1e-3 * theta.abs() * torch.sign(theta.grad)
        L2 = arb.adjoint_loss(theta - step, m, group, obs, target, scale, K, spec.dt, 100)
    assert float(L2.detach()) < float(L.detach())


def test_adjoint_full_size_sampled_cells():
    # 256 cells x ~300 CVs x 8,000 steps with a checkpoint every 500 steps; each cell's
    # gradient depends on that cell alone, so sampled cells are checked with the oracle
    import paper_1901_07454_b300 as arb
    from inputs.sample import submodel
    m, spec = make_config(4)
    tgt, _ = make_config(4, variant="target")
    K = spec.n_steps
    obs = m.cv_offset[:-1].copy()
    _, target = oracle.simulate(tgt, spec, probes=obs)     # the hidden parameters' soma traces
    scale = 1.0 / (K * obs.size)
    group, ng = m.param_groups()
    sim = arb.Simulation(m, dt=spec.dt, epoch_steps=spec.epoch_steps)
    loss, g = sim.adjoint(K, obs, target, scale, group, ng, checkpoint_every=500)
    g = g.cpu().numpy()
    assert np.isfinite(loss) and loss > 0
    cells = np.array([0, 101, 255])
    sm, ss, cv_old = submodel(m, spec, cells)
    sg, sng = sm.param_groups()
    nb = ng // m.n_cells
    so = sm.cv_offset[:-1].copy()
    lo, go = oracle.OracleSim(sm, spec.dt, spec.epoch_steps).adjoint(K, so, target[:, cells], scale, sg, sng)
    gg = g.reshape(m.n_cells, nb, 4)[cells].reshape(-1, 4)
    _close(gg, go, rel=1e-7)


def test_adjoint_refuses_synapses_and_the_explicit_scheme():
    import paper_1901_07454_b300 as arb
    m, spec, obs, target = _case()
    group, ng = m.param_groups()
    with pytest.raises(arb.ArbError):
        arb.Simulation(m, dt=spec.dt, scheme="explicit").adjoint(10, obs, target[:10], 1.0, group, ng)
    m2, _ = make_config(0)
    with pytest.raises(arb.ArbError) as ei:
        g2, n2 = m2.param_groups()
        arb.Simulation(m2, dt=0.025).adjoint(10, m2.cv_offset[:-1], np.zeros((10, m2.n_cells)), 1.0, g2, n2)
    assert "synapses" in str(ei.value)


def test_adjoint_ragged_trees_passive_dendrites_partial_groups():
    # HH soma and passive dendrites on ragged random trees (3 to 55 CVs per cell), a clamp,
    # observations on the soma and one dendritic CV, and CVs left out of every group
    import paper_1901_07454_b300 as arb
    from inputs import small_tree_model
    m = small_tree_model(8, n_cells=6, n_branches=7, cv_range=(1, 12), n_syn=0)
    m.stim_cv = m.cv_offset[:-1].copy()
    k = m.stim_cv.size
    m.stim_t_on, m.stim_dur, m.stim_amp = np.full(k, 0.5), np.full(k, 1e9), np.linspace(0.05, 0.6, k)
    m.__post_init__()
    spec = SimSpec(dt=0.025, t_end=6.0, epoch_steps=400)
    K = spec.n_steps
    obs = np.concatenate([m.cv_offset[:-1], m.cv_offset[1:] - 1])
    obs = np.unique(obs)
    rng = np.random.default_rng(3)
    target = -65.0 + 20.0 * rng.random((K, obs.size))
    group, ng = m.param_groups()
    group = group.copy()
    group[rng.random(group.size) < 0.2] = -1
    lo, go = oracle.OracleSim(m, spec.dt, 400).adjoint(K, obs, target, 1.0 / K, group, ng)
    sim = arb.Simulation(m, dt=spec.dt)
    lg, gg = sim.adjoint(K, obs, target, 1.0 / K, group, ng, checkpoint_every=37)
    assert abs(lg - lo) <= 1e-10 * lo
    gg = gg.cpu().numpy()
    for p in range(4):
        scale = max(np.max(np.abs(go[:, p])), 1e-300)
        assert np.max(np.abs(gg[:, p] - go[:, p])) <= 1e-8 * scale, p
    # no observations: zero loss, zero gradient
    l0, g0 = sim.adjoint(10, np.zeros(0, np.int64), np.zeros((10, 0)), 1.0, group, ng)
    assert l0 == 0.0 and not np.any(g0.cpu().numpy())


def test_adjoint_long_cable_cut_into_several_chains():
    # One unbranched 900-CV cable: along a chain the scaled pivots of the tree solve grow by
    # about a factor 2 per CV here, so the host cuts the cable into four chains (about every
    # 280-300 CVs) to keep them inside 2^{+-300}; each cut part hands its elimination to the
    # next like a child chain. HH on the first 100 CVs, a current pulse at the root,
    # observations along the cable, nine parameter groups of 100 CVs.
    import paper_1901_07454_b300 as arb
    from inputs.configs import uniform_cable_model
    m = uniform_cable_model(900, 4500.0, 1.0)
    m.hh_cv = np.arange(100)
    m.gnabar, m.gkbar, m.gl = np.full(100, 0.12), np.full(100, 0.036), np.full(100, 3e-4)
    m.pas_cv = np.arange(100, 900)
    m.g_pas, m.e_pas = np.full(800, 1e-4), np.full(800, -65.0)
    m.stim_cv = np.array([0])
    m.stim_t_on, m.stim_dur, m.stim_amp = np.array([1.0]), np.array([2.0]), np.array([1.5])
    m.branch_of_cv = (np.arange(900) // 100).astype(np.int32)
    m.__post_init__()
    spec = SimSpec(dt=0.025, t_end=12.0, epoch_steps=400)
    K = spec.n_steps
    obs = np.array([0, 50, 300, 600, 899])
    rng = np.random.default_rng(11)
    target = -65.0 + 30.0 * rng.random((K, obs.size))
    group, ng = m.param_groups()
    assert ng == 9
    lo, go = oracle.OracleSim(m, spec.dt, 400).adjoint(K, obs, target, 1.0 / K, group, ng)
    sim = arb.Simulation(m, dt=spec.dt)
    lg, gg = sim.adjoint(K, obs, target, 1.0 / K, group, ng, checkpoint_every=64)
    gg = gg.cpu().numpy()
    errs = [float(np.max(np.abs(gg[:, p] - go[:, p])) / max(np.max(np.abs(go[:, p])), 1e-300)) for p in range(4)]
    print("long cable: loss rel err %.2e, gradient rel errs %s" % (abs(lg - lo) / lo, ["%.1e" % e for e in errs]))
    assert abs(lg - lo) <= 1e-10 * lo, (lg, lo)
    # the passive groups have no HH: their gna/gk/gl gradients are zero on both sides
    assert np.all(gg[1:, :3] == 0.0) and np.all(go[1:, :3] == 0.0)
    for p in range(4):
        assert errs[p] <= 1e-8, (p, errs[p])
