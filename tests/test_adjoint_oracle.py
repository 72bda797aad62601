"""Pins of the oracle's discrete adjoint (no GPU).

The adjoint is checked against central finite differences of the oracle's forward
simulation (the same step that tests/test_oracle_pins.py pins), parameter by parameter,
for per-branch gbar_na, gbar_k, g_leak and cm; its rate derivatives against a
high-precision derivative and against differences of the oracle's own rate functions.
"""
import numpy as np
import pytest

import oracle
from inputs import SimSpec, make_config


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def test_exprelr_derivative_against_high_precision():
    import mpmath
    mpmath.mp.dps = 50
    f = lambda x: x / (mpmath.exp(x) - 1)
    for x in (-8.0, -2.5, -0.3, -0.1 - 1e-12, -0.1 + 1e-12, -2e-3, -1e-5, 0.0, 3e-7, 1.01e-3, 0.07, 0.0999, 0.1001, 1.5, 9.0):
        ref = mpmath.mpf(-0.5) if x == 0.0 else mpmath.diff(f, mpmath.mpf(x))
        got = oracle.exprelr_deriv(x)
        assert abs(got - float(ref)) <= 2e-14 * max(1.0, abs(float(ref))), (x, got, float(ref))


def test_rate_derivatives_against_differences_of_the_rates():
    h = 1e-3
    for v in np.linspace(-100.0, 40.0, 57):
        d = oracle.hh_rate_derivs(v)
        # fourth-order central difference of the oracle's own rates
        fd = (-oracle.hh_rates(v + 2 * h) + 8 * oracle.hh_rates(v + h) - 8 * oracle.hh_rates(v - h)
              + oracle.hh_rates(v - 2 * h)) / (12 * h)
        assert np.all(np.abs(d - fd) <= 1e-9 * np.maximum(np.abs(fd), 1e-3)), (v, d, fd)


def _small_case():
    # two config-4 cells (24 branches, HH everywhere, per-branch densities), clamp from 1 ms
    m, _ = make_config(4, n_cells=2, t_end=5.0)
    m.stim_t_on = np.full(m.stim_cv.size, 1.0)
    m.__post_init__()
    tgt, _ = make_config(4, n_cells=2, t_end=5.0, variant="target")
    tgt.stim_t_on = np.full(tgt.stim_cv.size, 1.0)
    tgt.__post_init__()
    spec = SimSpec(dt=0.025, t_end=5.0, epoch_steps=400)
    obs = m.cv_offset[:-1].copy()
    _, target = oracle.simulate(tgt, spec, probes=obs)
    return m, spec, obs, target


def _loss(model, spec, obs, target):
    _, tr = oracle.simulate(model, spec, probes=obs)
    return float(np.sum((tr - target) ** 2)) / (target.shape[0] * obs.size)


def test_adjoint_against_central_differences():
    m, spec, obs, target = _small_case()
    K = spec.n_steps
    scale = 1.0 / (K * obs.size)
    group, ng = m.param_groups()
    sim = oracle.OracleSim(m, spec.dt, spec.epoch_steps)
    loss, grad = sim.adjoint(K, obs, target, scale, group, ng)
    assert abs(loss - _loss(m, spec, obs, target)) <= 1e-12 * loss
    assert sim.steps == 0                       # the adjoint leaves the simulation untouched
    theta = m.group_params()
    fd = np.zeros_like(grad)
    for gi in range(ng):
        for p in range(4):
            h = 1e-6 * abs(theta[gi, p])
            tp, tm = theta.copy(), theta.copy()
            tp[gi, p] += h
            tm[gi, p] -= h
            fd[gi, p] = (_loss(m.with_group_params(tp), spec, obs, target)
                         - _loss(m.with_group_params(tm), spec, obs, target)) / (2 * h)
    for p in range(4):
        err = np.abs(grad[:, p] - fd[:, p])
        bar = 1e-4 * np.abs(fd[:, p]) + 1e-7 * np.max(np.abs(fd[:, p]))
        assert np.all(err <= bar), (m.PARAM_NAMES[p], float(np.max(err / np.maximum(bar, 1e-300))))
    assert np.all(np.abs(fd).max(axis=0) > 0)


def test_adjoint_is_linear_in_the_loss_scale_and_zero_on_target():
    m, spec, obs, target = _small_case()
    K = spec.n_steps
    group, ng = m.param_groups()
    sim = oracle.OracleSim(m, spec.dt, spec.epoch_steps)
    l1, g1 = sim.adjoint(K, obs, target, 1.0, group, ng)
    l2, g2 = sim.adjoint(K, obs, target, 0.5, group, ng)
    assert abs(l2 - 0.5 * l1) <= 1e-14 * l1 and np.allclose(g2, 0.5 * g1, rtol=1e-14, atol=0)
    # at the target's own parameters the loss and every gradient vanish
    _, own = oracle.simulate(m, spec, probes=obs)
    l0, g0 = sim.adjoint(K, obs, own, 1.0, group, ng)
    assert l0 == 0.0 and np.all(g0 == 0.0)
