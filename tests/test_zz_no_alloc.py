"""The allocation-free tree solve (arb_solve_trees_noalloc), checked against the library's
ordinary time step.

Callers that cannot allocate device memory where they need a solve (for example while a
stream is being captured into a CUDA graph, or with a device memory pool fixed up front) use
this entry point: it takes only their device arrays and keeps its scratch in a fixed array
inside the library. This test calls it through the C ABI twice in a row and compares each
result with the voltage that arb_advance (the existing entry point) computes for the same
implicit Euler system. This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from inputs import small_tree_model

pytestmark = pytest.mark.gpu
TOL = 1e-9


def _rel(x, y):
    return float(np.max(np.abs(x - y) / np.maximum(np.abs(y), 1.0)))


def test_noalloc_solve_matches_the_implicit_step_twice():
    import torch

    import oracle
    import paper_1901_07454_b300 as arb
    from paper_1901_07454_b300 import _build
    _build.build()
    assert torch.cuda.is_available()
    lib = arb.load()

    # passive random trees with clamps: one implicit step is exactly one tree solve
    m = small_tree_model(21, n_cells=40, n_branches=9, cv_range=(1, 14), passive_only=True)
    rng = np.random.default_rng(4)
    m.stim_cv = m.cv_offset[:-1:2].copy()
    k = m.stim_cv.size
    m.stim_t_on, m.stim_dur, m.stim_amp = np.zeros(k), np.full(k, 1e9), rng.uniform(-0.5, 0.5, k)
    m.__post_init__()
    dt = 0.025
    sim = arb.Simulation(m, dt=dt, epoch_steps=10)
    st = sim.get_state()
    st["V"] = rng.uniform(-80.0, -40.0, m.n_cv)
    sim.set_state(st)

    # the same system, assembled on the host
    area, cap, sigma = oracle.cv_geometry(m)
    G = np.zeros(m.n_cv)
    GE = np.zeros(m.n_cv)
    np.add.at(G, m.pas_cv, m.g_pas * area[m.pas_cv] * 1e-2)
    np.add.at(GE, m.pas_cv, m.g_pas * area[m.pas_cv] * 1e-2 * m.e_pas)
    inj = np.zeros(m.n_cv)
    np.add.at(inj, m.stim_cv, m.stim_amp)
    cell = np.repeat(np.arange(m.n_cells), np.diff(m.cv_offset))
    d = cap / dt + G
    a = np.zeros(m.n_cv)
    for i in range(m.n_cv):
        pl = m.parent[i]
        if pl >= 0:
            p = m.cv_offset[cell[i]] + pl
            d[i] += sigma[i]
            d[p] += sigma[i]
            a[i] = -sigma[i]

    dev = torch.device("cuda", torch.cuda.current_device())
    t_off = torch.from_numpy(m.cv_offset.astype(np.int64)).to(dev)
    t_par = torch.from_numpy(m.parent.astype(np.int32)).to(dev)
    t_d = torch.from_numpy(d).to(dev)
    t_a = torch.from_numpy(a).to(dev)
    x = torch.empty(m.n_cv, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    V = st["V"].copy()
    for call in range(2):
        b = cap / dt * V + GE + inj
        t_b = torch.from_numpy(b).to(dev)
        x.fill_(float("nan"))
        rc = lib.arb_solve_trees_noalloc(m.n_cells, m.n_cv, C.c_void_p(t_off.data_ptr()), C.c_void_p(t_par.data_ptr()),
                                         C.c_void_p(t_d.data_ptr()), C.c_void_p(t_a.data_ptr()),
                                         C.c_void_p(t_b.data_ptr()), C.c_void_p(x.data_ptr()),
                                         C.c_void_p(stream.cuda_stream))
        assert rc == 0, lib.arb_last_error(None)
        torch.cuda.synchronize()
        sim.advance((call + 1) * dt)             # the existing entry point, one step
        V = sim.voltage()
        assert _rel(x.cpu().numpy(), V) <= TOL, (call, _rel(x.cpu().numpy(), V))

    # sizes beyond the fixed scratch are refused before any launch
    rc = lib.arb_solve_trees_noalloc(1, 262145, C.c_void_p(t_off.data_ptr()), C.c_void_p(t_par.data_ptr()),
                                     C.c_void_p(t_d.data_ptr()), C.c_void_p(t_a.data_ptr()), C.c_void_p(t_d.data_ptr()),
                                     C.c_void_p(x.data_ptr()), None)
    assert rc == -1 and b"exceed" in lib.arb_last_error(None)
