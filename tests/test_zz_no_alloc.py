"""The allocation-free tree solve (arb_solve_trees_noalloc), checked against the oracle's solve
of the same host-assembled system and against the library's ordinary time step.

Callers that cannot allocate device memory where they need a solve (for example while a
stream is being captured into a CUDA graph, or with a device memory pool fixed up front) use
this entry point: it takes only their device arrays and keeps its scratch in a fixed array
inside the library. This test calls it through the C ABI twice in a row and compares each
result with the oracle's elimination of the system assembled here on the host, and with the
voltage that arb_advance (the existing entry point) computes for the same implicit Euler
step. It also checks the two ways a call can be malformed on the device: a cell whose parent
indices break the ordering rule (NaN over that cell only) and a cv_offset that is not a CSR
(NaN everywhere). This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from inputs import small_tree_model

pytestmark = pytest.mark.gpu
TOL = 1e-9


def _rel(x, y):
    return float(np.max(np.abs(x - y) / np.maximum(np.abs(y), 1.0)))


def _assemble(m, dt, oracle):
    """Diagonal, off-diagonal and the constant part of the right-hand side of one implicit
    step of passive cells, built here from the oracle's geometry."""
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
    return cap / dt, d, a, GE + inj


def _oracle_solve(m, d, a, b, oracle):
    x = np.zeros(m.n_cv)
    for c in range(m.n_cells):
        lo, hi = m.cv_offset[c], m.cv_offset[c + 1]
        x[lo:hi] = oracle.hines_solve(m.parent[lo:hi], d[lo:hi], a[lo:hi], b[lo:hi])
    return x


def test_noalloc_solve_matches_the_oracle_and_the_implicit_step_twice():
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
    cdt, d, a, b0 = _assemble(m, dt, oracle)

    dev = torch.device("cuda", torch.cuda.current_device())
    t_off = torch.from_numpy(m.cv_offset.astype(np.int64)).to(dev)
    t_par = torch.from_numpy(m.parent.astype(np.int32)).to(dev)
    t_d = torch.from_numpy(d).to(dev)
    t_a = torch.from_numpy(a).to(dev)
    x = torch.empty(m.n_cv, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def call(off, par, t_b):
        x.fill_(0.0)
        rc = lib.arb_solve_trees_noalloc(m.n_cells, m.n_cv, C.c_void_p(off.data_ptr()), C.c_void_p(par.data_ptr()),
                                         C.c_void_p(t_d.data_ptr()), C.c_void_p(t_a.data_ptr()),
                                         C.c_void_p(t_b.data_ptr()), C.c_void_p(x.data_ptr()),
                                         C.c_void_p(stream.cuda_stream))
        assert rc == 0, lib.arb_last_error(None)
        torch.cuda.synchronize()
        return x.cpu().numpy()

    V = st["V"].copy()
    for step in range(2):
        b = cdt * V + b0
        got = call(t_off, t_par, torch.from_numpy(b).to(dev))
        want = _oracle_solve(m, d, a, b, oracle)
        e_orc = _rel(got, want)
        sim.advance((step + 1) * dt)             # the existing entry point, one step
        V = sim.voltage()
        e_step = _rel(got, V)
        print("call %d: max rel err %.2e vs the oracle's solve, %.2e vs arb_advance" % (step, e_orc, e_step))
        assert e_orc <= TOL and e_step <= TOL, (step, e_orc, e_step)

    # a cell whose parents break the ordering rule gets NaN over its own CVs only
    b = cdt * V + b0
    want = _oracle_solve(m, d, a, b, oracle)
    t_b = torch.from_numpy(b).to(dev)
    bad_cell = 5
    lo, hi = int(m.cv_offset[bad_cell]), int(m.cv_offset[bad_cell + 1])
    assert hi - lo >= 2
    par_bad = m.parent.astype(np.int32).copy()
    par_bad[lo + 1] = 1                          # its own index: not below it
    got = call(t_off, torch.from_numpy(par_bad).to(dev), t_b)
    assert np.all(np.isnan(got[lo:hi]))
    keep = np.ones(m.n_cv, bool)
    keep[lo:hi] = False
    assert _rel(got[keep], want[keep]) <= TOL

    # an offset array that is not a CSR (a decreasing entry) makes every x NaN
    off_bad = m.cv_offset.astype(np.int64).copy()
    off_bad[7] = off_bad[9]
    got = call(torch.from_numpy(off_bad).to(dev), t_par, t_b)
    assert np.all(np.isnan(got))
    # ... and the next well-formed call is unaffected by it
    got = call(t_off, t_par, t_b)
    assert _rel(got, want) <= TOL

    # sizes beyond the fixed scratch are refused before any launch
    rc = lib.arb_solve_trees_noalloc(1, 262145, C.c_void_p(t_off.data_ptr()), C.c_void_p(t_par.data_ptr()),
                                     C.c_void_p(t_d.data_ptr()), C.c_void_p(t_a.data_ptr()), C.c_void_p(t_d.data_ptr()),
                                     C.c_void_p(x.data_ptr()), None)
    assert rc == -1 and b"exceed" in lib.arb_last_error(None)
