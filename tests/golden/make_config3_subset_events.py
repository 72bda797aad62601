"""Writes config3_subset_network_events.npz: the network events that the FP64 oracle delivers
to cells 0-1023 of the mixed-precision workload (65,536 cells, closed loop) during its first
100 ms. Calls only the oracle and the seeded input generators.

The open-loop comparison of the mixed-precision form drives those 1,024 cells with their own
external (Poisson) events, which the generator reproduces, plus these recorded network events.
With step-start events an event acts at the start of step ceil(t/dt) whatever its time inside
the step, so an event is stored as (connection, step): its synapse and weight are the
connection's, and it is replayed at t = (step - 1/2) dt. The connections into cells 0-1023 are
the first 102,400 of the workload; the file holds, per connection, its number of events (counts)
and their steps in increasing order as differences (dstep: the first step, then the gaps).

    python tests/golden/make_config3_subset_events.py      # about 7 minutes on 8 host cores
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, os.path.dirname(ROOT))

T_END = 100.0
N_SUBSET = 1024
OUT = os.path.join(HERE, "config3_subset_network_events.npz")


def subset_connections(m, n_subset=N_SUBSET):
    """Indices of the connections whose target synapse lies on cells 0 .. n_subset-1."""
    syn_cell = np.searchsorted(m.cv_offset, m.syn_cv, "right") - 1
    return np.nonzero(syn_cell[m.conn_dst_syn] < n_subset)[0]


def main():
    import oracle
    from inputs import make_config
    oracle.build()
    t0 = time.time()
    m, spec = make_config(3, t_end=T_END)
    sim = oracle.OracleSim(m, spec.dt, spec.epoch_steps, record_delivered=True)
    sim.enqueue(spec.ev_syn, spec.ev_t, spec.ev_w)
    sim.run_steps(spec.n_steps)
    d = sim.delivered()
    conn = subset_connections(m)
    keep = d["src"] >= 0
    keep[keep] = np.isin(d["idx"][keep], conn)
    idx, step = d["idx"][keep], d["step"][keep]
    assert np.array_equal(m.conn_dst_syn[idx], d["syn"][keep]) and np.array_equal(m.conn_weight[idx], d["w"][keep])
    o = np.lexsort((step, idx))
    idx, step = idx[o], step[o]
    pos = np.searchsorted(conn, idx)
    counts = np.bincount(pos, minlength=conn.size)
    first = np.r_[True, pos[1:] != pos[:-1]]
    dstep = np.where(first, step, np.r_[0, np.diff(step)])
    assert counts.max() < 256 and dstep.max() < 65536
    gid, _ = sim.spikes()
    np.savez_compressed(OUT, counts=counts.astype(np.uint8), dstep=dstep.astype(np.uint16), t_end=T_END,
                        dt=spec.dt, n_subset=N_SUBSET, n_connections=conn.size, network_spikes=gid.size)
    print("%d network events into cells 0-%d over %.0f ms (%d spikes in the network), %.0f s"
          % (idx.size, N_SUBSET - 1, T_END, gid.size, time.time() - t0))


if __name__ == "__main__":
    main()
