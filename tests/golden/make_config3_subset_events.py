"""Writes config3_subset_network_events.npz: the network events that the FP64 oracle delivers
to cells 0-1023 of the mixed-precision workload (65,536 cells, closed loop) during its first
100 ms. Calls only the oracle and the seeded input generators.

The open-loop comparison of the mixed-precision form drives those 1,024 cells with their own
external (Poisson) events, which the generator reproduces, plus these recorded network events,
each stored as (connection index, event time): its synapse and weight are the connection's.

    python tests/golden/make_config3_subset_events.py      # about 7 minutes on 8 host cores
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

T_END = 100.0
N_SUBSET = 1024
OUT = os.path.join(HERE, "config3_subset_network_events.npz")


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
    syn_cell = np.searchsorted(m.cv_offset, m.syn_cv, "right") - 1
    keep = (d["src"] >= 0) & (syn_cell[d["syn"]] < N_SUBSET)
    idx = d["idx"][keep].astype(np.int32)
    t = d["t"][keep]
    assert np.array_equal(m.conn_dst_syn[idx], d["syn"][keep]) and np.array_equal(m.conn_weight[idx], d["w"][keep])
    gid, _ = sim.spikes()
    np.savez_compressed(OUT, conn_idx=idx, t=t, t_end=T_END, n_subset=N_SUBSET, n_cells=m.n_cells,
                        network_spikes=gid.size)
    print("%d network events into cells 0-%d over %.0f ms (%d spikes in the network), %.0f s"
          % (idx.size, N_SUBSET - 1, T_END, gid.size, time.time() - t0))


if __name__ == "__main__":
    main()
