"""Dry run (Sec. "Scalability": one rank runs its own cells and mimics a large cluster by
generating proxy spikes for the cells of the other ranks) on the GPU against the oracle's dry
run, and against rank 0 of the full tiled network that it stands for.
"""
import dataclasses

import numpy as np
import pytest

from inputs import make_config
from parity_util import check_end, compare_spikes, rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-9


def _gpu(m, spec, **kw):
    import paper_1901_07454_b300 as arb
    sim = arb.Simulation(m, dt=spec.dt, epoch_steps=kw.pop("epoch_steps", spec.epoch_steps), **kw)
    sim.enqueue(spec.ev_syn, spec.ev_t, spec.ev_w)
    sim.advance(spec.t_end)
    return sim.voltage(), sim.spikes()


def _oracle(m, spec, R, **kw):
    import oracle
    o = oracle.simulate(m, spec, dry_run_ranks=R, **kw)[0]
    return o.voltage(), o.spikes()


@pytest.mark.parametrize("R,cells_per_pack", [(4, 0), (4, 32), (64, 32)])
def test_dry_run_matches_the_oracle(R, cells_per_pack):
    # 256 local cells of the batched workload as rank 0 of R ranks: 100 synapses per cell fed
    # from all R * 256 gids, so most events come from proxy spikes
    m, spec = make_config(2, n_cells=256, t_end=40.0, virtual_ranks=R)
    vg, sg = _gpu(m, spec, dry_run_ranks=R, cells_per_pack=cells_per_pack)
    vo, so = _oracle(m, spec, R)
    compare_spikes(sg, so)
    assert len(so[1]) > 100
    check_end(vg, vo)


def test_dry_run_is_rank_0_of_the_tiled_network():
    # the full network of 4 copies (1,024 cells) on the GPU: its copy 0 is what the dry run
    # stands for (equal to rounding: the copies are packed differently, which changes the
    # order in which a parent sums its children in the tree solve)
    R = 4
    m, spec = make_config(2, n_cells=256, t_end=40.0, virtual_ranks=R)
    full = m.tiled(R)
    fs = dataclasses.replace(spec, ev_syn=np.concatenate([spec.ev_syn + r * m.n_syn for r in range(R)]),
                             ev_t=np.tile(spec.ev_t, R), ev_w=np.tile(spec.ev_w, R))
    vd, sd = _gpu(m, spec, dry_run_ranks=R)
    vf, sf = _gpu(full, fs)
    check_end(vd, vf[:m.n_cv])
    for r in range(1, R):
        check_end(vf[r * m.n_cv:(r + 1) * m.n_cv], vf[:m.n_cv])
    sel = sf[0] < m.n_cells
    compare_spikes(sd, (sf[0][sel], sf[1][sel]))
    assert len(sf[1]) == R * len(sd[1])


def test_dry_run_with_overlapped_exchange_and_exact_events():
    R = 16
    m, spec = make_config(2, n_cells=256, t_end=40.0, virtual_ranks=R)
    vo, so = _oracle(m, spec, R)
    vg, sg = _gpu(m, spec, dry_run_ranks=R, epoch_overlap=True, epoch_steps=0)
    compare_spikes(sg, so)
    check_end(vg, vo)
    vo, so = _oracle(m, spec, R, exact_events=True)
    vg, sg = _gpu(m, spec, dry_run_ranks=R, exact_events=True, cells_per_pack=32)
    compare_spikes(sg, so)
    check_end(vg, vo)
