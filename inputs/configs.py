"""Seeded generators for the five benchmark workloads and for small test morphologies.

Morphologies are random trees of unbranched cables ("branches"). Branch 0 is the root
(the soma); each further branch attaches to the distal end of a uniformly chosen earlier
branch that has fewer than two children. Branch length ~ U(50, 300) um and radius
~ U(0.5, 2) um are drawn per branch; a branch of n compartments is cut into n equal
cylinders, numbered proximal to distal, branch after branch in creation order, so that
every parent index is smaller than its child's.

Seeds: numpy PCG64 with seed 190107454 + 100*config + block, blocks of 1024 cells.
Poisson trains: a count per synapse ~ Poisson(rate*T), then uniform times on [0, T)
sorted (the order-statistics construction of a homogeneous Poisson process).
"""
from __future__ import annotations

import numpy as np

from .model import Model, SimSpec

SEED_BASE = 190107454
BLOCK = 1024

# Default channel parameters of the workloads (S/cm^2, uF/cm^2, Ohm*cm, mV, ms, uS).
CM = 1.0
RA = 100.0
GNABAR, GKBAR, GL = 0.12, 0.036, 3e-4
G_PAS, E_PAS = 1e-4, -65.0
SYN_TAU, SYN_E = 2.0, 0.0


def _rng(config: int, block: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + 100 * config + block))


def _attach_branches(rng: np.random.Generator, n_branches: int) -> np.ndarray:
    """Parent branch of each branch (-1 for branch 0): uniform over branches with < 2 children."""
    parent = np.full(n_branches, -1, dtype=np.int64)
    eligible = [0]
    nchild = [0] * n_branches
    u = rng.random(n_branches)
    for b in range(1, n_branches):
        k = int(u[b] * len(eligible))
        p = eligible[k]
        parent[b] = p
        nchild[p] += 1
        if nchild[p] == 2:
            eligible[k] = eligible[-1]
            eligible.pop()
        eligible.append(b)
    return parent


class _TreeBatch:
    """Branch-level description of many cells, expanded to CV arrays in one vectorised pass."""

    def __init__(self):
        self.cell_nb = []        # branches per cell
        self.b_ncv = []          # per branch: CV count
        self.b_len = []          # per branch: length um
        self.b_rad = []          # per branch: radius um
        self.b_par = []          # per branch: parent branch (cell-local, -1 root)

    def add_cell(self, ncv, length, radius, parent):
        self.cell_nb.append(len(ncv))
        self.b_ncv.append(np.asarray(ncv, np.int64))
        self.b_len.append(np.asarray(length, np.float64))
        self.b_rad.append(np.asarray(radius, np.float64))
        self.b_par.append(np.asarray(parent, np.int64))

    def expand(self):
        cell_nb = np.asarray(self.cell_nb, np.int64)
        ncv = np.concatenate(self.b_ncv)
        blen = np.concatenate(self.b_len)
        brad = np.concatenate(self.b_rad)
        bpar = np.concatenate(self.b_par)
        n_cells = cell_nb.size
        b_cell = np.repeat(np.arange(n_cells), cell_nb)
        b_first_of_cell = np.concatenate([[0], np.cumsum(cell_nb)[:-1]])
        b_local = np.arange(ncv.size) - b_first_of_cell[b_cell]
        cell_ncv = np.bincount(b_cell, weights=ncv, minlength=n_cells).astype(np.int64)
        cv_offset = np.concatenate([[0], np.cumsum(cell_ncv)])
        b_start = np.concatenate([[0], np.cumsum(ncv)[:-1]])          # global CV index of branch head
        b_start_local = b_start - cv_offset[b_cell]
        # parent CV of each branch head (cell-local): last CV of the parent branch
        pglob = np.where(bpar >= 0, bpar + b_first_of_cell[b_cell], 0)
        head_parent = np.where(bpar >= 0, b_start_local[pglob] + ncv[pglob] - 1, -1)
        cv_branch = np.repeat(np.arange(ncv.size), ncv)
        cv_global = np.arange(cv_offset[-1])
        cv_in_branch = cv_global - b_start[cv_branch]
        cv_local = cv_global - cv_offset[b_cell[cv_branch]]
        parent = np.where(cv_in_branch == 0, head_parent[cv_branch], cv_local - 1).astype(np.int32)
        length = (blen / ncv)[cv_branch]
        radius = brad[cv_branch]
        branch_of_cv = b_local[cv_branch].astype(np.int32)
        return cv_offset, parent, length, radius, branch_of_cv


def _random_cell_fixed(rng, n_branches, ncv_sampler, tb: _TreeBatch):
    par = _attach_branches(rng, n_branches)
    ncv = ncv_sampler(n_branches)
    length = rng.uniform(50.0, 300.0, n_branches)
    radius = rng.uniform(0.5, 2.0, n_branches)
    tb.add_cell(ncv, length, radius, par)


def _random_cell_total(rng, n_total, tb: _TreeBatch):
    """Branch sizes U{4..32} drawn until they reach n_total; the last one is truncated (>= 1)."""
    sizes = []
    s = 0
    while s < n_total:
        k = int(rng.integers(4, 33))
        k = min(k, n_total - s)
        sizes.append(k)
        s += k
    nb = len(sizes)
    par = _attach_branches(rng, nb)
    length = rng.uniform(50.0, 300.0, nb)
    radius = rng.uniform(0.5, 2.0, nb)
    tb.add_cell(np.asarray(sizes), length, radius, par)


def _poisson_events(rng, syn_ids, rate_hz, t_end_ms, weight_per_syn):
    """Homogeneous Poisson trains on each synapse; returns (syn, t, w) sorted by time."""
    lam = rate_hz * 1e-3 * t_end_ms
    counts = rng.poisson(lam, size=syn_ids.size)
    syn = np.repeat(syn_ids, counts)
    t = rng.uniform(0.0, t_end_ms, size=syn.size)
    w = np.repeat(weight_per_syn, counts)
    order = np.lexsort((syn, t))
    return syn[order], t[order], w[order]


def _mechanisms_soma_hh(cv_offset, branch_of_cv, all_hh=False):
    n_cv = branch_of_cv.size
    is_soma = branch_of_cv == 0
    hh_mask = np.ones(n_cv, bool) if all_hh else is_soma
    hh_cv = np.nonzero(hh_mask)[0]
    pas_cv = np.nonzero(~hh_mask)[0]
    return hh_cv, pas_cv


def _truncated_normal(rng, mean, sd, n):
    w = rng.normal(mean, sd, n)
    bad = w <= 0
    while bad.any():
        w[bad] = rng.normal(mean, sd, int(bad.sum()))
        bad = w <= 0
    return w


def make_config(config: int, n_cells: int | None = None, t_end: float | None = None,
                variant: str = "", syn_per_cell: int | None = None,
                virtual_ranks: int = 1) -> tuple[Model, SimSpec]:
    """Workload `config` (0..5); n_cells / t_end shrink it for tests; variant selects options.

    variant "ring_active" (config 1): the stimulus on cell 0 is raised so that the ring fires.
    variant "target" (config 4): the hidden parameter set that produces the target traces.
    syn_per_cell (config 5): synapses (and incoming connections) per cell, default 10,000.
    virtual_ranks (configs 2, 3): the cells are rank 0 of that many ranks holding copies of them
    (dry run); connection sources are drawn from all ranks' gids (virtual_ranks * n_cells).
    """
    if config == 0:
        n = 10 if n_cells is None else n_cells
        T = 100.0 if t_end is None else t_end
        tb = _TreeBatch()
        for blk in range((n + BLOCK - 1) // BLOCK):
            rng = _rng(0, blk)
            for _ in range(min(BLOCK, n - blk * BLOCK)):
                _random_cell_fixed(rng, 8, lambda nb: np.full(nb, 16), tb)
        cv_offset, parent, length, radius, bcv = tb.expand()
        hh_cv, pas_cv = _mechanisms_soma_hh(cv_offset, bcv)
        rng = _rng(0, 999)
        # one synapse per cell at a random dendritic CV
        syn_cv = []
        for c in range(n):
            lo, hi = cv_offset[c], cv_offset[c + 1]
            dend = np.nonzero(bcv[lo:hi] != 0)[0]
            syn_cv.append(lo + dend[int(rng.integers(0, dend.size))])
        syn_cv = np.asarray(syn_cv, np.int64)
        m = _assemble(cv_offset, parent, length, radius, bcv, hh_cv, pas_cv, syn_cv)
        ev = _poisson_events(rng, np.arange(n, dtype=np.int64), 20.0, T, np.full(n, 0.01))
        spec = SimSpec(dt=0.025, t_end=T, epoch_steps=400, ev_syn=ev[0], ev_t=ev[1], ev_w=ev[2],
                       name="plain-small-%dx128" % n)
        return m, spec

    if config == 1:
        n = 1024 if n_cells is None else n_cells
        T = 1000.0 if t_end is None else t_end
        tb = _TreeBatch()
        for blk in range((n + BLOCK - 1) // BLOCK):
            rng = _rng(1, blk)
            for _ in range(min(BLOCK, n - blk * BLOCK)):
                nb = int(rng.integers(16, 49))
                _random_cell_fixed(rng, nb, lambda k, r=rng: r.integers(8, 17, size=k), tb)
        cv_offset, parent, length, radius, bcv = tb.expand()
        hh_cv, pas_cv = _mechanisms_soma_hh(cv_offset, bcv)
        rng = _rng(1, 999)
        nsyn = 10
        syn_cv = _place_synapses(rng, cv_offset, nsyn)
        m = _assemble(cv_offset, parent, length, radius, bcv, hh_cv, pas_cv, syn_cv)
        # ring: every synapse of cell i listens to cell (i-1) mod n
        cell_of_syn = np.repeat(np.arange(n), nsyn)
        m.conn_src = ((cell_of_syn - 1) % n).astype(np.int32)
        m.conn_dst_syn = np.arange(n * nsyn, dtype=np.int64)
        m.conn_delay = np.full(n * nsyn, 5.0)
        m.conn_weight = np.full(n * nsyn, 0.05)
        active = variant == "ring_active"
        m.stim_cv = np.array([cv_offset[0]], np.int64)
        m.stim_t_on = np.array([0.0])
        m.stim_dur = np.array([2.0 if active else 1.0])
        m.stim_amp = np.array([2.0 if active else 0.2])
        m.__post_init__()
        spec = SimSpec(dt=0.025, t_end=T, epoch_steps=200,
                       name="ring-%d" % n + ("-active" if active else ""))
        return m, spec

    if config in (2, 3):
        n = 65536 if n_cells is None else n_cells
        T = 500.0 if t_end is None else t_end
        tb = _TreeBatch()
        for blk in range((n + BLOCK - 1) // BLOCK):
            rng = _rng(2, blk)
            cnt = min(BLOCK, n - blk * BLOCK)
            totals = np.rint(np.exp(rng.uniform(np.log(50.0), np.log(2000.0), cnt))).astype(np.int64)
            for c in range(cnt):
                _random_cell_total(rng, int(totals[c]), tb)
        cv_offset, parent, length, radius, bcv = tb.expand()
        hh_cv, pas_cv = _mechanisms_soma_hh(cv_offset, bcv)
        rng = _rng(2, 9999)
        nsyn = 100
        syn_cv = _place_synapses(rng, cv_offset, nsyn)
        m = _assemble(cv_offset, parent, length, radius, bcv, hh_cv, pas_cv, syn_cv)
        nsyn_tot = n * nsyn
        cell_of_syn = np.repeat(np.arange(n), nsyn)
        n_glob = n * int(virtual_ranks)
        if n_glob > 1:
            src = rng.integers(0, n_glob - 1, size=nsyn_tot)
            src = np.where(src >= cell_of_syn, src + 1, src)   # no self connections
        else:
            src = np.zeros(nsyn_tot, np.int64)
        m.conn_src = src.astype(np.int32)
        m.conn_dst_syn = np.arange(nsyn_tot, dtype=np.int64)
        m.conn_delay = rng.uniform(1.0, 10.0, nsyn_tot)
        m.conn_weight = _truncated_normal(rng, 0.01, 0.002, nsyn_tot)
        m.__post_init__()
        ev = _poisson_events(rng, np.arange(nsyn_tot, dtype=np.int64), 5.0, T, m.conn_weight)
        spec = SimSpec(dt=0.025, t_end=T, epoch_steps=40, ev_syn=ev[0], ev_t=ev[1], ev_w=ev[2],
                       name=("batched" if config == 2 else "mixed") + "-%d" % n +
                       ("" if virtual_ranks == 1 else " (rank 0 of %d)" % virtual_ranks))
        return m, spec

    if config == 4:
        n = 256 if n_cells is None else n_cells
        T = 200.0 if t_end is None else t_end
        tb = _TreeBatch()
        for blk in range((n + BLOCK - 1) // BLOCK):
            rng = _rng(4, blk)
            for _ in range(min(BLOCK, n - blk * BLOCK)):
                _random_cell_fixed(rng, 24, lambda k, r=rng: r.integers(8, 18, size=k), tb)
        cv_offset, parent, length, radius, bcv = tb.expand()
        hh_cv, pas_cv = _mechanisms_soma_hh(cv_offset, bcv, all_hh=True)
        m = _assemble(cv_offset, parent, length, radius, bcv, hh_cv, pas_cv,
                      np.zeros(0, np.int64))
        # per-branch parameters, defaults x U(0.7, 1.3)
        prng = _rng(4, 777 if variant != "target" else 778)
        nbr = int(bcv.max()) + 1
        scale = prng.uniform(0.7, 1.3, size=(4, n, nbr))
        cell = m.cell_of_cv()
        m.gnabar = GNABAR * scale[0, cell, bcv]
        m.gkbar = GKBAR * scale[1, cell, bcv]
        m.gl = GL * scale[2, cell, bcv]
        m.cm = CM * scale[3, cell, bcv]
        srng = _rng(4, 555)
        m.stim_cv = cv_offset[:-1].copy()
        m.stim_t_on = np.full(n, 5.0)
        m.stim_dur = np.full(n, 1e9)
        m.stim_amp = srng.uniform(0.1, 0.5, n)
        m.__post_init__()
        spec = SimSpec(dt=0.025, t_end=T, epoch_steps=400, name="adjoint-%d" % n)
        return m, spec

    if config == 5:
        # dense network after the paper's "10k connectivity" benchmark model: ring-model cells
        # (about 130 compartments: 6-16 branches of 8-16 CVs, HH soma, passive dendrites),
        # 10,000 excitatory exponential synapses per cell, each fed by one connection from a
        # uniformly chosen other cell, delays U(10, 20) ms (minimum delay 10 ms), weights
        # N(1e-6, 2e-7) uS; every cell is driven to spike synchronously at 50 Hz by a 1-ms, 2-nA
        # pulse every 20 ms on CV 0 (the network input depolarises, up to about -40 mV, without
        # adding spikes)
        n = 4096 if n_cells is None else n_cells
        T = 100.0 if t_end is None else t_end
        nsyn = 10000 if syn_per_cell is None else int(syn_per_cell)
        tb = _TreeBatch()
        for blk in range((n + BLOCK - 1) // BLOCK):
            rng = _rng(5, blk)
            for _ in range(min(BLOCK, n - blk * BLOCK)):
                nb = int(rng.integers(6, 17))
                _random_cell_fixed(rng, nb, lambda k, r=rng: r.integers(8, 17, size=k), tb)
        cv_offset, parent, length, radius, bcv = tb.expand()
        hh_cv, pas_cv = _mechanisms_soma_hh(cv_offset, bcv)
        rng = _rng(5, 9999)
        syn_cv = _place_synapses(rng, cv_offset, nsyn)
        m = _assemble(cv_offset, parent, length, radius, bcv, hh_cv, pas_cv, syn_cv)
        nsyn_tot = n * nsyn
        cell_of_syn = np.repeat(np.arange(n), nsyn)
        if n > 1:
            src = rng.integers(0, n - 1, size=nsyn_tot)
            src = np.where(src >= cell_of_syn, src + 1, src)   # no self connections
        else:
            src = np.zeros(nsyn_tot, np.int64)
        m.conn_src = src.astype(np.int32)
        m.conn_dst_syn = np.arange(nsyn_tot, dtype=np.int64)
        m.conn_delay = rng.uniform(10.0, 20.0, nsyn_tot)
        m.conn_weight = _truncated_normal(rng, 1e-6, 2e-7, nsyn_tot)
        pulses = np.arange(1.0, T, 20.0)
        m.stim_cv = np.repeat(cv_offset[:-1], pulses.size)
        m.stim_t_on = np.tile(pulses, n)
        m.stim_dur = np.full(m.stim_cv.size, 1.0)
        m.stim_amp = np.full(m.stim_cv.size, 2.0)
        m.__post_init__()
        spec = SimSpec(dt=0.025, t_end=T, epoch_steps=400, name="dense-%d" % n)
        return m, spec

    raise ValueError("unknown config %r" % config)


def _place_synapses(rng, cv_offset, nsyn):
    """Synapse 0 of each cell on CV 0, the others on uniformly random CVs of the cell."""
    n = cv_offset.size - 1
    sizes = np.diff(cv_offset)
    local = (rng.random((n, nsyn)) * sizes[:, None]).astype(np.int64)
    local[:, 0] = 0
    return (cv_offset[:-1, None] + local).reshape(-1)


def _assemble(cv_offset, parent, length, radius, bcv, hh_cv, pas_cv, syn_cv):
    n_cv = parent.size
    return Model(
        cv_offset=cv_offset, parent=parent, length_um=length, radius_um=radius,
        cm=np.full(n_cv, CM), Ra=np.full(n_cv, RA), branch_of_cv=bcv,
        hh_cv=hh_cv, gnabar=np.full(hh_cv.size, GNABAR), gkbar=np.full(hh_cv.size, GKBAR),
        gl=np.full(hh_cv.size, GL),
        pas_cv=pas_cv, g_pas=np.full(pas_cv.size, G_PAS), e_pas=np.full(pas_cv.size, E_PAS),
        syn_cv=syn_cv, syn_tau=np.full(syn_cv.size, SYN_TAU), syn_e=np.full(syn_cv.size, SYN_E),
        detector_cv=cv_offset[:-1].copy(), threshold=-10.0)


def config_names():
    return {0: "plain-small", 1: "plain-ring", 2: "batched", 3: "mixed", 4: "adjoint", 5: "dense"}


def small_tree_model(seed: int, n_cells: int = 1, n_branches: int = 5, cv_range=(1, 6),
                     hh_soma: bool = True, n_syn: int = 0, passive_only: bool = False,
                     ragged: bool = True) -> Model:
    """Tiny random trees for pin and parity tests (seed-controlled, any sizes)."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 7 * seed + 3))
    tb = _TreeBatch()
    for _ in range(n_cells):
        nb = int(rng.integers(1, n_branches + 1)) if ragged else n_branches
        _random_cell_fixed(rng, nb, lambda k: rng.integers(cv_range[0], cv_range[1] + 1, size=k), tb)
    cv_offset, parent, length, radius, bcv = tb.expand()
    if passive_only or not hh_soma:
        hh_cv = np.zeros(0, np.int64)
        pas_cv = np.arange(parent.size, dtype=np.int64)
    else:
        hh_cv, pas_cv = _mechanisms_soma_hh(cv_offset, bcv)
    syn_cv = _place_synapses(rng, cv_offset, n_syn) if n_syn > 0 else np.zeros(0, np.int64)
    return _assemble(cv_offset, parent, length, radius, bcv, hh_cv, pas_cv, syn_cv)


def uniform_cable_model(n_cv: int, length_um: float, radius_um: float, cm: float = 1.0,
                        Ra: float = 100.0, g_pas: float = 1e-4, e_pas: float = -65.0) -> Model:
    """One unbranched sealed cable of n_cv equal compartments (passive everywhere)."""
    parent = np.arange(-1, n_cv - 1, dtype=np.int32)
    return Model(
        cv_offset=np.array([0, n_cv]), parent=parent,
        length_um=np.full(n_cv, length_um / n_cv), radius_um=np.full(n_cv, radius_um),
        cm=np.full(n_cv, cm), Ra=np.full(n_cv, Ra), branch_of_cv=np.zeros(n_cv, np.int32),
        pas_cv=np.arange(n_cv), g_pas=np.full(n_cv, g_pas), e_pas=np.full(n_cv, e_pas),
        detector_cv=np.array([0]))
