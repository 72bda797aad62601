"""Plain-array description of a batch of multicompartment cells.

Units (used by every consumer): V mV, t ms, length and radius um, cm uF/cm^2,
Ra Ohm*cm, channel densities S/cm^2, synaptic weights uS, currents nA.

A cell is a tree of compartments (control volumes, CVs). Each CV is a cylinder with
its own length, radius, specific capacitance and axial resistivity, and a parent CV
inside the same cell (-1 for the root, parent index < own index). All index arrays
that name a CV use the global CV index (cell offset + local index).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np


def _f64(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _i64(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.int64))


def _i32(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.int32))


@dataclass
class Model:
    # morphology
    cv_offset: np.ndarray            # int64 [n_cells+1]
    parent: np.ndarray               # int32 [n_cv], cell-local parent, -1 at the root
    length_um: np.ndarray            # float64 [n_cv]
    radius_um: np.ndarray            # float64 [n_cv]
    cm: np.ndarray                   # float64 [n_cv] uF/cm^2
    Ra: np.ndarray                   # float64 [n_cv] Ohm*cm
    branch_of_cv: np.ndarray         # int32 [n_cv], cell-local branch id (for per-branch parameters)
    # Hodgkin-Huxley instances (at most one per CV)
    hh_cv: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    gnabar: np.ndarray = field(default_factory=lambda: np.zeros(0))
    gkbar: np.ndarray = field(default_factory=lambda: np.zeros(0))
    gl: np.ndarray = field(default_factory=lambda: np.zeros(0))
    # passive instances
    pas_cv: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    g_pas: np.ndarray = field(default_factory=lambda: np.zeros(0))
    e_pas: np.ndarray = field(default_factory=lambda: np.zeros(0))
    # exponential synapses
    syn_cv: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    syn_tau: np.ndarray = field(default_factory=lambda: np.zeros(0))
    syn_e: np.ndarray = field(default_factory=lambda: np.zeros(0))
    # current clamps (positive = depolarising)
    stim_cv: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    stim_t_on: np.ndarray = field(default_factory=lambda: np.zeros(0))
    stim_dur: np.ndarray = field(default_factory=lambda: np.zeros(0))
    stim_amp: np.ndarray = field(default_factory=lambda: np.zeros(0))
    # one threshold detector per cell
    detector_cv: np.ndarray = None   # int64 [n_cells]
    threshold: float = -10.0
    # connections (source cell gid -> target synapse)
    conn_src: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    conn_dst_syn: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    conn_delay: np.ndarray = field(default_factory=lambda: np.zeros(0))
    conn_weight: np.ndarray = field(default_factory=lambda: np.zeros(0))

    def __post_init__(self):
        self.cv_offset = _i64(self.cv_offset)
        self.parent = _i32(self.parent)
        self.length_um = _f64(self.length_um)
        self.radius_um = _f64(self.radius_um)
        self.cm = _f64(self.cm)
        self.Ra = _f64(self.Ra)
        self.branch_of_cv = _i32(self.branch_of_cv)
        self.hh_cv = _i64(self.hh_cv)
        self.gnabar, self.gkbar, self.gl = _f64(self.gnabar), _f64(self.gkbar), _f64(self.gl)
        self.pas_cv = _i64(self.pas_cv)
        self.g_pas, self.e_pas = _f64(self.g_pas), _f64(self.e_pas)
        self.syn_cv = _i64(self.syn_cv)
        self.syn_tau, self.syn_e = _f64(self.syn_tau), _f64(self.syn_e)
        self.stim_cv = _i64(self.stim_cv)
        self.stim_t_on, self.stim_dur, self.stim_amp = _f64(self.stim_t_on), _f64(self.stim_dur), _f64(self.stim_amp)
        if self.detector_cv is None:
            self.detector_cv = self.cv_offset[:-1].copy()
        self.detector_cv = _i64(self.detector_cv)
        self.conn_src = _i32(self.conn_src)
        self.conn_dst_syn = _i64(self.conn_dst_syn)
        self.conn_delay, self.conn_weight = _f64(self.conn_delay), _f64(self.conn_weight)

    @property
    def n_cells(self) -> int:
        return int(self.cv_offset.shape[0] - 1)

    @property
    def n_cv(self) -> int:
        return int(self.parent.shape[0])

    @property
    def n_syn(self) -> int:
        return int(self.syn_cv.shape[0])

    def cell_of_cv(self) -> np.ndarray:
        return np.repeat(np.arange(self.n_cells, dtype=np.int64), np.diff(self.cv_offset))

    def cell_sizes(self) -> np.ndarray:
        return np.diff(self.cv_offset)

    def tiled(self, ranks: int):
        """The network of `ranks` copies of this model: copy r holds cells r*n .. r*n+n-1 (CVs,
        synapses and clamps shifted by r times the counts), and each connection (s -> synapse j)
        of the model is repeated in copy r as ((s + r*n) mod (ranks*n) -> synapse j of copy r).
        Connection sources of the model may be any of the ranks*n gids; copy 0's connections
        come first, in the model's order. Index shifting only."""
        R = int(ranks)
        n, ncv, nsyn = self.n_cells, self.n_cv, self.n_syn
        rr = np.arange(R, dtype=np.int64)

        def shift(idx, step):
            return (np.asarray(idx, np.int64)[None, :] + rr[:, None] * step).ravel()

        def tile(a):
            return np.tile(np.asarray(a), R)

        off = np.concatenate([[0], shift(self.cv_offset[1:], ncv)])
        m = Model(cv_offset=off, parent=tile(self.parent), length_um=tile(self.length_um),
                  radius_um=tile(self.radius_um), cm=tile(self.cm), Ra=tile(self.Ra),
                  branch_of_cv=tile(self.branch_of_cv),
                  hh_cv=shift(self.hh_cv, ncv), gnabar=tile(self.gnabar), gkbar=tile(self.gkbar), gl=tile(self.gl),
                  pas_cv=shift(self.pas_cv, ncv), g_pas=tile(self.g_pas), e_pas=tile(self.e_pas),
                  syn_cv=shift(self.syn_cv, ncv), syn_tau=tile(self.syn_tau), syn_e=tile(self.syn_e),
                  stim_cv=shift(self.stim_cv, ncv), stim_t_on=tile(self.stim_t_on), stim_dur=tile(self.stim_dur),
                  stim_amp=tile(self.stim_amp), detector_cv=shift(self.detector_cv, ncv), threshold=self.threshold,
                  conn_src=(shift(self.conn_src, n) % (R * n)).astype(np.int32),
                  conn_dst_syn=shift(self.conn_dst_syn, nsyn),
                  conn_delay=tile(self.conn_delay), conn_weight=tile(self.conn_weight))
        return m

    # per-branch parameter groups: group = cell * (branches per cell) + branch
    PARAM_NAMES = ("gnabar", "gkbar", "gl", "cm")

    def param_groups(self):
        """(group_of_cv int32 [n_cv], n_groups) with one group per (cell, branch)."""
        nb = int(self.branch_of_cv.max()) + 1 if self.n_cv else 0
        group = (self.cell_of_cv() * nb + self.branch_of_cv).astype(np.int32)
        return group, self.n_cells * nb

    def group_params(self):
        """theta [n_groups, 4] = (gnabar, gkbar, gl, cm), read from the first CV / HH
        instance of each group (groups are assumed uniform)."""
        group, ng = self.param_groups()
        th = np.zeros((ng, 4))
        th[group[::-1], 3] = self.cm[::-1]
        hg = group[self.hh_cv]
        th[hg[::-1], 0] = self.gnabar[::-1]
        th[hg[::-1], 1] = self.gkbar[::-1]
        th[hg[::-1], 2] = self.gl[::-1]
        return th

    def with_group_params(self, theta):
        """A copy whose per-instance densities and per-CV cm are taken from theta [n_groups, 4]."""
        import copy
        theta = np.asarray(theta, np.float64)
        group, ng = self.param_groups()
        assert theta.shape == (ng, 4)
        m = copy.copy(self)
        hg = group[self.hh_cv]
        m.gnabar, m.gkbar, m.gl = theta[hg, 0].copy(), theta[hg, 1].copy(), theta[hg, 2].copy()
        m.cm = theta[group, 3].copy()
        return m


@dataclass
class SimSpec:
    """Run settings that go with a model: time step, duration, epoch and external events."""
    dt: float = 0.025
    t_end: float = 100.0
    epoch_steps: int = 0                 # 0: derived from the minimum connection delay
    ev_syn: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    ev_t: np.ndarray = field(default_factory=lambda: np.zeros(0))
    ev_w: np.ndarray = field(default_factory=lambda: np.zeros(0))
    name: str = ""

    def __post_init__(self):
        self.ev_syn = _i64(self.ev_syn)
        self.ev_t = _f64(self.ev_t)
        self.ev_w = _f64(self.ev_w)

    @property
    def n_steps(self) -> int:
        return int(round(self.t_end / self.dt))
