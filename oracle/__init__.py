"""ORACLE -- test infrastructure only.

A plain FP64 CPU implementation of the cable-equation time stepper (arb_oracle.c). Only
tests/, the smoke check and the CPU-baseline leg of bench.py import this package; the
product path never does, and it shares no code with the CUDA library.

parity unpinned: full closed-loop network rasters (ring and random networks over many
epochs) have no external reference; they are compared GPU-vs-oracle only. Every building
block (solve, discretisation, splitting, gates, events, spike interpolation, epochs) is
pinned by tests/test_oracle_pins.py.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "arb_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with plain -O2, no fast-math and no FMA contraction."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Model(C.Structure):
    _fields_ = [
        ("n_cells", C.c_int32), ("cv_offset", C.c_void_p), ("parent", C.c_void_p),
        ("length_um", C.c_void_p), ("radius_um", C.c_void_p), ("cm", C.c_void_p), ("Ra", C.c_void_p),
        ("n_hh", C.c_int64), ("hh_cv", C.c_void_p), ("gnabar", C.c_void_p), ("gkbar", C.c_void_p),
        ("gl", C.c_void_p),
        ("n_pas", C.c_int64), ("pas_cv", C.c_void_p), ("g_pas", C.c_void_p), ("e_pas", C.c_void_p),
        ("n_syn", C.c_int64), ("syn_cv", C.c_void_p), ("syn_tau", C.c_void_p), ("syn_e", C.c_void_p),
        ("n_stim", C.c_int64), ("stim_cv", C.c_void_p), ("stim_t_on", C.c_void_p),
        ("stim_dur", C.c_void_p), ("stim_amp", C.c_void_p),
        ("detector_cv", C.c_void_p), ("threshold", C.c_double),
        ("n_conn", C.c_int64), ("conn_src", C.c_void_p), ("conn_dst_syn", C.c_void_p),
        ("conn_delay", C.c_void_p), ("conn_weight", C.c_void_p),
    ]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        vp, i64, dbl, i32 = C.c_void_p, C.c_int64, C.c_double, C.c_int
        L.orc_create.restype = vp
        L.orc_create.argtypes = [vp, dbl, i64, i32]
        L.orc_create_dry.restype = vp
        L.orc_create_dry.argtypes = [vp, dbl, i64, i32, i64]
        L.orc_destroy.argtypes = [vp]
        L.orc_enqueue.restype = i32
        L.orc_enqueue.argtypes = [vp, i64, vp, vp, vp]
        L.orc_run.restype = i32
        L.orc_run.argtypes = [vp, i64]
        L.orc_steps.restype = i64
        L.orc_steps.argtypes = [vp]
        L.orc_get_voltage.argtypes = [vp, vp]
        L.orc_num_spikes.restype = i64
        L.orc_num_spikes.argtypes = [vp]
        L.orc_get_spikes.argtypes = [vp, vp, vp]
        L.orc_set_probes.argtypes = [vp, i64, vp, vp, i64]
        L.orc_get_state.argtypes = [vp, vp, vp, vp, vp, vp]
        L.orc_set_state.argtypes = [vp, vp, vp, vp, vp, vp]
        L.orc_record_delivered.argtypes = [vp, i32]
        L.orc_set_explicit.argtypes = [vp, i32]
        L.orc_set_exact_events.argtypes = [vp, i32]
        L.orc_num_delivered.restype = i64
        L.orc_num_delivered.argtypes = [vp]
        L.orc_get_delivered.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.orc_cv_geometry.argtypes = [vp, vp, vp, vp]
        L.orc_hines_solve.restype = i32
        L.orc_hines_solve.argtypes = [i64, vp, vp, vp, vp, vp]
        L.orc_hh_rates.argtypes = [dbl, vp]
        L.orc_exprelr.restype = dbl
        L.orc_exprelr.argtypes = [dbl]
        L.orc_exprelr_deriv.restype = dbl
        L.orc_exprelr_deriv.argtypes = [dbl]
        L.orc_hh_rate_derivs.argtypes = [dbl, vp]
        L.orc_adjoint.restype = i32
        L.orc_adjoint.argtypes = [vp, i64, i64, vp, vp, dbl, vp, i32, vp, C.POINTER(dbl)]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None and a.size else None


class _Bound:
    """Keeps the NumPy arrays behind a _Model alive."""

    def __init__(self, m):
        self.m = m
        s = _Model()
        s.n_cells = m.n_cells
        s.cv_offset, s.parent = _p(m.cv_offset), _p(m.parent)
        s.length_um, s.radius_um, s.cm, s.Ra = _p(m.length_um), _p(m.radius_um), _p(m.cm), _p(m.Ra)
        s.n_hh = m.hh_cv.size
        s.hh_cv, s.gnabar, s.gkbar, s.gl = _p(m.hh_cv), _p(m.gnabar), _p(m.gkbar), _p(m.gl)
        s.n_pas = m.pas_cv.size
        s.pas_cv, s.g_pas, s.e_pas = _p(m.pas_cv), _p(m.g_pas), _p(m.e_pas)
        s.n_syn = m.syn_cv.size
        s.syn_cv, s.syn_tau, s.syn_e = _p(m.syn_cv), _p(m.syn_tau), _p(m.syn_e)
        s.n_stim = m.stim_cv.size
        s.stim_cv, s.stim_t_on, s.stim_dur, s.stim_amp = (_p(m.stim_cv), _p(m.stim_t_on),
                                                          _p(m.stim_dur), _p(m.stim_amp))
        s.detector_cv = _p(m.detector_cv)
        s.threshold = float(m.threshold)
        s.n_conn = m.conn_src.size
        s.conn_src, s.conn_dst_syn = _p(m.conn_src), _p(m.conn_dst_syn)
        s.conn_delay, s.conn_weight = _p(m.conn_delay), _p(m.conn_weight)
        self.s = s


def cv_geometry(m):
    """Per-CV (area um^2, capacitance nF, axial conductance to parent uS)."""
    b = _Bound(m)
    area, cap, sig = (np.zeros(m.n_cv) for _ in range(3))
    lib().orc_cv_geometry(C.byref(b.s), _p(area), _p(cap), _p(sig))
    return area, cap, sig


def hines_solve(parent, d, a, b):
    parent = np.ascontiguousarray(parent, np.int32)
    d, a, b = (np.ascontiguousarray(x, np.float64) for x in (d, a, b))
    x = np.zeros_like(b)
    rc = lib().orc_hines_solve(parent.size, _p(parent), _p(d), _p(a), _p(b), _p(x))
    assert rc == 0
    return x


def hh_rates(v):
    r = np.zeros(6)
    lib().orc_hh_rates(float(v), _p(r))
    return r


def exprelr(x):
    return lib().orc_exprelr(float(x))


def exprelr_deriv(x):
    return lib().orc_exprelr_deriv(float(x))


def hh_rate_derivs(v):
    r = np.zeros(6)
    lib().orc_hh_rate_derivs(float(v), _p(r))
    return r


class OracleSim:
    """FP64 CPU simulation of a Model; mirrors the library's create/enqueue/advance/read cycle."""

    def __init__(self, model, dt: float, epoch_steps: int, nthreads: int = 0, record_delivered=False,
                 explicit=False, exact_events=False, dry_run_ranks=1):
        """explicit=False: fully implicit voltage step (membrane conductance on the diagonal);
        explicit=True: the printed linear system with the membrane current at V(t).
        exact_events=True: steps are cut at the times of the events inside them.
        dry_run_ranks=R > 1: the model is rank 0 of R ranks holding copies of its cells;
        connection sources are global gids < R * n_cells, and every local spike also stands
        for the spikes of its copies on the other ranks (proxy spikes)."""
        self.model = model
        self.dt = float(dt)
        self.epoch_steps = int(epoch_steps)
        R = int(dry_run_ranks)
        if R < 1 or (model.conn_src.size and int(model.conn_src.max()) >= R * model.n_cells):
            raise ValueError("oracle: connection source outside the R * n_cells global gids")
        self._b = _Bound(model)
        self.h = lib().orc_create_dry(C.byref(self._b.s), self.dt, self.epoch_steps, int(nthreads), R)
        if record_delivered:
            lib().orc_record_delivered(self.h, 1)
        if explicit:
            lib().orc_set_explicit(self.h, 1)
        if exact_events:
            lib().orc_set_exact_events(self.h, 1)
        self._probe_buf = None

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().orc_destroy(h)
            self.h = None

    def enqueue(self, syn, t, w):
        syn = np.ascontiguousarray(syn, np.int64)
        t = np.ascontiguousarray(t, np.float64)
        w = np.ascontiguousarray(w, np.float64)
        if syn.size == 0:
            return
        rc = lib().orc_enqueue(self.h, syn.size, _p(syn), _p(t), _p(w))
        if rc != 0:
            raise ValueError("oracle: event in the past or bad synapse index")

    def set_probes(self, cvs, max_steps):
        cvs = np.ascontiguousarray(cvs, np.int64)
        self._probe_cvs = cvs
        self._probe_buf = np.full((int(max_steps), cvs.size), np.nan)
        lib().orc_set_probes(self.h, cvs.size, _p(cvs), _p(self._probe_buf), int(max_steps))
        return self._probe_buf

    def run_steps(self, n_steps: int):
        rc = lib().orc_run(self.h, int(n_steps))
        if rc != 0:
            raise RuntimeError("oracle: late event")

    def run(self, t_end: float):
        k_end = int(round(t_end / self.dt))
        self.run_steps(k_end - self.steps)

    @property
    def steps(self) -> int:
        return lib().orc_steps(self.h)

    def voltage(self):
        v = np.zeros(self.model.n_cv)
        lib().orc_get_voltage(self.h, _p(v))
        return v

    def spikes(self):
        n = lib().orc_num_spikes(self.h)
        gid = np.zeros(n, np.int32)
        t = np.zeros(n)
        if n:
            lib().orc_get_spikes(self.h, _p(gid), _p(t))
        return gid, t

    def get_state(self):
        m = self.model
        nh = m.hh_cv.size
        V, mm, hh, nn, g = np.zeros(m.n_cv), np.zeros(nh), np.zeros(nh), np.zeros(nh), np.zeros(m.n_syn)
        lib().orc_get_state(self.h, _p(V), _p(mm), _p(hh), _p(nn), _p(g))
        return dict(V=V, m=mm, h=hh, n=nn, g=g)

    def set_state(self, st):
        arrs = [np.ascontiguousarray(st[k], np.float64) for k in ("V", "m", "h", "n", "g")]
        lib().orc_set_state(self.h, *[_p(a) for a in arrs])

    def adjoint(self, n_steps, obs_cv, target, loss_scale, group_of_cv, n_groups):
        """Discrete adjoint over the next n_steps from the current state (which it leaves
        unchanged): returns (loss, grad [n_groups, 4] = dL/d(gnabar, gkbar, gl, cm))."""
        obs_cv = np.ascontiguousarray(obs_cv, np.int64)
        target = np.ascontiguousarray(target, np.float64).reshape(int(n_steps), obs_cv.size)
        group_of_cv = np.ascontiguousarray(group_of_cv, np.int32)
        grad = np.zeros((int(n_groups), 4))
        loss = C.c_double()
        rc = lib().orc_adjoint(self.h, int(n_steps), obs_cv.size, _p(obs_cv), _p(target), float(loss_scale),
                               _p(group_of_cv), int(n_groups), _p(grad), C.byref(loss))
        if rc != 0:
            raise ValueError("oracle adjoint: models with synapses are not supported")
        return loss.value, grad

    def delivered(self):
        n = lib().orc_num_delivered(self.h)
        syn, step, idx = np.zeros(n, np.int64), np.zeros(n, np.int64), np.zeros(n, np.int64)
        t, w, src = np.zeros(n), np.zeros(n), np.zeros(n, np.int32)
        if n:
            lib().orc_get_delivered(self.h, _p(syn), _p(t), _p(w), _p(step), _p(src), _p(idx))
        return dict(syn=syn, t=t, w=w, step=step, src=src, idx=idx)


def simulate(model, spec, nthreads: int = 0, probes=None, record_delivered=False, n_steps=None, explicit=False,
             exact_events=False, dry_run_ranks=1):
    """Run a whole SimSpec (or its first n_steps); returns (sim, probe trace or None)."""
    steps = spec.n_steps if n_steps is None else int(n_steps)
    sim = OracleSim(model, spec.dt, spec.epoch_steps or 400, nthreads, record_delivered, explicit, exact_events,
                    dry_run_ranks)
    sim.enqueue(spec.ev_syn, spec.ev_t, spec.ev_w)
    trace = sim.set_probes(probes, steps) if probes is not None else None
    sim.run_steps(steps)
    return sim, trace
