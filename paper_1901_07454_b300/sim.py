"""Python front end of the C ABI: torch provides the device workspace and the stream.

Every step of the simulation runs in the library's CUDA kernels; this module only marshals
arrays and owns the torch buffers.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None and a.size else None


def _model_struct(m):
    """Builds an arb_model from an inputs.Model (or any object with the same array fields)."""
    keep = {}

    def arr(name, dtype):
        a = np.ascontiguousarray(getattr(m, name), dtype=dtype)
        keep[name] = a
        return _p(a)

    s = L.arb_model()
    s.n_cells = int(np.asarray(m.cv_offset).size - 1)
    s.cv_offset = arr("cv_offset", np.int64)
    s.parent = arr("parent", np.int32)
    s.length_um, s.radius_um = arr("length_um", np.float64), arr("radius_um", np.float64)
    s.cm, s.Ra = arr("cm", np.float64), arr("Ra", np.float64)
    s.n_hh = int(np.asarray(m.hh_cv).size)
    s.hh_cv = arr("hh_cv", np.int64)
    s.gnabar, s.gkbar, s.gl = arr("gnabar", np.float64), arr("gkbar", np.float64), arr("gl", np.float64)
    s.n_pas = int(np.asarray(m.pas_cv).size)
    s.pas_cv, s.g_pas, s.e_pas = arr("pas_cv", np.int64), arr("g_pas", np.float64), arr("e_pas", np.float64)
    s.n_syn = int(np.asarray(m.syn_cv).size)
    s.syn_cv, s.syn_tau, s.syn_e = arr("syn_cv", np.int64), arr("syn_tau", np.float64), arr("syn_e", np.float64)
    s.n_stim = int(np.asarray(m.stim_cv).size)
    s.stim_cv = arr("stim_cv", np.int64)
    s.stim_t_on, s.stim_dur, s.stim_amp = arr("stim_t_on", np.float64), arr("stim_dur", np.float64), arr("stim_amp", np.float64)
    s.detector_cv = arr("detector_cv", np.int64)
    s.threshold = float(m.threshold)
    s.n_conn = int(np.asarray(m.conn_src).size)
    s.conn_src, s.conn_dst_syn = arr("conn_src", np.int32), arr("conn_dst_syn", np.int64)
    s.conn_delay, s.conn_weight = arr("conn_delay", np.float64), arr("conn_weight", np.float64)
    return s, keep


def default_params():
    p = L.arb_params()
    L.check(L.load().arb_default_params(C.byref(p)))
    return p


class Plan:
    """Host-side preparation only (arb_create): usable without a GPU."""

    def __init__(self, model, dt=0.025, epoch_steps=0, precision="fp64", cells_per_pack=0, smem_budget=0,
                 event_capacity=None, ext_event_capacity=None, spike_capacity=None, bucket_capacity=None,
                 stream=None, scheme="implicit", split_cvs=0, coalesce_synapses=False, exact_events=False,
                 epoch_overlap=False, dry_run_ranks=1, kernel_variant=-1, spread_rows=0, debug=False):
        """debug=True runs on the debug build (device index checks, workspace guard words)."""
        lib = L.load(debug)
        self.lib = lib
        self.model = model
        p = default_params()
        p.dt = float(dt)
        p.epoch_steps = int(epoch_steps)
        p.precision = L.ARB_MIXED if precision == "mixed" else L.ARB_FP64
        p.cells_per_pack = int(cells_per_pack)
        p.smem_budget = int(smem_budget)
        p.split_cvs = int(split_cvs)
        p.coalesce_synapses = 1 if coalesce_synapses else 0
        p.event_timing = L.ARB_EVENTS_EXACT if exact_events else L.ARB_EVENTS_STEP_START
        p.epoch_overlap = 1 if epoch_overlap else 0
        p.dry_run_ranks = int(dry_run_ranks)
        p.kernel_variant = int(kernel_variant)
        p.spread_rows = int(spread_rows)
        if scheme not in ("implicit", "explicit"):
            raise ValueError("scheme must be 'implicit' or 'explicit'")
        p.scheme = L.ARB_EXPLICIT if scheme == "explicit" else L.ARB_IMPLICIT
        if event_capacity is not None:
            p.event_capacity = int(event_capacity)
        if ext_event_capacity is not None:
            p.ext_event_capacity = int(ext_event_capacity)
        if spike_capacity is not None:
            p.spike_capacity = int(spike_capacity)
        if bucket_capacity is not None:
            p.bucket_capacity = int(bucket_capacity)
        p.stream = stream
        self.params = p
        self._ms, self._keep = _model_struct(model)
        h = C.c_void_p()
        st = lib.arb_create(C.byref(self._ms), C.byref(p), C.byref(h))
        L.check(st, None, lib)
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.arb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace_bytes(self) -> int:
        n = C.c_int64()
        L.check(self.lib.arb_workspace_bytes(self.h, C.byref(n)), self.h, self.lib)
        return n.value

    def workspace_region(self, name):
        """(byte offset, bytes) of a named plan array in the workspace (arb_workspace_region)."""
        off, nb = C.c_int64(), C.c_int64()
        L.check(self.lib.arb_workspace_region(self.h, name.encode(), C.byref(off), C.byref(nb)), self.h, self.lib)
        return off.value, nb.value

    def check_canaries(self):
        """Debug builds: raises ArbError when a guard word after a workspace region was overwritten."""
        L.check(self.lib.arb_check_canaries(self.h), self.h, self.lib)

    def plan_packs(self):
        """Per pack, in the persistent kernel's order: (solve rows, kind, mechanism rows) arrays;
        kind 0 streamed one cell per lane, 1 streamed spread over lanes, 2/3 tile packs."""
        lib = self.lib
        n = C.c_int64()
        L.check(lib.arb_plan_packs(self.h, 0, None, None, None, C.byref(n)), self.h, self.lib)
        rows, kind, mech = (np.zeros(n.value, np.int32) for _ in range(3))
        L.check(lib.arb_plan_packs(self.h, n.value, _p(rows), _p(kind), _p(mech), C.byref(n)), self.h, self.lib)
        return rows, kind, mech

    def plan_info(self):
        npk, rows, smem, mxr, split, srows = (C.c_int64() for _ in range(6))
        eff, ep, kpp, kv = C.c_double(), C.c_int32(), C.c_int32(), C.c_int32()
        L.check(self.lib.arb_plan_info(self.h, C.byref(npk), C.byref(rows), C.byref(smem), C.byref(eff), C.byref(ep),
                                       C.byref(mxr), C.byref(kpp), C.byref(split), C.byref(srows), C.byref(kv)), self.h,
                self.lib)
        return dict(n_packs=npk.value, total_rows=rows.value, smem_packs=smem.value, lane_efficiency=eff.value,
                    epoch_steps=ep.value, max_pack_rows=mxr.value, cells_per_pack=kpp.value, split_cvs=split.value,
                    spread_rows=srows.value, kernel_variant=kv.value)


class Simulation(Plan):
    """A bound handle: device workspace from torch, all stepping in the CUDA library."""

    def __init__(self, model, dt=0.025, device="cuda", stream=None, **kw):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        if self.device.type != "cuda":
            raise RuntimeError("Simulation needs a CUDA device; there is no CPU fallback")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        torch.cuda.set_device(self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        super().__init__(model, dt=dt, stream=C.c_void_p(self.stream.cuda_stream), **kw)
        nbytes = self.workspace_bytes()
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self._ws.data_ptr()
        aligned = (base + 255) & ~255
        self._ws_shift = aligned - base          # the bound workspace starts here in self._ws
        L.check(self.lib.arb_bind_workspace(self.h, C.c_void_p(aligned), nbytes), self.h, self.lib)
        self.dt = float(dt)
        self._trace = None

    # --- events and time
    def enqueue(self, syn, t, w):
        syn = np.ascontiguousarray(syn, np.int64)
        t = np.ascontiguousarray(t, np.float64)
        w = np.ascontiguousarray(w, np.float64)
        if syn.size:
            L.check(self.lib.arb_enqueue_events(self.h, syn.size, _p(syn), _p(t), _p(w)), self.h, self.lib)

    def advance(self, t_end: float):
        L.check(self.lib.arb_advance(self.h, float(t_end)), self.h, self.lib)

    def time(self):
        t, k = C.c_double(), C.c_int64()
        L.check(self.lib.arb_time(self.h, C.byref(t), C.byref(k)), self.h, self.lib)
        return t.value, k.value

    # --- outputs
    def voltage(self, out=None):
        """Voltages in model CV order: a numpy array, or into a given CUDA float64 tensor."""
        n = int(self.model.n_cv)
        if out is not None:
            assert out.is_cuda and out.dtype == self.torch.float64 and out.numel() == n
            L.check(self.lib.arb_read_voltage(self.h, C.c_void_p(out.data_ptr()), n, 1), self.h, self.lib)
            return out
        v = np.zeros(n)
        L.check(self.lib.arb_read_voltage(self.h, _p(v), n, 0), self.h, self.lib)
        return v

    def num_spikes(self) -> int:
        n = C.c_int64()
        L.check(self.lib.arb_num_spikes(self.h, C.byref(n)), self.h, self.lib)
        return n.value

    def spikes(self, first=0):
        """Spikes recorded after the first `first` ones, sorted by (time, gid): (gid, t)."""
        n = max(0, self.num_spikes() - int(first))
        gid = np.zeros(max(n, 1), np.int32)
        t = np.zeros(max(n, 1))
        got = C.c_int64()
        L.check(self.lib.arb_read_spikes_from(self.h, int(first), _p(gid), _p(t), n, C.byref(got)), self.h, self.lib)
        return gid[:got.value], t[:got.value]

    def new_spikes(self):
        """Spikes recorded since the previous new_spikes() call (all of them on the first
        call), sorted by (time, gid); the per-epoch spike export."""
        first = getattr(self, "_spike_cursor", 0)
        gid, t = self.spikes(first)
        self._spike_cursor = first + gid.size
        return gid, t

    def set_probes(self, cvs, max_steps):
        cvs = np.ascontiguousarray(cvs, np.int64)
        self._trace = self.torch.full((int(max_steps), cvs.size), float("nan"), dtype=self.torch.float64, device=self.device)
        L.check(self.lib.arb_set_probes(self.h, cvs.size, _p(cvs), C.c_void_p(self._trace.data_ptr()), int(max_steps)), self.h, self.lib)
        return self._trace

    def get_state(self):
        m = self.model
        nh = np.asarray(m.hh_cv).size
        V, mm, hh, nn, g = np.zeros(m.n_cv), np.zeros(nh), np.zeros(nh), np.zeros(nh), np.zeros(m.n_syn)
        L.check(self.lib.arb_get_state(self.h, _p(V), _p(mm), _p(hh), _p(nn), _p(g)), self.h, self.lib)
        return dict(V=V, m=mm, h=hh, n=nn, g=g)

    def set_state(self, st):
        arrs = [np.ascontiguousarray(st[k], np.float64) for k in ("V", "m", "h", "n", "g")]
        L.check(self.lib.arb_set_state(self.h, *[_p(a) for a in arrs]), self.h, self.lib)

    def last_timing(self):
        ms, n = C.c_double(), C.c_int64()
        L.check(self.lib.arb_last_timing(self.h, C.byref(ms), C.byref(n)), self.h, self.lib)
        return ms.value, n.value

    # --- discrete adjoint
    def adjoint(self, n_steps, obs_cv, target, loss_scale, group_of_cv, n_groups, checkpoint_every=500):
        """Loss and gradient over the next n_steps from the current state (arb_adjoint); the
        state is left unchanged. target: [n_steps, n_obs] (host or device); returns
        (loss float, grad float64 tensor [n_groups, 4] on the device)."""
        torch = self.torch
        lib = self.lib
        n_steps, n_groups = int(n_steps), int(n_groups)
        obs_cv = np.ascontiguousarray(obs_cv, np.int64)
        group = np.ascontiguousarray(group_of_cv, np.int32)
        tgt = torch.as_tensor(target, dtype=torch.float64).to(self.device).reshape(n_steps, obs_cv.size).contiguous()
        nbytes = C.c_int64()
        L.check(lib.arb_adjoint_workspace_bytes(self.h, n_steps, int(checkpoint_every), obs_cv.size, n_groups,
                                                C.byref(nbytes)), self.h, self.lib)
        ws = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=self.device)
        aligned = (ws.data_ptr() + 255) & ~255
        grad = torch.zeros((n_groups, 4), dtype=torch.float64, device=self.device)
        loss = C.c_double()
        L.check(lib.arb_adjoint(self.h, n_steps, int(checkpoint_every), obs_cv.size, _p(obs_cv),
                                C.c_void_p(tgt.data_ptr()), float(loss_scale), _p(group), n_groups,
                                C.c_void_p(aligned), nbytes.value, C.c_void_p(grad.data_ptr()), C.byref(loss)), self.h,
                self.lib)
        self._adj_keep = (ws, tgt)     # freed with the next call or the handle
        return loss.value, grad
