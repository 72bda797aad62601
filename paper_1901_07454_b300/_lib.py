"""ctypes binding of include/arb.h (same names, argument marshalling only).

Loading fails loudly when the in-tree CUDA library is missing: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libarb_b300.so")

ARB_OK, ARB_E_ARG, ARB_E_CUDA, ARB_E_OVERFLOW, ARB_E_NONFINITE, ARB_E_STATE, ARB_E_NOMEM = 0, -1, -2, -3, -4, -5, -6
ARB_FP64, ARB_MIXED = 0, 1
ARB_IMPLICIT, ARB_EXPLICIT = 0, 1
ARB_EVENTS_STEP_START, ARB_EVENTS_EXACT = 0, 1
STATUS_NAMES = {0: "ARB_OK", -1: "ARB_E_ARG", -2: "ARB_E_CUDA", -3: "ARB_E_OVERFLOW", -4: "ARB_E_NONFINITE",
                -5: "ARB_E_STATE", -6: "ARB_E_NOMEM"}

# Every symbol declared in include/arb.h.
EXPORTED = ["arb_default_params", "arb_create", "arb_destroy", "arb_workspace_bytes", "arb_bind_workspace",
            "arb_enqueue_events", "arb_advance", "arb_time", "arb_read_voltage", "arb_num_spikes",
            "arb_read_spikes", "arb_read_spikes_from", "arb_hh_gate_table", "arb_set_probes", "arb_get_state", "arb_set_state", "arb_plan_info",
            "arb_last_timing", "arb_last_error", "arb_solve_trees_noalloc", "arb_adjoint_workspace_bytes",
            "arb_adjoint", "arb_math_eval", "arb_kernel_variants", "arb_plan_packs", "arb_check_canaries",
            "arb_debug_build", "arb_workspace_region"]


class arb_params(C.Structure):
    _fields_ = [("dt", C.c_double), ("epoch_steps", C.c_int32), ("precision", C.c_int32),
                ("cells_per_pack", C.c_int32), ("smem_budget", C.c_int32),
                ("scheme", C.c_int32), ("split_cvs", C.c_int32),
                ("coalesce_synapses", C.c_int32), ("event_timing", C.c_int32), ("epoch_overlap", C.c_int32),
                ("dry_run_ranks", C.c_int32), ("spread_rows", C.c_int32), ("kernel_variant", C.c_int32),
                ("event_capacity", C.c_int64), ("ext_event_capacity", C.c_int64),
                ("spike_capacity", C.c_int64), ("bucket_capacity", C.c_int64), ("stream", C.c_void_p)]


class arb_model(C.Structure):
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


LIB_DEBUG_PATH = os.path.join(HERE, "libarb_b300_debug.so")
_libs = {}


def load(debug=False):
    """Loads libarb_b300.so (or, with debug, libarb_b300_debug.so: device index checks and
    workspace guard words); raises if it has not been built (no CPU fallback exists)."""
    key = bool(debug)
    if key in _libs:
        return _libs[key]
    path = LIB_DEBUG_PATH if debug else LIB_PATH
    if not os.path.exists(path):
        raise ImportError("%s is missing: build it with __graft_entry__.build() or "
                          "python paper_1901_07454_b300/_build.py (there is no CPU fallback)" % os.path.basename(path))
    L = C.CDLL(path)
    vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_double
    sig = {
        "arb_default_params": (i32, [vp]),
        "arb_create": (i32, [vp, vp, C.POINTER(vp)]),
        "arb_destroy": (None, [vp]),
        "arb_workspace_bytes": (i32, [vp, C.POINTER(i64)]),
        "arb_bind_workspace": (i32, [vp, vp, i64]),
        "arb_enqueue_events": (i32, [vp, i64, vp, vp, vp]),
        "arb_advance": (i32, [vp, dbl]),
        "arb_time": (i32, [vp, C.POINTER(dbl), C.POINTER(i64)]),
        "arb_read_voltage": (i32, [vp, vp, i64, i32]),
        "arb_num_spikes": (i32, [vp, C.POINTER(i64)]),
        "arb_read_spikes": (i32, [vp, vp, vp, i64, C.POINTER(i64)]),
        "arb_read_spikes_from": (i32, [vp, i64, vp, vp, i64, C.POINTER(i64)]),
        "arb_hh_gate_table": (i32, [dbl, vp, i64, C.POINTER(i64), C.POINTER(dbl), C.POINTER(dbl)]),
        "arb_set_probes": (i32, [vp, i64, vp, vp, i64]),
        "arb_get_state": (i32, [vp, vp, vp, vp, vp, vp]),
        "arb_set_state": (i32, [vp, vp, vp, vp, vp, vp]),
        "arb_plan_info": (i32, [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.POINTER(dbl), C.POINTER(i32),
                               C.POINTER(i64), C.POINTER(i32), C.POINTER(i64), C.POINTER(i64), C.POINTER(i32)]),
        "arb_last_timing": (i32, [vp, C.POINTER(dbl), C.POINTER(i64)]),
        "arb_last_error": (C.c_char_p, [vp]),
        "arb_solve_trees_noalloc": (i32, [i32, i64, vp, vp, vp, vp, vp, vp, vp]),
        "arb_adjoint_workspace_bytes": (i32, [vp, i64, i32, i64, i32, C.POINTER(i64)]),
        "arb_adjoint": (i32, [vp, i64, i32, i64, vp, vp, dbl, vp, i32, vp, i64, vp, C.POINTER(dbl)]),
        "arb_math_eval": (i32, [i32, i64, vp, vp, vp]),
        "arb_kernel_variants": (i32, [i32, vp, vp, vp]),
        "arb_plan_packs": (i32, [vp, i64, vp, vp, vp, C.POINTER(i64)]),
        "arb_check_canaries": (i32, [vp]),
        "arb_debug_build": (i32, []),
        "arb_workspace_region": (i32, [vp, C.c_char_p, C.POINTER(i64), C.POINTER(i64)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _libs[key] = L
    return L


class ArbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def check(status, handle=None, lib=None):
    if status != ARB_OK:
        msg = (lib or load()).arb_last_error(handle)
        raise ArbError(status, msg.decode() if msg else "")


def kernel_variants():
    """The compiled variants of the streamed epoch kernel: [(warps per SM, forward rows in
    flight, back-substitution rows in flight)], indexed by arb_params.kernel_variant."""
    import numpy as np
    lib = load()
    n = lib.arb_kernel_variants(0, None, None, None)
    w, f, b = (np.zeros(n, np.int32) for _ in range(3))
    lib.arb_kernel_variants(n, w.ctypes.data_as(C.c_void_p), f.ctypes.data_as(C.c_void_p), b.ctypes.data_as(C.c_void_p))
    return [(int(w[i]), int(f[i]), int(b[i])) for i in range(n)]

