"""C-ABI library: load, exported symbols, host-side validation and planning (no GPU)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from inputs import make_config, small_tree_model

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def arb():
    from paper_1901_07454_b300 import _build
    _build.build()
    import paper_1901_07454_b300 as m
    return m


def _header_symbols():
    txt = open(os.path.join(ROOT, "include", "arb.h")).read()
    return sorted(set(re.findall(r"\b(arb_[a-z_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(arb):
    declared = _header_symbols()
    assert len(declared) >= 15
    lib = arb.load()
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(arb.EXPORTED) == declared


def test_default_params(arb):
    p = arb.default_params()
    assert p.dt == 0.025 and p.precision == 0 and p.epoch_steps == 0


def _expect_error(arb, model, match, **kw):
    with pytest.raises(arb.ArbError) as ei:
        arb.Plan(model, **kw)
    assert "ARB_E_ARG" in str(ei.value)
    assert re.search(match, str(ei.value)), str(ei.value)


def test_validation_errors(arb):
    m = small_tree_model(1, n_cells=2, n_branches=4, cv_range=(2, 4))
    bad = small_tree_model(1, n_cells=2, n_branches=4, cv_range=(2, 4))
    bad.parent[3] = 5
    _expect_error(arb, bad, "parent")
    bad = small_tree_model(1, n_cells=2, n_branches=4, cv_range=(2, 4))
    bad.length_um[0] = -1.0
    _expect_error(arb, bad, "length")
    bad = small_tree_model(1, n_cells=2, n_branches=4, cv_range=(2, 4))
    bad.detector_cv = np.array([bad.cv_offset[1], 0])
    _expect_error(arb, bad, "detector")
    _expect_error(arb, m, "dt", dt=0.0)
    # delays shorter than the requested epoch
    r, spec = make_config(1, n_cells=4, t_end=10.0)
    _expect_error(arb, r, "epoch", dt=0.025, epoch_steps=400)
    # two HH instances on one CV
    bad = small_tree_model(2, n_cells=1, n_branches=2, cv_range=(2, 3))
    bad.hh_cv = np.array([0, 0])
    bad.gnabar = bad.gkbar = bad.gl = np.array([0.1, 0.1])
    _expect_error(arb, bad, "Hodgkin")


def test_planning_covers_every_cv(arb):
    for kpp in (32, 8, 3, 1):
        m = small_tree_model(5, n_cells=40, n_branches=9, cv_range=(1, 12), n_syn=3)
        p = arb.Plan(m, cells_per_pack=kpp)
        info = p.plan_info()
        assert info["total_rows"] * 32 >= m.n_cv
        assert 0 < info["lane_efficiency"] <= 1.0
        assert p.workspace_bytes() > 0


def test_streamed_plan_spreads_large_cells(arb):
    m = small_tree_model(11, n_cells=37, n_branches=9, cv_range=(1, 12), n_syn=4)
    one = arb.Plan(m, cells_per_pack=32, split_cvs=-1).plan_info()
    assert one["split_cvs"] == -1 and one["smem_packs"] == 0
    assert one["n_packs"] == 2 and one["max_pack_rows"] == int(np.diff(m.cv_offset).max())
    big = int((np.diff(m.cv_offset) > 40).sum())
    shared = arb.Plan(m, cells_per_pack=32, split_cvs=40).plan_info()
    assert shared["split_cvs"] == 40 and shared["smem_packs"] >= 1
    assert shared["max_pack_rows"] < one["max_pack_rows"]
    assert 1 <= shared["smem_packs"] <= big
    auto = arb.Plan(m, cells_per_pack=32).plan_info()      # a small batch: every cell is spread
    assert auto["split_cvs"] > 0 and auto["max_pack_rows"] <= shared["max_pack_rows"]
    _expect_error(arb, m, "split_cvs", cells_per_pack=32, split_cvs=-2)


def test_spread_schedules_keep_the_hand_over_rounds(arb):
    """Cells spread over lanes hand their contributions over through shared memory in rounds of
    rows. arb_create refuses a schedule in which such a write does not land in an earlier round
    than its parent reads it, or in which two lanes add to one slot in a round; on the implicit
    scheme's row-ring path the write lands one row after the child's last row, so a child on a
    round's last row writes in the next round. Plans of the batched workload's cells with most of
    them spread, for both schemes, every kernel variant and several split thresholds, pass."""
    m, spec = make_config(2, n_cells=1200, t_end=10.0)
    nv = len(arb.kernel_variants())
    for scheme in ("implicit", "explicit"):
        for split in (40, 150, 500):
            for v in range(nv):
                info = arb.Plan(m, dt=spec.dt, cells_per_pack=32, split_cvs=split, spread_rows=400,
                                kernel_variant=v, scheme=scheme).plan_info()
                assert info["split_cvs"] == split and info["smem_packs"] >= 1, (scheme, split, v, info)
                assert 0.5 < info["lane_efficiency"] <= 1.0, (scheme, split, v, info)


def test_epoch_is_derived_from_min_delay(arb):
    m, spec = make_config(1, n_cells=8, t_end=10.0)
    assert arb.Plan(m, dt=0.025).plan_info()["epoch_steps"] == 200
    m, spec = make_config(2, n_cells=64, t_end=10.0)
    assert arb.Plan(m, dt=0.025).plan_info()["epoch_steps"] == 40


def test_bind_requires_device_pointer(arb):
    m = small_tree_model(1, n_cells=1)
    p = arb.Plan(m)
    buf = (C.c_char * 1024)()
    st = arb.load().arb_bind_workspace(p.h, C.cast(buf, C.c_void_p), 1024)
    assert st != 0


def test_adjoint_workspace_query_and_unbound_handle(arb):
    lib = arb.load()
    m, _ = make_config(4, n_cells=2, t_end=1.0)
    p = arb.Plan(m)
    group, ng = m.param_groups()

    def ws(n_steps, ck):
        b = C.c_int64()
        assert lib.arb_adjoint_workspace_bytes(p.h, n_steps, ck, 2, ng, C.byref(b)) == 0
        return b.value

    # checkpoints grow with n_steps / ckpt, the two segment buffers with ckpt
    assert ws(8000, 500) > ws(4000, 500) > 0
    assert ws(8000, 100) < ws(8000, 500)
    assert ws(8000, 1) > ws(8000, 100)
    b = C.c_int64()
    assert lib.arb_adjoint_workspace_bytes(p.h, 0, 500, 2, ng, C.byref(b)) == -1
    assert lib.arb_adjoint_workspace_bytes(p.h, 10, 0, 2, ng, C.byref(b)) == -1
    # without a bound workspace the call is refused before any CUDA work
    loss = C.c_double()
    rc = lib.arb_adjoint(p.h, 10, 5, 0, None, None, 1.0, None, 0, None, 0, None, C.byref(loss))
    assert rc == -5 and b"bind" in lib.arb_last_error(p.h)
    # spike reads: a negative start is an argument error, an unbound handle a state error
    n = C.c_int64()
    assert lib.arb_read_spikes_from(p.h, -1, None, None, 0, C.byref(n)) == -1
    assert lib.arb_read_spikes_from(p.h, 0, None, None, 0, C.byref(n)) == -5


def test_exact_event_times_validation_and_plan(arb):
    m = small_tree_model(1, n_cells=40, n_branches=5, cv_range=(2, 8), n_syn=3)
    info = arb.Plan(m, exact_events=True).plan_info()
    assert info["cells_per_pack"] == 32 and info["split_cvs"] == -1
    _expect_error(arb, m, "exact event times", exact_events=True, scheme="explicit")
    _expect_error(arb, m, "exact event times", exact_events=True, precision="mixed")
    _expect_error(arb, m, "one cell per lane", exact_events=True, cells_per_pack=8)


def test_overlapped_exchange_epoch_rule_and_workspace(arb):
    # ring of 16 cells, every delay 5 ms: serial epochs may be 200 steps of 0.025 ms, overlapped
    # ones (half the minimum delay) at most 100
    from inputs import make_config
    m, _ = make_config(1, n_cells=16, t_end=10.0)
    assert arb.Plan(m).plan_info()["epoch_steps"] == 200
    assert arb.Plan(m, epoch_overlap=True).plan_info()["epoch_steps"] == 100
    assert arb.Plan(m, epoch_overlap=True, epoch_steps=100).plan_info()["epoch_steps"] == 100
    arb.Plan(m, epoch_steps=150)
    _expect_error(arb, m, "half the minimum delay", epoch_overlap=True, epoch_steps=150)
    _expect_error(arb, m, "bucket capacity", epoch_overlap=True, bucket_capacity=1 << 30)
    # two delivery-list buffers
    b_ser = arb.Plan(m, epoch_steps=100).workspace_bytes()
    b_ovl = arb.Plan(m, epoch_overlap=True).workspace_bytes()
    assert b_ovl > b_ser


def test_dry_run_sources_and_validation(arb):
    # 16 local cells as rank 0 of 8 ranks: sources may be any of the 128 global gids
    from inputs import make_config
    m, _ = make_config(2, n_cells=16, t_end=5.0, virtual_ranks=8)
    assert m.conn_src.max() >= 16
    _expect_error(arb, m, "source gid out of range")                        # not a dry run
    _expect_error(arb, m, "dry_run_ranks", dry_run_ranks=4)                  # too few ranks
    _expect_error(arb, m, "dry_run_ranks must be", dry_run_ranks=-1)
    _expect_error(arb, m, "2\\^31", dry_run_ranks=1 << 28)
    b8 = arb.Plan(m, dry_run_ranks=8).workspace_bytes()
    b64 = arb.Plan(m, dry_run_ranks=64).workspace_bytes()
    assert b64 - b8 >= 8 * 16 * 56        # one out-list offset per global gid


def test_connection_checks_report_the_first_failing_connection(arb):
    # more than 2^20 connections: checked in parallel parts, and the lowest failing index
    # decides the message, as a serial check would
    m = small_tree_model(3, n_cells=2, n_branches=4, cv_range=(2, 4), n_syn=2)
    n = (1 << 20) + 7
    m.conn_src = np.zeros(n, np.int32)
    m.conn_dst_syn = np.zeros(n, np.int64)
    m.conn_delay = np.full(n, 1.0)
    m.conn_weight = np.full(n, 0.01)
    m.__post_init__()
    assert arb.Plan(m).plan_info()["epoch_steps"] == 40
    m.conn_delay[700001] = -1.0
    m.conn_src[900000] = 5
    _expect_error(arb, m, "delays must be finite and > 0")
    m.conn_src[600000] = 5
    _expect_error(arb, m, "source gid out of range")
    m.conn_src[:] = 0
    m.conn_delay[:] = 1.0
    m.conn_weight[n - 1] = np.nan
    _expect_error(arb, m, "weights must be finite")
