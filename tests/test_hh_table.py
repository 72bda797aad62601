"""The tabulated HH gate update of the streamed FP64 kernel (host-built, no GPU) against the
gate update formed from the oracle's rates: x_inf = alpha / (alpha + beta) and
e = exp(-dt (alpha + beta)) for m, h and n (the exact update at frozen V, Sec. "Model")."""
import ctypes as C

import numpy as np
import pytest


@pytest.fixture(scope="module")
def table():
    import paper_1901_07454_b300 as arb
    lib = arb.load()
    n, vlo, pm = C.c_int64(), C.c_double(), C.c_double()
    assert lib.arb_hh_gate_table(0.025, None, 0, C.byref(n), C.byref(vlo), C.byref(pm)) == 0
    tab = np.zeros(n.value * 24)
    assert lib.arb_hh_gate_table(0.025, C.c_void_p(tab.ctypes.data), tab.size, C.byref(n), C.byref(vlo),
                                 C.byref(pm)) == 0
    assert lib.arb_hh_gate_table(0.0, None, 0, C.byref(n), C.byref(vlo), C.byref(pm)) == -1
    assert b"dt" in lib.arb_last_error(None)
    # a buffer too small for the table is refused and left untouched
    small = np.full(24, 7.0)
    assert lib.arb_hh_gate_table(0.025, C.c_void_p(small.ctypes.data), small.size, None, None, None) == -1
    assert b"needs" in lib.arb_last_error(None) and np.all(small == 7.0)
    return tab.reshape(n.value, 6, 4), vlo.value, pm.value


def _eval(table, V):
    coef, vlo, pm = table
    t = (V - vlo) * pm
    i = np.floor(t).astype(np.int64)
    s = (t - i)[:, None]
    c = coef[i]                                           # [n, 6, 4]
    return ((c[..., 3] * s + c[..., 2]) * s + c[..., 1]) * s + c[..., 0]


def _direct(oracle_lib, V, dt=0.025):
    out = np.zeros((V.size, 6))
    for k, v in enumerate(V):
        r = oracle_lib.hh_rates(v)                        # alpha_m, beta_m, alpha_h, beta_h, alpha_n, beta_n
        for q in range(3):
            a, b = r[2 * q], r[2 * q + 1]
            out[k, 2 * q] = a / (a + b)
            out[k, 2 * q + 1] = np.exp(-dt * (a + b))
    return out


def test_table_matches_the_gate_update_from_the_rates(table, oracle_lib):
    coef, vlo, pm = table
    assert vlo <= -120.0 and vlo + coef.shape[0] / pm >= 60.0
    rng = np.random.default_rng(190107454)
    V = np.concatenate([rng.uniform(vlo, vlo + coef.shape[0] / pm - 1e-9, 20000), np.linspace(-90.0, 50.0, 2801),
                        [-40.0, -55.0, -35.0, -65.0, vlo]])
    err = np.abs(_eval(table, V) - _direct(oracle_lib, V))
    # a few ulp of values in (0, 1]; a wrong coefficient, slope or scale is off by far more
    assert err.max() <= 1e-15, (err.max(), V[np.argmax(err.max(axis=1))])


def test_table_pieces_join(table):
    # each cubic ends where the next one starts (values agree to rounding)
    coef, _, _ = table
    end = coef.sum(axis=2)[:-1]
    start = coef[1:, :, 0]
    assert np.max(np.abs(end - start)) <= 1e-15


def test_table_slopes_match_the_derivatives_of_the_gate_update(table, oracle_lib):
    # the discrete adjoint takes dPhi/dV from the slopes of the cubics: x_inf' and e' against
    # the same formed from the oracle's rate derivatives
    coef, vlo, pm = table
    dt = 0.025
    rng = np.random.default_rng(7)
    V = rng.uniform(vlo + 1e-6, vlo + coef.shape[0] / pm - 1e-6, 4000)
    t = (V - vlo) * pm
    i = np.floor(t).astype(np.int64)
    s = (t - i)[:, None]
    c = coef[i]
    slope = (3.0 * c[..., 3] * s + 2.0 * c[..., 2]) * s + c[..., 1]
    slope *= pm
    ref = np.zeros_like(slope)
    for k, v in enumerate(V):
        r = oracle_lib.hh_rates(v)
        dr = oracle_lib.hh_rate_derivs(v)
        for q in range(3):
            a, b, da, db = r[2 * q], r[2 * q + 1], dr[2 * q], dr[2 * q + 1]
            ref[k, 2 * q] = (da * b - a * db) / (a + b) ** 2
            ref[k, 2 * q + 1] = -dt * (da + db) * np.exp(-dt * (a + b))
    err = np.abs(slope - ref)
    assert err.max() <= 1e-11 * max(1.0, np.abs(ref).max()), err.max()
