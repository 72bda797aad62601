"""The library's FP64 elementary functions (arb_math_eval) against CUDA's exp/expm1 and
against the oracle's Hodgkin-Huxley rates (needs a B300); the table generator is checked on
CPU."""
import ctypes as C
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1901_07454_b300", "csrc")


def test_exp_table_header_is_what_the_generator_writes():
    r = subprocess.run([sys.executable, os.path.join(CSRC, "gen_exp_table.py")], capture_output=True, text=True,
                       check=True)
    with open(os.path.join(CSRC, "arb_exp_table.h")) as f:
        assert f.read() == r.stdout
    # spot values: 2^(1/2) and 2^(1/64), and the split of ln(2)/64
    assert "0x1.6a09e667f3bcdp+0" in r.stdout and "0x1.02c9a3e778061p+0" in r.stdout


def _eval(fn, x):
    import torch
    import paper_1901_07454_b300 as arb
    lib = arb.load()
    xt = torch.as_tensor(np.ascontiguousarray(x, np.float64), device="cuda")
    out = torch.empty(xt.numel() * (6 if fn == 2 else 1), dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream()
    rc = lib.arb_math_eval(fn, xt.numel(), C.c_void_p(xt.data_ptr()), C.c_void_p(out.data_ptr()),
                           C.c_void_p(s.cuda_stream))
    assert rc == 0, lib.arb_last_error(None)
    torch.cuda.synchronize()
    return xt, out


@pytest.mark.gpu
def test_table_exp_within_two_ulp_of_cuda_exp():
    import torch
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-30, 30, 400000), rng.uniform(-1e-3, 1e-3, 50000),
                        np.arange(-20, 21) * np.log(2) / 64, [0.0, -0.0, 1e-300, -700.0 + 1, 699.0]])
    xt, y = _eval(0, x)
    ref = torch.exp(xt)
    ulp = torch.abs(y - ref) / torch.from_numpy(np.spacing(np.abs(ref.cpu().numpy()))).cuda()
    assert float(ulp.max()) <= 2.0, float(ulp.max())   # each within about an ulp of exp


@pytest.mark.gpu
def test_expm1_and_hh_rates():
    import torch
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-15, 15, 200000), rng.uniform(-0.2, 0.2, 50000), [0.0, 0.1, -0.1]])
    xt, y = _eval(1, x)
    ref = torch.expm1(xt)
    rel = torch.abs(y - ref) / torch.clamp(torch.abs(ref), min=1e-300)
    # for |x| >= 0.1 the difference exp(x) - 1 loses log2(e^x / |e^x - 1|) <= 3.4 bits
    assert float(rel.max()) <= 5e-15, float(rel.max())
    # the FP64 rates as the kernels compute them, against the oracle's direct formulas
    oracle.build()
    v = np.concatenate([np.linspace(-120.0, 60.0, 20001), [-40.0, -55.0, -35.0, -65.0, -40.0 + 1e-9]])
    _, r = _eval(2, v)
    r = r.cpu().numpy().reshape(-1, 6)
    ro = np.array([oracle.hh_rates(x) for x in v])
    assert np.max(np.abs(r - ro) / np.abs(ro)) <= 1e-14
