"""The 200x100 sessile-drop sweep (BGK; MRT with both readings of the Step-2
momentum rates; viscosity ratio 1 and 10; target angles 60, 90 and 120
degrees; 20000 steps) on the GPU in FP32 and FP64 against the FP64 oracle's
stored results (tests/golden/sweep_200x100.json, written by
tests/golden/make_sweep_200x100.py, which calls only the oracle).

FP32 runs in both g storages (full, and the compact form the bench times).
Bars: contact angle within 0.5 degrees (FP32) and 1e-6 degrees (FP64); the
spurious-current norm max |u| within 2 % (FP32).  A case whose oracle run
turned non-finite must turn non-finite on the GPU too (and be reported by the
statistics, not by a fault)."""
import json
import os

import numpy as np
import pytest

import lbinputs

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sweep_200x100.json")


@pytest.fixture(scope="module")
def lbf():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_0812_1282_gb300 as m

    return m


def _cases():
    if not os.path.exists(GOLDEN):
        return []
    with open(GOLDEN) as fh:
        return json.load(fh)["cases"]


def _id(c):
    name = c["collision"] + ("-relaxj" if c["step2_relax_momentum"] else "")
    return "%s-R%d-%g" % (name, c["ratio"], c["theta_target"])


def _run(lbf, case, precision, compact=False):
    c = lbinputs.SWEEP_200x100
    p = lbf.params(**lbinputs.BASE, precision=precision, collision=case["collision"],
                   tau_alpha=case["tau_alpha"], tau_beta=case["tau_beta"], h_bottom=case["h"],
                   h_top=0.0, step2_relax_momentum=case["step2_relax_momentum"],
                   compact_g=compact)
    sim = lbf.Lattice(p, c["nx"], c["ny"])
    try:
        sim.init_drop(c["R"], c["cx"], c["cy"])
        sim.step(c["steps"])
        _, _, ux, uy, st = sim.moments()
        if st["nonfinite"]:
            return None, None, st
        th = sim.contact_angle()[0]
        return th, float(np.hypot(ux, uy).max()), st
    finally:
        sim.close()


def test_golden_present():
    assert os.path.exists(GOLDEN), "run tests/golden/make_sweep_200x100.py"


@pytest.mark.parametrize("compact", [False, True], ids=["full-g", "compact-g"])
@pytest.mark.parametrize("case", _cases(), ids=_id)
def test_sweep_fp32_angle_within_half_degree(lbf, case, compact):
    """FP32 in both g storages (the compact one is the storage the bench
    times) against the FP64 oracle's 20000-step run."""
    th, umax, st = _run(lbf, case, "fp32", compact)
    if case["diverged_at"]:
        assert st["nonfinite"] > 0
        return
    print("%s compact=%s: oracle %.4f  gpu-fp32 %.4f  max|u| oracle %.3e gpu %.3e"
          % (_id(case), compact, case["theta"], th, case["max_u"], umax))
    assert st["nonfinite"] == 0
    assert abs(th - case["theta"]) <= 0.5
    assert umax == pytest.approx(case["max_u"], rel=0.02)


@pytest.mark.parametrize("case", [c for c in _cases() if c["theta_target"] == 120.0], ids=_id)
def test_sweep_fp64_matches_oracle(lbf, case):
    th, umax, st = _run(lbf, case, "fp64")
    if case["diverged_at"]:
        assert st["nonfinite"] > 0
        return
    assert st["nonfinite"] == 0
    assert abs(th - case["theta"]) <= 1e-6
    assert umax == pytest.approx(case["max_u"], rel=1e-9)
    assert st["mass"] == pytest.approx(case["mass"], rel=1e-12)
