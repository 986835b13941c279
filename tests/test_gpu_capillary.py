"""Capillary filling (Sec. VI) on the GPU against the FP64 oracle's run stored
in tests/golden/capillary_1000x120.json (written by
tests/golden/make_capillary_1000x120.py, which calls only the oracle): the
1000 x 120 set-up, 100000 steps, front position and advancing angle every
500 steps, both readings of the Step-2 momentum rates.

Bars: FP64 front within 1e-6 lattice units and angle within 1e-6 degrees at
every checkpoint; FP32 front within 0.1 lattice units and angle within 0.5
degrees.  A run whose oracle fields turned non-finite must turn non-finite
on the GPU as well, reported by the statistics."""
import json
import os

import pytest

import lbinputs

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "capillary_1000x120.json")


@pytest.fixture(scope="module")
def lbf():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_0812_1282_gb300 as m

    return m


def _runs():
    if not os.path.exists(GOLDEN):
        return []
    with open(GOLDEN) as fh:
        return json.load(fh)["runs"]


def test_golden_present():
    assert os.path.exists(GOLDEN), "run tests/golden/make_capillary_1000x120.py"


def _track(lbf, precision, relax, until):
    c = lbinputs.CAPILLARY_1000x120
    p = lbf.params(precision=precision, step2_relax_momentum=relax, **c["params"])
    sim = lbf.Lattice(p, c["nx"], c["ny"])
    sim.init_channel(c["res_len"], c["ch_w"], lbf.lb_wetting_h(c["theta"]), c["h_block"])
    y0 = (c["ny"] - c["ch_w"]) // 2
    out = []
    while sim.step_count < until:
        sim.step(c["every"])
        st = sim.stats()
        if st["nonfinite"]:
            out.append(None)
            break
        xf, th, _ = sim.meniscus(c["res_len"], c["nx"], y0, y0 + c["ch_w"])
        out.append((sim.step_count, xf, th))
    sim.close()
    return out


@pytest.mark.parametrize("run", _runs(), ids=lambda r: "relax" if r["step2_relax_momentum"]
                         else "literal")
@pytest.mark.parametrize("precision,tol_x,tol_th", [("fp64", 1e-6, 1e-6), ("fp32", 0.1, 0.5)])
def test_capillary_front_matches_oracle(lbf, run, precision, tol_x, tol_th):
    c = lbinputs.CAPILLARY_1000x120
    div = run["diverged_at"]
    until = div + 10 * c["every"] if div else c["steps"]
    got = _track(lbf, precision, run["step2_relax_momentum"], until)
    if div:
        assert got[-1] is None  # the GPU run goes non-finite too
        # compare well before the blow-up, where both runs are still smooth
        got = [g for g in got[:-1] if g[0] <= div - 10 * c["every"]]
    else:
        assert len(got) == len(run["t"])
    worst_x = worst_th = 0.0
    for (t, xf, th), t_ref, xf_ref, th_ref in zip(got, run["t"], run["x_front"], run["theta"]):
        assert t == t_ref
        worst_x = max(worst_x, abs(xf - xf_ref))
        worst_th = max(worst_th, abs(th - th_ref))
    print("%s %s: %d checkpoints, worst |dx_front| %.3e, worst |dtheta| %.3e"
          % (precision, "relax" if run["step2_relax_momentum"] else "literal", len(got),
             worst_x, worst_th))
    assert worst_x <= tol_x and worst_th <= tol_th
