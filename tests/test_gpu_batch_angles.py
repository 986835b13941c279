"""Per-instance contact-angle accuracy of the batched workload: all 256
sessile drops (sides 64..512, theta 30..150 degrees, viscosity ratio 1, 3 or
10; MRT, FP32) advance 10000 steps in one batched handle, in both g
storages (the compact one is the storage the bench times); the 16 smallest
domains are compared with the FP64 oracle's angles stored in
tests/golden/batch_angles.json (written by tests/golden/make_batch_angles.py,
which calls only the oracle).  Bar: 0.5 degrees.  A domain whose oracle run
went non-finite must be reported non-finite by the GPU statistics too.
Batched and single-domain results are bit-identical (test_gpu_parity), so
a per-domain launch loop has the same accuracy."""
import json
import os

import pytest

import lbinputs

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "batch_angles.json")


@pytest.fixture(scope="module")
def lbf():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_0812_1282_gb300 as m

    return m


def test_golden_present():
    assert os.path.exists(GOLDEN), "run tests/golden/make_batch_angles.py"


@pytest.mark.parametrize("compact", [False, True], ids=["full-g", "compact-g"])
@pytest.mark.parametrize("reading", ["literal", "relax"])
def test_batched_angles_match_oracle(lbf, reading, compact):
    with open(GOLDEN) as fh:
        gold = json.load(fh)
    specs = lbinputs.batch_specs()
    plist = [lbf.params(**lbinputs.BASE, collision="mrt", precision="fp32",
                        tau_alpha=s["tau_alpha"], tau_beta=s["tau_beta"],
                        h_bottom=lbf.lb_wetting_h(s["theta"]), h_top=0.0,
                        step2_relax_momentum=(reading == "relax"), compact_g=compact)
             for s in specs]
    batch = lbf.Batch(plist, [s["nx"] for s in specs], [s["ny"] for s in specs])
    for d, s in enumerate(specs):
        batch.init_drop(s["R"], s["cx"], s["cy"], dom=d)
    batch.step(gold["steps"])
    nonfinite = [d for d in range(len(specs)) if batch.stats(dom=d)["nonfinite"] > 0]
    print("%s compact=%s: %d of %d domains non-finite after %d steps"
          % (reading, compact, len(nonfinite), len(specs), gold["steps"]))
    worst = 0.0
    for rec in gold["domains"]:
        d, ref = rec["dom"], rec[reading]
        if ref["diverged"]:
            assert d in nonfinite, d
            continue
        assert d not in nonfinite, d
        th = batch.contact_angle(dom=d)[0]
        worst = max(worst, abs(th - ref["theta"]))
        assert abs(th - ref["theta"]) <= 0.5, (d, th, ref["theta"])
    print("%s compact=%s: worst angle error %.4f degrees over %d domains"
          % (reading, compact, worst, len(gold["domains"])))
    batch.close()
