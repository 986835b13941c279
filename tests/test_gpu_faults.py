"""Failure detection on the GPU without faulting it.

The step kernel's producer / consumer pipeline waits on mbarriers; each wait
is bounded in wall time and reports through a device error word.  Here a
warp waits on a barrier that nothing completes: the wait must give up
within its bound, the host must see LB_ERR_TIMEOUT, and the context must
stay usable afterwards.  Invalid host input must never reach the device.
"""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbf():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_0812_1282_gb300 as m

    return m


def test_bounded_wait_gives_up_and_reports(lbf):
    import torch

    stream = torch.cuda.current_stream().cuda_stream
    t0 = time.time()
    rc = lbf.lb_check_wait_timeout(stream)
    dt = time.time() - t0
    assert rc == lbf.LB_ERR_TIMEOUT
    assert dt < 10.0
    # the context is still usable: a lattice steps and reports finite moments
    sim = lbf.Lattice(lbf.params(precision="fp32", collision="mrt", tau_alpha=1.5, tau_beta=0.6),
                      64, 32)
    sim.init_drop(10.0, 32.0, -0.5)
    sim.step(20)
    sim.sync()
    st = sim.stats()
    assert st["nonfinite"] == 0 and np.isfinite(st["mass"])


def test_nonfinite_state_is_reported(lbf):
    """A NaN planted in the populations (host side) is counted by the
    diagnostics and surfaces as LB_ERR_NONFINITE, not as a device fault."""
    sim = lbf.Lattice(lbf.params(precision="fp64"), 40, 20)
    sim.init_drop(8.0, 20.0, -0.5)
    f, g = sim.populations()
    f[3, 10, 7] = np.nan
    sim.set_populations(f, g)
    _, _, _, _, st = sim.moments()
    assert st["nonfinite"] >= 1
    sim.step(2)
    _, _, _, _, st = sim.moments()
    assert st["nonfinite"] >= 1
