"""lb_stats_noalloc against lb_moments.

Some callers cannot allocate device memory at the moment they want the
diagnostics -- for example an application whose own memory pool owns every
byte of the device, or a service that must keep a fixed memory footprint.
For them the library offers lb_stats_noalloc, whose scratch space is a fixed
device array inside the library instead of an allocation.  It must report
the same mass, order parameter, momentum and spurious-current norm as the
allocating path (lb_moments), also when called twice in a row on different
states (the scratch array is shared between calls).
"""
import ctypes

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


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_stats_noalloc_matches_lb_moments_on_two_calls(lbf, precision):
    import torch

    nx, ny = 77, 41
    p = lbf.params(precision=precision, collision="mrt", tau_alpha=1.5, tau_beta=0.6,
                   h_bottom=lbf.lb_wetting_h(60.0))
    sim = lbf.Lattice(p, nx, ny)
    sim.init_drop(15.0, 38.0, -0.5)
    dtype = torch.float64 if precision == "fp64" else torch.float32
    prec = lbf.LB_FP64 if precision == "fp64" else lbf.LB_FP32
    stream = torch.cuda.current_stream().cuda_stream
    for call, steps in enumerate((50, 87)):
        sim.step(steps)
        ref = sim.stats()                       # allocating path
        f, g = sim.populations()                # absolute populations, FP64 host arrays
        fd = torch.from_numpy(f).to("cuda", dtype)
        gd = torch.from_numpy(g).to("cuda", dtype)
        out = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
        lbf.lb_stats_noalloc(fd.data_ptr(), gd.data_ptr(), nx, ny, prec, out.data_ptr(), stream)
        torch.cuda.synchronize()
        mass, order, mx, my, umax, bad = out.cpu().numpy().tolist()
        if precision == "fp64":
            # same numbers, different summation order only
            assert mass == pytest.approx(ref["mass"], rel=1e-12), call
            assert order == pytest.approx(ref["order"], abs=1e-10), call
            assert mx == pytest.approx(ref["mom_x"], abs=1e-12), call
            assert my == pytest.approx(ref["mom_y"], abs=1e-12), call
            assert umax == pytest.approx(ref["max_u"], rel=1e-10), call
        else:
            # the FP32 input arrays round each absolute population (|f| < 1)
            # to 6e-8, which bounds the differences below
            assert mass == pytest.approx(ref["mass"], rel=1e-7), call
            assert order == pytest.approx(ref["order"], abs=1e-4), call
            assert mx == pytest.approx(ref["mom_x"], abs=1e-4), call
            assert my == pytest.approx(ref["mom_y"], abs=1e-4), call
            assert umax == pytest.approx(ref["max_u"], abs=1e-6), call
        assert bad == 0.0
    sim.close()


def test_stats_noalloc_rejects_bad_sizes(lbf):
    """Sizes beyond the stated maximum are refused before any device work."""
    import torch

    buf = torch.zeros(64, dtype=torch.float64, device="cuda")
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    with pytest.raises(lbf.LBError) as e:
        lbf.lb_stats_noalloc(buf.data_ptr(), buf.data_ptr(), 20000, 20000, lbf.LB_FP64,
                             out.data_ptr())
    assert e.value.code == lbf.LB_ERR_INVALID_ARG
    with pytest.raises(lbf.LBError):
        lbf.lb_stats_noalloc(buf.data_ptr(), buf.data_ptr(), 0, 4, lbf.LB_FP64, out.data_ptr())
    with pytest.raises(lbf.LBError):
        lbf.lb_stats_noalloc(buf.data_ptr(), buf.data_ptr(), 4, 4, 7, out.data_ptr())


def test_stats_noalloc_rejects_host_arrays(lbf):
    """Every array must be device memory of one device; a host array is
    refused before any launch."""
    import torch

    # populations of a uniform state at rest (rho = 1 at every node)
    dev = torch.full((9 * 16,), 1.0 / 9.0, dtype=torch.float64, device="cuda")
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    host = np.zeros(9 * 16)
    for args in ((dev.data_ptr(), host.ctypes.data, out.data_ptr()),
                 (dev.data_ptr(), dev.data_ptr(), host.ctypes.data),
                 (host.ctypes.data, dev.data_ptr(), out.data_ptr())):
        with pytest.raises(lbf.LBError) as e:
            lbf.lb_stats_noalloc(args[0], args[1], 4, 4, lbf.LB_FP64, args[2])
        assert e.value.code == lbf.LB_ERR_INVALID_ARG
    # a valid call afterwards still works (nothing was left half set up)
    lbf.lb_stats_noalloc(dev.data_ptr(), dev.data_ptr(), 4, 4, lbf.LB_FP64, out.data_ptr(),
                         torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    mass, order, mx, my, umax, bad = out.cpu().numpy().tolist()
    assert mass == pytest.approx(16.0, rel=1e-14) and umax == 0.0 and bad == 0.0
