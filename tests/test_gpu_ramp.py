"""Quasi-static ramp of the wetting gradient (Sec. IV): the paper equilibrates
a drop at h = 0 and then changes h slowly, reading the angle along the way,
and finds MRT on the curve of Eq. (theory) while BGK at viscosity ratio 12.5
reads too high.

- lb_set_wetting changes h between steps with the state kept: FP64 parity
  with the oracle (whose parameters change at the same steps) to 1e-12.
- A shortened ramp of the paper's set-up (300 x 100, R = 35, Gamma = 0.5,
  tau 3 / 0.7, 3e4 steps at h = 0, then h lowered to h(50 deg) over 3e5
  steps): MRT within 3 degrees of Eq. (theory) along the way, BGK at least
  3 degrees further above it than MRT between 60 and 85 degrees."""
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


@pytest.fixture(scope="module")
def orc():
    import oracle

    oracle.build()
    return oracle


@pytest.mark.parametrize("coll", ["bgk", "mrt"])
def test_set_wetting_matches_oracle(lbf, orc, coll):
    nx, ny = 96, 40
    kw = dict(collision=coll, tau_alpha=3.0, tau_beta=0.7, gamma_mob=0.5)
    sim = lbf.Lattice(lbf.params(precision="fp64", **kw), nx, ny)
    ref = orc.OracleLattice(orc.params(**kw), nx, ny)
    sim.init_drop(18.0, 48.0, -0.5)
    ref.init_drop(18.0, 48.0, -0.5)
    for hb, ht in ((orc.wetting_h(70.0), 0.0), (orc.wetting_h(110.0), orc.wetting_h(80.0)),
                   (0.0, 0.0)):
        sim.set_wetting(hb, ht)
        ref.p.h_bottom, ref.p.h_top = hb, ht
        sim.step(201)
        ref.step(201)
    f, g = sim.populations()
    assert np.abs(f - ref.f).max() <= 1e-12 and np.abs(g - ref.g).max() <= 1e-12
    sim.close()


def _ramp(lbf, orc, coll, theta_end=50.0, n_eq=30000, n_ramp=300000, every=1000, meas=30000):
    p = lbf.params(a=0.04, kappa=0.04, gamma_mob=0.5, tau_alpha=3.0, tau_beta=0.7,
                   collision=coll, precision="fp32")
    sim = lbf.Lattice(p, 300, 100)
    sim.init_drop(35.0, 150.0, -0.5)
    sim.step(n_eq)
    h_end = lbf.lb_wetting_h(theta_end)
    out = []
    t = 0
    while t < n_ramp:
        sim.step(every)
        t += every
        h = h_end * t / n_ramp
        sim.set_wetting(h, 0.0)
        if t % meas == 0:
            assert sim.stats()["nonfinite"] == 0
            out.append((orc.theta_from_h(h), sim.contact_angle()[0]))
    sim.close()
    return out


def test_ramp_mrt_follows_theory_bgk_reads_high(lbf, orc):
    mrt = _ramp(lbf, orc, "mrt")
    bgk = _ramp(lbf, orc, "bgk")
    for (th, m), (_, b) in zip(mrt, bgk):
        print("theory %.2f  mrt %.2f  bgk %.2f" % (th, m, b))
    for th, m in mrt:
        assert abs(m - th) <= 3.0, (th, m)
    for (th, m), (_, b) in zip(mrt, bgk):
        if 60.0 <= th <= 85.0:
            assert b - th >= (m - th) + 3.0, (th, m, b)
