"""Compact g storage (FP32, tau_phi = 1): the state keeps phi, Gamma mu and
u_eq per node instead of nine g values (the post-collision g is the
equilibrium they fix, Eq. gevo and Appendix A).  Same method, other
rounding, so the FP32 bars against the FP64 oracle apply unchanged:
phi and u within 1e-5 after 1000 steps; reconstructed populations of one
step at full size within 2e-6 of the oracle's step from the same state.
Launch shape does not change the bits; a batch equals its domains stepped
alone."""
import numpy as np
import pytest

import lbinputs

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


def max_diff(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max())


def pair(lbf, orc, nx, ny, **kw):
    sim = lbf.Lattice(lbf.params(precision="fp32", compact_g=True, **kw), nx, ny)
    ref = orc.OracleLattice(orc.params(**kw), nx, ny)
    return sim, ref


@pytest.mark.parametrize("coll,taus,relax", [("bgk", (1.0, 1.0), False),
                                             ("mrt", (1.5, 0.6), False),
                                             ("mrt", (1.5, 0.6), True),
                                             ("bgk", (1.5, 0.6), False)])
@pytest.mark.parametrize("theta", [60.0, 120.0])
def test_compact_phi_within_1e5_after_1000_steps(lbf, orc, coll, taus, relax, theta):
    c = lbinputs.SWEEP_200x100
    kw = dict(lbinputs.BASE, collision=coll, tau_alpha=taus[0], tau_beta=taus[1],
              h_bottom=orc.wetting_h(theta), h_top=0.0, step2_relax_momentum=relax)
    sim, ref = pair(lbf, orc, c["nx"], c["ny"], **kw)
    sim.init_drop(c["R"], c["cx"], c["cy"])
    ref.init_drop(c["R"], c["cx"], c["cy"])
    f, g = sim.populations()
    assert max_diff(f, ref.f) <= 1e-7 and max_diff(g, ref.g) <= 1e-7
    sim.step(1000)
    ref.step(1000)
    _, phi, ux, uy, st = sim.moments()
    _, rphi, rux, ruy = ref.moments()
    assert max_diff(phi, rphi) <= 1e-5
    assert max_diff(ux, rux) <= 1e-5 and max_diff(uy, ruy) <= 1e-5
    assert st["nonfinite"] == 0
    sim.close()


def test_compact_agrees_with_full_storage(lbf, orc):
    """Both FP32 storages of the same scheme after 500 steps of a spinodal
    start (rounding-level differences only)."""
    n = 256
    c = lbinputs.SPINODAL_8192
    a = lbf.Lattice(lbf.params(precision="fp32", **c["params"]), n, n)
    b = lbf.Lattice(lbf.params(precision="fp32", compact_g=True, **c["params"]), n, n)
    for s in (a, b):
        s.init_random(c["amp"], c["seed"])
        s.step(500)
    fa, ga = a.populations()
    fb, gb = b.populations()
    assert max_diff(fa, fb) <= 1e-6 and max_diff(ga, gb) <= 1e-6
    sa, sb = a.stats(), b.stats()
    assert sb["mass"] == pytest.approx(sa["mass"], rel=1e-9)
    assert sb["order"] == pytest.approx(sa["order"], abs=1e-4)
    a.close()
    b.close()


@pytest.mark.parametrize("nx,ny,walls", [(3, 3, True), (37, 5, True), (129, 67, False),
                                         (130, 66, True), (33, 4, False), (200, 9, False)])
def test_compact_ragged_sizes_and_tile_independence(lbf, orc, nx, ny, walls):
    kw = dict(collision="mrt", tau_alpha=1.5, tau_beta=0.6, walls=walls,
              h_bottom=orc.wetting_h(70.0), h_top=orc.wetting_h(100.0))
    phi0 = lbinputs.smooth_random_field(nx, ny, 0.9, 5)
    ref = orc.OracleLattice(orc.params(**kw), nx, ny)
    ref.init_phi(phi0)
    ref.step(40)
    outs = []
    for bx, rows in [(32, 1), (64, 3), (128, 7), (256, 128), (96, 2), (128, 16)]:
        sim = lbf.Lattice(lbf.params(precision="fp32", compact_g=True, **kw), nx, ny)
        sim.set_tile(bx, rows)
        sim.init_phi(phi0)
        sim.step(40)
        outs.append(sim.save_state())
        f, g = sim.populations()
        assert max_diff(f, ref.f) <= 1e-6 and max_diff(g, ref.g) <= 1e-6, (bx, rows)
        sim.close()
    assert all(o == outs[0] for o in outs[1:])


@pytest.mark.parametrize("walls,rule", [(True, 0), (False, 0), (True, 1)])
def test_compact_batch_is_bitwise_equal_to_single_domains(lbf, walls, rule):
    specs = lbinputs.batch_specs(n=12, seed=7, lo=40, hi=200)
    plist = [lbf.params(**lbinputs.BASE, collision="mrt", precision="fp32", compact_g=True,
                        tau_alpha=s["tau_alpha"], tau_beta=s["tau_beta"], walls=walls,
                        h_bottom=lbf.lb_wetting_h(s["theta"]), wetting_rule=rule)
             for s in specs]
    batch = lbf.Batch(plist, [s["nx"] for s in specs], [s["ny"] for s in specs])
    batch.set_tile(128, 8)
    for d, s in enumerate(specs):
        batch.init_drop(s["R"], s["cx"], s["cy"], dom=d)
    batch.step(123)
    for d, s in enumerate(specs):
        sim = lbf.Lattice(plist[d], s["nx"], s["ny"])
        sim.init_drop(s["R"], s["cx"], s["cy"])
        sim.step(123)
        fs, gs = sim.populations()
        fb, gb = batch.populations(dom=d)
        assert np.array_equal(fs, fb) and np.array_equal(gs, gb), d
        sim.close()
    batch.close()


def test_compact_checkpoint_angle_and_refusals(lbf, orc):
    import paper_0812_1282_gb300 as m

    kw = dict(collision="mrt", tau_alpha=1.5, tau_beta=0.6, h_bottom=orc.wetting_h(60.0))
    sim, ref = pair(lbf, orc, 200, 100, **kw)
    sim.init_drop(40.0, 100.0, -0.5)
    ref.init_drop(40.0, 100.0, -0.5)
    sim.step(700)
    blob = sim.save_state()
    sim.step(300)
    a = sim.save_state()
    sim.load_state(blob)
    sim.step(300)
    assert sim.save_state()[32:] == a[32:]
    ref.step(1000)
    _, rphi, _, _ = ref.moments()
    assert sim.contact_angle()[0] == pytest.approx(orc.contact_angle(rphi)[0], abs=0.01)
    f, g = sim.populations()
    with pytest.raises(m.LBError):
        sim.set_populations(f, g)
    with pytest.raises(m.LBError):
        sim.set_geometry(np.zeros((100, 200), np.uint8), [0.0])
    sim.close()
    with pytest.raises(m.LBError):
        lbf.Lattice(lbf.params(precision="fp64", compact_g=True), 40, 20)
    with pytest.raises(m.LBError):
        lbf.Lattice(lbf.params(precision="fp32", compact_g=True, tau_phi=0.8), 40, 20)


def test_compact_full_size_8192_sampled_windows(lbf, orc):
    """One step of the 8192^2 FP32 MRT workload with compact storage in the
    benchmark's launch shape: sampled windows recomputed by the oracle from
    the GPU's own (reconstructed) state, plus global conservation."""
    c = lbinputs.SPINODAL_8192
    n = c["nx"]
    sim = lbf.Lattice(lbf.params(precision="fp32", compact_g=True, **c["params"]), n, n)
    sim.init_random(c["amp"], c["seed"])
    sim.step(3)
    st0 = sim.stats()
    windows = [(0, 64, 0, 3), (n - 64, n, n - 3, n), (4000, 4100, 4000, 4004), (n - 40, n, 0, 2),
               (0, 40, n - 2, n)]
    bands = []
    for (x0, x1, y0, y1) in windows:
        b0, b1 = max(0, y0 - 2), min(n, y1 + 2)
        bands.append((b0, *sim.populations_rows(b0, b1 - b0)))
    sim.step(1)
    st1 = sim.stats()
    op = orc.params(**c["params"])
    for (x0, x1, y0, y1), (b0, fb, gb) in zip(windows, bands):
        fo, go = orc.step_window(op, n, n, b0, fb, gb, x0, x1, y0, y1)
        f1, g1 = sim.populations_rows(y0, y1 - y0)
        assert max_diff(f1[:, :, x0:x1], fo) <= 2e-6
        assert max_diff(g1[:, :, x0:x1], go) <= 2e-6
    assert abs(st1["mass"] - st0["mass"]) <= 1e-9 * st0["mass"]
    assert abs(st1["order"] - st0["order"]) <= 1e-9 * st0["mass"]
    sim.close()
