"""GPU obstacle path (capillary filling, Sec. VI) against the FP64 oracle.

FP64: populations within 1e-12 of the oracle after hundreds of steps on a
block geometry (convex and concave corners, a gap) and on the capillary
set-up; FP32: phi and u within 1e-5 after 1000 steps.  The channel map the
library builds equals the oracle's own, bit for bit; an obstacle-free map
reproduces the staged plain kernel to rounding; a batch mixing plain and
obstacle domains is bit-identical to the domains stepped alone."""
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


def blocks_geometry(nx, ny):
    cls = np.zeros((ny, nx), np.uint8)
    cls[0:6, 8:14] = 1
    cls[10:16, 20:27] = 2
    cls[0:7, 30:34] = 3
    return cls


def max_diff(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max())


def _kw(orc, coll, relax=False, rule=0):
    return dict(collision=coll, tau_alpha=1.4, tau_beta=0.7, h_bottom=orc.wetting_h(65.0),
                h_top=orc.wetting_h(115.0), gamma_mob=0.3, step2_relax_momentum=relax,
                wetting_rule=rule)


@pytest.mark.parametrize("coll,relax,rule", [("bgk", False, 0), ("mrt", False, 0),
                                             ("mrt", True, 0), ("mrt", False, 1),
                                             ("bgk", False, 1)])
def test_fp64_blocks_match_oracle(lbf, orc, coll, relax, rule):
    nx, ny = 40, 24
    kw = _kw(orc, coll, relax, rule)
    cls = blocks_geometry(nx, ny)
    hc = [0.0, orc.wetting_h(50.0), orc.wetting_h(130.0), 0.1]
    phi0 = lbinputs.smooth_random_field(nx, ny, 0.9, 14)
    ref = orc.OracleLattice(orc.params(**kw), nx, ny)
    ref.set_geometry(cls, hc)
    ref.init_phi(phi0)
    sim = lbf.Lattice(lbf.params(precision="fp64", **kw), nx, ny)
    sim.set_geometry(cls, hc)
    assert np.array_equal(sim.geometry(), cls)
    sim.init_phi(phi0)
    f, g = sim.populations()
    assert max_diff(f, ref.f) <= 1e-14 and max_diff(g, ref.g) <= 1e-14
    for n in (1, 1, 50, 149):
        sim.step(n)
        ref.step(n)
    f, g = sim.populations()
    fl = cls == 0
    assert max_diff(f[:, fl], ref.f[:, fl]) <= 1e-12
    assert max_diff(g[:, fl], ref.g[:, fl]) <= 1e-12
    # solid nodes hold the rest state in both buffers
    assert max_diff(f[:, ~fl], ref.f[:, ~fl]) <= 1e-15 and max_diff(g[:, ~fl], 0.0) == 0.0
    rho, phi, ux, uy, st = sim.moments()
    assert np.all(rho[~fl] == 0.0) and np.all(phi[~fl] == 0.0)
    rrho, rphi, _, _ = ref.moments()
    assert st["mass"] == pytest.approx(rrho[fl].sum(), rel=1e-13)
    assert st["order"] == pytest.approx(rphi[fl].sum(), abs=1e-11)
    sim.close()


def test_channel_map_and_init_match_oracle(lbf, orc):
    nx, ny, res, w = 96, 40, 32, 12
    for prec, tol in (("fp64", 1e-14), ("fp32", 1e-7)):
        sim = lbf.Lattice(lbf.params(precision=prec, collision="mrt"), nx, ny)
        sim.init_channel(res, w, orc.wetting_h(60.0), 0.05)
        assert np.array_equal(sim.geometry(), orc.channel_geometry(nx, ny, res, w))
        ref = orc.OracleLattice(orc.params(collision="mrt"), nx, ny)
        ref.init_channel(res, w, orc.wetting_h(60.0), 0.05)
        f, g = sim.populations()
        assert max_diff(f, ref.f) <= tol and max_diff(g, ref.g) <= tol
        sim.close()


@pytest.mark.parametrize("relax", [False, True])
def test_fp64_channel_and_meniscus_match_oracle(lbf, orc, relax):
    nx, ny, res, w = 96, 40, 32, 12
    kw = dict(collision="mrt", tau_alpha=1.5, tau_beta=0.6, step2_relax_momentum=relax)
    sim = lbf.Lattice(lbf.params(precision="fp64", **kw), nx, ny)
    ref = orc.OracleLattice(orc.params(**kw), nx, ny)
    for lat in (sim, ref):
        lat.init_channel(res, w, orc.wetting_h(60.0), 0.0)
    sim.step(1500)
    ref.step(1500)
    f, g = sim.populations()
    fl = ref.cls == 0
    assert max_diff(f[:, fl], ref.f[:, fl]) <= 1e-12
    assert max_diff(g[:, fl], ref.g[:, fl]) <= 1e-12
    y0 = (ny - w) // 2
    xf, th, R = sim.meniscus(res, nx, y0, y0 + w)
    _, rphi, _, _ = ref.moments()
    rxf, rth, rR = orc.meniscus(rphi, ref.cls, res, nx, y0, y0 + w)
    assert xf == pytest.approx(rxf, abs=1e-8)
    assert th == pytest.approx(rth, abs=1e-7)
    assert xf > res  # the channel has started to fill
    sim.close()


def test_fp32_channel_within_1e5_after_1000_steps(lbf, orc):
    nx, ny, res, w = 96, 40, 32, 12
    kw = dict(collision="mrt", tau_alpha=1.5, tau_beta=0.6)
    sim = lbf.Lattice(lbf.params(precision="fp32", **kw), nx, ny)
    ref = orc.OracleLattice(orc.params(**kw), nx, ny)
    for lat in (sim, ref):
        lat.init_channel(res, w, orc.wetting_h(60.0), 0.0)
    sim.step(1000)
    ref.step(1000)
    _, phi, ux, uy, st = sim.moments()
    _, rphi, rux, ruy = ref.moments()
    fl = ref.cls == 0
    assert max_diff(phi[fl], rphi[fl]) <= 1e-5
    assert max_diff(ux[fl], rux[fl]) <= 1e-5 and max_diff(uy[fl], ruy[fl]) <= 1e-5
    assert st["nonfinite"] == 0
    sim.close()


@pytest.mark.parametrize("rule", [0, 1])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
def test_obstacle_free_map_equals_plain_kernel(lbf, orc, prec, tol, rule):
    """The obstacle kernel on an all-fluid map and the staged plain kernel
    compute the same arithmetic (the compiler may contract products into
    fused multiply-adds differently in the two kernels, so agreement is to
    rounding, not bitwise)."""
    nx, ny = 70, 33
    kw = dict(_kw(orc, "mrt", rule=rule), precision=prec)
    phi0 = lbinputs.smooth_random_field(nx, ny, 0.9, 21)
    a = lbf.Lattice(lbf.params(**kw), nx, ny)
    b = lbf.Lattice(lbf.params(**kw), nx, ny)
    b.set_geometry(np.zeros((ny, nx), np.uint8), [0.0])
    for s in (a, b):
        s.init_phi(phi0)
        s.step(77)
    fa, ga = a.populations()
    fb, gb = b.populations()
    print("%s: max |f diff| %.3e  max |g diff| %.3e" % (prec, max_diff(fa, fb), max_diff(ga, gb)))
    assert max_diff(fa, fb) <= tol and max_diff(ga, gb) <= tol
    a.close()
    b.close()


def test_mixed_batch_is_bitwise_equal_to_single_domains(lbf, orc):
    sizes = [(64, 40), (96, 40), (40, 24), (80, 50)]
    kws = [dict(collision="mrt", precision="fp32", tau_alpha=1.5, tau_beta=0.6,
                h_bottom=lbf.lb_wetting_h(t)) for t in (70.0, 90.0, 100.0, 120.0)]
    plist = [lbf.params(**k) for k in kws]

    def setup(lat, d, dom=0):
        nx, ny = sizes[d]
        if d == 1:
            lat.init_channel(32, 12, lbf.lb_wetting_h(60.0), 0.0, dom=dom)
        elif d == 2:
            lat.set_geometry(blocks_geometry(nx, ny), [0.0, 0.0, 0.1, -0.1], dom=dom)
            lat.init_phi(lbinputs.smooth_random_field(nx, ny, 0.9, 3), dom=dom)
        else:
            lat.init_drop(0.3 * nx, nx / 2, -0.5, dom=dom)

    batch = lbf.Batch(plist, [s[0] for s in sizes], [s[1] for s in sizes])
    for d in range(4):
        setup(batch, d, dom=d)
    batch.step(301)
    for d in range(4):
        sim = lbf.Lattice(plist[d], *sizes[d])
        setup(sim, d)
        sim.step(301)
        fs, gs = sim.populations()
        fb, gb = batch.populations(dom=d)
        assert np.array_equal(fs, fb) and np.array_equal(gs, gb), d
        sim.close()
    batch.close()


def test_geometry_errors(lbf):
    import paper_0812_1282_gb300 as m

    sim = lbf.Lattice(lbf.params(), 20, 12)
    cls = np.zeros((12, 20), np.uint8)
    cls[3:9, 5:8] = 1
    cls[3:9, 9:12] = 1  # one-node gap
    with pytest.raises(m.LBError):
        sim.set_geometry(cls, [0.0, 0.0])
    cls[:, 9:12] = 0
    with pytest.raises(m.LBError):
        sim.set_geometry(cls, [0.0])  # class 1 without a gradient
    with pytest.raises(m.LBError):
        sim.set_geometry(np.ones((12, 20), np.uint8), [0.0, 0.0])  # no fluid
    sim.set_geometry(cls, [0.0, 0.0])
    sim.set_geometry(None, None)
    assert not sim.geometry().any()
    sim.close()
    periodic = lbf.Lattice(lbf.params(walls=False), 40, 20)
    with pytest.raises(m.LBError):
        periodic.init_channel(10, 8, 0.0)
    periodic.close()


@pytest.mark.parametrize("walls,nx,ny,block", [(True, 13, 9, (3, 6, 4, 7)),
                                               (False, 11, 10, (2, 5, 3, 6)),
                                               (True, 37, 11, (4, 7, 30, 34))])
def test_small_obstacle_domains_match_oracle(lbf, orc, walls, nx, ny, block):
    """Obstacle domains narrower or shorter than the step's tile and its
    halos (a CTA covers 32 x 8 nodes plus three rings of phi), where the
    halos wrap around the lattice several times: FP64 within 1e-12 of the
    oracle."""
    kw = dict(_kw(orc, "mrt"), walls=walls)
    cls = np.zeros((ny, nx), np.uint8)
    y0, y1, x0, x1 = block
    cls[y0:y1, x0:x1] = 1
    hc = [0.0, orc.wetting_h(70.0)]
    phi0 = lbinputs.smooth_random_field(nx, ny, 0.9, 8)
    ref = orc.OracleLattice(orc.params(**kw), nx, ny)
    ref.set_geometry(cls, hc)
    ref.init_phi(phi0)
    sim = lbf.Lattice(lbf.params(precision="fp64", **kw), nx, ny)
    sim.set_geometry(cls, hc)
    sim.init_phi(phi0)
    sim.step(211)
    ref.step(211)
    f, g = sim.populations()
    fl = cls == 0
    assert max_diff(f[:, fl], ref.f[:, fl]) <= 1e-12
    assert max_diff(g[:, fl], ref.g[:, fl]) <= 1e-12
    sim.close()


def _persistent_case(lbf, orc, prec, nx, ny, walls, make_cls, node_walls=False):
    kw = dict(_kw(orc, "mrt"), walls=walls)
    cls = make_cls(nx, ny)
    hc = [0.0, orc.wetting_h(70.0), orc.wetting_h(110.0), 0.1]
    phi0 = lbinputs.smooth_random_field(nx, ny, 0.9, 21)
    out = []
    for persist, spl in ((0, 1), (1, 1), (0, 2)):
        sim = lbf.Lattice(lbf.params(precision=prec, **kw), nx, ny)
        sim.set_schedule(lbf.schedule(128, 16, ctas_per_sm=0, persist=persist,
                                      steps_per_launch=spl))
        sim.set_geometry(cls, hc)
        sim.init_phi(phi0)
        sim.step(131)  # a 64-step graph twice, a 2-step graph and one single step
        out.append(sim.populations())
        sim.close()
    return out


def _blocks(nx, ny):
    cls = np.zeros((ny, nx), np.uint8)
    cls[2:6, 8:14] = 1
    cls[ny - 7:ny - 3, nx // 2:nx // 2 + 5] = 2
    cls[ny // 2 - 1:ny // 2 + 2, 3:6] = 3
    return cls


def _node_walls(nx, ny):
    cls = np.zeros((ny, nx), np.uint8)
    cls[0] = 8
    cls[-1] = 8
    cls[4:8, 8:14] = 1
    cls[ny // 2 - 1:ny // 2 + 2, 30:36] = 2
    return cls


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("nx,ny,walls,cls_fn", [
    (40, 24, True, _blocks),
    (97, 25, False, _blocks),    # short last tiles in x and y: halos reach two tiles on
    (65, 17, False, _blocks),    # the far side of the periodic wrap
    (13, 9, True, lambda nx, ny: _small(nx, ny)),
    (200, 60, True, _node_walls),
    # FP32: 480 tiles, all resident; FP64 (two CTAs per SM): too many, so a
    # launch per step whatever the schedule says
    (1000, 120, True, _blocks),
])
def test_persistent_obstacle_steps_are_bitwise_equal(lbf, orc, prec, nx, ny, walls, cls_fn):
    """One cooperative launch of all of a domain's tiles per graph of steps,
    each tile waiting only for the tiles under its halo, and two steps per
    launch (each tile stepping a four-node halo first) give the state of a
    launch per step bit for bit: walls and periodic rows, tiles shorter than
    the halo, node walls, FP32 and FP64."""
    (f0, g0), (f1, g1), (f2, g2) = _persistent_case(lbf, orc, prec, nx, ny, walls, cls_fn)
    assert np.array_equal(f0, f1) and np.array_equal(g0, g1)
    assert np.array_equal(f0, f2) and np.array_equal(g0, g2)


def test_two_step_launches_switched_midrun_keep_the_state(lbf, orc):
    """A two-step launch flips the current buffer once: switching between
    one and two steps per launch mid-run, odd step counts and a checkpoint
    keep the run identical to one stepped a launch per step."""
    nx, ny = 200, 60
    kw = dict(_kw(orc, "mrt"), walls=True)
    cls = _node_walls(nx, ny)
    hc = [0.0, orc.wetting_h(70.0), orc.wetting_h(110.0)]
    phi0 = lbinputs.smooth_random_field(nx, ny, 0.9, 33)
    ref = lbf.Lattice(lbf.params(precision="fp32", **kw), nx, ny)
    ref.set_geometry(cls, hc)
    ref.init_phi(phi0)
    ref.step(200)
    sim = lbf.Lattice(lbf.params(precision="fp32", **kw), nx, ny)
    sim.set_geometry(cls, hc)
    sim.init_phi(phi0)
    two = lbf.schedule(128, 16, ctas_per_sm=0, steps_per_launch=2)
    one = lbf.schedule(128, 16, ctas_per_sm=0)
    sim.set_schedule(two)
    sim.step(67)
    sim.set_schedule(one)
    sim.step(3)
    blob = sim.save_state()
    sim.set_schedule(two)
    sim.step(11)
    sim.load_state(blob)
    sim.step(130)
    assert sim.step_count == ref.step_count == 200
    assert sim.save_state()[32:] == ref.save_state()[32:]
    sim.close()
    ref.close()


def _small(nx, ny):
    cls = np.zeros((ny, nx), np.uint8)
    cls[3:6, 4:7] = 1
    return cls


def test_capillary_autotune_keeps_state(lbf, orc):
    """The autotuner of a domain with obstacles times a launch per step
    against one persistent launch per graph and leaves the state alone."""
    sim = lbf.Lattice(lbf.params(precision="fp32", collision="mrt", tau_alpha=1.0, tau_beta=0.6),
                      300, 60)
    sim.init_channel(100, 20, orc.wetting_h(60.0), 0.05)
    sim.step(5)
    before = sim.save_state()
    sim.autotune(reps=1)
    assert sim.save_state() == before
    assert sim.schedule()["persist"] in (0, 1)
    sim.close()
