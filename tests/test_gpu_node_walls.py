"""Node bounce-back on the GPU (class 8: wall nodes in the outer rows of a
walled domain, the full-way scheme of Fig. 4b read as in the oracle) against
the FP64 oracle: FP64 within 1e-12, FP32 phi and u within 1e-5 after 1000
steps; invalid maps are refused as the oracle refuses them."""
import numpy as np
import pytest

import lbinputs

pytestmark = pytest.mark.gpu
NODE_WALL = 8


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


def node_wall_map(nx, ny):
    cls = np.zeros((ny, nx), np.uint8)
    cls[0] = NODE_WALL
    cls[-1] = NODE_WALL
    return cls


def _kw(orc, coll, relax=False):
    return dict(collision=coll, tau_alpha=1.4, tau_beta=0.7, h_bottom=orc.wetting_h(60.0),
                h_top=orc.wetting_h(110.0), step2_relax_momentum=relax)


def _pair(lbf, orc, nx, ny, prec, kw, cls, hc, phi0):
    sim = lbf.Lattice(lbf.params(precision=prec, **kw), nx, ny)
    sim.set_geometry(cls, hc)
    sim.init_phi(phi0)
    ref = orc.OracleLattice(orc.params(**kw), nx, ny)
    ref.set_geometry(cls, hc)
    ref.init_phi(phi0)
    return sim, ref


@pytest.mark.parametrize("coll,relax", [("bgk", False), ("mrt", False), ("mrt", True)])
def test_fp64_node_walls_match_oracle(lbf, orc, coll, relax):
    """A drop on the bottom wall-node row plus a small block (the wall nodes
    and obstacles together): every population, wall nodes included, within
    1e-12 of the oracle after 300 steps."""
    nx, ny = 70, 34
    cls = node_wall_map(nx, ny)
    cls[14:20, 50:56] = 1
    hc = [0.0, orc.wetting_h(80.0)]
    x, y = np.meshgrid(np.arange(nx), np.arange(ny))
    phi0 = np.tanh((14.0 - np.hypot(x - 25.0, y - 0.5)) / np.sqrt(2.0))
    sim, ref = _pair(lbf, orc, nx, ny, "fp64", _kw(orc, coll, relax), cls, hc, phi0)
    f, g = sim.populations()
    assert np.abs(f - ref.f).max() <= 1e-14 and np.abs(g - ref.g).max() <= 1e-14
    sim.step(300)
    ref.step(300)
    f, g = sim.populations()
    live = cls != 1  # fluid and wall nodes (solid obstacle nodes hold the rest state)
    assert np.abs(f[:, live] - ref.f[:, live]).max() <= 1e-12
    assert np.abs(g[:, live] - ref.g[:, live]).max() <= 1e-12
    # the totals over all live nodes are conserved
    assert f[:, live].sum() == pytest.approx(ref.f[:, live].sum(), rel=1e-13)
    sim.close()


def test_fp32_node_walls_within_1e5_after_1000_steps(lbf, orc):
    nx, ny = 64, 30
    cls = node_wall_map(nx, ny)
    phi0 = lbinputs.smooth_random_field(nx, ny, 0.9, 17)
    kw = _kw(orc, "mrt")
    sim, ref = _pair(lbf, orc, nx, ny, "fp32", kw, cls, [0.0], phi0)
    sim.step(1000)
    ref.step(1000)
    _, phi, ux, uy, st = sim.moments()
    _, rphi, rux, ruy = ref.moments()
    fl = cls == 0
    assert np.abs(phi[fl] - rphi[fl]).max() <= 1e-5
    assert max(np.abs(ux[fl] - rux[fl]).max(), np.abs(uy[fl] - ruy[fl]).max()) <= 1e-5
    assert st["nonfinite"] == 0
    # wall nodes carry no fluid of their own: reported as zero
    assert np.all(phi[~fl] == 0.0)
    sim.close()


def test_invalid_node_wall_maps_are_refused(lbf, orc):
    nx, ny = 20, 10
    bad_row = node_wall_map(nx, ny)
    bad_row[4, 3] = NODE_WALL
    mirror_on_wall = node_wall_map(nx, ny)
    mirror_on_wall[2:4, 5:8] = 1
    for cls, walls in ((bad_row, True), (node_wall_map(nx, ny), False),
                       (mirror_on_wall, True)):
        sim = lbf.Lattice(lbf.params(precision="fp64", walls=walls), nx, ny)
        with pytest.raises(lbf.LBError) as e:
            sim.set_geometry(cls, [0.0, 0.1])
        assert e.value.code == lbf.LB_ERR_INVALID_ARG
        ref = orc.OracleLattice(orc.params(walls=walls), nx, ny)
        with pytest.raises(Exception):
            ref.set_geometry(cls, [0.0, 0.1])
        sim.close()
