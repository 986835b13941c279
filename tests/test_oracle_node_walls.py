"""Pins of the oracle's node bounce-back (Fig. 4b of the paper: the wall lies
on the boundary nodes; the paper gives no further detail).

Read as the full-way scheme: wall nodes (class 8 in rows 0 and ny - 1)
stream like fluid nodes, reverse every population instead of colliding, and
show their fluid neighbours the one-sided wetting value phi(x, 0) =
phi(x, 1) - h.  Pinned against what that scheme fixes independently of the
code: exact conservation of the totals (streaming and reversal only move
populations), a fluid at rest that stays at rest, the reversal itself on a
brute-force replay, the mirror symmetry of a symmetric channel, and the
hydrodynamic wall position of full-way bounce-back (no-slip planes half a
spacing inside the wall-node rows)."""
import math

import numpy as np
import pytest

import lbinputs

NODE_WALL = 8
EX = [0, 1, -1, 0, 0, 1, -1, -1, 1]
EY = [0, 0, 0, 1, -1, 1, -1, 1, -1]
OPP = [0, 2, 1, 4, 3, 6, 5, 8, 7]
# e_i -> e_i mirrored in y: 3<->4, 5<->8, 6<->7
MIRROR_Y = [0, 1, 2, 4, 3, 8, 7, 6, 5]


def node_wall_map(nx, ny):
    cls = np.zeros((ny, nx), np.uint8)
    cls[0] = NODE_WALL
    cls[-1] = NODE_WALL
    return cls


def _lattice(orc, nx, ny, coll="mrt", phi0=None, **kw):
    base = dict(tau_alpha=1.4, tau_beta=0.7, h_bottom=orc.wetting_h(65.0),
                h_top=orc.wetting_h(115.0), gamma_mob=0.3, collision=coll, walls=True)
    base.update(kw)
    lat = orc.OracleLattice(orc.params(**base), nx, ny)
    lat.set_geometry(node_wall_map(nx, ny), [0.0])
    lat.init_phi(phi0 if phi0 is not None else lbinputs.smooth_random_field(nx, ny, 0.9, 31))
    return lat


@pytest.mark.parametrize("coll", ["bgk", "mrt"])
def test_node_walls_conserve_the_totals(oracle_mod, coll):
    """Streaming and reversal permute populations and the fluid-node
    collisions conserve rho and phi, so the sums over all nodes (wall nodes
    included) are constant."""
    lat = _lattice(oracle_mod, 31, 17, coll)
    m0, p0 = lat.f.sum(), lat.g.sum()
    lat.step(400)
    assert lat.f.sum() == pytest.approx(m0, rel=1e-13)
    assert lat.g.sum() == pytest.approx(p0, abs=1e-10)
    assert np.isfinite(lat.f).all()


@pytest.mark.parametrize("coll", ["bgk", "mrt"])
def test_fluid_at_rest_stays_at_rest(oracle_mod, coll):
    """Uniform phi, no flow, neutral walls: every node holds its rest
    equilibrium, which the reversal leaves unchanged (it is parity
    symmetric), so nothing moves (to the rounding of the per-step sums)."""
    nx, ny = 12, 9
    lat = _lattice(oracle_mod, nx, ny, coll, phi0=np.full((ny, nx), 0.37), h_bottom=0.0,
                   h_top=0.0)
    f0, g0 = lat.f.copy(), lat.g.copy()
    lat.step(200)
    assert np.abs(lat.f - f0).max() <= 1e-13
    assert np.abs(lat.g - g0).max() <= 1e-13


def test_wall_nodes_reverse_their_pulled_populations(oracle_mod):
    """Brute-force replay of one step at the wall nodes: each stored
    population is the opposite one it pulled (a pull from beyond the lattice
    takes the node's own opposite population)."""
    nx, ny = 9, 7
    lat = _lattice(oracle_mod, nx, ny, "mrt")
    lat.step(3)
    f0, g0 = lat.f.copy(), lat.g.copy()
    lat.step(1)
    for y in (0, ny - 1):
        for x in range(nx):
            for i in range(9):
                j = OPP[i]  # the pulled population that becomes i
                sx, sy = (x - EX[j]) % nx, y - EY[j]
                if 0 <= sy < ny:
                    ef, eg = f0[j, sy, sx], g0[j, sy, sx]
                else:
                    ef, eg = f0[OPP[j], y, x], g0[OPP[j], y, x]
                assert lat.f[i, y, x] == ef and lat.g[i, y, x] == eg, (x, y, i)


def test_symmetric_channel_stays_mirror_symmetric(oracle_mod):
    """Equal wetting gradients at both node walls and a phi field symmetric
    about the channel centre: the run stays symmetric under y -> ny - 1 - y
    (with e_i mirrored), to rounding."""
    nx, ny = 20, 14
    h = oracle_mod.wetting_h(70.0)
    base = lbinputs.smooth_random_field(nx, ny, 0.9, 4)
    phi0 = 0.5 * (base + base[::-1])
    lat = _lattice(oracle_mod, nx, ny, "mrt", phi0=phi0, h_bottom=h, h_top=h)
    lat.step(300)
    fm = lat.f[MIRROR_Y][:, ::-1, :]
    gm = lat.g[MIRROR_Y][:, ::-1, :]
    assert np.abs(lat.f - fm).max() <= 1e-12
    assert np.abs(lat.g - gm).max() <= 1e-12


def _decay_rate(amps, ts):
    return -np.polyfit(ts, np.log(np.abs(amps)), 1)[0]


@pytest.mark.parametrize("tau", [0.8, 1.0, 1.5])
def test_full_way_wall_sits_half_a_spacing_inside(oracle_mod, tau):
    """Full-way bounce-back puts the no-slip planes halfway between the
    wall-node rows and the first fluid rows (the textbook result for the
    scheme): the lowest shear mode over the ny - 2 fluid rows,
    u_x = U sin(pi (y - 1/2) / (ny - 2)), decays at nu (pi / (ny - 2))^2,
    nu = (tau - 1/2)/3 (a = kappa = 0: plain D2Q9)."""
    nx, ny = 4, 42
    lat = _lattice(oracle_mod, nx, ny, "bgk", phi0=np.zeros((ny, nx)), a=0.0, kappa=0.0,
                   tau_alpha=tau, tau_beta=tau, h_bottom=0.0, h_top=0.0)
    L = ny - 2
    prof = np.sin(math.pi * (np.arange(ny) - 0.5) / L)
    p = lat.p
    for y in range(1, ny - 1):
        feq, geq = oracle_mod.node_equilibrium(p, 1.0, 0.0, 1e-4 * prof[y], 0.0, 0, 0, 0)
        lat.f[:, y, :] = feq[:, None]
        lat.g[:, y, :] = geq[:, None]
    lat.step(200)
    fl = np.arange(1, ny - 1)
    amps, ts = [], []
    for _ in range(10):
        lat.step(100)
        _, _, ux, _ = lat.moments()
        amps.append(ux[fl, 0] @ prof[fl] / (prof[fl] @ prof[fl]))
        ts.append(lat.t)
    nu = _decay_rate(np.array(amps), np.array(ts)) / (math.pi / L) ** 2
    assert nu == pytest.approx((tau - 0.5) / 3, rel=0.01)


def test_node_wall_maps_are_checked(oracle_mod):
    """Class 8 only in the outer rows of a walled lattice of at least four
    rows; an obstacle's mirror node may not be a wall node."""
    nx, ny = 12, 10
    p = oracle_mod.params(walls=True)
    lat = oracle_mod.OracleLattice(p, nx, ny)
    bad = node_wall_map(nx, ny)
    bad[4, 3] = NODE_WALL
    with pytest.raises(Exception):
        lat.set_geometry(bad, [0.0])
    q = oracle_mod.OracleLattice(oracle_mod.params(walls=False), nx, ny)
    with pytest.raises(Exception):
        q.set_geometry(node_wall_map(nx, ny), [0.0])
    near = node_wall_map(nx, ny)
    near[2:4, 5:8] = 1  # its mirror below is the wall-node row
    with pytest.raises(Exception):
        lat.set_geometry(near, [0.0, 0.1])
