"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: printed
numbers, closed forms derived independently, exact identities of the scheme,
or long-wavelength hydrodynamic limits.  A dropped term, a wrong sign, a
transposed stencil or a misplaced wall fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import lbinputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EX = np.array([0, 1, -1, 0, 0, 1, -1, -1, 1], dtype=float)
EY = np.array([0, 0, 0, 1, -1, 1, -1, 1, -1], dtype=float)


def _read_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# --------------------------------------------------------------- inputs
def test_splitmix64_reference_vector(oracle_mod):
    """Published SplitMix64 outputs; both generators (oracle C and the shared
    numpy input module) must reproduce them."""
    for seed, k, out in _read_table("splitmix64.txt"):
        assert oracle_mod.splitmix64(int(seed), int(k)) == int(out)
        assert int(lbinputs.splitmix64(int(seed), int(k))) == int(out)


def test_random_field_matches_input_module(oracle_mod):
    a = oracle_mod.phi_random(37, 11, 0.1, 12345)
    b = lbinputs.random_field(37, 11, 0.1, 12345)
    assert np.array_equal(a, b)
    assert a.min() >= -0.1 and a.max() < 0.1
    assert abs(a.mean()) < 0.02


def test_paper_printed_constants():
    """W = 2 sqrt(2 kappa/a) = 2.8, gamma = sqrt(8 kappa a/9) = 0.038 and
    R_nu = 12.5, as printed in Sec. IV (values rounded as printed)."""
    tab = {r[0]: float(r[1]) for r in _read_table("paper_constants.txt")}
    a = kappa = 0.04
    assert round(2 * math.sqrt(2 * kappa / a), 1) == tab["interface_width_W"]
    assert round(math.sqrt(8 * kappa * a / 9), 3) == tab["interfacial_tension_gamma"]
    assert (3 - 0.5) / (0.7 - 0.5) == pytest.approx(tab["viscosity_ratio_R_nu"])


# ---------------------------------------------------------- MRT matrix
def test_mrt_rows_are_moment_polynomials(oracle_mod):
    """Each printed row of Eq. (Matrix) is a velocity-moment polynomial of the
    standard D2Q9 moment basis (density, energy, energy squared, momentum,
    heat flux, stress): rebuild it from e_i and compare."""
    M, Minv = oracle_mod.mrt_matrix()
    e2 = EX ** 2 + EY ** 2
    basis = np.stack([
        np.ones(9),
        3 * e2 - 4,
        4.5 * e2 ** 2 - 10.5 * e2 + 4,
        EX,
        (3 * e2 - 5) * EX,
        EY,
        (3 * e2 - 5) * EY,
        EX ** 2 - EY ** 2,
        EX * EY,
    ])
    assert np.array_equal(M, basis)
    assert np.allclose(M @ M.T, np.diag(np.diag(M @ M.T)))  # mutually orthogonal rows
    assert np.allclose(Minv @ M, np.eye(9), atol=1e-15)
    assert np.allclose(M @ Minv, np.eye(9), atol=1e-15)


def _random_node_state(rng, oracle_mod, p):
    rho = 1.0 + 0.05 * rng.standard_normal()
    phi = rng.uniform(-1.2, 1.2)
    ux, uy = 0.05 * rng.standard_normal(2)
    dx, dy, lap = 0.3 * rng.standard_normal(3)
    feq, geq = oracle_mod.node_equilibrium(p, rho, phi, ux, uy, dx, dy, lap)
    f = feq + 1e-3 * rng.standard_normal(9)
    # keep rho and j of f equal to those of feq (what a real node has)
    M, Minv = oracle_mod.mrt_matrix()
    m = M @ f
    meq = M @ feq
    m[[0, 3, 5]] = meq[[0, 3, 5]]
    f = Minv @ m
    return f, feq


def test_mrt_with_all_rates_equal_is_bgk(oracle_mod):
    """S = omega * I gives M^-1 S M = omega I: MRT must equal BGK (Sec. III.B)."""
    rng = np.random.default_rng(1)
    pm = oracle_mod.params(collision="mrt", mrt_all_rates=True)
    pb = oracle_mod.params(collision="bgk")
    for _ in range(20):
        f, feq = _random_node_state(rng, oracle_mod, pb)
        f = f + 1e-3 * rng.standard_normal(9)  # also off the conserved manifold
        omega = rng.uniform(0.3, 1.9)
        assert np.allclose(oracle_mod.node_collide_f(pm, f, feq, omega),
                           oracle_mod.node_collide_f(pb, f, feq, omega),
                           atol=1e-15, rtol=0)


def test_mrt_relaxes_each_moment_at_its_rate(oracle_mod):
    """Eq. (diag): conserved moments untouched, ghost moments (rows 1, 2, 4,
    6) relax fully (rate 1), stress moments (rows 7, 8) relax at omega."""
    rng = np.random.default_rng(2)
    p = oracle_mod.params(collision="mrt")
    M, _ = oracle_mod.mrt_matrix()
    for _ in range(20):
        f, feq = _random_node_state(rng, oracle_mod, p)
        f = f + 1e-4 * rng.standard_normal(9)
        omega = rng.uniform(0.3, 1.9)
        fo = oracle_mod.node_collide_f(p, f, feq, omega)
        m, meq, mo = M @ f, M @ feq, M @ fo
        for k in (0, 3, 5):
            assert mo[k] == pytest.approx(m[k], abs=1e-15)
        for k in (1, 2, 4, 6):
            assert mo[k] == pytest.approx(meq[k], abs=1e-14)
        for k in (7, 8):
            assert mo[k] == pytest.approx(m[k] - omega * (m[k] - meq[k]), abs=1e-14)


def test_step2_boundary_collision_moments(oracle_mod):
    """Step 2 zeroes the equilibrium velocity at boundary nodes.  With MRT the
    momentum rows have S = 0, so the post-collision momentum equals the
    pre-collision one; with BGK it decays by (1 - omega)."""
    rng = np.random.default_rng(3)
    M, _ = oracle_mod.mrt_matrix()
    for coll in ("mrt", "bgk"):
        p = oracle_mod.params(collision=coll)
        for _ in range(10):
            rho = 1.0 + 0.01 * rng.standard_normal()
            phi = rng.uniform(-1, 1)
            u = 0.02 * rng.standard_normal(2)
            d = 0.2 * rng.standard_normal(3)
            feq_true, _ = oracle_mod.node_equilibrium(p, rho, phi, u[0], u[1], *d)
            feq0, _ = oracle_mod.node_equilibrium(p, rho, phi, 0.0, 0.0, *d)
            f = feq_true + 1e-4 * rng.standard_normal(9)
            m = M @ f
            m[[0, 3, 5]] = (M @ feq_true)[[0, 3, 5]]
            f = np.linalg.solve(M, m)
            omega = rng.uniform(0.5, 1.8)
            fo = oracle_mod.node_collide_f(p, f, feq0, omega)
            j, jo = (M @ f)[[3, 5]], (M @ fo)[[3, 5]]
            if coll == "mrt":
                assert np.allclose(jo, j, atol=1e-15)
            else:
                assert np.allclose(jo, (1 - omega) * j, atol=1e-15)


def test_step2_relax_momentum_reading(oracle_mod):
    """Alternative reading of Eq. (diag) on Step-2 nodes: the two momentum
    rows relax at rate 1, so the node leaves the collision with zero momentum
    (the no-slip condition Step 2 is said to express), while rho is conserved
    and the non-conserved moments are exactly those of the literal reading.
    Away from Step-2 nodes the flag changes nothing."""
    rng = np.random.default_rng(31)
    M, _ = oracle_mod.mrt_matrix()
    lit = oracle_mod.params(collision="mrt")
    alt = oracle_mod.params(collision="mrt", step2_relax_momentum=True)
    for _ in range(20):
        rho = 1.0 + 0.01 * rng.standard_normal()
        phi = rng.uniform(-1, 1)
        u = 0.02 * rng.standard_normal(2)
        d = 0.2 * rng.standard_normal(3)
        feq_true, _ = oracle_mod.node_equilibrium(lit, rho, phi, u[0], u[1], *d)
        feq0, _ = oracle_mod.node_equilibrium(lit, rho, phi, 0.0, 0.0, *d)
        f = feq_true + 1e-3 * rng.standard_normal(9)
        m = M @ f
        m[[0, 3, 5]] = (M @ feq_true)[[0, 3, 5]]
        f = np.linalg.solve(M, m)
        omega = rng.uniform(0.5, 1.8)
        fl = oracle_mod.node_collide_f(lit, f, feq0, omega, step2_node=True)
        fa = oracle_mod.node_collide_f(alt, f, feq0, omega, step2_node=True)
        ml, ma = M @ fl, M @ fa
        assert abs(ma[0] - rho) < 1e-14
        assert np.allclose(ma[[3, 5]], 0.0, atol=1e-16)
        assert np.allclose(ml[[3, 5]], (M @ f)[[3, 5]], atol=1e-15)
        keep = [0, 1, 2, 4, 6, 7, 8]
        assert np.allclose(ma[keep], ml[keep], atol=1e-15)
        # interior node: identical
        fi = oracle_mod.node_collide_f(alt, f, feq_true, omega, step2_node=False)
        assert np.array_equal(fi, oracle_mod.node_collide_f(lit, f, feq_true, omega))


# ------------------------------------------------------- equilibria
def test_equilibrium_moments_reproduce_pressure_tensor(oracle_mod):
    """Appendix A: the equilibria are built so that sum f = rho,
    sum f e = rho u, sum f e e = P + rho u u with P of Eq. (pressten) and p0
    of Eq. (p0); sum g = phi, sum g e = phi u, sum g e e = Gamma mu I + phi u u
    with mu of Eq. (chempot)."""
    rng = np.random.default_rng(4)
    p = oracle_mod.params(a=0.037, kappa=0.051, gamma_mob=0.3)
    for _ in range(50):
        rho = 1 + 0.1 * rng.standard_normal()
        phi = rng.uniform(-1.3, 1.3)
        u = 0.1 * rng.standard_normal(2)
        d = 0.4 * rng.standard_normal(2)
        lap = 0.4 * rng.standard_normal()
        feq, geq = oracle_mod.node_equilibrium(p, rho, phi, u[0], u[1], d[0], d[1], lap)
        E = np.stack([EX, EY])
        a, kappa = p.a, p.kappa
        p0 = rho / 3 + a * (-0.5 * phi ** 2 + 0.75 * phi ** 4)
        P = (p0 - kappa * phi * lap - 0.5 * kappa * (d @ d)) * np.eye(2) + kappa * np.outer(d, d)
        mu = a * (-phi + phi ** 3) - kappa * lap
        assert feq.sum() == pytest.approx(rho, abs=1e-14)
        assert np.allclose(E @ feq, rho * u, atol=1e-14)
        assert np.allclose((E * feq) @ E.T, P + rho * np.outer(u, u), atol=1e-14)
        assert geq.sum() == pytest.approx(phi, abs=1e-14)
        assert np.allclose(E @ geq, phi * u, atol=1e-14)
        assert np.allclose((E * geq) @ E.T, p.gamma_mob * mu * np.eye(2) + phi * np.outer(u, u),
                           atol=1e-14)


def test_equilibrium_reduces_to_standard_d2q9(oracle_mod):
    """With a = kappa = 0 the equilibrium is the textbook D2Q9 one,
    t_i rho (1 + 3 e.u + 9/2 (e.u)^2 - 3/2 u^2), t = 4/9, 1/9, 1/36."""
    p = oracle_mod.params(a=0.0, kappa=0.0)
    t = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    rng = np.random.default_rng(5)
    for _ in range(10):
        rho = 1 + 0.1 * rng.standard_normal()
        u = 0.1 * rng.standard_normal(2)
        feq, _ = oracle_mod.node_equilibrium(p, rho, 0.3, u[0], u[1], 0.1, 0.2, 0.3)
        eu = EX * u[0] + EY * u[1]
        ref = t * rho * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * (u @ u))
        assert np.allclose(feq, ref, atol=1e-15)


# -------------------------------------------------------- stencils
def test_stencils_exact_on_quadratics(oracle_mod):
    """Eq. (best): the 1/12 gradient and 1/6 Laplacian are exact for
    quadratic fields (checked away from the periodic seam)."""
    p = oracle_mod.params(walls=False)
    ny, nx = 12, 14
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    c = [0.3, -0.7, 0.2, 0.11, -0.05, 0.07]
    phi = c[0] + c[1] * x + c[2] * y + c[3] * x * x + c[4] * y * y + c[5] * x * y
    dx, dy, lap = oracle_mod.phi_derivatives(p, phi)
    s = (slice(1, ny - 1), slice(1, nx - 1))
    assert np.allclose(dx[s], (c[1] + 2 * c[3] * x + c[5] * y)[s], atol=1e-13)
    assert np.allclose(dy[s], (c[2] + 2 * c[4] * y + c[5] * x)[s], atol=1e-13)
    assert np.allclose(lap[s], 2 * c[3] + 2 * c[4], atol=1e-13)


def test_stencil_fourier_symbols(oracle_mod):
    """On a periodic lattice a plane wave is an eigenfunction: the Laplacian
    symbol of Eq. (best) is -(2/3)(4 - 2cos kx - 2cos ky - cos kx cos ky)
    ... evaluated directly from the printed weights."""
    p = oracle_mod.params(walls=False)
    nx, ny = 16, 12
    kx, ky = 2 * np.pi * 3 / nx, 2 * np.pi * 2 / ny
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    phi = np.cos(kx * x + ky * y)
    dx, dy, lap = oracle_mod.phi_derivatives(p, phi)
    # printed 1/6 [1 4 1; 4 -20 4; 1 4 1] and 1/12 [-1 0 1; -4 0 4; -1 0 1]
    lam = (8 * np.cos(kx) + 8 * np.cos(ky) + 4 * np.cos(kx) * np.cos(ky) - 20) / 6
    sx = (8 * np.sin(kx) + 4 * np.sin(kx) * np.cos(ky)) / 12
    sy = (8 * np.sin(ky) + 4 * np.sin(ky) * np.cos(kx)) / 12
    assert np.allclose(lap, lam * phi, atol=1e-13)
    assert np.allclose(dx, -sx * np.sin(kx * x + ky * y), atol=1e-13)
    assert np.allclose(dy, -sy * np.sin(kx * x + ky * y), atol=1e-13)


def test_wetting_ghost_rows_impose_the_gradient(oracle_mod):
    """The wetting condition of Sec. II (inward normal derivative = h at the
    wall) holds exactly for the discrete y-gradient on both boundary rows."""
    rng = np.random.default_rng(6)
    p = oracle_mod.params(h_bottom=-0.2368, h_top=0.1234)
    phi = rng.uniform(-1, 1, size=(9, 13))
    _, dy, _ = oracle_mod.phi_derivatives(p, phi)
    assert np.allclose(dy[0], p.h_bottom, atol=1e-15)
    assert np.allclose(dy[-1], -p.h_top, atol=1e-15)


def test_one_sided_wetting_rule_sets_the_wall_plane_difference(oracle_mod):
    """The alternative discretisation of the wetting condition (reading 2):
    the ghost row takes phi(x,-1) = phi(x,0) - h, so the one-sided
    difference across the wall plane y = -1/2 equals h.  On a field linear
    in y (slope g) the isotropic y-gradient of the boundary row is then
    (g + h)/2 at the bottom and (g - h_top)/2 at the top; the mirror rule
    would give h and -h_top."""
    g = 0.037
    p = oracle_mod.params(h_bottom=-0.2368, h_top=0.1234, wetting_rule=1)
    y = np.arange(9, dtype=float)[:, None]
    phi = 0.3 + g * y + 0.0 * np.arange(13)[None, :]
    _, dy, _ = oracle_mod.phi_derivatives(p, phi)
    assert np.allclose(dy[0], 0.5 * (g + p.h_bottom), atol=1e-15)
    assert np.allclose(dy[-1], 0.5 * (g - p.h_top), atol=1e-15)
    assert np.allclose(dy[1:-1], g, atol=1e-15)


@pytest.mark.parametrize("theta", [60.0, 120.0])
def test_one_sided_wetting_rule_drop_angle(oracle_mod, theta):
    """With the one-sided ghost the sessile drop also settles near Eq.
    (theory): 60 -> 57.3 and 120 -> 121.9 degrees on this 2.8-node-wide
    interface after 9000 steps (the mirror rule gives 58.2 and 123.8)."""
    nx, ny, R = 120, 60, 25.0
    p = oracle_mod.params(tau_alpha=1.0, tau_beta=1.0, h_bottom=oracle_mod.wetting_h(theta),
                          h_top=0.0, gamma_mob=0.5, wetting_rule=1)
    lat = oracle_mod.OracleLattice(p, nx, ny)
    lat.init_drop(R, nx / 2, -0.5)
    lat.step(9000)
    _, ph, _, _ = lat.moments()
    th, *_ = oracle_mod.contact_angle(ph)
    assert th == pytest.approx(theta, abs=4.5)


# ------------------------------------------------- contact-angle theory
def _young_cos_theta(h, a, kappa):
    """cos(theta) from Young's law (Eq. Young) with Cahn wall tensions: the
    wall free energy xi*phi_s + |int_{phi_s}^{phi_bulk} sqrt(2 kappa dpsi)|
    minimised over the surface value phi_s (grid search, then a bounded
    refinement), for each bulk phase; xi = kappa*h."""
    from scipy.integrate import quad
    from scipy.optimize import minimize_scalar

    xi = kappa * h

    def dpsi(ph):  # bulk free energy above the coexistence value (Eq. bulkfe)
        return a * (-0.5 * ph ** 2 + 0.25 * ph ** 4) + 0.25 * a

    def grad_energy(p0, p1):
        return abs(quad(lambda s: math.sqrt(max(2 * kappa * dpsi(s), 0.0)), p0, p1,
                        epsabs=1e-14, epsrel=1e-13)[0])

    def wall_tension(bulk):
        def energy(s):
            return xi * s + grad_energy(s, bulk)

        grid = np.linspace(-1.9, 1.9, 761)
        vals = [energy(s) for s in grid]
        s0 = grid[int(np.argmin(vals))]
        res = minimize_scalar(energy, bounds=(s0 - 0.01, s0 + 0.01), method="bounded",
                              options={"xatol": 1e-12})
        return res.fun

    gamma = math.sqrt(8 * kappa * a / 9)
    return (wall_tension(-1.0) - wall_tension(1.0)) / gamma


@pytest.mark.parametrize("theta", [15.0, 30.0, 60.0, 75.0, 90.0, 110.0, 120.0, 150.0, 170.0])
def test_theta_closed_form_agrees_with_young_cahn(oracle_mod, theta):
    """Eq. (theory) versus an independent evaluation of Young's law with
    numerically minimised wall free energies: fixes both the formula and the
    sign convention (h > 0 -> theta > 90)."""
    a, kappa = 0.04, 0.04
    h = oracle_mod.wetting_h(theta, a, kappa)
    assert _young_cos_theta(h, a, kappa) == pytest.approx(math.cos(math.radians(theta)), abs=2e-6)
    assert oracle_mod.theta_from_h(h, a, kappa) == pytest.approx(theta, abs=1e-6)


def test_wetting_h_values():
    import oracle

    assert oracle.wetting_h(90.0) == 0.0
    assert oracle.wetting_h(60.0) == pytest.approx(-oracle.wetting_h(120.0), abs=1e-15)
    # complete wetting / drying bound: sqrt(2 kappa/a)|h| = 2 sqrt(cos30 (1-cos30))
    c = math.cos(math.pi / 6)
    assert oracle.wetting_h(0.0) == pytest.approx(-2 * math.sqrt(c * (1 - c)) / math.sqrt(2), abs=1e-12)


# ------------------------------------------------------ circle fit
def test_circle_fit_on_exact_arc(oracle_mod):
    rng = np.random.default_rng(7)
    for theta in (40.0, 90.0, 135.0):
        R, xc, wall = 23.0, 50.0, -0.5
        yc = wall + R * math.sin(math.radians(theta - 90.0))
        ang = rng.uniform(0, 2 * np.pi, 400)
        pts = np.stack([xc + R * np.cos(ang), yc + R * np.sin(ang)], axis=1)
        pts = pts[pts[:, 1] > wall + 2]
        fx, fy, fR = oracle_mod.fit_circle(pts)
        assert (fx, fy, fR) == pytest.approx((xc, yc, R), abs=1e-9)


def test_contact_angle_of_synthetic_drop_field(oracle_mod):
    """A tanh drop profile whose phi = 0 contour is an exact circle cut by the
    wall plane: the crossing + fit pipeline recovers its angle."""
    for theta in (60.0, 90.0, 120.0):
        R, xc, wall = 30.0, 80.0, -0.5
        yc = wall + R * math.sin(math.radians(theta - 90.0))
        y, x = np.mgrid[0:80, 0:160].astype(float)
        phi = np.tanh((R - np.hypot(x - xc, y - yc)) / math.sqrt(2))
        th, fR, fx, fy = oracle_mod.contact_angle(phi, wall_y=wall)
        assert th == pytest.approx(theta, abs=0.3)
        assert fR == pytest.approx(R, abs=0.1)


# --------------------------------------------------- whole-step pins
def test_one_step_phi_update_is_laplacian_of_mu(oracle_mod):
    """With tau_phi = 1 and u = 0, one step gives
    phi(t+1) = phi(t) + (Gamma/2) lap(mu) exactly: the pull of the g
    equilibria (Eq. equilibrium, Eq. feq0) from the eight neighbours."""
    p = oracle_mod.params(walls=False, gamma_mob=0.37, a=0.05, kappa=0.03)
    nx, ny = 24, 20
    phi0 = lbinputs.smooth_random_field(nx, ny, 0.9, seed=11)
    lat = oracle_mod.OracleLattice(p, nx, ny)
    lat.init_phi(phi0)
    lat.step(1)
    _, phi1, _, _ = lat.moments()
    _, _, lap = oracle_mod.phi_derivatives(p, phi0)
    mu = p.a * (-phi0 + phi0 ** 3) - p.kappa * lap
    _, _, lap_mu = oracle_mod.phi_derivatives(p, mu)
    assert np.allclose(phi1, phi0 + 0.5 * p.gamma_mob * lap_mu, atol=1e-14, rtol=0)


@pytest.mark.parametrize("coll,taus", [("bgk", (1.0, 1.0)), ("mrt", (3.0, 0.7)),
                                       ("bgk", (1.5, 0.6))])
def test_conservation_of_mass_and_order_parameter(oracle_mod, coll, taus):
    """Collision conserves rho and phi (Eq. feq0) and streaming with
    bounce-back permutes populations: totals constant to rounding."""
    p = oracle_mod.params(collision=coll, tau_alpha=taus[0], tau_beta=taus[1],
                          h_bottom=oracle_mod.wetting_h(60.0), h_top=0.0)
    lat = oracle_mod.OracleLattice(p, 100, 50)
    lat.init_drop(20.0, 50.0, -0.5)
    r0, ph0, _, _ = lat.moments()
    lat.step(300)
    r1, ph1, ux, uy = lat.moments()
    assert abs(r1.sum() - r0.sum()) <= 1e-12 * r0.sum()
    assert abs(ph1.sum() - ph0.sum()) <= 1e-12 * r0.sum()
    assert np.isfinite(ux).all() and np.abs(ux).max() < 0.05


def _decay_rate(series, t):
    return -np.polyfit(t, np.log(series), 1)[0]


@pytest.mark.parametrize("coll,tau", [("bgk", 0.8), ("mrt", 0.8), ("mrt", 1.4)])
def test_shear_wave_viscosity(oracle_mod, coll, tau):
    """Eq. (kine): a shear wave u_x = U sin(k y) decays as exp(-nu k^2 t) with
    nu = (tau - 1/2)/3 (a = kappa = 0 reduces the fluid to plain D2Q9)."""
    nx, ny = 4, 64
    p = oracle_mod.params(a=0.0, kappa=0.0, walls=False, collision=coll,
                          tau_alpha=tau, tau_beta=tau)
    lat = oracle_mod.OracleLattice(p, nx, ny)
    k = 2 * np.pi / ny
    U = 1e-4
    for y in range(ny):
        feq, geq = oracle_mod.node_equilibrium(p, 1.0, 0.0, U * math.sin(k * y), 0.0, 0, 0, 0)
        lat.f[:, y, :] = feq[:, None]
        lat.g[:, y, :] = geq[:, None]
    amps, ts = [], []
    basis = np.sin(k * np.arange(ny))
    for s in range(10):
        lat.step(60)
        _, _, ux, _ = lat.moments()
        amps.append(ux[:, 0] @ basis / (basis @ basis))
        ts.append(lat.t)
    nu = _decay_rate(np.array(amps), np.array(ts)) / k ** 2
    assert nu == pytest.approx((tau - 0.5) / 3, rel=0.01)


def test_bounce_back_wall_sits_mid_link(oracle_mod):
    """Mid-link bounce-back puts the no-slip planes half a spacing outside
    rows 0 and ny-1: the lowest shear mode between them,
    u_x = U sin(pi (y + 1/2) / ny), decays at nu (pi / ny)^2."""
    nx, ny, tau = 4, 40, 1.0
    p = oracle_mod.params(a=0.0, kappa=0.0, walls=True, collision="bgk",
                          tau_alpha=tau, tau_beta=tau)
    lat = oracle_mod.OracleLattice(p, nx, ny)
    k = np.pi / ny
    prof = np.sin(k * (np.arange(ny) + 0.5))
    for y in range(ny):
        feq, geq = oracle_mod.node_equilibrium(p, 1.0, 0.0, 1e-4 * prof[y], 0.0, 0, 0, 0)
        lat.f[:, y, :] = feq[:, None]
        lat.g[:, y, :] = geq[:, None]
    amps, ts = [], []
    lat.step(100)
    for s in range(10):
        lat.step(80)
        _, _, ux, _ = lat.moments()
        amps.append(ux[:, 0] @ prof / (prof @ prof))
        ts.append(lat.t)
    nu = _decay_rate(np.array(amps), np.array(ts)) / k ** 2
    assert nu == pytest.approx((tau - 0.5) / 3, rel=0.01)


@pytest.mark.parametrize("tau_phi,nx,rel", [(1.0, 16, 1e-6), (0.8, 64, 0.02)])
def test_spinodal_mode_growth_rate(oracle_mod, tau_phi, nx, rel):
    """Eqs. (nsfinal23), (chempot), (Mobility): about phi = 0 a small mode
    grows at M k^2 (a - kappa k^2), M = Gamma (tau_phi - 1/2), decoupled from
    the flow at linear order.  With tau_phi = 1 the per-step factor is exactly
    1 + (Gamma/2) L (a - kappa L), L = -lap symbol = 2(1 - cos k); for
    tau_phi != 1 the long-wave continuum rate holds to the discretisation
    error."""
    ny = 3
    p = oracle_mod.params(walls=False, tau_phi=tau_phi, gamma_mob=0.5)
    k = 2 * np.pi / nx
    x = np.arange(nx)
    lat = oracle_mod.OracleLattice(p, nx, ny)
    lat.init_phi(np.tile(1e-7 * np.cos(k * x), (ny, 1)))
    amps, ts = [], []
    lat.step(10)
    for s in range(8):
        lat.step(25)
        _, ph, _, _ = lat.moments()
        amps.append(ph[0] @ np.cos(k * x) / (nx / 2))
        ts.append(lat.t)
    rate = -_decay_rate(np.array(amps), np.array(ts))
    L = 2 * (1 - np.cos(k))
    if tau_phi == 1.0:
        expect = math.log(1 + 0.5 * p.gamma_mob * L * (p.a - p.kappa * L))
    else:
        M = p.gamma_mob * (tau_phi - 0.5)
        expect = M * L * (p.a - p.kappa * L)
    assert rate == pytest.approx(expect, rel=rel)


def _discrete_flat_profile(p, phi_guess):
    """Newton solve of a(phi^3 - phi) - kappa lap1(phi) = mu0 on a periodic
    1-D lattice with sum(phi) fixed (the discrete chemical-potential
    balance that a static LB interface must satisfy)."""
    n = phi_guess.size
    phi = phi_guess.copy()
    mu0 = 0.0
    target = phi_guess.sum()
    for _ in range(50):
        lap = np.roll(phi, 1) + np.roll(phi, -1) - 2 * phi
        res = np.concatenate([p.a * (phi ** 3 - phi) - p.kappa * lap - mu0, [phi.sum() - target]])
        J = np.zeros((n + 1, n + 1))
        idx = np.arange(n)
        J[idx, idx] = p.a * (3 * phi ** 2 - 1) + 2 * p.kappa
        J[idx, (idx + 1) % n] -= p.kappa
        J[idx, (idx - 1) % n] -= p.kappa
        J[idx, n] = -1.0
        J[n, :n] = 1.0
        d = np.linalg.solve(J, -res)
        phi += d[:n]
        mu0 += d[n]
        if np.abs(d).max() < 1e-15:
            break
    return phi, mu0


def test_flat_interface_is_the_discrete_equilibrium(oracle_mod):
    """A flat stripe relaxes to the profile with uniform discrete chemical
    potential (Eq. chempot with the stencil of Eq. best, which reduces to
    the 1-D three-point Laplacian for an x-only profile), at rest."""
    nx, ny = 24, 3
    p = oracle_mod.params(walls=False, gamma_mob=1.0)
    ell = math.sqrt(2 * p.kappa / p.a)
    x = np.arange(nx)
    prof = np.tanh((x - 6.3) / ell) - np.tanh((x - 17.7) / ell) - 1.0
    lat = oracle_mod.OracleLattice(p, nx, ny)
    lat.init_phi(np.tile(prof, (ny, 1)))
    lat.step(20000)
    _, ph, ux, uy = lat.moments()
    ref, mu0 = _discrete_flat_profile(p, ph[0].copy())
    assert np.abs(ph - ph[0]).max() < 1e-13
    assert np.abs(ph[0] - ref).max() < 1e-9
    assert np.abs(ux).max() < 1e-9 and np.abs(uy).max() < 1e-12
    # and the continuum tanh profile to the discretisation error
    assert np.abs(ref - prof).max() < 0.05


def _laplace_slope(oracle_mod, p, n, radii, steps):
    inv_r, dp = [], []
    for R in radii:
        lat = oracle_mod.OracleLattice(p, n, n)
        lat.init_drop(R, n / 2 - 0.5, n / 2 - 0.5)
        lat.step(steps)
        rho, ph, _, _ = lat.moments()
        p0 = rho / 3 + p.a * (-0.5 * ph ** 2 + 0.75 * ph ** 4)  # Eq. (p0)
        c = n // 2
        p_in = p0[c - 2:c + 2, c - 2:c + 2].mean()
        p_out = p0[:3, :3].mean()
        _, _, Rf = oracle_mod.fit_circle(oracle_mod.interface_points(ph))
        inv_r.append(1.0 / Rf)
        dp.append(p_in - p_out)
    return np.polyfit(inv_r, dp, 1)[0]


def test_laplace_law(oracle_mod):
    """2-D Laplace law p_in - p_out = gamma / R, gamma = sqrt(8 kappa a/9)
    (Sec. II), from the slope over three radii.  At a = kappa = 0.04 the
    interface is only 2.8 nodes wide and the lattice tension sits about 6 %
    under the continuum value, hence the 8 % band; the wide-interface test
    below closes it to 2 %."""
    p = oracle_mod.params(walls=False)
    slope = _laplace_slope(oracle_mod, p, 64, (10.0, 14.0, 20.0), 3000)
    assert slope == pytest.approx(math.sqrt(8 * p.kappa * p.a / 9), rel=0.08)


@pytest.mark.slow
def test_laplace_law_wide_interface(oracle_mod):
    """Same law with a = 0.01 (interface width 5.7 nodes): within 2 %."""
    p = oracle_mod.params(walls=False, a=0.01, kappa=0.04, gamma_mob=1.0)
    slope = _laplace_slope(oracle_mod, p, 100, (16.0, 22.0, 30.0), 10000)
    assert slope == pytest.approx(math.sqrt(8 * p.kappa * p.a / 9), rel=0.02)


@pytest.mark.parametrize("theta,coll", [(90.0, "bgk"), (60.0, "bgk"), (120.0, "mrt")])
def test_sessile_drop_angle_matches_theory(oracle_mod, theta, coll):
    """Sec. IV: with tau = 1 the measured equilibrium angle follows Eq.
    (theory).  On this 2.8-node-wide interface the converged angles sit
    within about 4 degrees of the continuum curve (60 -> 58.0, 90 -> 90.7,
    120 -> 123.9); a sign error in h (60 <-> 120) or a factor two in the
    ghost rule (60 -> ~75) falls far outside the 4.5 degree band."""
    nx, ny, R = 120, 60, 25.0
    p = oracle_mod.params(collision=coll, tau_alpha=1.0, tau_beta=1.0,
                          h_bottom=oracle_mod.wetting_h(theta), h_top=0.0, gamma_mob=0.5)
    lat = oracle_mod.OracleLattice(p, nx, ny)
    lat.init_drop(R, nx / 2, -0.5)
    lat.step(9000)
    _, ph, _, _ = lat.moments()
    th, *_ = oracle_mod.contact_angle(ph)
    assert th == pytest.approx(theta, abs=4.5)


def test_mrt_with_unit_rate_equals_bgk_tau_one(oracle_mod):
    """With tau = 1 every non-conserved rate of Eq. (diag) is 1, so MRT
    without Step 2 is BGK at tau = 1 at every node (whole-step check)."""
    common = dict(tau_alpha=1.0, tau_beta=1.0, h_bottom=oracle_mod.wetting_h(70.0),
                  zero_u_at_walls=False)
    pb = oracle_mod.params(collision="bgk", **common)
    pm = oracle_mod.params(collision="mrt", **common)
    lats = []
    for p in (pb, pm):
        lat = oracle_mod.OracleLattice(p, 40, 24)
        lat.init_drop(10.0, 20.0, -0.5)
        lat.step(200)
        lats.append(lat)
    assert np.abs(lats[0].f - lats[1].f).max() < 1e-13
    assert np.abs(lats[0].g - lats[1].g).max() < 1e-13


def test_step_window_matches_full_step(oracle_mod):
    """The windowed evaluation used for sampled checks of large lattices
    gives the same post-collision values as a full step."""
    p = oracle_mod.params(collision="mrt", tau_alpha=1.5, tau_beta=0.6,
                          h_bottom=0.1, h_top=-0.05)
    nx, ny = 30, 20
    lat = oracle_mod.OracleLattice(p, nx, ny)
    lat.init_phi(lbinputs.smooth_random_field(nx, ny, 0.8, seed=3))
    lat.step(5)
    f0, g0 = lat.f.copy(), lat.g.copy()
    lat.step(1)
    for (x0, x1, y0, y1) in [(0, 5, 0, 3), (25, 30, 17, 20), (10, 20, 8, 12)]:
        b0 = max(0, y0 - 2)
        b1 = min(ny, y1 + 2)
        fo, go = oracle_mod.step_window(p, nx, ny, b0, f0[:, b0:b1], g0[:, b0:b1], x0, x1, y0, y1)
        assert np.array_equal(fo, lat.f[:, y0:y1, x0:x1])
        assert np.array_equal(go, lat.g[:, y0:y1, x0:x1])


# ------------------------------------------------- lookup-table MRT, Sec. V
def test_lookup_table_tau(oracle_mod):
    """Sec. V replaces the per-node collision matrix by the nearest of ~1e4
    tabulated viscosities: tau takes exactly n values, the bulk values at the
    table ends, within half a table step of Eq. (tau) inside [-1, 1],
    monotone in phi, clamped beyond the bulk values; BGK ignores the table."""
    for ta, tb in ((3.0, 0.7), (0.6, 1.5)):
        n = 101
        p = oracle_mod.params(collision="mrt", tau_alpha=ta, tau_beta=tb, mrt_lut=n)
        exact = oracle_mod.params(collision="mrt", tau_alpha=ta, tau_beta=tb)
        step = abs(ta - tb) / (n - 1)
        assert oracle_mod.node_tau(p, 1.0) == ta and oracle_mod.node_tau(p, -1.0) == tb
        phis = np.linspace(-1.0, 1.0, 20001)
        taus = np.array([oracle_mod.node_tau(p, v) for v in phis])
        ex = np.array([oracle_mod.node_tau(exact, v) for v in phis])
        assert np.abs(taus - ex).max() <= step / 2 + 1e-13
        assert len(np.unique(np.round(taus, 12))) == n
        d = np.diff(taus) * np.sign(ta - tb)
        assert (d >= -1e-15).all()
        assert oracle_mod.node_tau(p, 1.3) == oracle_mod.node_tau(p, 1.0)
        assert oracle_mod.node_tau(p, -1.3) == oracle_mod.node_tau(p, -1.0)
        bgk = oracle_mod.params(collision="bgk", tau_alpha=ta, tau_beta=tb, mrt_lut=n)
        assert oracle_mod.node_tau(bgk, 0.3) == oracle_mod.node_tau(exact, 0.3)


def test_lookup_table_run_converges_to_exact(oracle_mod):
    """A 1e4-entry table changes a drop run by far less than a coarse one."""
    nx, ny = 48, 24
    kw = dict(collision="mrt", tau_alpha=3.0, tau_beta=0.7, h_bottom=oracle_mod.wetting_h(70.0))
    runs = {}
    for n in (0, 10000, 3):
        lat = oracle_mod.OracleLattice(oracle_mod.params(mrt_lut=n, **kw), nx, ny)
        lat.init_drop(10.0, 24.0, -0.5)
        lat.step(400)
        runs[n] = lat.moments()[1]
    fine = np.abs(runs[10000] - runs[0]).max()
    coarse = np.abs(runs[3] - runs[0]).max()
    assert fine < 1e-3 and coarse > 20 * fine


# ---------------------------------------------------- stripe (Sec. IV.A)
def _stripe_phi0(c, p):
    """tanh edges at xa (rising) and xb (falling), each over its half of the
    period, so that the profile shifted by half the period is exactly its
    negative."""
    ell = math.sqrt(2 * p.kappa / p.a)
    x = np.arange(c["nx"], dtype=float)
    half = c["nx"] // 2
    prof = np.where(x < half, np.tanh((x - c["xa"]) / ell), -np.tanh((x - c["xb"]) / ell))
    return np.tile(prof, (c["ny"], 1))


def _left_edge(row):
    """x of the phi = 0 crossing of the stripe's left edge (linear between
    the two nodes around it)."""
    for i in range(1, row.size // 2):
        if row[i - 1] < 0.0 <= row[i]:
            return i - 1 + (-row[i - 1]) / (row[i] - row[i - 1])
    return float("nan")


def stripe_run(oracle_mod, coll, ta, tb, steps=None):
    """Steady state of the stripe: (phi, max |u|, bulge), the bulge being
    the left edge's x at mid-height less its x on the wall row (negative:
    the alpha stripe is wider in the middle, barrel shaped)."""
    c = lbinputs.STRIPE_28x15
    p = oracle_mod.params(collision=coll, tau_alpha=ta, tau_beta=tb, **c["params"])
    lat = oracle_mod.OracleLattice(p, c["nx"], c["ny"])
    lat.init_phi(_stripe_phi0(c, p))
    lat.step(steps or c["steps"])
    _, ph, ux, uy = lat.moments()
    bulge = _left_edge(ph[c["ny"] // 2]) - _left_edge(ph[0])
    return ph, float(np.hypot(ux, uy).max()), bulge


def test_stripe_spurious_current_is_of_order_1e_3(oracle_mod):
    """Sec. IV.A: the 28 x 15 stripe at tau = 10 between neutral walls
    settles with spurious velocities of order 10^-3 c, and with equal
    viscosities its edges stay straight (the 90 degree angle)."""
    _, umax, bulge = stripe_run(oracle_mod, "bgk", 10.0, 10.0)
    assert 1e-4 < umax < 1e-2
    assert abs(bulge) < 1e-4


def test_stripe_barrel_shape_bgk_not_mrt(oracle_mod):
    """Sec. IV.A: with tau_alpha > tau_beta the BGK stripe becomes barrel
    shaped (at the paper's ratio 12.5).  MRT with Step 2, the paper's cure,
    keeps the edges much straighter."""
    _, _, b_bgk = stripe_run(oracle_mod, "bgk", 3.0, 0.7)
    _, _, b_mrt = stripe_run(oracle_mod, "mrt", 3.0, 0.7)
    assert b_bgk < -0.2
    assert abs(b_mrt) < 0.5 * abs(b_bgk)


@pytest.mark.parametrize("coll", ["bgk", "mrt"])
def test_stripe_phase_swap_antisymmetry(oracle_mod, coll):
    """phi -> -phi with tau_alpha <-> tau_beta maps the stripe onto its
    complement (both 14 columns wide): mu and g^eq are odd in phi, f^eq is
    even, so the two runs are mirror images (to the rounding of the two
    forms of tau(phi)) and the bulge changes sign."""
    c = lbinputs.STRIPE_28x15
    ph1, u1, b1 = stripe_run(oracle_mod, coll, 1.5, 0.6, steps=4000)
    ph2, u2, b2 = stripe_run(oracle_mod, coll, 0.6, 1.5, steps=4000)
    shift = int(c["xb"] - c["xa"])
    assert np.abs(np.roll(ph1, shift, axis=1) + ph2).max() < 1e-10
    assert abs(b1 + b2) < 1e-9 and abs(b1) > 1e-3
    assert u1 == pytest.approx(u2, rel=1e-9)
