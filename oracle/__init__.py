"""FP64 CPU oracle for the free-energy binary-fluid lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg are the only callers.  The product
library never imports this package and this package never imports the
product library.

The time step itself lives in ``lb_oracle.c`` (plain C, double precision,
compiled with ``-ffp-contract=off`` so that x86-64 and aarch64 hosts agree
bit for bit).  This module adds:

* a ctypes wrapper around it (``OracleLattice`` and node-level helpers);
* the closed-form equilibrium contact angle of Eq. (theory) and its inverse
  (Sec. IV);
* the circle-fit contact-angle measurement of Sec. IV written with numpy.

Function -> paper passage:
  node_equilibrium      Appendix A, Eqs. (equilibrium), (feq0)
  node_collide_f        Eqs. (latbolt), (mrtlb), (Matrix), (diag)
  phi_derivatives       Eq. (best) + wetting ghost rows (Sec. II, IV)
  OracleLattice.step    Steps 1-4 of Sec. V with Eqs. (stream1-2)
  theta_from_h / wetting_h   Eq. (theory)
  contact_angle         circle fit of Sec. IV (Fig. 1)
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lb_oracle.c")
_LIBDIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIBDIR, "liblboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile lb_oracle.c into a shared library (plain gcc, OpenMP)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-ffp-contract=off", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("a", ctypes.c_double), ("kappa", ctypes.c_double),
        ("gamma_mob", ctypes.c_double), ("tau_phi", ctypes.c_double),
        ("tau_alpha", ctypes.c_double), ("tau_beta", ctypes.c_double),
        ("h_bottom", ctypes.c_double), ("h_top", ctypes.c_double),
        ("collision", ctypes.c_int), ("zero_u_at_walls", ctypes.c_int),
        ("walls", ctypes.c_int), ("mrt_all_rates", ctypes.c_int),
        ("step2_relax_momentum", ctypes.c_int), ("mrt_lut", ctypes.c_int),
        ("wetting_rule", ctypes.c_int),
    ]


def params(a=0.04, kappa=0.04, gamma_mob=0.1, tau_phi=1.0, tau_alpha=1.0,
           tau_beta=1.0, h_bottom=0.0, h_top=0.0, collision="bgk",
           zero_u_at_walls=None, walls=True, mrt_all_rates=False,
           step2_relax_momentum=False, mrt_lut=0, wetting_rule=0) -> OrcParams:
    """Parameter block.  ``zero_u_at_walls`` defaults to on for MRT (the
    proposed algorithm of Sec. V) and off for BGK."""
    coll = {"bgk": 0, "mrt": 1}[collision] if isinstance(collision, str) else int(collision)
    if zero_u_at_walls is None:
        zero_u_at_walls = coll == 1
    return OrcParams(a, kappa, gamma_mob, tau_phi, tau_alpha, tau_beta, h_bottom,
                     h_top, coll, int(bool(zero_u_at_walls)), int(bool(walls)),
                     int(bool(mrt_all_rates)), int(bool(step2_relax_momentum)), int(mrt_lut),
                     int(wetting_rule))


_D = ctypes.POINTER(ctypes.c_double)
_U8 = ctypes.POINTER(ctypes.c_uint8)


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _ptr8(a: np.ndarray):
    assert a.dtype == np.uint8 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_U8)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P = ctypes.POINTER(OrcParams)
            i, d, u64 = ctypes.c_int, ctypes.c_double, ctypes.c_uint64
            sig = {
                "orc_set_threads": (None, [i]),
                "orc_get_threads": (i, []),
                "orc_mrt_matrix": (None, [_D, _D]),
                "orc_node_equilibrium": (None, [P, d, d, d, d, d, d, d, _D, _D]),
                "orc_node_collide_f": (None, [P, _D, _D, d, i, _D]),
                "orc_phi_derivatives": (None, [P, i, i, _D, _D, _D, _D]),
                "orc_phi_drop": (None, [P, i, i, d, d, d, _D]),
                "orc_splitmix64": (u64, [u64, u64]),
                "orc_phi_random": (None, [i, i, d, u64, _D]),
                "orc_init": (None, [P, i, i, _D, _D, _D]),
                "orc_step": (None, [P, i, i, _D, _D, i]),
                "orc_moments": (None, [i, i, _D, _D, _D, _D, _D, _D]),
                "orc_step_window": (i, [P, i, i, i, i, _D, _D, i, i, i, i, _D, _D]),
                "orc_geo_check": (i, [P, i, i, _U8]),
                "orc_node_tau": (d, [P, d]),
                "orc_phi_derivatives_geo": (None, [P, i, i, _U8, _D, _D, _D, _D, _D]),
                "orc_init_geo": (i, [P, i, i, _U8, _D, _D, _D, _D]),
                "orc_step_geo": (i, [P, i, i, _U8, _D, _D, _D, i]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


# ----------------------------------------------------------- node helpers
def mrt_matrix():
    m = np.zeros(81)
    minv = np.zeros(81)
    lib().orc_mrt_matrix(_ptr(m), _ptr(minv))
    return m.reshape(9, 9), minv.reshape(9, 9)


def node_equilibrium(p: OrcParams, rho, phi, ux, uy, dphix, dphiy, lap):
    feq = np.zeros(9)
    geq = np.zeros(9)
    lib().orc_node_equilibrium(ctypes.byref(p), rho, phi, ux, uy, dphix, dphiy, lap,
                               _ptr(feq), _ptr(geq))
    return feq, geq


def node_collide_f(p: OrcParams, f, feq, omega, step2_node=False):
    """Collision of one node; step2_node marks a Step-2 boundary node (it
    matters only for MRT with step2_relax_momentum)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    feq = np.ascontiguousarray(feq, dtype=np.float64)
    out = np.zeros(9)
    lib().orc_node_collide_f(ctypes.byref(p), _ptr(f), _ptr(feq), float(omega),
                             int(bool(step2_node)), _ptr(out))
    return out


def node_tau(p: OrcParams, phi: float) -> float:
    """tau_rho the step uses at a node of order parameter phi (Eq. tau, or
    the nearest tabulated value with the lookup table of Sec. V)."""
    return float(lib().orc_node_tau(ctypes.byref(p), float(phi)))


def phi_derivatives(p: OrcParams, phi: np.ndarray):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    ny, nx = phi.shape
    dx = np.zeros_like(phi)
    dy = np.zeros_like(phi)
    lap = np.zeros_like(phi)
    lib().orc_phi_derivatives(ctypes.byref(p), nx, ny, _ptr(phi), _ptr(dx), _ptr(dy), _ptr(lap))
    return dx, dy, lap


# --------------------------------------------------------- initial fields
def phi_drop(p: OrcParams, nx, ny, R, cx, cy):
    phi = np.zeros((ny, nx))
    lib().orc_phi_drop(ctypes.byref(p), nx, ny, R, cx, cy, _ptr(phi))
    return phi


def splitmix64(seed: int, k: int) -> int:
    return int(lib().orc_splitmix64(seed, k))


def phi_random(nx, ny, amp, seed):
    phi = np.zeros((ny, nx))
    lib().orc_phi_random(nx, ny, amp, seed, _ptr(phi))
    return phi


class OracleLattice:
    """Full lattice state (post-collision f', g') advanced by the oracle.
    With a geometry (``set_geometry``) the lattice holds solid obstacles."""

    def __init__(self, p: OrcParams, nx: int, ny: int):
        if nx < 3 or ny < 3:
            raise ValueError("lattice must be at least 3x3")
        self.p = p
        self.nx, self.ny = nx, ny
        self.f = np.zeros((9, ny, nx))
        self.g = np.zeros((9, ny, nx))
        self.t = 0
        self.cls = None
        self.hcls = None

    def set_geometry(self, cls: np.ndarray, hcls) -> None:
        """cls: (ny, nx) uint8, 0 fluid, k in 1..7 solid of wetting class k,
        8 a node-bounce-back wall node (rows 0 and ny - 1 of a walled
        lattice only; its wetting gradient is h_bottom / h_top); hcls: the
        wetting gradient of each solid class (index 0 unused)."""
        cls = np.ascontiguousarray(cls, dtype=np.uint8)
        assert cls.shape == (self.ny, self.nx)
        h = np.zeros(8)
        h[:len(hcls)] = hcls
        if lib().orc_geo_check(ctypes.byref(self.p), self.nx, self.ny, _ptr8(cls)) != 0:
            raise ValueError("geometry rejected (feature thinner than two nodes or bad class)")
        self.cls, self.hcls = cls, h

    def init_phi(self, phi0: np.ndarray) -> None:
        phi0 = np.ascontiguousarray(phi0, dtype=np.float64)
        assert phi0.shape == (self.ny, self.nx)
        if self.cls is None:
            lib().orc_init(ctypes.byref(self.p), self.nx, self.ny, _ptr(phi0),
                           _ptr(self.f), _ptr(self.g))
        else:
            lib().orc_init_geo(ctypes.byref(self.p), self.nx, self.ny, _ptr8(self.cls),
                               _ptr(self.hcls), _ptr(phi0), _ptr(self.f), _ptr(self.g))
        self.t = 0

    def init_channel(self, res_len: int, ch_w: int, h_channel: float, h_block: float) -> None:
        """Capillary filling set-up (Sec. VI): see channel_geometry and
        channel_phi0."""
        self.set_geometry(channel_geometry(self.nx, self.ny, res_len, ch_w),
                          [0.0, h_channel, h_block])
        self.init_phi(channel_phi0(self.p, self.nx, self.ny, res_len, ch_w))

    def init_drop(self, R, cx, cy):
        self.init_phi(phi_drop(self.p, self.nx, self.ny, R, cx, cy))

    def init_random(self, amp, seed):
        self.init_phi(phi_random(self.nx, self.ny, amp, seed))

    def step(self, n: int = 1) -> None:
        if self.cls is None:
            lib().orc_step(ctypes.byref(self.p), self.nx, self.ny, _ptr(self.f),
                           _ptr(self.g), int(n))
        else:
            rc = lib().orc_step_geo(ctypes.byref(self.p), self.nx, self.ny, _ptr8(self.cls),
                                    _ptr(self.hcls), _ptr(self.f), _ptr(self.g), int(n))
            assert rc == 0
        self.t += int(n)

    def moments(self):
        """(rho, phi, ux, uy) of the stored post-collision populations."""
        out = [np.zeros((self.ny, self.nx)) for _ in range(4)]
        lib().orc_moments(self.nx, self.ny, _ptr(self.f), _ptr(self.g), *[_ptr(o) for o in out])
        return tuple(out)


def step_window(p: OrcParams, nx, ny, band_y0, fband, gband, x0, x1, y0, y1):
    """One step on the window [x0,x1)x[y0,y1) of a lattice (nx, ny) whose
    rows [band_y0, band_y0 + band_rows) are given as ``fband``/``gband``
    with shape (9, band_rows, nx)."""
    fband = np.ascontiguousarray(fband, dtype=np.float64)
    gband = np.ascontiguousarray(gband, dtype=np.float64)
    rows = fband.shape[1]
    fo = np.zeros((9, y1 - y0, x1 - x0))
    go = np.zeros((9, y1 - y0, x1 - x0))
    rc = lib().orc_step_window(ctypes.byref(p), nx, ny, band_y0, rows, _ptr(fband),
                               _ptr(gband), x0, x1, y0, y1, _ptr(fo), _ptr(go))
    if rc != 0:
        raise ValueError("window / band mismatch")
    return fo, go


# ------------------------------------------------- contact angle, Sec. IV
def theta_from_h(h, a=0.04, kappa=0.04):
    """Equilibrium angle (degrees) for an inward wetting gradient h, by
    solving Eq. (theory) for theta (bisection on the monotone right side)."""
    target = math.sqrt(2.0 * kappa / a) * h
    if target == 0.0:
        return 90.0

    def rhs(theta_deg):
        th = math.radians(theta_deg)
        alpha = math.acos(math.sin(th) ** 2)
        c = math.cos(alpha / 3.0)
        sgn = (theta_deg > 90.0) - (theta_deg < 90.0)
        return 2.0 * sgn * math.sqrt(max(c * (1.0 - c), 0.0))

    lo, hi = 0.0, 180.0
    if target <= rhs(lo):
        return 0.0
    if target >= rhs(hi):
        return 180.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if rhs(mid) < target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def wetting_h(theta_deg, a=0.04, kappa=0.04):
    """Inward wetting gradient h that Eq. (theory) assigns to theta."""
    th = math.radians(theta_deg)
    alpha = math.acos(math.sin(th) ** 2)
    c = math.cos(alpha / 3.0)
    sgn = (theta_deg > 90.0) - (theta_deg < 90.0)
    return 2.0 * sgn * math.sqrt(max(c * (1.0 - c), 0.0)) / math.sqrt(2.0 * kappa / a)


def interface_points(phi: np.ndarray, periodic_x: bool = True):
    """phi = 0 crossings on every horizontal and vertical link whose ends have
    phi > 0 and phi < 0, by linear interpolation along the link (Sec. IV).
    Returns an (n, 2) array of (x, y), sorted."""
    ny, nx = phi.shape
    pts = []
    for y in range(ny):
        for x in range(nx):
            a = phi[y, x]
            # horizontal link (x, y) - (x+1, y)
            if x + 1 < nx or periodic_x:
                b = phi[y, (x + 1) % nx]
                if (a > 0.0 and b < 0.0) or (a < 0.0 and b > 0.0):
                    t = a / (a - b)
                    pts.append((x + t, float(y)))
            # vertical link (x, y) - (x, y+1)
            if y + 1 < ny:
                b = phi[y + 1, x]
                if (a > 0.0 and b < 0.0) or (a < 0.0 and b > 0.0):
                    t = a / (a - b)
                    pts.append((float(x), y + t))
    pts = np.array(sorted(pts), dtype=np.float64).reshape(-1, 2)
    return pts


def fit_circle(pts: np.ndarray, iters: int = 10):
    """Least-squares circle through the points: algebraic (Kasa) start, then
    Gauss-Newton on the geometric residuals |p - c| - R."""
    x, y = pts[:, 0], pts[:, 1]
    A = np.stack([x, y, np.ones_like(x)], axis=1)
    rhs = x * x + y * y
    sol, *_ = np.linalg.lstsq(A, rhs, rcond=None)
    xc, yc = sol[0] / 2.0, sol[1] / 2.0
    R = math.sqrt(max(sol[2] + xc * xc + yc * yc, 0.0))
    for _ in range(iters):
        dx, dy = x - xc, y - yc
        d = np.sqrt(dx * dx + dy * dy)
        r = d - R
        J = np.stack([-dx / d, -dy / d, -np.ones_like(d)], axis=1)
        step, *_ = np.linalg.lstsq(J, -r, rcond=None)
        xc, yc, R = xc + step[0], yc + step[1], R + step[2]
    return xc, yc, R


def contact_angle(phi: np.ndarray, wall_y: float = -0.5, exclude: float = 2.0):
    """Contact angle (degrees, measured through the phi > 0 drop) of a drop
    sitting on the wall plane y = wall_y: crossings closer than ``exclude``
    to the wall are dropped, a circle is fitted and its angle with the plane
    is 90 + asin((yc - wall_y) / R).  Returns (theta, R, xc, yc)."""
    pts = interface_points(phi)
    pts = pts[pts[:, 1] >= wall_y + exclude]
    if pts.shape[0] < 3:
        raise ValueError("fewer than three interface points")
    xc, yc, R = fit_circle(pts)
    s = max(-1.0, min(1.0, (yc - wall_y) / R))
    return 90.0 + math.degrees(math.asin(s)), R, xc, yc


# ------------------------------------------------ capillary filling, Sec. VI
def channel_geometry(nx: int, ny: int, res_len: int, ch_w: int) -> np.ndarray:
    """Solid classes of the capillary set-up: the columns x >= res_len are
    solid except the channel rows [y0, y0 + ch_w), y0 = (ny - ch_w) // 2.
    Class 1: the two solid rows that bound the channel (its walls); class 2:
    every other solid node (the block end faces and interiors)."""
    y0 = (ny - ch_w) // 2
    cls = np.zeros((ny, nx), dtype=np.uint8)
    cls[:, res_len:] = 2
    cls[y0:y0 + ch_w, res_len:] = 0
    cls[y0 - 1, res_len:] = 1
    cls[y0 + ch_w, res_len:] = 1
    return cls


def channel_phi0(p: OrcParams, nx: int, ny: int, res_len: int, ch_w: int) -> np.ndarray:
    """Initial order parameter of the capillary set-up: phase alpha (+1)
    fills the reservoir columns [res_len // 2, res_len), phase beta (-1) the
    rest (the other half of the reservoir, which the channel outlet reaches
    through the periodic x boundary, and the channel).  Flat tanh profiles
    of width sqrt(2 kappa / a) centred half a node before each interface
    column; solid nodes carry 0."""
    l = math.sqrt(2.0 * p.kappa / p.a)
    xa, xb = res_len // 2, res_len
    x = np.arange(nx, dtype=np.float64)
    d = np.minimum(x - (xa - 0.5), (xb - 0.5) - x)
    phi = np.tile(np.tanh(d / l), (ny, 1))
    phi[channel_geometry(nx, ny, res_len, ch_w) != 0] = 0.0
    return phi


def meniscus(phi: np.ndarray, cls: np.ndarray, x_lo: int, x_hi: int, y_lo: int, y_hi: int,
             exclude: float = 2.0):
    """Meniscus of a channel whose walls are the planes y_lo - 1/2 and
    y_hi - 1/2, with phase alpha (phi > 0) behind it (smaller x).  The phi = 0
    crossings on fluid-fluid links inside [x_lo, x_hi) x [y_lo, y_hi),
    farther than `exclude` from both walls, are fitted with a circle.
    Returns (x_front, theta_deg, R): x_front is the circle's x on the channel
    centre line (on the branch facing the points); theta is the angle
    through alpha at the two walls (mean of both), from the circle."""
    pts = []
    for y in range(y_lo, y_hi):
        for x in range(x_lo, x_hi):
            if cls[y, x]:
                continue
            a = phi[y, x]
            if x + 1 < x_hi and not cls[y, x + 1]:
                b = phi[y, x + 1]
                if (a > 0 > b) or (a < 0 < b):
                    pts.append((x + a / (a - b), float(y)))
            if y + 1 < y_hi and not cls[y + 1, x]:
                c = phi[y + 1, x]
                if (a > 0 > c) or (a < 0 < c):
                    pts.append((float(x), y + a / (a - c)))
    wb, wt = y_lo - 0.5, y_hi - 0.5
    pts = np.array([q for q in pts if wb + exclude <= q[1] <= wt - exclude])
    if len(pts) < 3:
        raise ValueError("fewer than three meniscus points")
    xc, yc, R = fit_circle(pts)
    # centre ahead of the points (on the beta side): alpha wets, theta < 90
    s = 1.0 if xc > pts[:, 0].mean() else -1.0
    th_b = math.degrees(math.acos(max(-1.0, min(1.0, s * (yc - wb) / R))))
    th_t = math.degrees(math.acos(max(-1.0, min(1.0, s * (wt - yc) / R))))
    ym = 0.5 * (wb + wt)
    x_front = xc - s * math.sqrt(max(R * R - (ym - yc) ** 2, 0.0))
    return x_front, 0.5 * (th_b + th_t), R
