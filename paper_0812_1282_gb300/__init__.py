"""Python binding of the GB300 binary-fluid lattice Boltzmann library.

Argument marshalling only: every step of the method runs in the CUDA
kernels of ``csrc/`` behind the C ABI of ``include/lbfe.h``.  PyTorch
provides device memory (the state buffer is a uint8 CUDA tensor handed to
``lb_create``) and the CUDA stream.  There is no CPU fallback: without the
compiled library or a CUDA device, calls raise ``LBError``.

Functions carry the C names (``lb_create``, ``lb_step``, ...); ``Lattice``
and ``Batch`` wrap a handle for convenience.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "liblbfe.so")

LB_OK = 0
LB_ERR_INVALID_ARG = -1
LB_ERR_CUDA = -2
LB_ERR_NONFINITE = -3
LB_ERR_TIMEOUT = -4
LB_ERR_NO_INTERFACE = -5
LB_ERR_CAPACITY = -6
LB_BGK, LB_MRT = 0, 1
LB_FP32, LB_FP64 = 0, 1

# Every symbol declared in include/lbfe.h.
EXPORTS = (
    "lb_device_bytes", "lb_create", "lb_create_batch", "lb_destroy", "lb_init_drop",
    "lb_init_random", "lb_init_phi", "lb_step", "lb_moments", "lb_contact_angle",
    "lb_wetting_h", "lb_get_populations", "lb_get_populations_rows", "lb_set_populations", "lb_state_bytes",
    "lb_save_state", "lb_load_state", "lb_set_tile", "lb_get_tile", "lb_autotune",
    "lb_step_count", "lb_sync", "lb_launch_count", "lb_error_string", "lb_last_error",
    "lb_stats_noalloc", "lb_check_wait_timeout", "lb_set_geometry", "lb_get_geometry",
    "lb_init_channel", "lb_meniscus", "lb_set_wetting", "lb_set_schedule", "lb_get_schedule",
    "lb_fp64_peak",
)
LB_MAX_SCHED_CLASSES = 8


class LBError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (code %d)" % (msg, code))
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [
        ("a", ctypes.c_double), ("kappa", ctypes.c_double),
        ("gamma_mob", ctypes.c_double), ("tau_phi", ctypes.c_double),
        ("tau_alpha", ctypes.c_double), ("tau_beta", ctypes.c_double),
        ("h_bottom", ctypes.c_double), ("h_top", ctypes.c_double),
        ("collision", ctypes.c_int), ("zero_u_at_walls", ctypes.c_int),
        ("precision", ctypes.c_int), ("walls", ctypes.c_int),
        ("step2_relax_momentum", ctypes.c_int), ("mrt_lut", ctypes.c_int),
        ("compact_g", ctypes.c_int), ("wetting_rule", ctypes.c_int),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("mass", ctypes.c_double), ("order", ctypes.c_double),
        ("mom_x", ctypes.c_double), ("mom_y", ctypes.c_double),
        ("max_u", ctypes.c_double), ("nonfinite", ctypes.c_longlong),
        ("step", ctypes.c_longlong),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Schedule(ctypes.Structure):
    """lb_schedule: how a batch's work is cut and spread (include/lbfe.h)."""
    _fields_ = [
        ("n_class", ctypes.c_int),
        ("max_nx", ctypes.c_int * LB_MAX_SCHED_CLASSES),
        ("block_x", ctypes.c_int * LB_MAX_SCHED_CLASSES),
        ("rows", ctypes.c_int * LB_MAX_SCHED_CLASSES),
        ("ctas_per_sm", ctypes.c_int * LB_MAX_SCHED_CLASSES),
        ("order", ctypes.c_int), ("chains", ctypes.c_int), ("persist", ctypes.c_int),
        ("fill_pct", ctypes.c_int), ("steps_per_launch", ctypes.c_int),
        ("seal_edges", ctypes.c_int * LB_MAX_SCHED_CLASSES),
    ]

    def as_dict(self):
        n = self.n_class
        return {"n_class": n, "max_nx": list(self.max_nx)[:max(n - 1, 0)],
                "block_x": list(self.block_x)[:n], "rows": list(self.rows)[:n],
                "ctas_per_sm": list(self.ctas_per_sm)[:n], "order": self.order,
                "chains": self.chains, "persist": self.persist, "fill_pct": self.fill_pct,
                "steps_per_launch": self.steps_per_launch,
                "seal_edges": list(self.seal_edges)[:n]}


def schedule(block_x, rows, ctas_per_sm=8, max_nx=(), order=0, chains=1, persist=0,
             fill_pct=0, seal_edges=0, steps_per_launch=0) -> Schedule:
    """Schedule block; block_x, rows and ctas_per_sm are per class (an int
    applies to every class); max_nx gives the class limits (n_class - 1
    values); persist=1 runs each class's steps in one persistent launch
    (fill_pct: the share of the GPU its CTAs fill); seal_edges (per class)
    =1 makes whole-domain strips write whole sectors; steps_per_launch=2 steps a
    single domain with obstacles twice per launch."""
    n = len(max_nx) + 1

    def per_class(v):
        v = list(v) if isinstance(v, (list, tuple)) else [v] * n
        assert len(v) == n
        return v + [v[0]] * (LB_MAX_SCHED_CLASSES - n)

    arr = ctypes.c_int * LB_MAX_SCHED_CLASSES
    return Schedule(n, arr(*(list(max_nx) + [0] * (LB_MAX_SCHED_CLASSES - len(max_nx)))),
                    arr(*per_class(block_x)), arr(*per_class(rows)), arr(*per_class(ctas_per_sm)),
                    int(order), int(chains), int(persist), int(fill_pct),
                    int(steps_per_launch), arr(*per_class(seal_edges)))


def params(a=0.04, kappa=0.04, gamma_mob=0.1, tau_phi=1.0, tau_alpha=1.0, tau_beta=1.0,
           h_bottom=0.0, h_top=0.0, collision="bgk", zero_u_at_walls=None,
           precision="fp64", walls=True, step2_relax_momentum=False, mrt_lut=0,
           compact_g=False, wetting_rule=0) -> Params:
    """Parameter block (lattice units).  Step 2 of the proposed algorithm
    (zero equilibrium velocity on wall rows) defaults to on for MRT and off
    for BGK; step2_relax_momentum selects the alternative reading of the
    momentum rates on those rows (see include/lbfe.h)."""
    coll = {"bgk": LB_BGK, "mrt": LB_MRT}[collision] if isinstance(collision, str) else int(collision)
    prec = {"fp32": LB_FP32, "fp64": LB_FP64}[precision] if isinstance(precision, str) else int(precision)
    if zero_u_at_walls is None:
        zero_u_at_walls = coll == LB_MRT
    return Params(a, kappa, gamma_mob, tau_phi, tau_alpha, tau_beta, h_bottom, h_top, coll,
                  int(bool(zero_u_at_walls)), prec, int(bool(walls)),
                  int(bool(step2_relax_momentum)), int(mrt_lut), int(bool(compact_g)),
                  int(wetting_rule))


_lib = None
_lock = threading.Lock()
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_H = ctypes.c_void_p


def lib():
    """Load the compiled library (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise LBError(LB_ERR_CUDA, "CUDA library not built: %s (run "
                              "__graft_entry__.build())" % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            P = ctypes.POINTER(Params)
            i, d, sz, vp, ll = ctypes.c_int, ctypes.c_double, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_longlong
            sig = {
                "lb_device_bytes": (sz, [i, i, _I, _I]),
                "lb_create": (i, [P, i, i, vp, vp, sz, ctypes.POINTER(_H)]),
                "lb_create_batch": (i, [P, _I, _I, i, vp, vp, sz, ctypes.POINTER(_H)]),
                "lb_destroy": (None, [_H]),
                "lb_init_drop": (i, [_H, i, d, d, d]),
                "lb_init_random": (i, [_H, i, d, ctypes.c_ulonglong]),
                "lb_init_phi": (i, [_H, i, vp, i]),
                "lb_step": (i, [_H, i]),
                "lb_moments": (i, [_H, i, i, vp, vp, vp, vp, ctypes.POINTER(Stats)]),
                "lb_contact_angle": (i, [_H, i, d, _D, _D, _D, _D]),
                "lb_wetting_h": (d, [d, d, d]),
                "lb_get_populations": (i, [_H, i, vp, vp]),
                "lb_get_populations_rows": (i, [_H, i, i, i, vp, vp]),
                "lb_set_populations": (i, [_H, i, vp, vp]),
                "lb_state_bytes": (sz, [_H]),
                "lb_save_state": (i, [_H, vp, sz]),
                "lb_load_state": (i, [_H, vp, sz]),
                "lb_set_tile": (i, [_H, i, i]),
                "lb_get_tile": (i, [_H, _I, _I]),
                "lb_autotune": (i, [_H, i, _I, _I, _D]),
                "lb_step_count": (ll, [_H]),
                "lb_sync": (i, [_H]),
                "lb_launch_count": (ll, [_H]),
                "lb_error_string": (ctypes.c_char_p, [i]),
                "lb_last_error": (ctypes.c_char_p, []),
                "lb_stats_noalloc": (i, [vp, vp, i, i, i, vp, vp]),
                "lb_check_wait_timeout": (i, [vp]),
                "lb_set_geometry": (i, [_H, i, vp, _D, i]),
                "lb_get_geometry": (i, [_H, i, vp]),
                "lb_init_channel": (i, [_H, i, i, i, d, d]),
                "lb_meniscus": (i, [_H, i, i, i, i, i, d, _D, _D, _D]),
                "lb_set_wetting": (i, [_H, i, d, d]),
                "lb_set_schedule": (i, [_H, ctypes.POINTER(Schedule)]),
                "lb_get_schedule": (i, [_H, ctypes.POINTER(Schedule)]),
                "lb_fp64_peak": (i, [i, vp, _D]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(rc):
    if rc != LB_OK:
        L = lib()
        raise LBError(rc, "%s: %s" % (L.lb_error_string(rc).decode(), L.lb_last_error().decode()))
    return rc


def _np_ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------ C-name API
def lb_wetting_h(theta_deg, a=0.04, kappa=0.04) -> float:
    return float(lib().lb_wetting_h(float(theta_deg), float(a), float(kappa)))


def lb_device_bytes(precision, nx, ny) -> int:
    nx = np.ascontiguousarray(np.atleast_1d(nx), dtype=np.int32)
    ny = np.ascontiguousarray(np.atleast_1d(ny), dtype=np.int32)
    return int(lib().lb_device_bytes(int(precision), len(nx), nx.ctypes.data_as(_I),
                                     ny.ctypes.data_as(_I)))


def lb_stats_noalloc(f_dev_ptr, g_dev_ptr, nx, ny, precision, stats_dev_ptr, stream_ptr=0):
    """Diagnostics of caller-owned device population arrays into a
    caller-owned device buffer of 6 doubles, without allocating (see
    include/lbfe.h).  Pointers are integers (e.g. tensor.data_ptr())."""
    L = lib()
    rc = L.lb_stats_noalloc(ctypes.c_void_p(f_dev_ptr), ctypes.c_void_p(g_dev_ptr), int(nx),
                            int(ny), int(precision), ctypes.c_void_p(stats_dev_ptr),
                            ctypes.c_void_p(stream_ptr))
    if rc != LB_OK:  # this entry point leaves no message behind (it allocates nothing)
        raise LBError(rc, "lb_stats_noalloc: %s" % L.lb_error_string(rc).decode())
    return rc


def lb_fp64_peak(kind=0, stream_ptr=0) -> float:
    """Measured FP64 operations per second of the current device (kind 0
    DFMA, 1 DADD, 2 DMUL; see include/lbfe.h)."""
    v = ctypes.c_double()
    _check(lib().lb_fp64_peak(int(kind), ctypes.c_void_p(stream_ptr), ctypes.byref(v)))
    return v.value


def lb_check_wait_timeout(stream_ptr=0) -> int:
    """Run the bounded-wait self-check; returns the status code
    (LB_ERR_TIMEOUT is the expected, healthy answer)."""
    return int(lib().lb_check_wait_timeout(ctypes.c_void_p(stream_ptr)))


def _torch():
    import torch

    if not torch.cuda.is_available():
        raise LBError(LB_ERR_CUDA, "no CUDA device")
    return torch


class _HandleBase:
    """Owns an lb_handle plus the torch tensor backing its device memory."""

    def __init__(self, plist, nxs, nys, device=None, stream=None):
        torch = _torch()
        self.torch = torch
        self.device = torch.device(device if device is not None else "cuda")
        prec = plist[0].precision
        nbytes = lb_device_bytes(prec, nxs, nys)
        if nbytes == 0:
            raise LBError(LB_ERR_INVALID_ARG, "invalid domain sizes")
        with torch.cuda.device(self.device):
            self.mem = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            h = _H()
            if len(plist) == 1:
                rc = lib().lb_create(ctypes.byref(plist[0]), int(nxs[0]), int(nys[0]),
                                     ctypes.c_void_p(self.stream.cuda_stream),
                                     ctypes.c_void_p(self.mem.data_ptr()), nbytes, ctypes.byref(h))
            else:
                arr = (Params * len(plist))(*plist)
                nx = np.ascontiguousarray(nxs, dtype=np.int32)
                ny = np.ascontiguousarray(nys, dtype=np.int32)
                rc = lib().lb_create_batch(arr, nx.ctypes.data_as(_I), ny.ctypes.data_as(_I),
                                           len(plist), ctypes.c_void_p(self.stream.cuda_stream),
                                           ctypes.c_void_p(self.mem.data_ptr()), nbytes,
                                           ctypes.byref(h))
            _check(rc)
        self.h = h
        self.plist = list(plist)
        self.nxs = [int(v) for v in nxs]
        self.nys = [int(v) for v in nys]

    def close(self):
        if getattr(self, "h", None):
            lib().lb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- per-domain operations
    def init_drop(self, R, cx, cy=-0.5, dom=0):
        _check(lib().lb_init_drop(self.h, dom, float(R), float(cx), float(cy)))

    def init_random(self, amp, seed, dom=0):
        _check(lib().lb_init_random(self.h, dom, float(amp), int(seed)))

    def init_phi(self, phi0, dom=0):
        phi0 = np.ascontiguousarray(phi0, dtype=np.float64)
        assert phi0.shape == (self.nys[dom], self.nxs[dom])
        _check(lib().lb_init_phi(self.h, dom, _np_ptr(phi0), 0))

    def set_geometry(self, cls, h_class, dom=0):
        """Obstacle map (ny, nx) uint8 (0 fluid, k solid of class k) and the
        classes' wetting gradients; None removes the obstacles."""
        if cls is None:
            _check(lib().lb_set_geometry(self.h, dom, None, None, 0))
            return
        cls = np.ascontiguousarray(cls, dtype=np.uint8)
        assert cls.shape == (self.nys[dom], self.nxs[dom])
        hc = np.ascontiguousarray(h_class, dtype=np.float64)
        _check(lib().lb_set_geometry(self.h, dom, _np_ptr(cls), hc.ctypes.data_as(_D), len(hc)))

    def set_wetting(self, h_bottom, h_top, dom=0):
        _check(lib().lb_set_wetting(self.h, dom, float(h_bottom), float(h_top)))

    def geometry(self, dom=0):
        cls = np.empty((self.nys[dom], self.nxs[dom]), dtype=np.uint8)
        _check(lib().lb_get_geometry(self.h, dom, _np_ptr(cls)))
        return cls

    def init_channel(self, res_len, ch_w, h_channel, h_block=0.0, dom=0):
        _check(lib().lb_init_channel(self.h, dom, int(res_len), int(ch_w), float(h_channel),
                                     float(h_block)))

    def meniscus(self, x_lo, x_hi, y_lo, y_hi, exclude=2.0, dom=0):
        """(x_front, theta_deg, R) of a channel meniscus (see lb_meniscus)."""
        xf, th, R = (ctypes.c_double() for _ in range(3))
        _check(lib().lb_meniscus(self.h, dom, int(x_lo), int(x_hi), int(y_lo), int(y_hi),
                                 float(exclude), ctypes.byref(xf), ctypes.byref(th),
                                 ctypes.byref(R)))
        return xf.value, th.value, R.value

    def step(self, n=1):
        _check(lib().lb_step(self.h, int(n)))

    def sync(self):
        _check(lib().lb_sync(self.h))

    def moments(self, dom=0, fields=True):
        """(rho, phi, ux, uy) as (ny, nx) float64 arrays and the stats dict."""
        ny, nx = self.nys[dom], self.nxs[dom]
        st = Stats()
        if fields:
            out = [np.empty((ny, nx)) for _ in range(4)]
            rc = lib().lb_moments(self.h, dom, 0, *[_np_ptr(o) for o in out], ctypes.byref(st))
        else:
            out = [None] * 4
            rc = lib().lb_moments(self.h, dom, 0, None, None, None, None, ctypes.byref(st))
        if rc not in (LB_OK, LB_ERR_NONFINITE):
            _check(rc)
        return (*out, st.as_dict())

    def stats(self, dom=0):
        return self.moments(dom, fields=False)[4]

    def contact_angle(self, dom=0, exclude=2.0):
        th, R, xc, yc = (ctypes.c_double() for _ in range(4))
        _check(lib().lb_contact_angle(self.h, dom, float(exclude), ctypes.byref(th), ctypes.byref(R),
                                      ctypes.byref(xc), ctypes.byref(yc)))
        return th.value, R.value, xc.value, yc.value

    def populations(self, dom=0):
        ny, nx = self.nys[dom], self.nxs[dom]
        f = np.empty((9, ny, nx))
        g = np.empty((9, ny, nx))
        _check(lib().lb_get_populations(self.h, dom, _np_ptr(f), _np_ptr(g)))
        return f, g

    def populations_rows(self, y0, nrows, dom=0):
        nx = self.nxs[dom]
        f = np.empty((9, nrows, nx))
        g = np.empty((9, nrows, nx))
        _check(lib().lb_get_populations_rows(self.h, dom, int(y0), int(nrows), _np_ptr(f), _np_ptr(g)))
        return f, g

    def set_populations(self, f, g, dom=0):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        _check(lib().lb_set_populations(self.h, dom, _np_ptr(f), _np_ptr(g)))

    def save_state(self) -> bytes:
        n = int(lib().lb_state_bytes(self.h))
        buf = ctypes.create_string_buffer(n)
        _check(lib().lb_save_state(self.h, buf, n))
        return buf.raw

    def load_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(lib().lb_load_state(self.h, buf, len(blob)))

    def set_tile(self, block_x, rows):
        _check(lib().lb_set_tile(self.h, int(block_x), int(rows)))

    def tile(self):
        bx, r = ctypes.c_int(), ctypes.c_int()
        _check(lib().lb_get_tile(self.h, ctypes.byref(bx), ctypes.byref(r)))
        return bx.value, r.value

    def set_schedule(self, sched: Schedule):
        _check(lib().lb_set_schedule(self.h, ctypes.byref(sched)))

    def schedule(self) -> dict:
        sc = Schedule()
        _check(lib().lb_get_schedule(self.h, ctypes.byref(sc)))
        return sc.as_dict()

    def autotune(self, reps=5):
        bx, r, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check(lib().lb_autotune(self.h, int(reps), ctypes.byref(bx), ctypes.byref(r), ctypes.byref(ms)))
        return bx.value, r.value, ms.value

    @property
    def step_count(self):
        return int(lib().lb_step_count(self.h))

    @property
    def launch_count(self):
        return int(lib().lb_launch_count(self.h))


class Lattice(_HandleBase):
    """One domain: ``Lattice(params(...), nx, ny)``."""

    def __init__(self, p: Params, nx: int, ny: int, device=None, stream=None):
        super().__init__([p], [nx], [ny], device=device, stream=stream)
        self.p = p
        self.nx, self.ny = int(nx), int(ny)


class Batch(_HandleBase):
    """Independent domains advanced together by one launch per step."""

    def __init__(self, plist, nxs, nys, device=None, stream=None):
        super().__init__(list(plist), list(nxs), list(nys), device=device, stream=stream)
        self.n_dom = len(self.plist)
