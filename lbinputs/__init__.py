"""Seeded synthetic inputs shared by the tests, the smoke check and bench.py.

This module holds no arithmetic of the lattice Boltzmann method: only
random draws (SplitMix64, Steele, Lea & Flood 2014, used counter-based) and
the numeric descriptions of the workloads (lattice sizes, parameters, target
angles).  Both the CUDA path and the oracle receive the same numbers from it;
each side turns them into populations with its own code.

Workloads (parameters a = kappa = 0.04, Gamma = 0.1, tau_phi = 1 unless
stated; x periodic; bounce-back walls at y = 0 and y = ny - 1):

  DROP_100x50      BGK, tau = 1, neutral walls, drop R = 20 centred on the
                   bottom wall plane; 2000 steps (FP64 parity case).
  SWEEP_200x100    BGK and MRT (both readings of the Step-2 momentum
                   rates), drop R = 40; viscosity ratio 1 (tau 1 / 1) and
                   10 (tau_alpha 1.5 drop, tau_beta 0.6 gas); target
                   angles 60, 90, 120 degrees; 20000 steps.
  CAPILLARY_1000x120  capillary filling: walled 1000 x 120 box, reservoir
                   columns 0..199 (alpha in 100..199), channel rows 40..79
                   from column 200 on, h(60 deg) on the channel walls,
                   neutral elsewhere; MRT, tau_alpha 1.5, tau_beta 0.6;
                   100000 steps, front tracked every 500.
  STRIPE_28x15     the spurious-current set-up of Sec. IV.A: a stripe of
                   alpha (columns 7..20, tanh edges of width sqrt(2 kappa/a))
                   across the channel between neutral walls; BGK and MRT at
                   tau 10 / 10 (the paper's case) and at viscosity ratios
                   12.5 (tau 3 / 0.7) and 10 (1.5 / 0.6); 20000 steps.
  SPINODAL_8192    MRT, tau_alpha 1.5, tau_beta 0.6, neutral walls,
                   phi uniform in [-0.1, 0.1) from SplitMix64 seed 12345
                   (node (x, y) takes draw y*nx + x); FP32 and FP64.
  BATCH_256        256 sessile drops, sides uniform in 64..512,
                   R = 0.3 min(nx, ny) (so the drop clears the top wall),
                   target angle uniform in [30, 150], viscosity ratio in
                   {1, 3, 10} (tau_beta 0.6, tau_alpha 0.5 + 0.1 R); MRT FP32.
"""
from __future__ import annotations

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, k) -> np.ndarray:
    """Draw(s) k of the SplitMix64 stream seeded with ``seed``:
    mix(seed + (k + 1) * golden_gamma), all arithmetic mod 2**64."""
    k = np.asarray(k, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (k + np.uint64(1)) * GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, k) -> np.ndarray:
    """Top 53 bits of draw k as a double in [0, 1)."""
    return (splitmix64(seed, k) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def random_field(nx: int, ny: int, amp: float, seed: int) -> np.ndarray:
    """(ny, nx) field uniform in [-amp, amp), node (x, y) from draw y*nx+x."""
    k = np.arange(nx * ny, dtype=np.uint64)
    return (amp * (2.0 * uniform01(seed, k) - 1.0)).reshape(ny, nx)


def smooth_random_field(nx: int, ny: int, amp: float, seed: int, modes: int = 4) -> np.ndarray:
    """Sum of a few random Fourier modes (periodic in x and y): a smooth
    seeded test field with values in roughly [-amp, amp]."""
    u = uniform01(seed, np.arange(4 * modes * modes, dtype=np.uint64)).reshape(modes, modes, 4)
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    out = np.zeros((ny, nx))
    for kx in range(modes):
        for ky in range(modes):
            c, s, px, py = u[kx, ky]
            out += (c - 0.5) * np.cos(2 * np.pi * (kx * x / nx + px)) * \
                   np.cos(2 * np.pi * (ky * y / ny + py)) + \
                   (s - 0.5) * np.sin(2 * np.pi * (kx * x / nx + ky * y / ny))
    return amp * out / max(np.abs(out).max(), 1e-300)


BASE = dict(a=0.04, kappa=0.04, gamma_mob=0.1, tau_phi=1.0)

DROP_100x50 = dict(nx=100, ny=50, R=20.0, cx=50.0, cy=-0.5, steps=2000,
                   params=dict(BASE, tau_alpha=1.0, tau_beta=1.0, h_bottom=0.0,
                               h_top=0.0, collision="bgk"))

SWEEP_200x100 = dict(nx=200, ny=100, R=40.0, cx=100.0, cy=-0.5, steps=20000,
                     angles=(60.0, 90.0, 120.0),
                     tau_pairs={1: (1.0, 1.0), 10: (1.5, 0.6)},
                     # (collision, step2_relax_momentum)
                     variants=(("bgk", False), ("mrt", False), ("mrt", True)),
                     check_every=500)

CAPILLARY_1000x120 = dict(nx=1000, ny=120, res_len=200, ch_w=40, theta=60.0, h_block=0.0,
                          steps=100000, every=500,
                          params=dict(BASE, collision="mrt", tau_alpha=1.5, tau_beta=0.6,
                                      h_bottom=0.0, h_top=0.0))

STRIPE_28x15 = dict(nx=28, ny=15, xa=7.0, xb=21.0, steps=20000,
                    taus=((10.0, 10.0), (3.0, 0.7), (1.5, 0.6)),
                    params=dict(BASE, h_bottom=0.0, h_top=0.0))

SPINODAL_8192 = dict(nx=8192, ny=8192, amp=0.1, seed=12345, steps=1000,
                     sub=512,
                     params=dict(BASE, tau_alpha=1.5, tau_beta=0.6, h_bottom=0.0,
                                 h_top=0.0, collision="mrt"))


def batch_specs(n: int = 256, seed: int = 2026, lo: int = 64, hi: int = 512):
    """Per-domain (nx, ny, R, theta_deg, ratio, tau_alpha, tau_beta) for the
    batched sessile-drop workload.  Draw 5*d + j of the stream feeds field j
    of domain d."""
    out = []
    ratios = (1, 3, 10)
    for d in range(n):
        u = uniform01(seed, np.arange(5 * d, 5 * d + 5, dtype=np.uint64))
        nx = lo + int(u[0] * (hi - lo + 1))
        ny = lo + int(u[1] * (hi - lo + 1))
        theta = 30.0 + 120.0 * float(u[2])
        ratio = ratios[int(u[3] * 3)]
        tau_beta = 0.6
        tau_alpha = 0.5 + 0.1 * ratio
        out.append(dict(nx=nx, ny=ny, R=0.3 * min(nx, ny), cx=nx / 2.0, cy=-0.5,
                        theta=theta, ratio=ratio, tau_alpha=tau_alpha,
                        tau_beta=tau_beta))
    return out
