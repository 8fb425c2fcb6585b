"""Seeded synthetic inputs for the MDF-LBM workloads.

This module produces initial pressure/velocity fields, body forces and batch
draws as plain FP64 numpy arrays.  It holds none of the lattice Boltzmann
arithmetic: both the CUDA library and the CPU oracle receive the very same
arrays from here and each turns them into populations on its own.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), implemented below from its
published definition so the draws are identical on every machine.

Array layout: node index n = x + nx*(y + ny*z); a vector field is [d][N].
Nodes sit at integer lattice coordinates x_j = j (lattice units).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Tuple

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    """SplitMix64: state += golden gamma, then a 3-step xor-shift-multiply mix."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def randint(self, lo: int, hi: int) -> int:
        """Integer in [lo, hi] (inclusive), by scaling a uniform draw."""
        return lo + min(int(self.uniform() * (hi - lo + 1)), hi - lo)


def grid_coords(n: Tuple[int, ...]):
    """Integer coordinates (x, y[, z]) of every node, x fastest, as FP64."""
    if len(n) == 2:
        nx, ny = n
        Y, X = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64),
                           indexing="ij")
        return X.ravel(), Y.ravel()
    nx, ny, nz = n
    Z, Y, X = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return X.ravel(), Y.ravel(), Z.ravel()


def taylor_green_2d(n: int, U0: float, P0: float = 1.0, offset: float = 0.0):
    """2D Taylor-Green vortex on an n x n periodic lattice, k = 2 pi / n.

    u = U0 ( sin kx cos ky, -cos kx sin ky ),
    P = P0 + (U0^2 / 4)(cos 2kx + cos 2ky)   (rho0 = 1).
    Returns (P [N], u [2][N]).
    """
    X, Y = grid_coords((n, n))
    X = X + offset
    Y = Y + offset
    k = 2.0 * math.pi / n
    u = np.stack([U0 * np.sin(k * X) * np.cos(k * Y), -U0 * np.cos(k * X) * np.sin(k * Y)])
    P = P0 + 0.25 * U0 * U0 * (np.cos(2 * k * X) + np.cos(2 * k * Y))
    return P, u


def taylor_green_3d(n: int, U0: float, P0: float = 1.0):
    """3D Taylor-Green vortex on an n^3 periodic lattice, k = 2 pi / n.

    u = U0 ( sin kx cos ky cos kz, -cos kx sin ky cos kz, 0 ),
    P = P0 + (U0^2 / 16)(cos 2kx + cos 2ky)(cos 2kz + 2).
    """
    X, Y, Z = grid_coords((n, n, n))
    k = 2.0 * math.pi / n
    u = np.stack([
        U0 * np.sin(k * X) * np.cos(k * Y) * np.cos(k * Z),
        -U0 * np.cos(k * X) * np.sin(k * Y) * np.cos(k * Z),
        np.zeros_like(X),
    ])
    P = P0 + (U0 * U0 / 16.0) * (np.cos(2 * k * X) + np.cos(2 * k * Y)) * (np.cos(2 * k * Z) + 2.0)
    return P, u


@dataclass
class FourierMode:
    mx: int
    my: int
    phase: float
    amp: float  # streamfunction amplitude a_m; velocity amplitude is a_m |k_m|


def random_modes(n: int, seed: int = 2108, count: int = 8, mmax: int = 8,
                 total_amp: float = 0.01) -> List[FourierMode]:
    """Seeded divergence-free modes psi_m = a_m cos(k_m . x + phi_m).

    Wave numbers (mx, my) are drawn uniformly from [-mmax, mmax]^2 without
    (0, 0); phases from [0, 2 pi).  Each mode's velocity amplitude is
    total_amp / count, so the sum never exceeds total_amp.
    """
    rng = SplitMix64(seed)
    modes = []
    while len(modes) < count:
        mx = rng.randint(-mmax, mmax)
        my = rng.randint(-mmax, mmax)
        phase = 2.0 * math.pi * rng.uniform()
        if mx == 0 and my == 0:
            continue
        kmag = 2.0 * math.pi / n * math.hypot(mx, my)
        modes.append(FourierMode(mx, my, phase, (total_amp / count) / kmag))
    return modes


def modes_velocity(n: int, modes: List[FourierMode], X=None, Y=None):
    """u = d psi / dy, v = -d psi / dx of the summed modes at the given nodes."""
    if X is None:
        X, Y = grid_coords((n, n))
    u = np.zeros((2, X.size))
    k0 = 2.0 * math.pi / n
    for m in modes:
        kx, ky = k0 * m.mx, k0 * m.my
        s = np.sin(kx * X + ky * Y + m.phase)
        u[0] += -m.amp * ky * s
        u[1] += m.amp * kx * s
    return u


def tg_plus_modes(n: int, U0: float = 0.01, seed: int = 2108, P0: float = 1.0):
    """Taylor-Green vortex plus 8 seeded divergence-free Fourier modes.

    The pressure is the Taylor-Green pressure alone.  Returns (P, u).
    """
    P, u = taylor_green_2d(n, U0, P0)
    u = u + modes_velocity(n, random_modes(n, seed))
    return P, u


def window(n: int, fields, cx: int, cy: int, half: int):
    """Periodic (2*half+1)^2 window of 2D fields centred on node (cx, cy)."""
    idx = (np.arange(-half, half + 1))
    ys = (cy + idx) % n
    xs = (cx + idx) % n
    sel = (ys[:, None] * n + xs[None, :]).ravel()
    return [f[..., sel] for f in fields]


def four_roll_mill_force(N: int, U0: float, nu: float, dx: float, offset: float = 0.0):
    """Body force of the simplified four-roll mill on [0, 2 pi]^2 (Sec. 4.2).

    F1 = U0^2 sin x cos x + 2 nu U0 sin x cos y,
    F2 = U0^2 sin y cos y - 2 nu U0 sin y cos x, at x_j = (j + offset) dx.
    """
    X, Y = grid_coords((N, N))
    X = (X + offset) * dx
    Y = (Y + offset) * dx
    F1 = U0 * U0 * np.sin(X) * np.cos(X) + 2 * nu * U0 * np.sin(X) * np.cos(Y)
    F2 = U0 * U0 * np.sin(Y) * np.cos(Y) - 2 * nu * U0 * np.sin(Y) * np.cos(X)
    return np.stack([F1, F2])


def cavity_batch(count: int = 64, seed: int = 2108, sides=(65, 129, 257, 513),
                 re_range=(100.0, 3200.0)):
    """Seeded batch of lid-driven cavities: (side, Re) pairs."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(count):
        side = sides[rng.randint(0, len(sides) - 1)]
        re = re_range[0] + (re_range[1] - re_range[0]) * rng.uniform()
        out.append((side, re))
    return out


def rest_state(N: int, d: int, P0: float = 1.0):
    return np.full(N, P0), np.zeros((d, N))


def smooth_fields(n: Tuple[int, ...], seed: int, amp: float = 0.02, mean_flow: bool = True):
    """Seeded smooth periodic (P, u) on any grid shape (2D or 3D).

    A few low Fourier modes with SplitMix64 phases; the velocity is not
    divergence-free on purpose (it exercises the pressure and the
    compressible transient of the scheme).  Returns (P [N], u [d][N]).
    """
    rng = SplitMix64(seed)
    d = len(n)
    C = grid_coords(tuple(n))
    two_pi = 2.0 * math.pi
    ph = [two_pi * rng.uniform() for _ in range(2 * d + 1)]
    P = 1.0 + 0.1 * amp * np.cos(two_pi * C[0] / n[0] + ph[0]) * np.cos(two_pi * C[1] / n[1] + ph[1])
    u = np.empty((d, C[0].size))
    for a in range(d):
        b = (a + 1) % d
        arg = two_pi * ((a + 1) * C[a] / n[a] + (2 - a % 2) * C[b] / n[b]) + ph[2 + a]
        u[a] = amp * np.sin(arg)
        if mean_flow:
            u[a] += 0.1 * amp * (1.0 - 2.0 * rng.uniform())
    return P, u
