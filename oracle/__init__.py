"""FP64 CPU oracle of the MDF-LBM (Chai, Shi & Zhan, arXiv 2108.08591).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library never does, and it shares no code with it.

The arithmetic lives in ``mdf_oracle.c`` (plain C, FP64); this module compiles
it with gcc and marshals numpy arrays through ctypes.  Arrays are FP64 and
x-fastest: a scalar field is ``[nz][ny][nx]`` flattened to ``N`` nodes, a
vector field ``[d][N]``, populations ``[nsets][q][N]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mdf_oracle.c")
_LIB = os.path.join(_HERE, "_mdf_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_mdf_oracle.so`` (gcc, OpenMP)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "mdf_oracle.h")))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fopenmp", "-fPIC",
               "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int), ("q", ctypes.c_int), ("with_rho", ctypes.c_int),
        ("n", ctypes.c_int * 3), ("wall", ctypes.c_int * 3), ("lid", ctypes.c_int),
        ("lid_u", ctypes.c_double * 3), ("dx", ctypes.c_double), ("dt", ctypes.c_double),
        ("s0", ctypes.c_double), ("s1", ctypes.c_double), ("s2", ctypes.c_double),
        ("rho0", ctypes.c_double), ("force", ctypes.POINTER(ctypes.c_double)),
        ("scheme", ctypes.c_int),
    ]


def _dptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER(_Problem)
        dp = ctypes.POINTER(ctypes.c_double)
        sig = {
            "orc_lattice": [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp, dp],
            "orc_moment_basis": [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double, dp, dp],
            "orc_collision_matrix": [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, dp],
            "orc_init": [P, dp, dp, dp],
            "orc_init_neq": [P, dp, dp, dp, dp],
            "orc_mask": [P, ctypes.POINTER(ctypes.c_ubyte)],
            "orc_step": [P, dp, dp, dp],
            "orc_run": [P, ctypes.c_long, dp],
            "orc_macro": [P, dp, dp, dp, dp],
            "orc_derived": [P, dp, dp, dp, dp, dp, dp],
            "orc_sums": [P, dp, dp],
            "orc_threads": [],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        _lib = L
    return _lib


def s2_rule(s1: float) -> float:
    """Default s2 = 8(2 - s1)/(8 - s1) of the paper's experiments (Sec. 4.1)."""
    return 8.0 * (2.0 - s1) / (8.0 - s1)


@dataclass
class Problem:
    """One MDF-LBM problem in physical units (lattice units: dx = dt = 1)."""
    d: int
    n: Sequence[int]
    s1: float
    s2: Optional[float] = None
    s0: float = 1.0
    with_rho: bool = True
    wall: Sequence[int] = (0, 0, 0)
    lid: bool = False
    lid_u: Sequence[float] = (0.0, 0.0, 0.0)
    dx: float = 1.0
    dt: float = 1.0
    rho0: float = 1.0
    force: Optional[np.ndarray] = None  # [d][N] body force at nodes
    scheme: int = 0  # forcing: 0 = Eq. 3-21, 2 = Scheme II (Eq. 2-3c, 2-7a; state is fbar)
    nq: int = 0  # directions: 0 = D2Q5 / D3Q7; 4 = D2Q4, 6 = D3Q6 (no rest direction)
    _c: _Problem = field(default=None, repr=False)

    @property
    def q(self) -> int:
        return self.nq if self.nq else (5 if self.d == 2 else 7)

    @property
    def N(self) -> int:
        n = list(self.n) + [1] * (3 - len(self.n))
        return int(n[0] * n[1] * n[2])

    @property
    def nsets(self) -> int:
        return self.d + 1 if self.with_rho else self.d

    def shape(self):
        n = list(self.n) + [1] * (3 - len(self.n))
        return (n[2], n[1], n[0]) if self.d == 3 else (n[1], n[0])

    def c_struct(self) -> _Problem:
        n = list(self.n) + [1] * (3 - len(self.n))
        pb = _Problem()
        pb.d, pb.q, pb.with_rho = self.d, self.q, int(bool(self.with_rho))
        pb.n[:] = [int(v) for v in n]
        w = list(self.wall) + [0] * (3 - len(self.wall))
        pb.wall[:] = [int(v) for v in w]
        pb.lid = int(bool(self.lid))
        lu = list(self.lid_u) + [0.0] * (3 - len(self.lid_u))
        pb.lid_u[:] = [float(v) for v in lu]
        pb.dx, pb.dt = float(self.dx), float(self.dt)
        pb.s0, pb.s1 = float(self.s0), float(self.s1)
        pb.s2 = float(s2_rule(self.s1) if self.s2 is None else self.s2)
        pb.rho0 = float(self.rho0)
        if self.force is not None:
            self.force = np.ascontiguousarray(self.force, dtype=np.float64).reshape(self.d, self.N)
            pb.force = _dptr(self.force)
        else:
            pb.force = None
        pb.scheme = int(self.scheme)
        self._c = pb
        return pb


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed ({rc})")


def lattice(d: int, q: int, c: float = 1.0):
    cv = np.zeros(21)
    w = np.zeros(7)
    cs2 = ctypes.c_double()
    _check(lib().orc_lattice(d, q, c, _dptr(cv), _dptr(w), ctypes.byref(cs2)), "lattice")
    return cv.reshape(7, 3)[:q, :d].copy(), w[:q].copy(), cs2.value


def moment_basis(d: int, q: int, c: float, s0: float, s1: float, s2: float):
    M = np.zeros(q * q)
    S = np.zeros(q)
    _check(lib().orc_moment_basis(d, q, c, s0, s1, s2, _dptr(M), _dptr(S)), "basis")
    return M.reshape(q, q), S


def collision_matrix(d: int, q: int, c: float, s0: float, s1: float, s2: float):
    L = np.zeros(q * q)
    _check(lib().orc_collision_matrix(d, q, c, s0, s1, s2, _dptr(L)), "collision matrix")
    return L.reshape(q, q)


def init(pb: Problem, P: np.ndarray, u: np.ndarray, G: Optional[np.ndarray] = None) -> np.ndarray:
    """f = f^eq(P, u) for every set, plus the first-order non-equilibrium part
    of the velocity gradient G [d][d][N] (G[a][b] = du_a/dx_b) when given;
    returns populations [nsets][q][N]."""
    P = np.ascontiguousarray(P, dtype=np.float64).reshape(pb.N)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(pb.d, pb.N)
    f = np.zeros((pb.nsets, pb.q, pb.N))
    if G is None:
        _check(lib().orc_init(ctypes.byref(pb.c_struct()), _dptr(P), _dptr(u), _dptr(f)), "init")
    else:
        G = np.ascontiguousarray(G, dtype=np.float64).reshape(pb.d, pb.d, pb.N)
        _check(lib().orc_init_neq(ctypes.byref(pb.c_struct()), _dptr(P), _dptr(u), _dptr(G),
                                  _dptr(f)), "init")
    return f


def run(pb: Problem, f: np.ndarray, nsteps: int) -> np.ndarray:
    """Advance ``f`` in place by ``nsteps`` time steps and return it."""
    assert f.shape == (pb.nsets, pb.q, pb.N) and f.dtype == np.float64
    _check(lib().orc_run(ctypes.byref(pb.c_struct()), int(nsteps), _dptr(f)), "run")
    return f


def macro(pb: Problem, f: np.ndarray):
    """(P, u, rho): pressure Eq. 3-15, velocity and rho from Eq. 2-7."""
    P = np.zeros(pb.N)
    u = np.zeros((pb.d, pb.N))
    rho = np.zeros(pb.N) if pb.with_rho else None
    _check(lib().orc_macro(ctypes.byref(pb.c_struct()), _dptr(f), _dptr(P), _dptr(u),
                           _dptr(rho)), "macro")
    return P, u, rho


def derived(pb: Problem, f: np.ndarray) -> dict:
    """Eq. 3-16 .. 3-19: G[a][b] = du_a/dx_b, div, S, sigma, omega."""
    d, N = pb.d, pb.N
    nsym = 3 if d == 2 else 6
    out = {
        "G": np.zeros((d, d, N)), "div": np.zeros(N), "S": np.zeros((nsym, N)),
        "sigma": np.zeros((nsym, N)), "omega": np.zeros((1 if d == 2 else 3, N)),
    }
    _check(lib().orc_derived(ctypes.byref(pb.c_struct()), _dptr(f), _dptr(out["G"]),
                             _dptr(out["div"]), _dptr(out["S"]), _dptr(out["sigma"]),
                             _dptr(out["omega"])), "derived")
    return out


def mask(pb: Problem) -> np.ndarray:
    m = np.zeros(pb.N, dtype=np.uint8)
    _check(lib().orc_mask(ctypes.byref(pb.c_struct()),
                          m.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))), "mask")
    return m


def sums(pb: Problem, f: np.ndarray) -> np.ndarray:
    s = np.zeros(pb.nsets)
    _check(lib().orc_sums(ctypes.byref(pb.c_struct()), _dptr(f), _dptr(s)), "sums")
    return s


def threads() -> int:
    return int(lib().orc_threads())


def rel_l2(ref: np.ndarray, num: np.ndarray) -> float:
    """E_L2 = ||ref - num||_2 / ||ref||_2 (Sec. 4)."""
    ref = np.asarray(ref, dtype=np.float64)
    num = np.asarray(num, dtype=np.float64)
    return float(np.linalg.norm((ref - num).ravel()) / np.linalg.norm(ref.ravel()))
