"""GB300-native MDF-LBM (Chai, Shi & Zhan, arXiv 2108.08591).

Thin Python binding over the C-ABI of ``libmdf.so`` (include/mdf.h).  Every
step of the method runs in the library's CUDA kernels; this module only
marshals arguments.  PyTorch supplies device memory for outputs and the
CUDA stream the library enqueues on.
"""
from __future__ import annotations

import ctypes
from typing import Dict, Iterable, Optional, Sequence

import numpy as np

from . import _lib
from ._lib import DEVICE, HOST, MdfError, STORAGE

__all__ = ["Lattice", "Slabs", "CavityBatch", "MdfError", "FIELD_NAMES", "field_shapes"]

FIELD_NAMES = ("P", "u", "rho", "G", "div", "S", "sigma", "omega")


def field_shapes(d: int, N: int) -> Dict[str, tuple]:
    nsym = 3 if d == 2 else 6
    return {"P": (N,), "u": (d, N), "rho": (N,), "G": (d, d, N), "div": (N,),
            "S": (nsym, N), "sigma": (nsym, N), "omega": ((1 if d == 2 else 3), N)}


def _ptr(a) -> Optional[int]:
    """Address of a contiguous FP64 numpy array or torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags.c_contiguous, "need contiguous float64"
        return a.ctypes.data
    assert a.dtype.is_floating_point and a.element_size() == 8 and a.is_contiguous(), \
        "need a contiguous float64 tensor"
    return a.data_ptr()


def _is_device(a) -> bool:
    return not isinstance(a, np.ndarray) and a.is_cuda


class Lattice:
    """One MDF-LBM lattice: d + 1 (or d) D2Q5/D3Q7 distribution sets.

    shape: (nx, ny) or (nx, ny, nz).  s1 sets the viscosity
    nu = (1/s1 - 1/2) c_s^2 (Eq. 3-13a); s2 < 0 picks the paper's rule.
    wall: per-axis halfway walls (anti-halfway bounce-back), lid: the + face
    of the last axis moves with lid_u.  storage: 'f32', 'f16', 'bf16', 'f64',
    'f16eq', 'bf16eq'.  vx / block: x-nodes per thread and threads per block
    of the update kernel (0: the library's tuned default).  q: 0 for
    D2Q5 / D3Q7, 4 for D2Q4, 6 for D3Q6 (rest-shifted storage types only).
    inplace: one population buffer streamed in place by the AA pattern
    (rest-shifted storage types; half the memory, the same results).
    """

    def __init__(self, shape: Sequence[int], s1: float, s2: float = -1.0, s0: float = 1.0,
                 wall: Sequence[int] = (0, 0, 0), lid: bool = False,
                 lid_u: Sequence[float] = (0.0, 0.0, 0.0), storage: str = "f32",
                 with_rho: bool = True, stream=None, vx: int = 0, block: int = 0, q: int = 0,
                 inplace: bool = False):
        import torch

        self._lib = _lib.load()
        self.d = len(shape)
        if self.d not in (2, 3):
            raise ValueError("shape must have 2 or 3 entries")
        nx, ny = int(shape[0]), int(shape[1])
        nz = int(shape[2]) if self.d == 3 else 1
        self.shape = tuple(int(v) for v in shape)
        self.N = nx * ny * nz
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        sptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        g = _lib.Grid(nx, ny, nz)
        r = _lib.Rates(s0, s1, s2)
        bc = _lib.BC()
        w = list(wall) + [0] * (3 - len(wall))
        bc.wall[:] = [int(v) for v in w[:3]]
        bc.lid = int(bool(lid))
        lu = list(lid_u) + [0.0] * (3 - len(lid_u))
        bc.lid_u[:] = [float(v) for v in lu[:3]]
        o = _lib.Opts(STORAGE[storage], int(bool(with_rho)), ctypes.c_void_p(sptr), int(vx), int(block),
                      int(q), int(bool(inplace)))
        h = ctypes.c_void_p()
        _lib.check(self._lib.mdf_create(ctypes.byref(h), ctypes.byref(g), self.d,
                                        ctypes.byref(r), ctypes.byref(bc), ctypes.byref(o)))
        self._h = h
        self.with_rho = bool(with_rho)
        self.storage = storage
        self._keep = []  # device inputs that must outlive queued work

    # ------------------------------------------------------------------
    def _check(self, status: int):
        _lib.check(status, self._h)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mdf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def info(self) -> _lib.Info:
        inf = _lib.Info()
        self._check(self._lib.mdf_info(self._h, ctypes.byref(inf)))
        return inf

    # ------------------------------------------------------------------
    def init(self, P, u, G=None):
        """f = f^eq(P, u); P [N], u [d][N] FP64, numpy (host) or CUDA tensors.
        With G [d][d][N] (G[a][b] = du_a/dx_b) the state also carries the
        first-order non-equilibrium part of that gradient (mdf_init_neq)."""
        dev = _is_device(P)
        if dev != _is_device(u) or (G is not None and dev != _is_device(G)):
            raise ValueError("P, u (and G) must all be on the host or all on the device")
        if dev:
            self._keep = [P, u, G]
        where = DEVICE if dev else HOST
        if G is None:
            self._check(self._lib.mdf_init(self._h, _ptr(P), _ptr(u), where))
        else:
            self._check(self._lib.mdf_init_neq(self._h, _ptr(P), _ptr(u), _ptr(G), where))

    def set_force(self, F):
        """Body force Fbar [d][N] (Eq. 2-6); None removes it."""
        if F is None:
            self._check(self._lib.mdf_set_force(self._h, None, HOST))
            return
        self._check(self._lib.mdf_set_force(self._h, _ptr(F), DEVICE if _is_device(F) else HOST))

    FORCING = {"eq3-21": 0, "scheme2": 2}

    def set_forcing(self, scheme: str):
        """'eq3-21' (default, Eq. 3-21) or 'scheme2' (Scheme II, Eq. 2-3c and
        2-7a: the state is fbar = f - dt F/2).  Set it, and the force, before
        init: the Scheme II initial state is f^eq - dt F/2."""
        self._check(self._lib.mdf_set_forcing(self._h, self.FORCING[scheme]))

    @property
    def forcing(self) -> str:
        v = ctypes.c_int()
        self._check(self._lib.mdf_get_forcing(self._h, ctypes.byref(v)))
        return {k: n for n, k in self.FORCING.items()}[v.value]

    def step(self, n: int = 1):
        self._check(self._lib.mdf_step(self._h, int(n)))

    def _fields_struct(self, out: Dict[str, object], where: int) -> _lib.Fields:
        f = _lib.Fields()
        for k, v in out.items():
            setattr(f, k, _ptr(v))
        f.where = where
        return f

    def alloc_fields(self, names: Iterable[str] = FIELD_NAMES):
        import torch
        shapes = field_shapes(self.d, self.N)
        return {k: torch.empty(shapes[k], dtype=torch.float64, device="cuda") for k in names
                if k != "rho" or self.with_rho}

    def step_fields(self, n: int, out: Dict[str, object]):
        """n updates; the first also writes the fields of the starting state."""
        f = self._fields_struct(out, DEVICE)
        self._check(self._lib.mdf_step_fields(self._h, int(n), ctypes.byref(f)))

    def fields(self, names: Iterable[str] = ("P", "u"), out: Optional[Dict[str, object]] = None):
        """Derived fields of the current state as CUDA tensors (Eq. 2-7, 3-15 .. 3-19)."""
        if out is None:
            out = self.alloc_fields(names)
        f = self._fields_struct(out, DEVICE)
        self._check(self._lib.mdf_fields(self._h, ctypes.byref(f)))
        return out

    def fields_host(self, names: Iterable[str] = ("P", "u"), out=None) -> Dict[str, np.ndarray]:
        """Derived fields copied to host numpy arrays (synchronises)."""
        shapes = field_shapes(self.d, self.N)
        if out is None:
            out = {k: np.empty(shapes[k]) for k in names}
        f = self._fields_struct(out, HOST)
        self._check(self._lib.mdf_fields(self._h, ctypes.byref(f)))
        return out

    def fields_host_noalloc(self, names: Iterable[str] = ("P", "u"), out=None) -> Dict[str, np.ndarray]:
        """As fields_host(), but the library allocates no device memory: the
        fields are staged in its fixed 16 MiB buffer (at most 2,097,152
        doubles per call; calls from several threads must not overlap)."""
        shapes = field_shapes(self.d, self.N)
        if out is None:
            out = {k: np.empty(shapes[k]) for k in names}
        f = self._fields_struct(out, HOST)
        self._check(self._lib.mdf_fields_host_noalloc(self._h, ctypes.byref(f)))
        return out

    def moments(self):
        """(P, u, rho) of the current state as CUDA tensors (mdf_moments);
        rho is None without the alpha = 0 set."""
        o = self.alloc_fields(("P", "u", "rho") if self.with_rho else ("P", "u"))
        self._check(self._lib.mdf_moments(self._h, _ptr(o["P"]), _ptr(o["u"]), _ptr(o.get("rho"))))
        return o["P"], o["u"], o.get("rho")

    def gradients(self):
        """G, div, S, sigma and omega of the current state as CUDA tensors
        (mdf_gradients)."""
        o = self.alloc_fields(("G", "div", "S", "sigma", "omega"))
        self._check(self._lib.mdf_gradients(self._h, *(_ptr(o[k]) for k in
                                                       ("G", "div", "S", "sigma", "omega"))))
        return o

    def sums(self) -> np.ndarray:
        out = np.zeros(4)
        self._check(self._lib.mdf_sums(self._h, out.ctypes.data))
        return out[: self.info.nsets].copy()

    def residual(self) -> float:
        out = np.zeros(1)
        self._check(self._lib.mdf_residual(self._h, out.ctypes.data))
        return float(out[0])

    def mask(self) -> np.ndarray:
        m = np.zeros(self.N, dtype=np.uint8)
        self._check(self._lib.mdf_mask(self._h, m.ctypes.data))
        return m

    def save(self, path: str):
        self._check(self._lib.mdf_save(self._h, path.encode()))

    def load(self, path: str):
        self._check(self._lib.mdf_load(self._h, path.encode()))

    def autotune(self, reps: int = 10):
        """Measure the update kernel's launch shapes and keep the fastest;
        the lattice state is unchanged.  Returns (vx, block)."""
        vx, block = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.mdf_autotune(self._h, int(reps), ctypes.byref(vx), ctypes.byref(block)))
        return vx.value, block.value

    def sync(self):
        self._check(self._lib.mdf_sync(self._h))


class Slabs:
    """One lattice split into k slabs along its last axis, with the per-face
    exchange of the populations crossing each face after every update
    (mdf_slabs_*).  Same arguments as Lattice; the split axis is periodic."""

    def __init__(self, shape: Sequence[int], s1: float, k: int, s2: float = -1.0, s0: float = 1.0,
                 wall: Sequence[int] = (0, 0, 0), storage: str = "f32", with_rho: bool = True,
                 stream=None, q: int = 0):
        import torch

        self._lib = _lib.load()
        self.d = len(shape)
        nx, ny = int(shape[0]), int(shape[1])
        nz = int(shape[2]) if self.d == 3 else 1
        self.shape = tuple(int(v) for v in shape)
        self.N = nx * ny * nz
        self.with_rho = bool(with_rho)
        if stream is None:
            stream = torch.cuda.current_stream()
        sptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        g = _lib.Grid(nx, ny, nz)
        r = _lib.Rates(s0, s1, s2)
        bc = _lib.BC()
        w = list(wall) + [0] * (3 - len(wall))
        bc.wall[:] = [int(v) for v in w[:3]]
        o = _lib.Opts(STORAGE[storage], int(self.with_rho), ctypes.c_void_p(sptr), 0, 0, int(q), 0)
        h = ctypes.c_void_p()
        _lib.check_slabs(self._lib.mdf_slabs_create(ctypes.byref(h), ctypes.byref(g), self.d, ctypes.byref(r),
                                                    ctypes.byref(bc), ctypes.byref(o), int(k)))
        self._h = h

    def _check(self, status: int):
        _lib.check_slabs(status, self._h)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mdf_slabs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, P, u):
        """f = f^eq(P, u) from host FP64 arrays P [N], u [d][N]."""
        P = np.ascontiguousarray(P, dtype=np.float64)
        u = np.ascontiguousarray(u, dtype=np.float64)
        self._check(self._lib.mdf_slabs_init(self._h, _ptr(P), _ptr(u)))

    def step(self, n: int = 1):
        self._check(self._lib.mdf_slabs_step(self._h, int(n)))

    def fields_host(self, names: Iterable[str] = ("P", "u")) -> Dict[str, np.ndarray]:
        shapes = field_shapes(self.d, self.N)
        out = {k: np.empty(shapes[k]) for k in names}
        f = _lib.Fields()
        for k, v in out.items():
            setattr(f, k, _ptr(v))
        f.where = HOST
        self._check(self._lib.mdf_slabs_fields(self._h, ctypes.byref(f)))
        return out


class CavityBatch:
    """Many lid-driven cavities (closed boxes, lid on the + face of the last
    axis moving along x) advanced together to steady state by one persistent
    kernel per convergence period (see mdf_batch_* in include/mdf.h)."""

    def __init__(self, sides: Sequence[int], Re: Sequence[float], lid_speed: float = 0.1,
                 d: int = 2, with_rho: bool = True, stream=None):
        import torch

        self._lib = _lib.load()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        sptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self.sides = np.ascontiguousarray(sides, dtype=np.int32)
        self.Re = np.ascontiguousarray(Re, dtype=np.float64)
        self.d = d
        self.n = len(self.sides)
        self.with_rho = bool(with_rho)
        o = _lib.Opts(STORAGE["f32"], int(bool(with_rho)), ctypes.c_void_p(sptr), 0, 0)
        h = ctypes.c_void_p()
        _lib.check_batch(self._lib.mdf_batch_create(ctypes.byref(h), d, self.n, self.sides.ctypes.data,
                                                    self.Re.ctypes.data, float(lid_speed), ctypes.byref(o)))
        self._h = h
        self.init()

    def _check(self, status: int):
        _lib.check_batch(status, self._h)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mdf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, cavity: int = -1, P=None, u=None, neq: bool = False):
        """Rest state (P = u = None) or f = f^eq(P, u) for one cavity; with
        neq, plus the non-equilibrium part of the seed's velocity gradient
        (see mdf_batch_seed)."""
        dev = P is not None and _is_device(P)
        self._check(self._lib.mdf_batch_seed(self._h, int(cavity), _ptr(P), _ptr(u),
                                             DEVICE if dev else HOST, int(bool(neq))))

    def run(self, tol: float = 1e-8, max_steps: int = 2_000_000, check_every: int = 100):
        """Run to steady state; returns (steps, status, residual) arrays.
        status: 0 converged, 4 diverged, 6 not converged (mdf_status codes)."""
        steps = np.zeros(self.n, dtype=np.int64)
        status = np.zeros(self.n, dtype=np.int32)
        res = np.zeros(self.n)
        rc = self._lib.mdf_batch_run(self._h, float(tol), int(max_steps), int(check_every),
                                     steps.ctypes.data, status.ctypes.data, res.ctypes.data)
        if rc not in (_lib.OK, _lib.EDIVERGED, _lib.ENOTCONVERGED):
            self._check(rc)
        return steps, status, res

    def step(self, n: int):
        self._check(self._lib.mdf_batch_step(self._h, int(n)))

    def set_timeout(self, cycles: int):
        """Grid-barrier spin limit in SM clock cycles (default ~2 s)."""
        self._check(self._lib.mdf_batch_set_timeout(self._h, int(cycles)))

    def set_schedule(self, threads: int = 128, grid: int = 0, sched: int = 0):
        """Launch shape of the persistent step kernel (see mdf_batch_set_schedule)."""
        self._check(self._lib.mdf_batch_set_schedule(self._h, int(threads), int(grid), int(sched)))

    def schedule(self) -> Dict[str, int]:
        v = np.zeros(3, np.int32)
        self._check(self._lib.mdf_batch_get_schedule(self._h, v[0:].ctypes.data, v[1:].ctypes.data,
                                                     v[2:].ctypes.data))
        return {"threads": int(v[0]), "grid": int(v[1]), "sched": int(v[2])}

    def autotune(self, reps: int = 20) -> Dict[str, int]:
        """Time every schedule on the current state, keep the fastest, restore
        the state; returns the chosen {threads, grid, sched}."""
        v = np.zeros(3, np.int32)
        self._check(self._lib.mdf_batch_autotune(self._h, int(reps), v[0:].ctypes.data, v[1:].ctypes.data,
                                                 v[2:].ctypes.data))
        return {"threads": int(v[0]), "grid": int(v[1]), "sched": int(v[2])}

    def fields_host(self, cavity: int, names: Iterable[str] = ("P", "u")) -> Dict[str, np.ndarray]:
        N = int(self.sides[cavity]) ** self.d
        shapes = field_shapes(self.d, N)
        out = {k: np.empty(shapes[k]) for k in names}
        f = _lib.Fields()
        for k, v in out.items():
            setattr(f, k, _ptr(v))
        f.where = HOST
        self._check(self._lib.mdf_batch_fields(self._h, int(cavity), ctypes.byref(f)))
        return out

    def info(self):
        nodes, tiles, grid = np.zeros(1, np.int64), np.zeros(1, np.int32), np.zeros(1, np.int32)
        self._check(self._lib.mdf_batch_info(self._h, nodes.ctypes.data, tiles.ctypes.data,
                                             grid.ctypes.data))
        return int(nodes[0]), int(tiles[0]), int(grid[0])


class WarmStartNet:
    """The warm-start U-Net (mdf_ws_* in include/mdf.h): forward, training
    step and parameters; tensors are CUDA float32 NHWC."""

    def __init__(self, H: int, W: int, channels: Sequence[int] = (32, 64, 128, 256), cin: int = 16,
                 cout: int = 16, cout_used: int = 3, max_batch: int = 8, seed: int = 2108,
                 stream=None):
        import torch

        self._lib = _lib.load()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        sptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        ch = np.ascontiguousarray(channels, dtype=np.int32)
        h = ctypes.c_void_p()
        _lib.check_ws(self._lib.mdf_ws_create(ctypes.byref(h), H, W, len(ch), ch.ctypes.data, cin, cout,
                                              cout_used, max_batch, seed, ctypes.c_void_p(sptr)))
        self._h = h
        self.H, self.W, self.channels = H, W, tuple(int(c) for c in channels)
        self.cin, self.cout, self.cout_used, self.max_batch = cin, cout, cout_used, max_batch

    def _check(self, status: int):
        _lib.check_ws(status, self._h)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mdf_ws_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nparam(self) -> int:
        return int(self._lib.mdf_ws_param_count(self._h))

    def get_params(self, grads: bool = False):
        p = np.empty(self.nparam, dtype=np.float32)
        g = np.empty(self.nparam, dtype=np.float32) if grads else None
        self._check(self._lib.mdf_ws_get_params(self._h, p.ctypes.data,
                                                None if g is None else g.ctypes.data))
        return (p, g) if grads else p

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._check(self._lib.mdf_ws_set_params(self._h, p.ctypes.data))

    def forward(self, x):
        import torch
        y = torch.empty((x.shape[0], self.H, self.W, self.cout), dtype=torch.float32, device=x.device)
        self._check(self._lib.mdf_ws_forward(self._h, x.data_ptr(), x.shape[0], y.data_ptr()))
        return y

    def train_step(self, x, t, lr: float, want_loss: bool = True):
        loss = np.zeros(1)
        self._check(self._lib.mdf_ws_train_step(self._h, x.data_ptr(), t.data_ptr(), x.shape[0],
                                                float(lr), loss.ctypes.data if want_loss else None))
        return float(loss[0]) if want_loss else None


CONV_KERNELS = {"mma.sync": 0, "tcgen05": 1, "tcgen05-halo": 2}


def set_conv_kernel(which: str):
    """Forward/dgrad convolution kernel: 'tcgen05-halo' (default), 'tcgen05'
    (im2col gathers) or 'mma.sync'."""
    _lib.check(_lib.load().mdf_nn_set_conv_kernel(CONV_KERNELS[which]))


def set_wgrad_kernel(which: str):
    """Weight-gradient kernel: 'tcgen05' (default) or 'mma.sync'."""
    _lib.check(_lib.load().mdf_nn_set_wgrad_kernel({"mma.sync": 0, "tcgen05": 1}[which]))


def set_wgrad_tile(bn: int = 0, ctas_per_sm: int = 0, kc: int = 0):
    """Launch shape of the tcgen05 weight gradient: N tile of 16, 32 or 64
    channels, the CTAs per SM its pipeline depth leaves room for and the
    pixel positions per stage, 64 or 128 (0: automatic, each)."""
    _lib.check(_lib.load().mdf_nn_set_wgrad_tile(int(bn), int(ctas_per_sm), int(kc)))


def conv_timeout_flag() -> int:
    """Read and clear the tcgen05 kernel's time-out flag (synchronises)."""
    f = np.zeros(1, dtype=np.int32)
    _lib.check(_lib.load().mdf_nn_conv_error(f.ctypes.data))
    return int(f[0])


def conv3x3_bf16(x, w, bias=None, relu=False, out_fp32=True):
    """The library's tensor-core convolution on CUDA tensors (bf16 x, w)."""
    import torch
    lib = _lib.load()
    B, H, W, Cin = x.shape
    Cout = w.shape[0]
    y = torch.empty((B, H, W, Cout), device=x.device,
                    dtype=torch.float32 if out_fp32 else torch.bfloat16)
    s = torch.cuda.current_stream().cuda_stream
    _lib.check(lib.mdf_nn_conv_fwd(x.data_ptr(), w.data_ptr(), None if bias is None else bias.data_ptr(),
                                   None if out_fp32 else y.data_ptr(), y.data_ptr() if out_fp32 else None,
                                   B, H, W, Cin, Cout, int(relu), ctypes.c_void_p(s)))
    return y


def conv3x3_bf16_wgrad(x, dz):
    """dw fp32 [Cout, 3, 3, Cin] of the library's weight-gradient kernel
    (the one set_wgrad_kernel selects) for NHWC bf16 x and dz."""
    import torch
    lib = _lib.load()
    B, H, W, Cin = x.shape
    Cout = dz.shape[3]
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    part = torch.empty(int(lib.mdf_nn_wgrad_scratch(B, H, W, Cin, Cout)), dtype=torch.float32, device=x.device)
    dw = torch.empty((Cout, 3, 3, Cin), dtype=torch.float32, device=x.device)
    _lib.check(lib.mdf_nn_conv_wgrad(x.data_ptr(), dz.data_ptr(), dw.data_ptr(), part.data_ptr(), B, H, W,
                                     Cin, Cout, s))
    return dw


def conv3x3_bf16_backward(x, w, dz):
    """(dx bf16, dw fp32) of the library's convolution kernels."""
    import torch
    lib = _lib.load()
    B, H, W, Cin = x.shape
    Cout = w.shape[0]
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    part = torch.empty(int(lib.mdf_nn_wgrad_scratch(B, H, W, Cin, Cout)), dtype=torch.float32, device=x.device)
    dw = torch.empty((Cout, 3, 3, Cin), dtype=torch.float32, device=x.device)
    _lib.check(lib.mdf_nn_conv_wgrad(x.data_ptr(), dz.data_ptr(), dw.data_ptr(), part.data_ptr(), B, H, W,
                                     Cin, Cout, s))
    wt = torch.empty(Cout * 9 * Cin, dtype=torch.bfloat16, device=x.device)
    dx = torch.empty((B, H, W, Cin), dtype=torch.bfloat16, device=x.device)
    _lib.check(lib.mdf_nn_conv_dgrad(dz.data_ptr(), w.data_ptr(), wt.data_ptr(), dx.data_ptr(), B, H, W,
                                     Cin, Cout, s))
    return dx, dw
