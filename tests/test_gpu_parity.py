"""GPU-vs-oracle parity of the MDF-LBM stepper through the C-ABI.

Tolerances (relative L2, Sec. 4's E_L2; the pressure by its fluctuation
P - mean(P)):
  * FP64 storage (FP64 arithmetic): u, P within 1e-10; derived fields within
    1e-8 (the oracle itself carries ~1e-12 cancellation noise in f^ne).
  * FP32 storage: u, P within 1e-5.  Derived fields within 1e-4: one FP32
    rounding of a shifted population (|g| ~ 3e-3, ulp ~ 2e-10) against the
    first moment of f^ne (~1e-4 .. 1e-5 at these sizes) gives ~1e-6 per node.
  * Equilibrium-shifted FP16 / BF16 storage (the 16-bit storage the
    contract names): u and P within 2e-3 (FP16: 1e-4 and 1e-3, below
    that).  Derived fields are reported per field, with bounds of 1e-2
    (FP16) and 5e-2 (BF16): the 16-bit rounding lands on f^ne itself, whose
    first moment they are.
  * Rest-shifted FP16 / BF16 storage: reported, no contract.  The pressure
    fluctuation P' ~ U^2 is carried by populations of size ~U, which
    rest-shifted 16-bit storage resolves only to ~2e-3 .. 5e-3 (FP16) or
    ~5e-2 (BF16, 8-bit significand) relative.  The bounds below (FP16: u
    2e-3, P 5e-3; BF16: u 2e-2, P 5e-2) guard against regressions; they are
    not the 2e-3 contract, which this storage does not meet for P.
Masks are compared byte for byte.
"""
import os
import tempfile

import numpy as np
import pytest

import oracle as O
import synth
from tests._harness import errors, rel, rel_p, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

NU = 0.01
S1_TG = 1.0 / (3 * NU + 0.5)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_08591_gb300 import _build
    _build.build()


def _tol(storage):
    """(u, P - mean P, derived fields) bounds per storage type; the
    rest-shifted f16 / bf16 rows are reported, not the contract."""
    return {"f64": (1e-10, 1e-10, 1e-8), "f32": (1e-5, 1e-5, 1e-4),
            "f16": (2e-3, 5e-3, 5e-2), "bf16": (2e-2, 5e-2, 3e-1),
            "f16eq": (1e-4, 1e-3, 1e-2), "bf16eq": (1e-3, 2e-3, 5e-2)}[storage]


# --------------------------------------------------------------------------
# 2D periodic
# --------------------------------------------------------------------------
@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_taylor_green_64_matches_oracle(storage):
    """64^2 Taylor-Green plus 8 seeded modes, 1000 steps (the small 2D case)."""
    n, steps = 64, 1000
    P, u = synth.tg_plus_modes(n, U0=0.01, seed=2108)
    got = run_gpu((n, n), P, u, steps, S1_TG, storage=storage)
    ref = run_oracle((n, n), P, u, steps, S1_TG)
    e = errors(ref, got)
    tu, tp, tg = _tol(storage)
    assert e["u"] < tu and e["P"] < tp, e
    for k in ("G", "S", "sigma", "omega"):
        assert e[k] < tg, (k, e)
    assert e["rho"] < (1e-12 if storage == "f64" else 1e-6)


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16", "f16eq", "bf16eq"])
def test_ragged_grid_2d(storage):
    """Grid spanning several 128-wide blocks with a ragged tail (nx = 300) and
    a padded pitch; smooth seeded fields with a mean flow."""
    shape, steps, s1 = (300, 37), 150, 1.55
    P, u = synth.smooth_fields(shape, seed=5, amp=0.02)
    got = run_gpu(shape, P, u, steps, s1, storage=storage)
    ref = run_oracle(shape, P, u, steps, s1)
    e = errors(ref, got)
    tu, tp, tg = _tol(storage)
    print(storage, e)
    assert e["u"] < tu and e["P"] < tp, e
    assert e["G"] < tg and e["omega"] < tg, e


@pytest.mark.parametrize("d", [2, 3])
def test_divergence_identity_fp64(d):
    """Eq. 3-15 with R = 0 makes Eq. 3-16a vanish at every node; with FP64
    storage and arithmetic the GPU fields show it to rounding."""
    shape = (128, 96) if d == 2 else (40, 24, 20)
    P, u = synth.smooth_fields(shape, seed=23)
    got = run_gpu(shape, P, u, 30, 1.7, storage="f64", names=("G", "div"))
    assert np.abs(got["G"]).max() > 1e-4
    assert np.abs(got["div"]).max() < 1e-12 * np.abs(got["G"]).max()


def test_without_continuity_set_is_identical():
    """u, P and every derived field do not depend on the alpha = 0 set."""
    shape = (70, 45)
    P, u = synth.smooth_fields(shape, seed=9)
    a = run_gpu(shape, P, u, 40, 1.3, with_rho=True)
    b = run_gpu(shape, P, u, 40, 1.3, with_rho=False)
    for k in ("P", "u", "G", "div", "S", "sigma", "omega"):
        assert np.array_equal(a[k], b[k]), k


# --------------------------------------------------------------------------
# 3D periodic
# --------------------------------------------------------------------------
@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "f16eq", "bf16eq"])
def test_d3q7_ragged_matches_oracle(storage):
    shape, steps, s1 = (150, 20, 18), 60, 1.45
    P, u = synth.smooth_fields(shape, seed=13)
    got = run_gpu(shape, P, u, steps, s1, storage=storage)
    ref = run_oracle(shape, P, u, steps, s1)
    e = errors(ref, got)
    tu, tp, tg = _tol(storage)
    print(storage, e)
    assert e["u"] < tu and e["P"] < tp, e
    for k in ("G", "S", "sigma", "omega"):
        assert e[k] < tg, (k, e)


def test_taylor_green_3d_matches_oracle():
    n, steps = 32, 200
    nu = 1.0 / 40
    s1 = 1.0 / (4 * nu + 0.5)
    P, u = synth.taylor_green_3d(n, U0=0.05)
    got = run_gpu((n, n, n), P, u, steps, s1, storage="f32")
    ref = run_oracle((n, n, n), P, u, steps, s1)
    e = errors(ref, got)
    assert e["u"] < 1e-5 and e["P"] < 1e-5, e
    assert e["omega"] < 1e-4, e


# --------------------------------------------------------------------------
# Walls, lid, force
# --------------------------------------------------------------------------
@pytest.mark.parametrize("storage", ["f64", "f32", "f16eq"])
def test_lid_driven_cavity_2d(storage):
    """Anti-halfway bounce-back walls and a moving lid on a 67 x 53 cavity."""
    shape, steps, s1 = (67, 53), 400, 1.6
    P, u = synth.rest_state(67 * 53, 2)
    kw = dict(wall=(1, 1, 0), lid=True, lid_u=(0.05, 0.0, 0.0))
    got = run_gpu(shape, P, u, steps, s1, storage=storage, **kw)
    ref = run_oracle(shape, P, u, steps, s1, **kw)
    assert np.array_equal(got["mask"], ref["mask"])
    e = errors(ref, got)
    tu, tp, tg = _tol(storage)
    assert e["u"] < tu and e["P"] < tp, e
    assert e["G"] < tg and e["omega"] < tg, e


def test_cavity_3d_and_non_rest_init():
    """3D box with walls on every face, lid on +z, from a non-rest state."""
    shape, steps, s1 = (37, 21, 19), 120, 1.4
    P, u = synth.smooth_fields(shape, seed=21, amp=0.01)
    kw = dict(wall=(1, 1, 1), lid=True, lid_u=(0.03, -0.01, 0.0))
    got = run_gpu(shape, P, u, steps, s1, storage="f64", **kw)
    ref = run_oracle(shape, P, u, steps, s1, **kw)
    assert np.array_equal(got["mask"], ref["mask"])
    e = errors(ref, got)
    assert e["u"] < 1e-10 and e["P"] < 1e-10, e


def test_mixed_walls_and_force():
    """Periodic x, walls on y, a non-uniform body force (Eq. 2-6)."""
    shape, steps, s1 = (40, 33), 500, 1.2
    X, Y = synth.grid_coords(shape)
    F = np.stack([1e-5 * (1.0 + 0.5 * np.cos(2 * np.pi * X / 40)), 2e-6 * np.sin(2 * np.pi * Y / 33)])
    P, u = synth.rest_state(shape[0] * shape[1], 2)
    # the pressure fluctuation of this flow is ~1e-7, so FP32 storage
    # rounding (~1e-11 absolute) leaves ~1e-5 relative on it: bound 5e-5
    for storage, tol, tolp in (("f64", 1e-10, 1e-10), ("f32", 1e-5, 5e-5)):
        got = run_gpu(shape, P, u, steps, s1, storage=storage, wall=(0, 1, 0), force=F)
        ref = run_oracle(shape, P, u, steps, s1, wall=(0, 1, 0), force=F)
        e = errors(ref, got)
        assert e["u"] < tol and e["P"] < tolp, (storage, e)


# --------------------------------------------------------------------------
# Scheme II forcing (Eq. 2-3c, 2-7a)
# --------------------------------------------------------------------------
def _scheme2_force(shape, amp):
    X = synth.grid_coords(shape)
    d = len(shape)
    return np.stack([amp * (1.0 + 0.7 * np.cos(2 * np.pi * X[(a + 1) % d] / shape[(a + 1) % d])
                            + 0.4 * np.sin(2 * np.pi * X[a] / shape[a]))
                     for a in range(d)])


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16", "f16eq", "bf16eq"])
@pytest.mark.parametrize("case", ["2d_walls_lid", "3d_walls"])
def test_scheme2_matches_oracle(storage, case):
    """Scheme II with a non-uniform force: walls and a lid in 2D (ragged
    67 x 45), walls on two axes in 3D, a non-rest start.  Fields, rho and
    the Eq. 2-7a sums against the oracle.  The same run under Eq. 3-21 is
    farther from the Scheme II oracle than the tolerance (the test tells
    the schemes apart)."""
    if case == "2d_walls_lid":
        shape, steps, s1 = (67, 45), 300, 1.3
        kw = dict(wall=(1, 1, 0), lid=True, lid_u=(0.02, 0.0, 0.0))
        amp = 2e-5
    else:
        shape, steps, s1 = (36, 19, 17), 80, 1.5
        kw = dict(wall=(1, 0, 1), lid=False)
        amp = 1e-5
    P, u = synth.smooth_fields(shape, seed=41, amp=0.01)
    F = _scheme2_force(shape, amp)
    ref = run_oracle(shape, P, u, steps, s1, force=F, scheme=2, **kw)
    got = run_gpu(shape, P, u, steps, s1, storage=storage, force=F, forcing="scheme2", **kw)
    assert np.array_equal(got["mask"], ref["mask"])
    e = errors(ref, got)
    tu, tp, tg = _tol(storage)
    assert e["u"] < tu and e["P"] < tp, e
    assert e["G"] < tg and e["S"] < tg and e["omega"] < tg, e
    if storage in ("f64", "f32"):
        other = run_oracle(shape, P, u, steps, s1, force=F, scheme=0, **kw)
        assert rel(ref["u"], other["u"]) > 20 * tu


@pytest.mark.parametrize("storage", ["f64", "f32", "f16eq"])
def test_scheme2_init_sums_and_residual(storage):
    """The Scheme II initial state is fbar = f^eq - F/2, so ubar (Eq. 2-7a)
    reads back the input u; sums of ubar and the residual follow the oracle."""
    from paper_2108_08591_gb300 import Lattice
    shape, s1 = (48, 40), 1.4
    P, u = synth.smooth_fields(shape, seed=5, amp=0.01)
    F = _scheme2_force(shape, 3e-5)
    lat = Lattice(shape, s1=s1, storage=storage)
    try:
        lat.set_forcing("scheme2")
        assert lat.forcing == "scheme2"
        lat.set_force(F)
        lat.init(P, u)
        tu = _tol(storage)[0]
        assert rel(u, lat.fields_host(("u",))["u"]) < tu
        lat.step(25)
        pb = O.Problem(d=2, n=shape, s1=s1, force=F, scheme=2)
        f = O.run(pb, O.init(pb, P, u), 25)
        want = O.sums(pb, f)
        got = lat.sums()
        tol_sum = {"f64": 1e-12, "f32": 1e-6, "f16eq": 1e-5}[storage] * pb.N
        assert np.abs(got - want).max() < tol_sum, (got, want)
        assert lat.residual() == np.inf
        lat.step(1)
        f1 = O.run(pb, f.copy(), 1)
        u0 = O.macro(pb, f)[1]
        u1 = O.macro(pb, f1)[1]
        r_ref = np.linalg.norm(u1 - u0) / np.linalg.norm(u1)
        assert lat.residual() == pytest.approx(r_ref, rel=1e-6 if storage == "f64" else 2e-2)
    finally:
        lat.close()


def test_forcing_scheme_is_checked():
    """Only Eq. 3-21 (0) and Scheme II (2) exist; Scheme I is refused."""
    from paper_2108_08591_gb300 import Lattice, _lib
    lat = Lattice((32, 32), s1=1.2)
    try:
        for bad in (1, 3, -1):
            assert lat._lib.mdf_set_forcing(lat._h, bad) == _lib.EINVAL
        assert lat.forcing == "eq3-21"
    finally:
        lat.close()


def test_scheme2_without_force_is_eq_3_21():
    """Without a force the two schemes are one update: same bits."""
    shape = (64, 33)
    P, u = synth.smooth_fields(shape, seed=9)
    a = run_gpu(shape, P, u, 40, 1.3, storage="f32", forcing="scheme2")
    b = run_gpu(shape, P, u, 40, 1.3, storage="f32")
    for k in ("P", "u", "G"):
        assert np.array_equal(a[k], b[k]), k


# --------------------------------------------------------------------------
# Non-equilibrium seeding (mdf_init_neq)
# --------------------------------------------------------------------------
def _seed_gradient(shape, seed, amp=1e-3):
    """A smooth, non-solenoidal gradient field [d][d][N] (its trace is
    dropped by the seed, which the comparison with the oracle covers)."""
    d = len(shape)
    X = synth.grid_coords(shape)
    rng = synth.SplitMix64(seed)
    G = np.zeros((d, d, int(np.prod(shape))))
    for a in range(d):
        for b in range(d):
            ph = 6 * rng.uniform()
            G[a, b] = amp * np.sin(2 * np.pi * X[(a + b) % d] / shape[(a + b) % d] + ph).ravel()
    return G


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "f16eq", "bf16eq"])
@pytest.mark.parametrize("case", ["2d_walls_lid", "3d_periodic", "2d_scheme2"])
@pytest.mark.parametrize("steps", [0, 40])
def test_neq_seed_matches_oracle(storage, case, steps):
    """f^eq + f^ne(G) at the start (steps = 0: the fields read back the
    traceless G) and after 40 updates, against the oracle."""
    kw = {}
    if case == "3d_periodic":
        shape, s1 = (24, 18, 14), 1.4
    else:
        shape, s1 = (45, 37), 1.3
        kw = dict(wall=(1, 1, 0), lid=True, lid_u=(0.02, 0.0, 0.0))
    P, u = synth.smooth_fields(shape, seed=17, amp=0.01)
    G = _seed_gradient(shape, 3)
    okw, gkw = dict(kw), dict(kw)
    if case == "2d_scheme2":
        F = _scheme2_force(shape, 2e-5)
        okw.update(force=F, scheme=2)
        gkw.update(force=F, forcing="scheme2")
    ref = run_oracle(shape, P, u, steps, s1, G=G, **okw)
    got = run_gpu(shape, P, u, steps, s1, storage=storage, G=G, **gkw)
    e = errors(ref, got)
    tu, tp, tg = _tol(storage)
    assert e["u"] < tu and e["P"] < tp, e
    assert e["G"] < tg and e["S"] < tg and e["omega"] < tg, e
    if steps == 0 and storage in ("f64", "f32"):
        d = len(shape)
        tr = np.einsum("aan->n", G)
        want = G - np.eye(d)[:, :, None] * tr[None, None, :] / d
        assert rel(want, got["G"]) < (1e-12 if storage == "f64" else 1e-4)


def test_neq_seed_removes_the_initial_layer_on_the_gpu():
    """2D Taylor-Green from its exact gradient (FP32 storage): the Eq. 3-16
    gradient after one update is within 1e-2 of the closed form, against
    ~0.2 from the equilibrium start."""
    from paper_2108_08591_gb300 import Lattice
    n, U0, s1 = 64, 0.01, 1.2
    nu = (1 / s1 - 0.5) / 3
    k = 2 * np.pi / n
    P, u = synth.taylor_green_2d(n, U0)
    X, Y = synth.grid_coords((n, n))
    cc, ss = (np.cos(k * X) * np.cos(k * Y)).ravel(), (np.sin(k * X) * np.sin(k * Y)).ravel()
    G0 = U0 * k * np.stack([np.stack([cc, -ss]), np.stack([ss, -cc])])
    err = {}
    for name, G in (("eq", None), ("neq", G0)):
        lat = Lattice((n, n), s1=s1)
        lat.init(P, u, G)
        lat.step(1)
        g01 = lat.fields_host(("G",))["G"][0, 1]
        lat.close()
        err[name] = rel(G0[0, 1] * np.exp(-2 * nu * k * k), g01)
    assert err["neq"] < 1e-2 and err["eq"] > 0.1, err


# --------------------------------------------------------------------------
# Lattices without a rest direction (D2Q4, D3Q6)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("case", ["2d_periodic", "2d_walls_lid_force", "3d_walls", "3d_periodic_force"])
def test_rest_free_lattice_matches_oracle(storage, case):
    """D2Q4 / D3Q6 against the oracle: ragged periodic grids, walls and a
    lid, a non-uniform force, a non-rest start; fields, rho and the mask."""
    d = 3 if case.startswith("3d") else 2
    q = 6 if d == 3 else 4
    kw, F = {}, None
    if d == 2:
        shape, steps, s1 = (67, 45), 300, 1.3
    else:
        shape, steps, s1 = (36, 19, 17), 80, 1.5
    if "walls" in case:
        kw = dict(wall=(1, 1, 0), lid=True, lid_u=(0.02, 0.0, 0.0)) if d == 2 else dict(wall=(1, 0, 1))
    if "force" in case:
        F = _scheme2_force(shape, 1e-5)
    P, u = synth.smooth_fields(shape, seed=23, amp=0.01)
    ref = run_oracle(shape, P, u, steps, s1, force=F, q=q, **kw)
    got = run_gpu(shape, P, u, steps, s1, storage=storage, force=F, q=q, **kw)
    assert np.array_equal(got["mask"], ref["mask"])
    e = errors(ref, got)
    tu, tp, tg = _tol(storage)
    assert e["u"] < tu and e["P"] < tp, e
    assert e["G"] < tg and e["S"] < tg and e["omega"] < tg, e
    assert e["rho"] < (1e-10 if storage == "f64" else 1e-2), e


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_rest_free_scheme2_and_neq_seed(storage):
    """D2Q4 with Scheme II forcing and a non-equilibrium start, with walls."""
    shape, steps, s1 = (45, 37), 60, 1.3
    kw = dict(wall=(0, 1, 0))
    P, u = synth.smooth_fields(shape, seed=29, amp=0.01)
    F = _scheme2_force(shape, 2e-5)
    G = _seed_gradient(shape, 7)
    ref = run_oracle(shape, P, u, steps, s1, force=F, scheme=2, G=G, q=4, **kw)
    got = run_gpu(shape, P, u, steps, s1, storage=storage, force=F, forcing="scheme2", G=G, q=4, **kw)
    e = errors(ref, got)
    tu, tp, tg = _tol(storage)
    assert e["u"] < tu and e["P"] < tp and e["G"] < tg, e


@pytest.mark.parametrize("d,storage,vx", [
    (2, "f32", 4), (2, "f32", 2), (2, "f16", 8), (2, "bf16", 4), (2, "f64", 2),
    (3, "f32", 2), (3, "f16", 4), (3, "bf16", 4), (3, "f64", 2),
])
@pytest.mark.parametrize("walls", [False, True])
def test_rest_free_vector_kernel_is_bitwise_the_scalar_kernel(d, storage, vx, walls):
    from paper_2108_08591_gb300 import Lattice
    shape = (264, 9) if d == 2 else (264, 5, 4)
    P, u = synth.smooth_fields(shape, seed=19)
    kw = {}
    if walls:
        kw = dict(wall=(1, 1, 1)[:d] + (0,) * (3 - d), lid=True, lid_u=(0.02, 0.01, 0.0))
    outs = []
    for v in (1, vx):
        lat = Lattice(shape, s1=1.35, storage=storage, vx=v, block=64, q=2 * d, **kw)
        lat.init(P, u)
        lat.step(9)
        outs.append(lat.fields_host(("P", "u", "G", "rho")))
        lat.close()
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[1][k]), k


def test_rest_free_lattice_rejections():
    """Equilibrium-shifted storage and the batch need D2Q5 / D3Q7; q must
    name a lattice of the dimension."""
    from paper_2108_08591_gb300 import CavityBatch, Lattice, MdfError
    for shape, q, storage in (((64, 32), 4, "f16eq"), ((32, 16, 8), 6, "bf16eq"),
                              ((32, 16, 8), 4, "f32"), ((64, 32), 6, "f32"), ((64, 32), 3, "f32")):
        with pytest.raises(MdfError):
            Lattice(shape, s1=1.2, storage=storage, q=q)
    lat = Lattice((64, 32), s1=1.2, q=4)
    assert lat.info.q == 4
    lat.close()


# --------------------------------------------------------------------------
# In-place AA pattern (one population buffer)
# --------------------------------------------------------------------------
def _run_pattern(shape, storage, inplace, steps_list, kw, q=0, forcing="eq3-21", F=None, G=None, vx=0):
    """Fields after each entry of steps_list, the fused-epilogue fields of
    the last update and the sums, from one lattice."""
    from paper_2108_08591_gb300 import Lattice
    P, u = synth.smooth_fields(shape, seed=31, amp=0.01)
    lat = Lattice(shape, s1=1.35, storage=storage, q=q, inplace=inplace, vx=vx, block=64, **kw)
    out = []
    try:
        lat.set_forcing(forcing)
        if F is not None:
            lat.set_force(F)
        lat.init(P, u, G)
        for n in steps_list:
            lat.step(n)
            out.append(lat.fields_host(("P", "u", "G", "omega") + (("rho",) if lat.with_rho else ())))
        fl = lat.alloc_fields(("P", "u", "S"))
        lat.step_fields(3, fl)
        out.append({k: t.cpu().numpy() for k, t in fl.items()})
        out.append({"sums": lat.sums()})
    finally:
        lat.close()
    return out


@pytest.mark.parametrize("storage", ["f32", "f64", "f16", "bf16"])
@pytest.mark.parametrize("case", ["2d_periodic", "2d_walls_lid", "3d_walls", "2d_q4_walls", "3d_q6_periodic"])
def test_inplace_aa_is_bitwise_the_pull_stream(storage, case):
    """The AA pattern moves the same values through one buffer: fields after
    odd and even step counts, a fused-epilogue update and the sums equal
    the two-buffer pull stream's bit for bit.  (With 16-bit storage and a
    moving lid the AA pattern stores the bounced value with its lid term
    and rounds once more; that case is compared against the oracle
    instead.)"""
    d = 3 if case.startswith("3d") else 2
    q = 4 if "q4" in case else 6 if "q6" in case else 0
    shape = (45, 37) if d == 2 else (24, 18, 14)
    kw = {}
    if "walls_lid" in case:
        kw = dict(wall=(1, 1, 0), lid=True, lid_u=(0.02, 0.0, 0.0))
    elif "walls" in case:
        kw = dict(wall=(1, 1, 0)) if d == 2 else dict(wall=(1, 0, 1))
    steps = [1, 2, 7, 10]
    if storage in ("f16", "bf16") and kw.get("lid"):
        ref = run_oracle(shape, *synth.smooth_fields(shape, seed=31, amp=0.01), sum(steps), 1.35, **kw)
        got = _run_pattern(shape, storage, True, steps, kw)[len(steps) - 1]
        e = errors(ref, got)
        tu, tp, tg = _tol(storage)
        assert e["u"] < tu and e["P"] < tp, e
        return
    a = _run_pattern(shape, storage, False, steps, kw, q=q)
    b = _run_pattern(shape, storage, True, steps, kw, q=q)
    for ra, rb in zip(a, b):
        for k in ra:
            assert np.array_equal(ra[k], rb[k]), (k, np.abs(ra[k] - rb[k]).max())


@pytest.mark.parametrize("d,storage,vx", [
    (2, "f32", 4), (2, "f32", 2), (2, "f16", 8), (2, "bf16", 4), (2, "f64", 2),
    (3, "f32", 2), (3, "f16", 4), (3, "bf16", 4), (3, "f64", 2),
])
@pytest.mark.parametrize("walls", [False, True])
def test_inplace_aa_vector_kernel_is_bitwise_the_pull_stream(d, storage, vx, walls):
    """The vector AA kernel (shuffled x-neighbours, scalar accesses at warp
    and row edges, per-node wall links) against the one-node-per-thread pull
    stream: x extents of several warps with a partial last block (264 = 33 x
    8), odd and even step counts, walls on every axis."""
    shape = (264, 9) if d == 2 else (264, 5, 4)
    kw = dict(wall=(1, 1, 1)[:d] + (0,) * (3 - d)) if walls else {}
    steps = [1, 2, 5, 6]
    a = _run_pattern(shape, storage, False, steps, kw, vx=1)
    b = _run_pattern(shape, storage, True, steps, kw, vx=vx)
    for ra, rb in zip(a, b):
        for k in ra:
            assert np.array_equal(ra[k], rb[k]), (k, np.abs(ra[k] - rb[k]).max())


def test_inplace_aa_with_force_scheme2_and_seed():
    """Force, Scheme II and a non-equilibrium start through the AA pattern."""
    shape = (45, 37)
    F = _scheme2_force(shape, 2e-5)
    G = _seed_gradient(shape, 11)
    kw = dict(wall=(0, 1, 0))
    a = _run_pattern(shape, "f32", False, [3, 4], kw, forcing="scheme2", F=F, G=G)
    b = _run_pattern(shape, "f32", True, [3, 4], kw, forcing="scheme2", F=F, G=G)
    for ra, rb in zip(a, b):
        for k in ra:
            assert np.array_equal(ra[k], rb[k]), k


def test_inplace_aa_checkpoint_keeps_the_parity(tmp_path):
    """A checkpoint taken in the odd layout resumes bit for bit; a
    two-buffer handle refuses it."""
    from paper_2108_08591_gb300 import Lattice, MdfError
    shape = (64, 33)
    P, u = synth.smooth_fields(shape, seed=5)
    path = str(tmp_path / "aa.ckpt")
    a = Lattice(shape, s1=1.3, inplace=True)
    a.init(P, u)
    a.step(5)  # odd layout
    a.save(path)
    a.step(6)
    want = a.fields_host(("P", "u", "G"))
    b = Lattice(shape, s1=1.3, inplace=True)
    b.load(path)
    b.step(6)
    got = b.fields_host(("P", "u", "G"))
    for k in want:
        assert np.array_equal(want[k], got[k]), k
    c = Lattice(shape, s1=1.3)
    with pytest.raises(MdfError):
        c.load(path)
    with pytest.raises(MdfError):
        a.autotune(reps=1)
    for lat in (a, b, c):
        lat.close()


def test_inplace_aa_halves_the_population_memory():
    """One buffer: the device memory a handle takes drops by one population
    buffer (2048^2 D2Q5 x 3 FP32: 252 MB per buffer)."""
    import torch
    from paper_2108_08591_gb300 import Lattice
    shape = (2048, 2048)
    used = {}
    for inplace in (False, True):
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        lat = Lattice(shape, s1=1.3, inplace=inplace)
        torch.cuda.synchronize()
        used[inplace] = free0 - torch.cuda.mem_get_info()[0]
        lat.close()
    buf = 2048 * 2048 * 15 * 4
    assert abs((used[False] - used[True]) - buf) < 0.05 * buf, used


# --------------------------------------------------------------------------
# Slab decomposition with the per-face exchange (mdf_slabs_*)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("case,storage,k", [
    ("2d", "f32", 1), ("2d", "f32", 2), ("2d", "f32", 3), ("2d", "f32", 4), ("2d", "f64", 4),
    ("2d", "f16", 4), ("2d", "bf16", 2), ("2d_xwalls", "f32", 4), ("2d_q4", "f32", 3),
    ("3d", "f32", 2), ("3d", "f32", 4), ("3d_q6_xwalls", "f64", 2),
])
def test_slabs_are_bitwise_the_undivided_lattice(case, storage, k):
    """k sub-domains along the last axis, each with ghost layers refilled by
    the face exchange after every update, give the undivided lattice's bits
    (the exchange is the whole coupling between slabs)."""
    from paper_2108_08591_gb300 import Lattice, Slabs
    d = 3 if case.startswith("3d") else 2
    q = 4 if "q4" in case else 6 if "q6" in case else 0
    shape = (40, 48) if d == 2 else (20, 14, 16)
    wall = (1, 0, 0) if "xwalls" in case else (0, 0, 0)
    P, u = synth.smooth_fields(shape, seed=37, amp=0.01)
    names = ("P", "u", "G", "omega", "rho")
    ref = Lattice(shape, s1=1.3, storage=storage, wall=wall, q=q)
    ref.init(P, u)
    sl = Slabs(shape, s1=1.3, k=k, storage=storage, wall=wall, q=q)
    sl.init(P, u)
    try:
        for n in (1, 6, 17):
            ref.step(n)
            sl.step(n)
            a = ref.fields_host(names)
            b = sl.fields_host(names)
            for key in names:
                assert np.array_equal(a[key], b[key]), (n, key, np.abs(a[key] - b[key]).max())
    finally:
        ref.close()
        sl.close()


# --------------------------------------------------------------------------
# Fused epilogue, reductions, checkpoints, edges
# --------------------------------------------------------------------------
def test_fused_fields_equal_separate_pass():
    import torch
    from paper_2108_08591_gb300 import Lattice
    shape = (129, 40)
    P, u = synth.smooth_fields(shape, seed=3)
    a = Lattice(shape, s1=1.3)
    b = Lattice(shape, s1=1.3)
    a.init(P, u)
    b.init(P, u)
    a.step(7)
    b.step(7)
    fa = a.alloc_fields()
    a.step_fields(5, fa)
    fb = b.fields(list(fa.keys()))
    b.step(5)
    torch.cuda.synchronize()
    for k in fa:
        assert torch.equal(fa[k], fb[k]), k
    ua = a.fields_host(("u",))["u"]
    ub = b.fields_host(("u",))["u"]
    assert np.array_equal(ua, ub)
    a.close()
    b.close()


@pytest.mark.parametrize("d", [2, 3])
def test_conservation_sums(d):
    from paper_2108_08591_gb300 import Lattice
    shape = (45, 38) if d == 2 else (20, 17, 12)
    P, u = synth.smooth_fields(shape, seed=4)
    pb = O.Problem(d=d, n=shape, s1=1.5)
    ref0 = O.sums(pb, O.init(pb, P, u))
    for storage, tol in (("f64", 1e-13), ("f32", 1e-6), ("f16eq", 1e-5)):
        lat = Lattice(shape, s1=1.5, storage=storage)
        lat.init(P, u)
        s0 = lat.sums()
        lat.step(200)
        s1 = lat.sums()
        lat.close()
        scale = np.abs(ref0).max()
        assert np.abs(s0 - ref0).max() < tol * scale, (storage, s0, ref0)
        assert np.abs(s1 - s0).max() < tol * scale, (storage, s1, s0)


def test_residual_matches_definition():
    from paper_2108_08591_gb300 import Lattice
    shape = (64, 48)
    P, u = synth.smooth_fields(shape, seed=8)
    lat = Lattice(shape, s1=1.7, storage="f64")
    lat.init(P, u)
    assert lat.residual() == float("inf")
    u0 = lat.fields_host(("u",))["u"]
    lat.step(10)
    r = lat.residual()
    u1 = lat.fields_host(("u",))["u"]
    want = np.linalg.norm(u1 - u0) / np.linalg.norm(u1)
    assert r == pytest.approx(want, rel=1e-10)
    lat.close()


def test_nonfinite_is_reported():
    from paper_2108_08591_gb300 import Lattice, MdfError
    shape = (32, 16)
    P, u = synth.rest_state(512, 2)
    P[77] = np.nan
    lat = Lattice(shape, s1=1.2)
    lat.init(P, u)
    with pytest.raises(MdfError, match="EDIVERGED"):
        lat.sums()
    lat.close()


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16eq"])
def test_checkpoint_resume_is_bit_identical(storage):
    from paper_2108_08591_gb300 import Lattice, MdfError
    shape = (50, 30)
    P, u = synth.smooth_fields(shape, seed=2)
    a = Lattice(shape, s1=1.4, storage=storage)
    a.init(P, u)
    a.step(33)
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "ck.mdf")
        a.save(path)
        a.step(40)
        b = Lattice(shape, s1=1.4, storage=storage)
        b.load(path)
        assert b.info.step == 33
        b.step(40)
        assert np.array_equal(a.fields_host(("u", "P", "G"))["G"], b.fields_host(("u", "P", "G"))["G"])
        # corrupt file is rejected
        raw = bytearray(open(path, "rb").read())
        raw[-5] ^= 0xFF
        open(path, "wb").write(bytes(raw))
        with pytest.raises(MdfError, match="EIO"):
            b.load(path)
        # a handle of another configuration refuses the file
        c = Lattice(shape, s1=1.41, storage=storage)
        a.save(path)
        with pytest.raises(MdfError, match="EIO"):
            c.load(path)
        b.close()
        c.close()
    a.close()


@pytest.mark.parametrize("shape", [(2, 2), (3, 2), (33, 2), (2, 2, 2), (5, 3, 2)])
def test_smallest_grids(shape):
    P, u = synth.smooth_fields(shape, seed=1)
    got = run_gpu(shape, P, u, 25, 1.1, storage="f64")
    ref = run_oracle(shape, P, u, 25, 1.1)
    e = errors(ref, got)
    assert e["u"] < 1e-10, e


def test_zero_steps_and_graph_chunks():
    """n = 0 is a no-op; long runs (graph chunks of 64 plus a remainder)
    equal the same number of single steps."""
    import torch
    from paper_2108_08591_gb300 import Lattice
    shape = (96, 20)
    P, u = synth.smooth_fields(shape, seed=6)
    s = torch.cuda.Stream()  # graphs are captured on a non-legacy stream only
    a = Lattice(shape, s1=1.3, stream=s)
    b = Lattice(shape, s1=1.3, stream=s)
    a.init(P, u)
    b.init(P, u)
    a.step(0)
    a.step(64 * 2 + 13)
    for _ in range(64 * 2 + 13):
        b.step(1)
    assert np.array_equal(a.fields_host(("u",))["u"], b.fields_host(("u",))["u"])
    assert a.info.step == b.info.step == 141
    a.close()
    b.close()


# --------------------------------------------------------------------------
# Full size (4096^2, the benchmark's configuration): sampled parity
# --------------------------------------------------------------------------
def _sample_points(n, d, count, seed):
    """Seeded nodes of an n^d lattice plus the nodes where the vector
    kernels change path: the first and last nodes of a row, of a warp's x
    span (32 threads x 1, 2 or 4 nodes) and of a block's (64 .. 256 threads),
    each at a seeded position along the other axes."""
    rng = synth.SplitMix64(seed)
    xs = [x for x in (0, 1, 2, 3, 4, 7, 8, 31, 32, 63, 64, 127, 128, 255, 256, 511, 512, 1023,
                      1024, n - 2, n - 1) if x < n]
    pts = []
    for x in sorted(set(xs)):
        pts.append([x] + [rng.randint(0, n - 1) for _ in range(d - 1)])
    pts.append([rng.randint(0, n - 1)] + [0] * (d - 1))
    pts.append([rng.randint(0, n - 1)] + [n - 1] * (d - 1))
    while len(pts) < count:
        pts.append([rng.randint(0, n - 1) for _ in range(d)])
    return pts


def _flat(c, n):
    return c[0] + n * (c[1] + (n * c[2] if len(c) == 3 else 0))


def _gather(out, pts, n):
    """Device fields at the sampled nodes only: {name: array[..., j]} for
    point j (copying whole 512^3 fields to the host would take minutes)."""
    import torch
    idx = torch.tensor([_flat(c, n) for c in pts], dtype=torch.long, device="cuda")
    return {k: v.index_select(v.dim() - 1, idx).cpu().numpy() for k, v in out.items()}


def _sampled_window_errors(shape, s1, P, u, got, steps, pts, s2=None):
    """Relative L2 of u, P - 1, G, S and omega on the given nodes of a
    periodic lattice, against the FP64 oracle on (2 steps + 1)^d windows
    (after `steps` updates a node depends only on nodes within that many
    links).  got: fields gathered at pts (column j = point j)."""
    d = len(shape)
    n = shape[0]
    W = 2 * steps + 1
    offs = np.arange(-steps, steps + 1)
    keys = ("u", "P", "G", "S", "omega")
    ref = {k: [] for k in keys}
    num = {k: [] for k in keys}
    for g, c in enumerate(pts):
        axes = [(c[b] + offs) % n for b in range(d)]
        if d == 2:
            sel = (axes[1][:, None] * n + axes[0][None, :]).ravel()
        else:
            sel = ((axes[2][:, None, None] * n + axes[1][None, :, None]) * n + axes[0][None, None, :]).ravel()
        pb = O.Problem(d=d, n=(W,) * d, s1=s1, s2=s2)
        f = O.run(pb, O.init(pb, P[sel], u[:, sel]), steps)
        Pr, ur, _ = O.macro(pb, f)
        D = O.derived(pb, f)
        mid = (W ** d) // 2
        ref["u"].append(ur[:, mid]); num["u"].append(got["u"][:, g])
        ref["P"].append(Pr[mid] - 1.0); num["P"].append(got["P"][g] - 1.0)
        for k in ("G", "S", "omega"):
            ref[k].append(D[k][..., mid]); num[k].append(got[k][..., g])
    return {k: rel(np.array(ref[k]), np.array(num[k])) for k in keys}


def test_full_size_4096_sampled_parity():
    """4096^2 D2Q5 x 3, FP32 storage, Taylor-Green + 8 modes, run as the
    benchmark runs it (fused epilogue update, then graph chunks), compared
    with the FP64 oracle at 64 nodes, including every row, warp and block
    edge of the vector kernel.  After n steps a node depends only on nodes
    within distance n, so the oracle runs a periodic (2n+1)^2 window around
    each sampled node."""
    import torch
    from paper_2108_08591_gb300 import Lattice
    n, steps = 4096, 71
    P, u = synth.tg_plus_modes(n, U0=0.01, seed=2108)
    lat = Lattice((n, n), s1=S1_TG, storage="f32")
    lat.init(P, u)
    fl = lat.alloc_fields(("P", "u", "G", "div"))
    lat.step_fields(steps, fl)
    out = lat.fields(("P", "u", "G", "S", "omega", "div"))
    torch.cuda.synchronize()
    # fields of the initial state from the fused update: f = f^eq there, so
    # f^ne and every gradient vanish up to FP32 storage rounding (~1e-9
    # against |grad u| ~ 1.5e-5 of the flow)
    assert np.abs(fl["G"].cpu().numpy()).max() < 1e-8
    assert np.abs(fl["div"].cpu().numpy()).max() < 1e-8
    # after 71 updates: divergence identity (exact in exact arithmetic; FP32
    # epilogue arithmetic leaves a few 1e-6 of |G|)
    gmax = float(out["G"].abs().max())
    assert gmax > 1e-6
    assert float(out["div"].abs().max()) < 5e-5 * gmax
    pts = _sample_points(n, 2, 64, 77)
    got = _gather(out, pts, n)
    lat.close()
    e = _sampled_window_errors((n, n), S1_TG, P, u, got, steps, pts)
    print("4096^2 f32", e)
    assert e["u"] < 1e-5 and e["P"] < 1e-5, e
    assert e["G"] < 1e-3 and e["S"] < 1e-3 and e["omega"] < 1e-3, e


@pytest.mark.parametrize("storage,tol", [("f16eq", (2e-3, 2e-3, 1e-2)), ("bf16eq", (2e-3, 2e-3, 5e-2))])
def test_full_size_4096_equilibrium_shifted_sampled_parity(storage, tol):
    """The 4096^2 workload with equilibrium-shifted 16-bit storage, in the
    benchmark's launch configuration, at 64 sampled nodes including the
    vector kernel's edges: u and P - mean P within the 2e-3 bound on 16-bit
    storage; G, S and omega reported per field."""
    from paper_2108_08591_gb300 import Lattice
    n, steps = 4096, 40
    P, u = synth.tg_plus_modes(n, U0=0.01, seed=2108)
    lat = Lattice((n, n), s1=S1_TG, storage=storage)
    lat.init(P, u)
    lat.step(steps)
    pts = _sample_points(n, 2, 64, 91)
    got = _gather(lat.fields(("P", "u", "G", "S", "omega")), pts, n)
    lat.close()
    e = _sampled_window_errors((n, n), S1_TG, P, u, got, steps, pts)
    print("4096^2", storage, e)
    assert e["u"] < tol[0] and e["P"] < tol[1], e
    assert e["G"] < tol[2] and e["S"] < tol[2] and e["omega"] < tol[2], e


@pytest.mark.parametrize("storage,tol", [("f32", (1e-5, 1e-5, 1e-3)), ("f16eq", (2e-3, 2e-3, 1e-2)),
                                         ("f16", (2e-3, 2e-2, 0.5))])
def test_full_size_512_cubed_sampled_parity(storage, tol):
    """512^3 D3Q7 x 4 3D Taylor-Green (U0 = 0.05, Re = 1600, s2 = 1: the
    s2 rule is unstable at these rates), in the benchmark's launch
    configuration, at 48 sampled nodes including the vector kernels' edges.  FP32 and equilibrium-shifted FP16 are held to
    the contract on u and P; the rest-shifted FP16 row is reported, not the
    contract (its P and gradient bounds only guard against regressions)."""
    from paper_2108_08591_gb300 import Lattice
    n, steps = 512, 12
    k = 2 * np.pi / n
    nu = 0.05 / (k * 1600.0)
    s1 = 1.0 / (4 * nu + 0.5)
    P, u = synth.taylor_green_3d(n, U0=0.05)
    lat = Lattice((n, n, n), s1=s1, s2=1.0, storage=storage)
    lat.init(P, u)
    lat.step(steps)
    pts = _sample_points(n, 3, 48, 93)
    got = _gather(lat.fields(("P", "u", "G", "S", "omega")), pts, n)
    lat.close()
    e = _sampled_window_errors((n, n, n), s1, P, u, got, steps, pts, s2=1.0)
    print("512^3", storage, e)
    assert e["u"] < tol[0] and e["P"] < tol[1], e
    assert e["G"] < tol[2] and e["omega"] < tol[2], e


# --------------------------------------------------------------------------
# Vector kernel (VX x-nodes per thread) against the one-node-per-thread kernel
# --------------------------------------------------------------------------
@pytest.mark.parametrize("d,storage,vx", [
    (2, "f32", 4), (2, "f32", 2), (2, "f16", 8), (2, "bf16", 4), (2, "f64", 2),
    (3, "f32", 2), (3, "f16", 4), (3, "bf16", 4), (3, "f64", 2),
    (2, "f16eq", 2), (2, "f16eq", 4), (2, "bf16eq", 4), (3, "f16eq", 2), (3, "bf16eq", 2),
])
@pytest.mark.parametrize("walls", [False, True])
def test_vector_kernel_is_bitwise_the_scalar_kernel(d, storage, vx, walls):
    """Same per-node arithmetic, so the same bits: x extents of several warps
    with a partial last warp (264 = 33 x 8), the row wrap, walls and lid."""
    from paper_2108_08591_gb300 import Lattice
    shape = (264, 9) if d == 2 else (264, 5, 4)
    P, u = synth.smooth_fields(shape, seed=17)
    kw = {}
    if walls:
        kw = dict(wall=(1, 1, 1)[:d] + (0,) * (3 - d), lid=True, lid_u=(0.02, 0.01, 0.0))
    outs = []
    for v in (1, vx):
        lat = Lattice(shape, s1=1.35, storage=storage, vx=v, block=64, **kw)
        lat.init(P, u)
        lat.step(5)
        f1 = lat.fields_host(("P", "u", "G", "rho"))
        fl = lat.alloc_fields(("P", "u", "omega"))
        lat.step_fields(7, fl)
        f2 = {k: t.cpu().numpy() for k, t in fl.items()}
        f3 = lat.fields_host(("P", "u", "G", "S", "sigma", "omega", "div"))
        outs.append((f1, f2, f3))
        lat.close()
    for a, b in zip(outs[0], outs[1]):
        for k in a:
            assert np.array_equal(a[k], b[k]), (k, np.abs(a[k] - b[k]).max())


def test_autotune_keeps_the_state_and_the_bits():
    from paper_2108_08591_gb300 import Lattice
    shape = (256, 40)
    P, u = synth.smooth_fields(shape, seed=29)
    a = Lattice(shape, s1=1.5, vx=1, block=128)
    b = Lattice(shape, s1=1.5)
    for lat in (a, b):
        lat.init(P, u)
        lat.step(3)
    before = b.fields_host(("u", "P"))
    vx, block = b.autotune(reps=3)
    assert vx in (1, 2, 4) and block in (64, 128, 256)
    assert (b.info.vx, b.info.block) == (vx, block)
    after = b.fields_host(("u", "P"))
    assert np.array_equal(before["u"], after["u"]) and np.array_equal(before["P"], after["P"])
    a.step(20)
    b.step(20)
    assert np.array_equal(a.fields_host(("u",))["u"], b.fields_host(("u",))["u"])
    a.close()
    b.close()
