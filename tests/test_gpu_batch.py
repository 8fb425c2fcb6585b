"""Batched lid-driven cavities (persistent cooperative kernel) through the
C-ABI: bitwise against the single-lattice path, against the FP64 oracle,
convergence bookkeeping and failure reporting."""
import numpy as np
import pytest

import synth
from tests._harness import errors, run_oracle

pytestmark = pytest.mark.gpu

U = 0.1


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_08591_gb300 import _build
    _build.build()


def _rates(N, Re, d=2):
    cs2 = 1.0 / 3.0 if d == 2 else 0.25
    nu = U * N / Re
    s1 = 1.0 / (nu / cs2 + 0.5)
    return s1, 8.0 * (2.0 - s1) / (8.0 - s1)


@pytest.mark.parametrize("d,sides,Res", [(2, [17, 24, 40], [100.0, 400.0, 1000.0]),
                                         (3, [10, 13], [50.0, 200.0])])
def test_batch_is_bitwise_the_single_lattice(d, sides, Res):
    from paper_2108_08591_gb300 import CavityBatch, Lattice
    names = ("P", "u", "G", "omega")
    b = CavityBatch(sides, Res, lid_speed=U, d=d)
    b.step(150)
    for c, (N, Re) in enumerate(zip(sides, Res)):
        s1, s2 = _rates(N, Re, d)
        wall = (1, 1, 1)[:d]
        lat = Lattice((N,) * d, s1=s1, s2=s2, wall=wall, lid=True, lid_u=(U, 0, 0))
        lat.init(*synth.rest_state(N ** d, d))
        lat.step(150)
        want = lat.fields_host(names)
        got = b.fields_host(c, names)
        lat.close()
        for k in names:
            assert np.array_equal(want[k], got[k]), (c, k, np.abs(want[k] - got[k]).max())
    b.close()


def test_batch_matches_oracle():
    from paper_2108_08591_gb300 import CavityBatch
    sides, Res, steps = [19, 26], [150.0, 600.0], 300
    b = CavityBatch(sides, Res, lid_speed=U)
    b.step(steps)
    for c, (N, Re) in enumerate(zip(sides, Res)):
        s1, s2 = _rates(N, Re)
        ref = run_oracle((N, N), *synth.rest_state(N * N, 2), steps, s1, s2=s2, wall=(1, 1, 0),
                         lid=True, lid_u=(U, 0, 0))
        got = b.fields_host(c, ("P", "u", "G", "S", "sigma", "omega"))
        e = errors(ref, got)
        assert e["u"] < 1e-5 and e["P"] < 1e-5, (c, e)
        assert e["G"] < 1e-4 and e["omega"] < 1e-4, (c, e)
    b.close()


@pytest.mark.parametrize("graph,sched", [(False, 0), (True, 0), (True, 2), (True, 3)])
def test_batch_run_to_steady_state(graph, sched):
    """Low-Re cavities converge; the residual and the step count follow the
    definition; the final state equals a plain run of the same length (with
    the grid-barrier, the neighbour-wait and the claimed-tail schedules,
    cavities retiring at different periods)."""
    import torch
    from paper_2108_08591_gb300 import CavityBatch, Lattice
    sides, Res = [12, 16, 21], [5.0, 10.0, 20.0]
    stream = torch.cuda.Stream() if graph else None
    b = CavityBatch(sides, Res, lid_speed=U, stream=stream)
    b.set_schedule(128, 0, sched)
    steps, status, res = b.run(tol=1e-7, max_steps=200000, check_every=50)
    assert (status == 0).all(), (steps, status, res)
    assert (steps % 50 == 0).all() and (steps > 0).all()
    assert (res < 1e-7).all()
    for c, (N, Re) in enumerate(zip(sides, Res)):
        s1, s2 = _rates(N, Re)
        lat = Lattice((N, N), s1=s1, s2=s2, wall=(1, 1), lid=True, lid_u=(U, 0, 0))
        lat.init(*synth.rest_state(N * N, 2))
        # the residual: mean per-step change of u over the last check period
        lat.step(int(steps[c]) - 50)
        u0 = lat.fields_host(("u",))["u"]
        lat.step(50)
        u1 = lat.fields_host(("u",))["u"]
        assert res[c] == pytest.approx(np.linalg.norm(u1 - u0) / (50 * np.linalg.norm(u1)), rel=1e-4)
        got = b.fields_host(c, ("u",))["u"]
        assert np.array_equal(got, u1), c
        lat.close()
    b.close()


def test_batch_reports_divergence_and_step_cap():
    from paper_2108_08591_gb300 import CavityBatch
    sides, Res = [14, 14], [50.0, 300.0]
    b = CavityBatch(sides, Res, lid_speed=U)
    P, u = synth.rest_state(14 * 14, 2)
    P[37] = np.nan
    b.init(0, P, u)
    steps, status, res = b.run(tol=1e-12, max_steps=400, check_every=100)
    assert status[0] == 4  # MDF_EDIVERGED
    assert status[1] == 6 and steps[1] == 400  # MDF_ENOTCONVERGED at the cap
    b.close()


def test_batch_rejects_bad_arguments():
    from paper_2108_08591_gb300 import CavityBatch, MdfError
    with pytest.raises(MdfError, match="EINVAL"):
        CavityBatch([1, 10], [100.0, 100.0])
    b = CavityBatch([10], [100.0])
    with pytest.raises(MdfError, match="EINVAL"):
        b.run(check_every=33)
    b.close()


def test_barrier_timeout_is_reported_not_hung():
    """A zero spin limit makes the first waiting block give up at once: every
    block returns, the host reads MDF_ETIMEOUT, and the GPU stays usable."""
    from paper_2108_08591_gb300 import CavityBatch, MdfError
    b = CavityBatch([40, 33, 50], [100.0, 200.0, 300.0])
    b.set_timeout(0)
    with pytest.raises(MdfError, match="ETIMEOUT"):
        b.step(20)
    b.set_timeout(4_000_000_000)
    b.init()
    b.step(20)  # usable again
    assert np.isfinite(b.fields_host(0, ("u",))["u"]).all()
    b.close()


@pytest.mark.parametrize("d,sides,Res", [(2, [17, 65, 40], [100.0, 400.0, 1000.0]),
                                         (3, [10, 13], [50.0, 200.0])])
def test_every_schedule_gives_the_same_bits(d, sides, Res):
    """Threads per block 128 / 64 / 32 (1, 2, 4 nodes per thread), both tile
    orders with a grid barrier, the claimed-tail order and the barrier-free
    neighbour-wait schedule,
    a one-block and the largest grid: the same arithmetic per node, so the
    same bits after 40 updates in one launch."""
    from paper_2108_08591_gb300 import CavityBatch
    names = ("P", "u", "G")
    ref = None
    for threads in (128, 64, 32):
        for sched in (0, 1, 2, 3):
            for grid in (1, 0):
                b = CavityBatch(sides, Res, lid_speed=U, d=d)
                b.set_schedule(threads, grid, sched)
                got = b.schedule()
                assert got["threads"] == threads and got["sched"] == sched
                assert got["grid"] >= 1 and (grid == 0 or got["grid"] == grid)
                b.step(40)
                out = [b.fields_host(c, names) for c in range(len(sides))]
                b.close()
                if ref is None:
                    ref = out
                    continue
                for c in range(len(sides)):
                    for k in names:
                        assert np.array_equal(ref[c][k], out[c][k]), (threads, sched, grid, c, k)


def test_autotune_keeps_the_state_and_the_bits():
    from paper_2108_08591_gb300 import CavityBatch
    sides, Res = [33, 48, 65], [200.0, 500.0, 800.0]
    a = CavityBatch(sides, Res, lid_speed=U)
    b = CavityBatch(sides, Res, lid_speed=U)
    for x in (a, b):
        x.step(30)
    before = [b.fields_host(c, ("P", "u")) for c in range(3)]
    best = b.autotune(reps=6)
    assert best == b.schedule()
    assert best["threads"] in (32, 64, 128) and best["sched"] in (0, 1, 2, 3) and best["grid"] >= 1
    after = [b.fields_host(c, ("P", "u")) for c in range(3)]
    for c in range(3):
        for k in ("P", "u"):
            assert np.array_equal(before[c][k], after[c][k]), (c, k)
    a.step(50)
    b.step(50)
    for c in range(3):
        fa, fb = a.fields_host(c, ("u",)), b.fields_host(c, ("u",))
        assert np.array_equal(fa["u"], fb["u"]), c
    steps, status, _ = b.run(tol=1e-5, max_steps=4000, check_every=100)
    assert (steps > 0).all()
    a.close()
    b.close()


def test_schedule_rejects_bad_arguments():
    from paper_2108_08591_gb300 import CavityBatch
    from paper_2108_08591_gb300._lib import MdfError
    b = CavityBatch([17], [100.0], lid_speed=U)
    for args in ((96, 0, 0), (128, 0, 4), (128, 0, -1), (128, -1, 0), (128, 10 ** 7, 0)):
        with pytest.raises(MdfError, match="EINVAL"):
            b.set_schedule(*args)
    b.close()


def _fd_grad(u, N, d, lid):
    """grad u by central differences, ghost 2 u_wall - u beyond the walls
    (lid on the + face of the last axis): G[a][b] = d u_a / d x_b."""
    G = np.zeros((d, d) + (N,) * d)
    for a in range(d):
        ua = u[a].reshape((N,) * d)  # [z][y][x] / [y][x]
        for b in range(d):
            ax = d - 1 - b  # numpy axis of lattice axis b
            lo_wall = 0.0
            hi_wall = lid[a] if b == d - 1 else 0.0
            first = np.take(ua, [0], axis=ax)
            last = np.take(ua, [N - 1], axis=ax)
            ext = np.concatenate([2 * lo_wall - first, ua, 2 * hi_wall - last], axis=ax)
            G[a, b] = 0.5 * (np.take(ext, np.arange(2, N + 2), axis=ax) - np.take(ext, np.arange(0, N), axis=ax))
    return G.reshape(d, d, -1)


@pytest.mark.parametrize("d,sides,Res", [(2, [24, 33], [150.0, 600.0]), (3, [12], [80.0])])
def test_nonequilibrium_seed_returns_the_seed_gradient(d, sides, Res):
    """With the f^ne seed, Eq. 3-16 on the initial state gives the traceless
    part of the seed's finite-difference gradient, Eq. 2-7 the seed velocity
    and Eq. 3-15 the seed pressure; without it the gradient is zero."""
    from paper_2108_08591_gb300 import CavityBatch
    lid = (U, 0.0, 0.0)
    b = CavityBatch(sides, Res, lid_speed=U, d=d)
    for c, N in enumerate(sides):
        P, u = synth.smooth_fields((N,) * d, seed=40 + c)
        G = _fd_grad(u, N, d, lid)
        div = sum(G[a, a] for a in range(d))
        for a in range(d):
            G[a, a] -= div / d
        b.init(c, P, u, neq=True)
        got = b.fields_host(c, ("P", "u", "G"))
        scale = np.abs(G).max()
        assert np.abs(got["G"] - G).max() < 2e-4 * scale, np.abs(got["G"] - G).max() / scale
        assert np.abs(got["u"] - u).max() < 1e-6 * np.abs(u).max()
        assert np.abs(got["P"] - P).max() < 1e-3 * np.abs(P - 1).max()
        b.init(c, P, u)
        g0 = b.fields_host(c, ("G",))["G"]
        assert np.abs(g0).max() < 1e-5 * scale
    b.close()


def test_divergence_step_matches_the_fp64_oracle():
    """The seeded 65^2 draws above cell Re 8 blow up in the FP32 batch at the
    same 100-step check as in the FP64 oracle, and the draws below the limit
    stay bounded in both: the divergence belongs to the method at that cell
    Reynolds number, not to the FP32 storage (Sec. 4.3 cavity, s2 rule of
    Sec. 4.1)."""
    import oracle as O
    from paper_2108_08591_gb300 import CavityBatch
    draws = synth.cavity_batch()
    idx = [15, 18, 17, 22, 46]
    sides = [draws[i][0] for i in idx]
    Res = [draws[i][1] for i in idx]
    assert set(sides) == {65}
    cap = 6000
    b = CavityBatch(sides, Res, lid_speed=U)
    steps, status, _ = b.run(tol=1e-14, max_steps=cap, check_every=100)
    b.close()
    for c, (N, Re) in enumerate(zip(sides, Res)):
        s1, s2 = _rates(N, Re)
        pb = O.Problem(d=2, n=(N, N), s1=s1, s2=s2, wall=(1, 1, 0), lid=True, lid_u=(U, 0, 0))
        f = O.init(pb, *synth.rest_state(N * N, 2))
        ref = None
        for k in range(100, cap + 1, 100):
            O.run(pb, f, 100)
            if not np.isfinite(f).all():
                ref = k
                break
        if ref is None:
            assert status[c] == 6 and steps[c] == cap, (c, Re, status[c], steps[c])
        else:
            assert status[c] == 4, (c, Re, status[c], steps[c], ref)
            assert abs(int(steps[c]) - ref) <= 100, (c, Re, int(steps[c]), ref)
