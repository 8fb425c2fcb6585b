"""Stability of the method at the workloads' relaxation rates, on the FP64
oracle alone.

1. The lid-driven cavity at high cell Reynolds number (Sec. 4.3 cavity; D2Q5
   MRT with the s2 rule of Sec. 4.1).  The paper runs its cavity at cell
   Re = U dx / nu <= 1.95.  The seeded batch of 64 cavities (sides from
   {65, 129, 257, 513}, Re from U[100, 3200], lid speed 0.1) reaches cell
   Re ~ 49, and the GPU batch reports many of those draws as diverged.  These
   tests settle whether the divergence belongs to the method or to the FP32
   path: the FP64 oracle, with the same geometry (anti-halfway bounce-back
   walls, lid on +y), the same s1 = 1/(3 nu + 1/2) and the same s2 rule,
   blows up on the same draws, and stays bounded on neighbouring draws of
   lower cell Re.  (tests/test_gpu_batch.py runs the same draws through the
   GPU batch and compares the step at which each is reported diverged.)  The
   batch checks for non-finite values every 100 steps; the oracle here is
   checked at the same cadence.

2. Linear stability of a uniform flow.  A uniform velocity U plus a 1e-7
   seeded perturbation on a small periodic box: the perturbation must decay
   where the scheme is stable.  With the 3D Taylor-Green rates (D3Q7, nu for
   Re = 1600 on U0 = 0.05 and k = 2 pi / 512, so s1 = 1.960), the s2 rule of
   Sec. 4.1 gives s2 = 0.053, and the perturbation grows without bound for
   U >= 0.015: the paper's rule, made for its D2Q5 wall experiments, leaves
   the D3Q7 scheme unstable at that workload's speeds.  With s2 = 1 (which
   leaves the viscosity, set by s1 through Eq. 3-13a, unchanged) it decays.
   The 2D Taylor-Green rates (D2Q5, nu = 0.01, s2 rule) are stable at the
   speeds of that workload.
"""
import numpy as np
import pytest

import oracle as O
import synth

U = 0.1
CHECK = 100


def _run_until_nonfinite(N, Re, max_steps):
    """Return (first 100-step check at which f holds a non-finite value or
    None, the final populations)."""
    nu = U * N / Re
    s1 = 1.0 / (3.0 * nu + 0.5)
    pb = O.Problem(d=2, n=(N, N), s1=s1, wall=(1, 1, 0), lid=True, lid_u=(U, 0.0, 0.0))
    f = O.init(pb, *synth.rest_state(N * N, 2))
    step = 0
    while step < max_steps:
        O.run(pb, f, CHECK)
        step += CHECK
        if not np.isfinite(f).all():
            return step, f
    return None, f


def _draw(side, index_hint):
    """The (side, Re) pair of the seeded 64-cavity batch at a given index."""
    draws = synth.cavity_batch()
    N, Re = draws[index_hint]
    assert N == side
    return N, Re


# (batch index, side) of draws above cell Re 8
DIVERGED = [(15, 65), (18, 65), (17, 65)]
# (batch index, side): bounded draws of lower cell Re on the same box size
BOUNDED = [(22, 65), (46, 65)]


@pytest.mark.parametrize("idx,side", DIVERGED)
def test_oracle_diverges_above_cell_re_8(idx, side):
    N, Re = _draw(side, idx)
    assert Re / N > 8.0
    step, _ = _run_until_nonfinite(N, Re, 10000)
    assert step is not None, f"FP64 oracle bounded after 10000 steps at Re {Re:.1f}"


@pytest.mark.parametrize("idx,side", BOUNDED)
def test_oracle_bounded_below_the_limit(idx, side):
    N, Re = _draw(side, idx)
    assert Re / N < 7.3
    step, f = _run_until_nonfinite(N, Re, 6000)
    assert step is None
    pb = O.Problem(d=2, n=(N, N), s1=1.0 / (3.0 * U * N / Re + 0.5), wall=(1, 1, 0), lid=True,
                   lid_u=(U, 0.0, 0.0))
    _, u, _ = O.macro(pb, f)
    assert np.abs(u).max() < 1.2 * U  # the flow stays of the lid's magnitude


def _perturbation_rms(d, n, s1, s2, U, steps, seed=1):
    """RMS of the velocity deviation from its mean after `steps` updates of a
    uniform flow U along x with a 1e-7 seeded perturbation of P and u."""
    rng = np.random.default_rng(seed)
    N = n ** d
    P = 1.0 + 1e-7 * rng.standard_normal(N)
    u = 1e-7 * rng.standard_normal((d, N))
    u[0] += U
    pb = O.Problem(d=d, n=(n,) * d, s1=s1, s2=s2)
    f = O.init(pb, P, u)
    O.run(pb, f, steps)
    _, un, _ = O.macro(pb, f)
    dev = un - un.mean(axis=1, keepdims=True)
    rms = float(np.sqrt((dev ** 2).mean()))
    return rms if np.isfinite(rms) else np.inf


S1_TG3D = 1.0 / (4.0 * (0.05 / (2 * np.pi / 512 * 1600.0)) + 0.5)
S1_TG2D = 1.0 / (3.0 * 0.01 + 0.5)


def test_d3q7_s2_rule_unstable_at_tg3d_rates():
    assert O.s2_rule(S1_TG3D) == pytest.approx(0.0533, abs=1e-3)
    assert _perturbation_rms(3, 16, S1_TG3D, None, 0.05, 2000) > 1e-3  # grew from 1e-7
    assert _perturbation_rms(3, 16, S1_TG3D, None, 0.015, 2000) > 1e-6
    # at rest the same rates are stable
    assert _perturbation_rms(3, 16, S1_TG3D, None, 0.0, 2000) < 1e-8


@pytest.mark.parametrize("s2", [1.0, 1.5])
def test_d3q7_stable_at_tg3d_rates_with_larger_s2(s2):
    assert _perturbation_rms(3, 16, S1_TG3D, s2, 0.05, 2000) < 1e-7


@pytest.mark.parametrize("U", [0.01, 0.02])
def test_d2q5_s2_rule_stable_at_tg2d_rates(U):
    assert _perturbation_rms(2, 32, S1_TG2D, None, U, 2000) < 1e-8
