"""The in-place AA access pattern as a plain CPU model, against the oracle.

The collision of one node is the oracle's own step on a one-node periodic
lattice (its stream maps every population back onto the node).  The model
keeps one array A[set][i][node] and alternates the two updates the GPU
kernels implement:
  even: f_i = A[i][x];                   collide;  A[opp(i)][x] = f*_i
  odd:  f_i = A[opp(i)][x - c_i]          collide;  A[i][x + c_i] = f*_i
with anti-halfway bounce-back inside the node:
  odd read,  link into x along c_i through a wall:   f_i = -A[i][x] + 2 w_i ubar_w
  odd write, link out of x along c_i through a wall: A[opp(i)][x] = -f*_i + 2 w_i ubar_w
(ubar_w: rho0 for the alpha = 0 set, the lid velocity on a lid link; the
GPU's rest-shifted storage cancels the rho0 term)
After every update the state it encodes must equal the oracle's (push
streaming over two arrays).  This pins the layout logic on the CPU; the GPU
kernels are then checked bit for bit against the pull stream."""
import numpy as np
import pytest

import oracle as O
import synth


def _collide(pb1, f_node, force_node):
    """Post-collision populations of one node [nsets][q]."""
    pb1.force = None if force_node is None else force_node.reshape(pb1.d, 1)
    g = f_node.reshape(pb1.nsets, pb1.q, 1).copy()
    O.run(pb1, g, 1)
    return g[:, :, 0]


def _model(d, n, q, wall, lid, lid_u, force, steps, s1=1.3):
    pb = O.Problem(d=d, n=n, s1=s1, wall=wall, lid=lid, lid_u=lid_u, force=force, nq=q)
    pb1 = O.Problem(d=d, n=(1,) * d, s1=s1, nq=q)
    cv, w, _ = O.lattice(d, pb.q, 1.0)
    c = cv.astype(int)
    opp = [int(np.flatnonzero((cv == -cv[i]).all(axis=1))[0]) for i in range(pb.q)]
    mask = O.mask(pb)
    N, ns, Q = pb.N, pb.nsets, pb.q
    shape = list(n)

    def node(xs):
        k, s = 0, 1
        for b in range(d):
            k += (xs[b] % shape[b]) * s
            s *= shape[b]
        return k

    def coords(k):
        out = []
        for b in range(d):
            out.append(k % shape[b])
            k //= shape[b]
        return out

    up = int(np.flatnonzero(c[:, d - 1] > 0)[0])
    alpha = [a + 1 - (1 if pb.with_rho else 0) for a in range(ns)]

    def lid_term(i_arrive, k):
        """2 w_i ubar_wall of the anti-halfway bounce-back (the oracle works
        with unshifted populations): rho0 = 1 for the alpha = 0 set, the lid
        velocity for a velocity set on a link through the lid, else 0."""
        out = np.zeros(ns)
        for a in range(ns):
            if alpha[a] == 0:
                out[a] = 2.0 * w[i_arrive] * 1.0
            elif lid and i_arrive == opp[up] and (mask[k] & 0x80):
                out[a] = 2.0 * w[i_arrive] * lid_u[alpha[a] - 1]
        return out

    P, u = synth.smooth_fields(tuple(n), seed=47, amp=0.01)
    ref = O.init(pb, P, u)
    A = ref.copy()  # even layout: slot i of x holds f_i(x)
    Fn = None if force is None else np.asarray(force).reshape(d, N)
    for t in range(steps):
        odd = t % 2 == 1
        # node by node in place, in a scrambled order: every node reads and
        # then writes its own set of locations, and no other node touches
        # them, so the order cannot matter
        order = np.random.default_rng(t).permutation(N)
        for k in order:
            x = coords(k)
            f = np.zeros((ns, Q))
            for i in range(Q):
                if not odd:
                    f[:, i] = A[:, i, k]
                elif i != opp[i] and (mask[k] >> opp[i]) & 1:
                    f[:, i] = -A[:, i, k] + lid_term(i, k)
                else:
                    f[:, i] = A[:, opp[i], node([x[b] - c[i, b] for b in range(d)])]
            fs = _collide(pb1, f, None if Fn is None else Fn[:, k])
            for i in range(Q):
                if not odd:
                    A[:, opp[i], k] = fs[:, i]
                elif i != opp[i] and (mask[k] >> i) & 1:
                    A[:, opp[i], k] = -fs[:, i] + lid_term(opp[i], k)
                else:
                    A[:, i, node([x[b] + c[i, b] for b in range(d)])] = fs[:, i]
        ref = O.run(pb, ref, 1)
        # decode the state the layout holds and compare with the oracle's
        got = np.zeros_like(ref)
        for k in range(N):
            x = coords(k)
            for i in range(Q):
                if not odd:  # left the odd layout
                    if i != opp[i] and (mask[k] >> opp[i]) & 1:
                        got[:, i, k] = -A[:, i, k] + lid_term(i, k)
                    else:
                        got[:, i, k] = A[:, opp[i], node([x[b] - c[i, b] for b in range(d)])]
                else:  # back in the even layout
                    got[:, i, k] = A[:, i, k]
        assert np.abs(got - ref).max() < 1e-14, (t, np.abs(got - ref).max())
    return A


@pytest.mark.parametrize("d,n,q,wall,lid", [
    (2, (5, 4), 0, (0, 0, 0), False),
    (2, (5, 4), 0, (1, 1, 0), True),
    (2, (4, 5), 4, (0, 1, 0), True),
    (3, (3, 4, 3), 0, (1, 0, 1), True),
    (3, (3, 3, 4), 6, (0, 1, 0), False),
])
def test_aa_pattern_reproduces_the_oracle_stream(d, n, q, wall, lid):
    N = int(np.prod(n))
    F = np.stack([1e-4 * np.linspace(1, 2, N) for _ in range(d)])
    _model(d, n, q, wall, lid, (0.02, -0.01, 0.0), F, steps=5)
