"""The slab decomposition's exchange plan on CPU, across processes: two gloo
ranks on 127.0.0.1 each advance one half of a periodic lattice (split along
its last axis, one ghost layer per side) with the FP64 oracle, and after
every step send each neighbour only the populations that cross the shared
face: one direction per face and set, one layer.  The halves must equal the
undivided oracle run.  This is the exchange that mdf_slabs_* performs
between sub-domains on one GPU (there with the post-collision slot before
streaming; here, since the oracle streams by push, with the streamed layer
that lands in the neighbour's ghost)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _shape(d):
    return (6, 12) if d == 2 else (4, 5, 8)


def _axis_dirs(d, q):
    """(up, down): the directions along + and - the last axis."""
    import oracle as O
    cv, _, _ = O.lattice(d, q, 1.0)
    up = int(np.flatnonzero(cv[:, d - 1] > 0)[0])
    dn = int(np.flatnonzero(cv[:, d - 1] < 0)[0])
    return up, dn


def _rank(rank, world, port, d, nq, steps, q_out):
    import torch
    import torch.distributed as dist

    import oracle as O
    import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    shape = _shape(d)
    n = shape[-1]
    nloc = n // world
    L = int(np.prod(shape[:-1]))  # nodes per layer
    P, u = synth.smooth_fields(shape, seed=43, amp=0.01)
    # local slab: global layers rank*nloc - 1 .. rank*nloc + nloc (periodic)
    layers = [(rank * nloc + l - 1) % n for l in range(nloc + 2)]
    sel = np.concatenate([np.arange(g * L, (g + 1) * L) for g in layers])
    lshape = tuple(shape[:-1]) + (nloc + 2,)
    pb = O.Problem(d=d, n=lshape, s1=1.3, nq=nq)
    f = O.init(pb, P[sel], u[:, sel])
    up, dn = _axis_dirs(d, pb.q)
    lo, hi = (rank - 1) % world, (rank + 1) % world
    Nl = L * (nloc + 2)
    for _ in range(steps):
        O.run(pb, f, 1)
        fr = f.reshape(pb.nsets, pb.q, Nl)
        # my top ghost layer received, by streaming, what my last real layer
        # sends up: it belongs to the upper neighbour's first real layer;
        # my bottom ghost layer holds what goes down to the lower neighbour
        send_up = torch.from_numpy(fr[:, up, (nloc + 1) * L:(nloc + 2) * L].copy())
        send_dn = torch.from_numpy(fr[:, dn, 0:L].copy())
        recv_lo = torch.empty_like(send_up)
        recv_hi = torch.empty_like(send_dn)
        reqs = [dist.isend(send_up, hi), dist.isend(send_dn, lo),
                dist.irecv(recv_lo, lo), dist.irecv(recv_hi, hi)]
        for r in reqs:
            r.wait()
        fr[:, up, L:2 * L] = recv_lo.numpy()                 # first real layer, moving up
        fr[:, dn, nloc * L:(nloc + 1) * L] = recv_hi.numpy()  # last real layer, moving down
    Pn, un, _ = O.macro(pb, f)
    q_out.put((rank, Pn[L:(nloc + 1) * L].copy(), un[:, L:(nloc + 1) * L].copy(),
               f.reshape(pb.nsets, pb.q, Nl)[:, :, L:(nloc + 1) * L].copy()))
    dist.destroy_process_group()


@pytest.mark.parametrize("d,nq", [(2, 0), (3, 0), (2, 4)])
def test_two_rank_slab_exchange_equals_the_undivided_lattice(d, nq):
    import oracle as O
    import synth
    steps = 9
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, d, nq, steps, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=120) for _ in range(2)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shape = _shape(d)
    P, u = synth.smooth_fields(shape, seed=43, amp=0.01)
    pb = O.Problem(d=d, n=shape, s1=1.3, nq=nq)
    f = O.run(pb, O.init(pb, P, u), steps)
    Pn, un, _ = O.macro(pb, f)
    got_P = np.concatenate([o[1] for o in out])
    got_u = np.concatenate([o[2] for o in out], axis=1)
    got_f = np.concatenate([o[3] for o in out], axis=2)
    assert np.abs(got_f - f).max() < 1e-15
    assert np.abs(got_P - Pn).max() < 1e-15 and np.abs(got_u - un).max() < 1e-15
