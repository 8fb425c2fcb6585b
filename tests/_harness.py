"""Shared plumbing of the GPU parity tests: run the CUDA library (through the
C-ABI binding) and the FP64 oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np

import oracle as O

FIELDS = ("P", "u", "rho", "G", "div", "S", "sigma", "omega")


def run_gpu(shape, P, u, steps, s1, s2=-1.0, storage="f32", wall=(0, 0, 0), lid=False,
            lid_u=(0.0, 0.0, 0.0), with_rho=True, force=None, names=FIELDS, forcing="eq3-21",
            G=None, q=0):
    from paper_2108_08591_gb300 import Lattice
    lat = Lattice(shape, s1=s1, s2=s2, storage=storage, wall=wall, lid=lid, lid_u=lid_u,
                  with_rho=with_rho, q=q)
    try:
        lat.set_forcing(forcing)
        if force is not None:  # before init: the Scheme II initial state depends on it
            lat.set_force(force)
        lat.init(P, u, G)
        lat.step(steps)
        names = [k for k in names if k != "rho" or with_rho]
        out = lat.fields_host(names)
        out["mask"] = lat.mask()
        return out
    finally:
        lat.close()


def run_oracle(shape, P, u, steps, s1, s2=None, wall=(0, 0, 0), lid=False,
               lid_u=(0.0, 0.0, 0.0), with_rho=True, force=None, scheme=0, G=None, q=0):
    d = len(shape)
    pb = O.Problem(d=d, n=tuple(shape), s1=s1, s2=s2, wall=wall, lid=lid, lid_u=lid_u,
                   with_rho=with_rho, force=force, scheme=scheme, nq=q)
    f = O.init(pb, P, u, G)
    O.run(pb, f, steps)
    Pn, un, rho = O.macro(pb, f)
    out = {"P": Pn, "u": un}
    if with_rho:
        out["rho"] = rho
    out.update(O.derived(pb, f))
    out["mask"] = O.mask(pb)
    out["_f"] = f
    out["_pb"] = pb
    return out


def rel(ref, num) -> float:
    return O.rel_l2(ref, num)


def rel_p(ref_P, num_P) -> float:
    """E_L2 of P - mean(P): the pressure is compared by its fluctuation."""
    return O.rel_l2(ref_P - ref_P.mean(), num_P - num_P.mean())


def errors(ref, got) -> dict:
    e = {"P": rel_p(ref["P"], got["P"]), "u": rel(ref["u"], got["u"])}
    for k in ("G", "S", "sigma", "omega"):
        if k in got:
            e[k] = rel(ref[k], got[k])
    if "rho" in got and "rho" in ref:
        e["rho"] = float(np.abs(ref["rho"] - got["rho"]).max())
    return e
