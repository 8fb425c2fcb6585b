"""The benchmark spec-named boundary calls mdf_moments and mdf_gradients, through
ctypes, against mdf_fields on the same state (Eq. 2-7, 3-15 .. 3-19)."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_08591_gb300 import _build
    _build.build()


@pytest.mark.parametrize("shape,storage", [((37, 29), "f32"), ((37, 29), "f16eq"),
                                           ((11, 9, 13), "f32"), ((11, 9, 13), "bf16eq")])
def test_moments_and_gradients_equal_fields(shape, storage):
    import torch
    from paper_2108_08591_gb300 import Lattice, MdfError
    P, u = synth.smooth_fields(shape, seed=7)
    lat = Lattice(shape, s1=1.6, storage=storage)
    try:
        lat.init(P, u)
        lat.step(23)
        want = {k: v.cpu().numpy() for k, v in lat.fields().items()}
        want.update({k: v.cpu().numpy() for k, v in
                     lat.fields(("rho", "G", "div", "S", "sigma", "omega")).items()})
        Pm, um, rho = lat.moments()
        gr = lat.gradients()
        torch.cuda.synchronize()
        assert np.array_equal(Pm.cpu().numpy(), want["P"])
        assert np.array_equal(um.cpu().numpy(), want["u"])
        assert np.array_equal(rho.cpu().numpy(), want["rho"])
        for k in ("G", "div", "S", "sigma", "omega"):
            assert np.array_equal(gr[k].cpu().numpy(), want[k]), k
        # the calls take no step: a second read gives the same bits
        P2, _, _ = lat.moments()
        assert torch.equal(P2, Pm)
        # null required outputs are rejected with a status, not a fault
        with pytest.raises(MdfError, match="EINVAL"):
            lat._check(lat._lib.mdf_moments(lat._h, None, um.data_ptr(), None))
        with pytest.raises(MdfError, match="EINVAL"):
            lat._check(lat._lib.mdf_gradients(lat._h, None, None, None, None, None))
    finally:
        lat.close()
