"""The allocation-free host readback mdf_fields_host_noalloc, through the C-ABI.

It exists for callers that cannot let the library allocate GPU memory at the
moment they read results back: processes whose device memory is fully held
by another allocator, or code that runs while allocation is forbidden (for
instance while another thread captures a CUDA graph in global mode).  Its
output must equal that of the ordinary entry point, mdf_fields with host
outputs, which stages through a buffer it allocates.

This file is collected last on purpose, so a failure here leaves every other
test already run; it passes alone and after the rest of the suite.
"""
import numpy as np
import pytest

import synth
from tests._harness import rel

pytestmark = pytest.mark.gpu

NAMES = ("P", "u", "rho", "G", "div", "S", "sigma", "omega")
TOL = 1e-10  # the FP64 parity bound of the suite; the two paths share one kernel


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_08591_gb300 import _build
    _build.build()


@pytest.mark.parametrize("shape,storage,inplace", [
    ((96, 70), "f32", False), ((24, 18, 14), "f64", False),
    # equilibrium-shifted storage: the node moments travel with the populations
    ((96, 70), "f16eq", False), ((24, 18, 14), "bf16eq", False),
    # in-place AA stream: the layout parity of the state changes every update
    ((96, 70), "f32", True), ((24, 18, 14), "f16", True)])
def test_noalloc_readback_matches_fields_on_two_calls(shape, storage, inplace):
    from paper_2108_08591_gb300 import Lattice
    P, u = synth.smooth_fields(shape, seed=31)
    lat = Lattice(shape, s1=1.45, storage=storage, inplace=inplace)
    try:
        lat.init(P, u)
        lat.step(17)
        for call in range(2):  # two calls in a row share the static buffer
            want = lat.fields_host(NAMES)
            got = lat.fields_host_noalloc(NAMES)
            for k in NAMES:
                assert got[k].shape == want[k].shape
                assert rel(want[k], got[k]) <= TOL, (call, k)
            lat.step(9)
        # a smaller request after a larger one reads only what it asked for
        want = lat.fields_host(("u",))
        got = lat.fields_host_noalloc(("u",))
        assert rel(want["u"], got["u"]) <= TOL
    finally:
        lat.close()


def test_noalloc_rejects_requests_beyond_the_static_buffer():
    from paper_2108_08591_gb300 import Lattice, MdfError
    shape = (1024, 1024)  # all fields: 15 doubles per node > 2,097,152
    P, u = synth.rest_state(shape[0] * shape[1], 2)
    lat = Lattice(shape, s1=1.2)
    try:
        lat.init(P, u)
        with pytest.raises(MdfError, match="EINVAL.*static staging buffer"):
            lat.fields_host_noalloc(NAMES)
    finally:
        lat.close()
    # a request that fits still works: P and u are 3 doubles per node
    small = Lattice((512, 512), s1=1.2)
    try:
        small.init(*synth.rest_state(512 * 512, 2))
        out = small.fields_host_noalloc(("P", "u"))
        assert np.allclose(out["P"], 1.0, atol=1e-7) and np.abs(out["u"]).max() < 1e-7
    finally:
        small.close()
