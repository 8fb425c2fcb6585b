"""CPU-side checks of the C-ABI library: it loads, exports every entry point
declared in include/*.h, and rejects bad arguments before touching a GPU."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(mdf_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2108_08591_gb300 import _build, _lib
    _build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("mdf_create", "mdf_init", "mdf_step", "mdf_moments", "mdf_gradients"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in sorted(_declared()):
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2108_08591_gb300 import _lib
    assert _declared() <= set(_lib.SIGNATURES)


def test_invalid_arguments_are_rejected_without_a_gpu(lib):
    from paper_2108_08591_gb300 import _lib
    h = ctypes.c_void_p()
    g = _lib.Grid(8, 8, 1)
    r = _lib.Rates(1.0, 1.2, -1.0)
    # bad dimension
    assert lib.mdf_create(ctypes.byref(h), ctypes.byref(g), 4, ctypes.byref(r), None, None) == _lib.EINVAL
    assert b"d must be" in lib.mdf_last_error(None)
    # relaxation rate outside (0, 2)
    bad = _lib.Rates(1.0, 2.5, -1.0)
    assert lib.mdf_create(ctypes.byref(h), ctypes.byref(g), 2, ctypes.byref(bad), None, None) == _lib.EINVAL
    # grid too small / nz mismatch
    g2 = _lib.Grid(1, 8, 1)
    assert lib.mdf_create(ctypes.byref(h), ctypes.byref(g2), 2, ctypes.byref(r), None, None) == _lib.EINVAL
    g3 = _lib.Grid(8, 8, 4)
    assert lib.mdf_create(ctypes.byref(h), ctypes.byref(g3), 2, ctypes.byref(r), None, None) == _lib.EINVAL
    # lid without walls on the last axis
    bc = _lib.BC()
    bc.lid = 1
    assert lib.mdf_create(ctypes.byref(h), ctypes.byref(g), 2, ctypes.byref(r), ctypes.byref(bc), None) == _lib.EINVAL
    # unknown storage
    o = _lib.Opts(9, 1, None)
    assert lib.mdf_create(ctypes.byref(h), ctypes.byref(g), 2, ctypes.byref(r), None, ctypes.byref(o)) == _lib.EUNSUPPORTED
    assert h.value is None
    # null handles
    assert lib.mdf_step(None, 1) == _lib.EINVAL
    assert lib.mdf_init(None, None, None, 0) == _lib.EINVAL
    lib.mdf_destroy(None)


def test_network_kernel_choices_are_checked_without_a_gpu(lib):
    """The process-wide kernel and tile setters validate their arguments on
    the host (they launch nothing)."""
    from paper_2108_08591_gb300 import _lib
    for bad in ((24, 0, 0), (128, 0, 0), (32, -1, 0), (32, 17, 0), (32, 0, 96), (0, 0, 32)):
        assert lib.mdf_nn_set_wgrad_tile(*bad) == _lib.EINVAL, bad
    for good in ((0, 0, 0), (16, 1, 64), (64, 4, 128)):
        assert lib.mdf_nn_set_wgrad_tile(*good) == _lib.OK, good
    assert lib.mdf_nn_set_wgrad_tile(0, 0, 0) == _lib.OK
    assert lib.mdf_nn_set_wgrad_kernel(2) == _lib.EINVAL
    assert lib.mdf_nn_set_wgrad_kernel(1) == _lib.OK
    assert lib.mdf_nn_set_conv_kernel(3) == _lib.EINVAL
    assert lib.mdf_nn_set_conv_kernel(2) == _lib.OK


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors have the header's sizes and field offsets (a C
    program built with gcc against include/mdf.h prints them)."""
    import shutil
    import subprocess
    from paper_2108_08591_gb300 import _lib
    if not shutil.which("gcc"):
        pytest.skip("gcc not found")
    mirrors = {"mdf_grid": _lib.Grid, "mdf_rates": _lib.Rates, "mdf_bc": _lib.BC,
               "mdf_opts": _lib.Opts, "mdf_fields_t": _lib.Fields, "mdf_info_t": _lib.Info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mdf.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_lattice_choice_is_checked_without_a_gpu(lib):
    """q names a lattice of the dimension; equilibrium-shifted storage needs
    D2Q5 / D3Q7."""
    from paper_2108_08591_gb300 import _lib
    h = ctypes.c_void_p()
    r = _lib.Rates(1.0, 1.2, -1.0)
    g2, g3 = _lib.Grid(8, 8, 1), _lib.Grid(8, 8, 8)
    for g, d, q, storage in ((g2, 2, 3, "f32"), (g2, 2, 6, "f32"), (g3, 3, 4, "f32"),
                             (g2, 2, 4, "f16eq"), (g3, 3, 6, "bf16eq")):
        o = _lib.Opts(_lib.STORAGE[storage], 1, None, 0, 0, q)
        assert lib.mdf_create(ctypes.byref(h), ctypes.byref(g), d, ctypes.byref(r), None,
                              ctypes.byref(o)) == _lib.EUNSUPPORTED, (d, q, storage)
    # the in-place AA pattern takes the rest-shifted storage types only
    for storage in ("f16eq", "bf16eq"):
        o = _lib.Opts(_lib.STORAGE[storage], 1, None, 0, 0, 0, 1)
        assert lib.mdf_create(ctypes.byref(h), ctypes.byref(g2), 2, ctypes.byref(r), None,
                              ctypes.byref(o)) == _lib.EUNSUPPORTED, storage


def test_slab_split_is_checked_without_a_gpu(lib):
    """The split axis must divide into k slabs and be periodic; slabs take
    the two-buffer rest-shifted storage types."""
    from paper_2108_08591_gb300 import _lib
    s = ctypes.c_void_p()
    g = _lib.Grid(16, 12, 1)
    r = _lib.Rates(1.0, 1.2, -1.0)
    assert lib.mdf_slabs_create(ctypes.byref(s), ctypes.byref(g), 2, ctypes.byref(r), None, None, 5) == _lib.EINVAL
    assert lib.mdf_slabs_create(ctypes.byref(s), ctypes.byref(g), 2, ctypes.byref(r), None, None, 0) == _lib.EINVAL
    bc = _lib.BC()
    bc.wall[:] = [0, 1, 0]
    assert lib.mdf_slabs_create(ctypes.byref(s), ctypes.byref(g), 2, ctypes.byref(r), ctypes.byref(bc), None,
                                3) == _lib.EUNSUPPORTED
    for storage, inplace in (("f16eq", 0), ("f32", 1)):
        o = _lib.Opts(_lib.STORAGE[storage], 1, None, 0, 0, 0, inplace)
        assert lib.mdf_slabs_create(ctypes.byref(s), ctypes.byref(g), 2, ctypes.byref(r), None, ctypes.byref(o),
                                    3) == _lib.EUNSUPPORTED
    assert b"periodic" in lib.mdf_slabs_last_error(None) or b"storage" in lib.mdf_slabs_last_error(None)


def test_batch_options_are_checked_without_a_gpu(lib):
    """Batched cavities take FP32 storage, D2Q5 / D3Q7 and two pools."""
    from paper_2108_08591_gb300 import _lib
    b = ctypes.c_void_p()
    side = (ctypes.c_int * 2)(65, 129)
    Re = (ctypes.c_double * 2)(100.0, 400.0)
    for storage, q, inplace in (("f16", 0, 0), ("f32", 4, 0), ("f32", 0, 1)):
        o = _lib.Opts(_lib.STORAGE[storage], 1, None, 0, 0, q, inplace)
        st = lib.mdf_batch_create(ctypes.byref(b), 2, 2, ctypes.cast(side, ctypes.c_void_p),
                                  ctypes.cast(Re, ctypes.c_void_p), 0.1, ctypes.byref(o))
        assert st == _lib.EUNSUPPORTED, (storage, q, inplace)
