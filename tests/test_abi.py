"""The C-ABI library loads without a GPU and exports every entry point that
include/*.h declares; host-side argument checks answer CLB_EINVAL."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(clb_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1603_01955_gb300 import clb

    return clb.lib


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("clb_create", "clb_step", "clb_observables", "clb_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_library_is_built_for_sm_103a_only():
    from paper_1603_01955_gb300 import build

    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_destroy_null_and_bad_arguments(lib):
    from paper_1603_01955_gb300 import clb

    assert lib.clb_destroy(None) == clb.CLB_OK
    h = C.c_void_p()
    # argument checks run before any CUDA call
    assert lib.clb_create(0, 8, 0.1, 2.0, -1.0, 0, 1e-6, None, C.byref(h)) == clb.CLB_EINVAL
    assert not h.value
    assert lib.clb_create(3, 8, 0.1, 2.0, -1.0, 1, 2.0, None, C.byref(h)) == clb.CLB_EINVAL
    assert lib.clb_create(8, 8, -0.1, 2.0, -1.0, 0, 1e-6, None, C.byref(h)) == clb.CLB_EINVAL
    assert lib.clb_create(8, 8, 0.1, 2.0, 1.5, 0, 1e-6, None, C.byref(h)) == clb.CLB_EINVAL
    assert lib.clb_create(8, 8, 0.1, 2.0, -1.0, 1, -2.0, None, C.byref(h)) == clb.CLB_EINVAL
    assert lib.clb_create(8, 70000, 0.1, 2.0, -1.0, 0, 0.0, None, C.byref(h)) == clb.CLB_EINVAL
    o = clb.clb_opts_default()
    o.storage = 7
    assert lib.clb_create(8, 8, 0.1, 2.0, -1.0, 0, 0.0, C.byref(o), C.byref(h)) == clb.CLB_EINVAL
    o = clb.clb_opts_default()
    o.block_x = 48
    assert lib.clb_create(8, 8, 0.1, 2.0, -1.0, 0, 0.0, C.byref(o), C.byref(h)) == clb.CLB_EINVAL
    assert b"block_x" in lib.clb_last_error()
    assert lib.clb_step(None, 1) == clb.CLB_EINVAL
    assert lib.clb_observables(None, 0, None, None, None, None, None, None) == clb.CLB_EINVAL


def test_opts_defaults_are_the_papers(lib):
    from paper_1603_01955_gb300 import clb

    o = clb.clb_opts_default()
    assert (o.b2, o.sigma, o.s3, o.s8, o.rho_out) == (0.55, 1.0, 1.1, 1.2, 1.0)
    assert o.storage == clb.CLB_FP32_SHIFTED
