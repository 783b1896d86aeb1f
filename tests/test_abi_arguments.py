"""Host-side argument checks of the batched, adjoint, checkpoint, peak and
allocation-free entry points.  Every case here is refused before the library
makes its first CUDA call, so the tests run without a GPU; each asserts the
status code and that the message names the entry point."""
import ctypes as C
import os
import struct

import pytest


@pytest.fixture(scope="module")
def clb():
    from paper_1603_01955_gb300 import clb

    return clb


def arr(ctype, values):
    return (ctype * len(values))(*values)


def refused(clb, status, who, code=None):
    code = clb.CLB_EINVAL if code is None else code
    assert status == code, (status, clb.lib.clb_last_error())
    assert who.encode() in clb.lib.clb_last_error()


def test_batch_create_arguments(clb):
    lib = clb.lib
    h = C.c_void_p()
    nx, ny, kn = arr(C.c_int, [8, 8]), arr(C.c_int, [8, 8]), arr(C.c_double, [0.1, 0.2])
    assert lib.clb_batch_create(2, nx, ny, kn, 2.0, -1.0, 1e-6, None, None) == clb.CLB_EINVAL
    refused(clb, lib.clb_batch_create(0, nx, ny, kn, 2.0, -1.0, 1e-6, None, C.byref(h)), "clb_batch_create")
    assert not h.value
    refused(clb, lib.clb_batch_create(2, None, ny, kn, 2.0, -1.0, 1e-6, None, C.byref(h)), "clb_batch_create")
    refused(clb, lib.clb_batch_create(2, nx, ny, kn, -1.0, -1.0, 1e-6, None, C.byref(h)), "clb_batch_create")
    refused(clb, lib.clb_batch_create(2, nx, ny, kn, 2.0, 1.5, 1e-6, None, C.byref(h)), "clb_batch_create")
    refused(clb, lib.clb_batch_create(2, nx, ny, kn, 2.0, -1.0, float("nan"), None, C.byref(h)),
            "clb_batch_create")
    bad_kn = arr(C.c_double, [0.1, 0.0])
    refused(clb, lib.clb_batch_create(2, nx, ny, bad_kn, 2.0, -1.0, 1e-6, None, C.byref(h)), "channel 1")
    # one block holds a whole channel: 4096 nodes at most
    big = arr(C.c_int, [8, 1024])
    refused(clb, lib.clb_batch_create(2, nx, big, kn, 2.0, -1.0, 1e-6, None, C.byref(h)), "shared memory")
    # sides whose product overflows a 32-bit int are refused, not wrapped
    wide = arr(C.c_int, [65536, 8])
    refused(clb, lib.clb_batch_create(2, wide, wide, kn, 2.0, -1.0, 1e-6, None, C.byref(h)), "channel 0")
    o = clb.clb_opts_default()
    o.storage = clb.CLB_FP16_SCALED
    refused(clb, lib.clb_batch_create(2, nx, ny, kn, 2.0, -1.0, 1e-6, C.byref(o), C.byref(h)), "storage")
    o = clb.clb_opts_default()
    o.block_x = 40
    refused(clb, lib.clb_batch_create(2, nx, ny, kn, 2.0, -1.0, 1e-6, C.byref(o), C.byref(h)), "block_x")
    assert not h.value
    for name in ("clb_batch_step", "clb_batch_tune", "clb_batch_set_schedule", "clb_batch_schedule",
                 "clb_batch_observables", "clb_batch_info"):
        fn = getattr(lib, name)
        args = [None] + [0] * (len(fn.argtypes) - 1)
        args = [a if t in (C.c_int, C.c_int64) else None for a, t in zip(args, fn.argtypes)]
        refused(clb, fn(*args), name)
    refused(clb, lib.clb_batch_get_state(None, 0, None), "clb_batch state")
    assert lib.clb_batch_destroy(None) == clb.CLB_OK


def test_adjoint_arguments(clb):
    lib = clb.lib
    h = C.c_void_p()
    j = C.c_double()
    ok = dict(nx=4, ny=8, kn=0.1, a=2.0, r=-1.0, g=1e-5, n=100, every=10)

    def fwd(**kw):
        p = dict(ok, **kw)
        return lib.clb_adjoint_forward(p["nx"], p["ny"], p["kn"], p["a"], p["r"], p["g"], p["n"], p["every"],
                                       kw.get("opts"), C.byref(h), C.byref(j))

    assert lib.clb_adjoint_forward(4, 8, 0.1, 2.0, -1.0, 1e-5, 100, 10, None, None, None) == clb.CLB_EINVAL
    for bad in (dict(nx=0), dict(ny=0), dict(nx=4096, ny=4096), dict(n=0), dict(kn=0.0), dict(a=-1.0),
                dict(r=1.5), dict(g=float("inf"))):
        refused(clb, fwd(**bad), "clb_adjoint_forward")
        assert not h.value
    o = clb.clb_opts_default()
    o.storage = clb.CLB_BF16_SCALED
    refused(clb, fwd(opts=C.byref(o)), "storage")
    grad = (C.c_double * 3)()
    refused(clb, lib.clb_adjoint_backward(None, 1.0, grad), "clb_adjoint_backward")
    refused(clb, lib.clb_adjoint_q(None, C.byref(j)), "clb_adjoint_q")
    refused(clb, lib.clb_adjoint_q_backward(None, 1.0, grad), "clb_adjoint_q_backward")
    assert lib.clb_adjoint_destroy(None) == clb.CLB_OK


def test_noalloc_and_peak_arguments(clb):
    lib = clb.lib
    s = clb.clb_scalars()
    fake = C.c_void_p(256)  # never dereferenced: every case below is refused first

    def call(f, nx, ny, drive, kn=0.1, rho_in=2.0, rho_out=1.0):
        return lib.clb_observables_noalloc(f, nx, ny, drive, 0.0, rho_in, rho_out, kn, -1, None, C.byref(s),
                                           None, None, None, None, None)

    refused(clb, call(None, 8, 8, clb.CLB_DRIVE_PRESSURE), "populations pointer")
    refused(clb, call(fake, 0, 8, clb.CLB_DRIVE_PRESSURE), "outside")
    refused(clb, call(fake, 65537, 8, clb.CLB_DRIVE_PRESSURE), "outside")
    refused(clb, call(fake, 8, 4097, clb.CLB_DRIVE_PRESSURE), "outside")
    refused(clb, call(fake, 8, 8, 5), "unknown drive")
    refused(clb, call(fake, 8, 8, clb.CLB_DRIVE_PRESSURE, kn=0.0), "pressure drive")
    refused(clb, call(fake, 8, 8, clb.CLB_DRIVE_PRESSURE, rho_out=-1.0), "pressure drive")
    t = C.c_double()
    refused(clb, lib.clb_peak_fma(clb.CLB_FP64, None, None), "clb_peak_fma")
    refused(clb, lib.clb_peak_fma(clb.CLB_FP16_SCALED, None, C.byref(t)), "clb_peak_fma")


def test_load_refuses_bad_files(clb, tmp_path):
    lib = clb.lib
    h = C.c_void_p()
    refused(clb, lib.clb_load(None, None, C.byref(h)), "clb_load")
    missing = os.fsencode(str(tmp_path / "missing.ckpt"))
    refused(clb, lib.clb_load(missing, None, C.byref(h)), "cannot open", clb.CLB_EIO)
    short = tmp_path / "short.ckpt"
    short.write_bytes(b"CLB")
    refused(clb, lib.clb_load(os.fsencode(str(short)), None, C.byref(h)), "truncated header", clb.CLB_EIO)
    other = tmp_path / "other.ckpt"
    other.write_bytes(struct.pack("<8s", b"NOTACLB!") + bytes(168))
    refused(clb, lib.clb_load(os.fsencode(str(other)), None, C.byref(h)), "not a CLB checkpoint", clb.CLB_EIO)
    assert not h.value


def ckpt_header(version=1, elem=4, buf_bytes=None, checksum=0):
    """A checkpoint header of a 4 x 2 FP32-shifted periodic channel, laid out
    as clb_save writes it (176 bytes, little-endian)."""
    nx, ny, storage, pitch, rc_stride = 4, 2, 1, 64, 32
    if buf_bytes is None:
        buf_bytes = 9 * ny * pitch * 4
    rc_bytes = 2 * rc_stride * 4
    ints = (nx, ny, 0, storage, 0, pitch, elem, rc_stride)
    doubles = (0.1, 2.0, 0.6, 1e-6, 0.55, 1.0, 1.1, 1.2, 1.0, 0.0)
    h = struct.pack("<8sII8iqii10d4Q", b"CLBCKPT1", version, 176, *ints, 0, 0, 0, *doubles, buf_bytes, rc_bytes,
                    checksum, 0)
    assert len(h) == 176
    return h, buf_bytes + rc_bytes


@pytest.mark.parametrize("case", ["version", "inconsistent", "payload", "checksum"])
def test_load_refuses_bad_headers_and_payloads(clb, tmp_path, case):
    lib = clb.lib
    h = C.c_void_p()
    if case == "version":
        head, n = ckpt_header(version=2)
        data, why = head + bytes(n), "unsupported checkpoint version"
    elif case == "inconsistent":
        head, n = ckpt_header(elem=2)  # FP32 storage stores 4-byte values
        data, why = head + bytes(n), "inconsistent header"
    elif case == "payload":
        head, n = ckpt_header()
        data, why = head + bytes(n - 1), "truncated payload"
    else:
        head, n = ckpt_header(checksum=12345)
        data, why = head + bytes(n), "checksum mismatch"
    p = tmp_path / f"{case}.ckpt"
    p.write_bytes(data)
    refused(clb, lib.clb_load(os.fsencode(str(p)), None, C.byref(h)), why, clb.CLB_EIO)
    assert not h.value
