"""clb_observables_noalloc: the allocation-free observable reduction.

Some callers cannot allocate device memory when they want the observables
(their device memory belongs to another allocator or is budgeted in advance),
so this entry point reduces a population array the caller already holds, with
its scratch in a fixed array inside the library.  Checked here through the C
ABI against clb_observables on the same state, on two calls in a row (the
shared scratch keeps the previous call's contents).  This file is collected
last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_01955_gb300 import clb

    return torch, clb


def compare(got, want):
    vel = max(np.abs(want["ux_prof"]).max(), 1e-300)
    floors = dict(ux_prof=vel, uy_prof=vel, p_centre=1.0, dp_nonlin=1.0,
                  m_of_x=max(np.abs(want["m_of_x"]).max(), 1e-300))
    for key, scale in floors.items():
        np.testing.assert_allclose(got[key], want[key], rtol=1e-10, atol=1e-12 * scale, err_msg=key)
    for key in ("mass_flow", "q_norm", "u_slip", "total_mass", "ux_max"):
        assert got[key] == pytest.approx(want[key], rel=1e-10, abs=1e-18), key


def noalloc(torch, clb, ch, f_dev, drive, g, kn, col, stream):
    info = ch.info()
    s = clb.clb_scalars()
    out = dict(ux_prof=np.zeros(ch.ny), uy_prof=np.zeros(ch.ny), p_centre=np.zeros(ch.nx),
               dp_nonlin=np.zeros(ch.nx), m_of_x=np.zeros(ch.nx))
    clb.clb_observables_noalloc(f_dev.data_ptr(), ch.nx, ch.ny, drive, g, info["rho_in"], info["rho_out"], kn, col,
                                stream.cuda_stream, s, out["ux_prof"], out["uy_prof"], out["p_centre"],
                                out["dp_nonlin"], out["m_of_x"])
    out.update({k: getattr(s, k) for k, _ in clb.clb_scalars._fields_})
    return out


@pytest.mark.parametrize("drive,value,nx,ny,kn,col", [
    ("pressure", 2.0, 160, 10, 0.15, -1),
    ("body_force", 1e-5, 6, 11, 0.3, 2),
])
def test_noalloc_matches_observables_twice(env, drive, value, nx, ny, kn, col):
    torch, clb = env
    ch = clb.Channel(nx, ny, kn, drive=drive, drive_value=value, storage="fp64")
    d = clb.CLB_DRIVE_PRESSURE if drive == "pressure" else clb.CLB_DRIVE_BODY_FORCE
    g = value if drive == "body_force" else 0.0
    stream = torch.cuda.current_stream()
    for steps in (300, 57):  # two calls in a row on different states
        ch.step(steps)
        want = ch.observables(col)
        f_dev = torch.from_numpy(ch.state()).to("cuda")  # the caller's own device buffer
        torch.cuda.synchronize()
        got = noalloc(torch, clb, ch, f_dev, d, g, kn, col, stream)
        compare(got, want)
        assert got["residual"] == -1.0


def test_noalloc_rejects_oversize(env):
    torch, clb = env
    f = torch.zeros(9 * 4, dtype=torch.float64, device="cuda")
    s = clb.clb_scalars()
    for nx, ny in ((65537, 1), (4, 4097), (0, 4)):
        st = clb.clb_observables_noalloc(f.data_ptr(), nx, ny, clb.CLB_DRIVE_BODY_FORCE, 0.0, 1.0, 1.0, 0.1, -1, 0,
                                         s, None, None, None, None, None, check=False)
        assert st == clb.CLB_EINVAL
        assert b"outside" in clb.lib.clb_last_error()
