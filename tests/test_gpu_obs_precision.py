"""The observable reduction's own error, apart from the storage's.

For FP32 and 16-bit storage the reduction forms each node's rho u in FP32
and sums a thread's rows in compensated FP32; only the sums across threads
are FP64.  Here the library's observables of a state are compared with the
same observables evaluated in FP64, from their definitions (Sec. 3.1, 3.2:
m(x) = sum_y rho u_x, m = mean_x m(x), p = rho/3 at the centreline,
dp = (p_c - p_l)/p_out, p_l linear from p_in to p_out), on exactly that state
as the library stores it (clb_get_state converts the stored values to FP64
without rounding).  The difference is the reduction's error alone.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])


@pytest.fixture(scope="module")
def clb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1603_01955_gb300.clb as clb

    return clb


@pytest.mark.parametrize("storage", ["fp32s", "fp16s", "bf16s", "fp64"])
def test_reduction_error_apart_from_storage(clb, storage):
    nx, ny, ratio = 25601, 256, 2.47
    ch = clb.Channel(nx, ny, 0.1, drive="pressure", drive_value=ratio, storage=storage)
    ch.step(300)
    o = ch.observables()
    f = ch.state()
    ch.close()
    rho = f.sum(axis=0)
    jx = np.tensordot(EX, f, axes=1)  # rho u_x (no body force in a pressure channel)
    m_x = jx.sum(axis=0)
    mbar = m_x.mean()
    rc = 0.5 * (rho[ny // 2 - 1] + rho[ny // 2])
    x = np.arange(nx)
    p_in, p_out = ratio / 3, 1 / 3
    dp = (rc / 3 - (p_in - (p_in - p_out) * x / (nx - 1))) / p_out
    ux_out = jx[:, -1] / rho[:, -1]
    e_m = abs(o["mass_flow"] / mbar - 1)
    e_mx = np.abs(o["m_of_x"] - m_x).max() / np.abs(m_x).max()
    e_dp = np.abs(o["dp_nonlin"] - dp).max()
    e_u = np.abs(o["ux_prof"] - ux_out).max() / np.abs(ux_out).max()
    e_mass = abs(o["total_mass"] / rho.sum() - 1)
    # FP64 storage reduces in FP64; the others form rho u per node in FP32 from
    # deviations no larger than max|d| ~ 1e-2 and sum a few hundred of them:
    # a few FP32 ulps of the column sums, relative to the largest of them
    tol = 1e-12 if storage == "fp64" else 2e-6
    assert e_m <= tol, e_m
    assert e_mx <= tol, e_mx
    assert e_u <= tol, e_u
    assert e_dp <= (1e-14 if storage == "fp64" else 1e-6), e_dp
    assert e_mass <= (1e-14 if storage == "fp64" else 1e-9), e_mass
