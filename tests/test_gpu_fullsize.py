"""Parity at the full benchmark size: the L/H = 100 pressure-driven channel with
Ny = 256, Nx = 25601 (6.55 M nodes), Kn_out = 0.1, p_in/p_out = 2.47, in the
launch configuration the benchmark times (library defaults).

The oracle cannot run thousands of steps on 6.55 M nodes within a test, so:
* one step is checked node by node on a sample (all corners, the inlet and
  outlet columns and their two neighbours, both wall rows, random interior
  nodes): the GPU's state after step n is handed to the oracle, which computes
  step n+1 at the sampled nodes;
* a short run of the whole grid is compared in full (FP64) and on the mass
  flow (FP32-shifted).
"""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu

C3 = inputs.PRESSURE_25601x256


@pytest.fixture(scope="module")
def clb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1603_01955_gb300.clb as clb

    return clb


def params(oracle_mod):
    return oracle_mod.OracleParams(nx=C3["nx"], ny=C3["ny"], pressure=True, kn=C3["kn_out"],
                                   rho_in=C3["ratio"], rho_out=1.0)


def sample_nodes(nx, ny, seed=5, n_interior=3000):
    r = inputs.rng(seed)
    xs, ys = [], []
    for x in (0, 1, 2, nx - 3, nx - 2, nx - 1):
        for y in list(range(0, 4)) + list(range(ny - 4, ny)) + list(r.integers(0, ny, 8)):
            xs.append(x)
            ys.append(int(y))
    for y in (0, 1, ny - 2, ny - 1):
        for x in r.integers(0, nx, 64):
            xs.append(int(x))
            ys.append(y)
    xs += list(r.integers(0, nx, n_interior))
    ys += list(r.integers(0, ny, n_interior))
    return np.array(xs, np.int32), np.array(ys, np.int32)


def reference_profile(nx):
    """R(x): the linear density between the end pressures (the initial state)."""
    x = np.arange(nx)
    return C3["ratio"] + (1.0 - C3["ratio"]) * x / (nx - 1)


@pytest.mark.parametrize("storage", ["fp64", "fp32s"])
def test_full_size_one_step_sampled(clb, oracle_mod, storage):
    nx, ny = C3["nx"], C3["ny"]
    ch = clb.Channel(nx, ny, C3["kn_out"], drive="pressure", drive_value=C3["ratio"], storage=storage)
    ch.step(60)
    f0 = ch.state()
    ch.step(1)
    f1 = ch.state()
    xs, ys = sample_nodes(nx, ny)
    want = oracle_mod.step_nodes(params(oracle_mod), f0, xs, ys)
    got = f1[:, ys, xs].T
    del f0, f1
    if storage == "fp64":
        assert (np.abs(got - want) / np.abs(want)).max() <= 1e-13
    else:
        w = oracle_mod.feq(1.0, 0.0, 0.0)
        dev = want - w[None, :] * reference_profile(nx)[xs][:, None]
        scale = np.abs(dev).max()
        assert scale > 0
        assert np.abs(got - want).max() <= 8 * 2.0**-24 * scale + 4 * 2.0**-24 * 1e-3


def test_full_size_short_run(clb, oracle_mod):
    nx, ny, n = C3["nx"], C3["ny"], 100
    orc = oracle_mod.OracleSim(params(oracle_mod))
    orc.step(n)
    o = orc.observables()
    so = orc.state()
    ch64 = clb.Channel(nx, ny, C3["kn_out"], drive="pressure", drive_value=C3["ratio"], storage="fp64")
    ch64.step(n)
    s64 = ch64.state()
    assert (np.abs(s64 - so) / np.abs(so)).max() <= 1e-12
    del s64
    g64 = ch64.observables()
    ch64.close()
    assert g64["mass_flow"] == pytest.approx(o["mass_flow"], rel=1e-11)
    ch32 = clb.Channel(nx, ny, C3["kn_out"], drive="pressure", drive_value=C3["ratio"], storage="fp32s")
    ch32.step(n)
    g32 = ch32.observables()
    # every population of the whole grid, within the FP32 bound of the parity
    # tests (c 2^-24 sqrt(n) max|d|, c = 4, d the deviation from w_i R(x))
    s32 = ch32.state()
    w = oracle_mod.feq(1.0, 0.0, 0.0)[:, None, None]
    scale = np.abs(so - w * reference_profile(nx)[None, None, :]).max()
    assert np.abs(s32 - so).max() <= 4 * 2.0**-24 * np.sqrt(n) * scale
    del s32
    ch32.close()
    # the 16-bit storages: the same bound with their unit round-off (FP16 x 2^14: 2^-11,
    # BF16: 2^-8); their mass flow is reported, not bounded at 1e-5
    for storage, u in (("fp16s", 2.0**-11), ("bf16s", 2.0**-8)):
        ch = clb.Channel(nx, ny, C3["kn_out"], drive="pressure", drive_value=C3["ratio"], storage=storage)
        ch.step(n)
        s16 = ch.state()
        ch.close()
        err = np.abs(s16 - so).max()
        del s16
        assert err <= 4 * u * np.sqrt(n) * scale, (storage, err / scale)
    assert g32["mass_flow"] == pytest.approx(o["mass_flow"], rel=1e-5)
    assert np.abs(g32["m_of_x"] - o["m_of_x"]).max() <= 1e-5 * np.abs(o["m_of_x"]).max()
    assert g32["total_mass"] == pytest.approx(o["total_mass"], rel=1e-9)


@pytest.mark.parametrize("storage,eps", [("fp16s", 2.0**-11), ("bf16s", 2.0**-8)])
def test_full_size_one_step_sampled_16bit(clb, oracle_mod, storage, eps):
    nx, ny = C3["nx"], C3["ny"]
    ch = clb.Channel(nx, ny, C3["kn_out"], drive="pressure", drive_value=C3["ratio"], storage=storage)
    ch.step(60)
    f0 = ch.state()
    ch.step(1)
    f1 = ch.state()
    xs, ys = sample_nodes(nx, ny)
    want = oracle_mod.step_nodes(params(oracle_mod), f0, xs, ys)
    got = f1[:, ys, xs].T
    w = oracle_mod.feq(1.0, 0.0, 0.0)
    dev = want - w[None, :] * reference_profile(nx)[xs][:, None]
    # one rounding of the stored output (half an ulp) plus the FP32 collision
    assert np.abs(got - want).max() <= eps * np.abs(dev).max() + 8 * 2.0**-24 * np.abs(dev).max()
