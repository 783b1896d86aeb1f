"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle
on the same seeded inputs.

Tolerances:
* FP64 storage: 1e-12 relative per population after 1000 steps (the target
  stated for the plain FP64 path); both sides evaluate the same formulas in
  FP64 in different orders, so only round-off separates them.
* FP32-shifted storage: the stored values are deviations d = f - w_i R(x) from
  the reference density R (the linear initial profile of a pressure channel,
  rho_out otherwise).  Each step rounds them once on store and the collision
  adds a few FP32 roundings on quantities no larger than max|d|; over n steps
  of a non-amplifying update these add up like a random walk, so the bound is
  c * 2^-24 * sqrt(n) * max|d| per population with c = 4 (observed c ~ 2),
  and the mass flow within 1e-5 relative (the target stated for this path).
"""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def tol32(n):
    return 4 * 2.0**-24 * np.sqrt(max(n, 1))


def rho_bound(n, scale):
    """Largest density error of a node implied by the per-population bound
    (a density is the sum of nine populations)."""
    return 9 * tol32(n) * scale


@pytest.fixture(scope="module")
def clb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1603_01955_gb300.clb as clb

    return clb


def oracle_params(oracle_mod, nx, ny, kn, drive, value, r=-1.0, a=2.0, sigma=1.0, rho_out=1.0):
    if drive == "pressure":
        return oracle_mod.OracleParams(nx=nx, ny=ny, pressure=True, kn=kn, a=a, sigma=sigma,
                                       r=None if r < 0 else r, rho_in=value * rho_out, rho_out=rho_out)
    return oracle_mod.OracleParams(nx=nx, ny=ny, kn=kn, a=a, sigma=sigma, r=None if r < 0 else r,
                                   gx=value, rho_out=rho_out)


def pair(clb, oracle_mod, nx, ny, kn, drive, value, storage="fp64", r=-1.0, **launch):
    ch = clb.Channel(nx, ny, kn, r=r, drive=drive, drive_value=value, storage=storage, **launch)
    orc = oracle_mod.OracleSim(oracle_params(oracle_mod, nx, ny, kn, drive, value, r=r))
    return ch, orc


def rel_err(got, want):
    return np.abs(got - want).max() / np.abs(want).max()


def per_pop_rel(got, want):
    return (np.abs(got - want) / np.abs(want)).max()


def dev_scale(orc_state, oracle_mod, drive, ratio=1.0):
    """max |f - w_i R(x)| of an oracle state: the size of the FP32-stored
    deviations (R linear from ratio to 1 in a pressure channel, 1 otherwise)."""
    nx = orc_state.shape[2]
    w = oracle_mod.feq(1.0, 0.0, 0.0)[:, None, None]
    if drive == "pressure":
        R = ratio + (1.0 - ratio) * np.arange(nx) / (nx - 1)
    else:
        R = np.ones(nx)
    return np.abs(orc_state - w * R[None, None, :]).max() + 1e-30


# ------------------------------------------------------------- FP64 parity

def test_fp64_initial_state_matches(clb, oracle_mod):
    ch, orc = pair(clb, oracle_mod, 37, 9, 0.2, "pressure", 2.0)
    assert per_pop_rel(ch.state(), orc.state()) <= 1e-15


def test_fp64_periodic_channel_4x32_1000_steps(clb, oracle_mod):
    c = inputs.PERIODIC_4x32
    ch, orc = pair(clb, oracle_mod, c["nx"], c["ny"], c["kn"], "body_force", c["gx"])
    ch.step(1000)
    orc.step(1000)
    assert per_pop_rel(ch.state(), orc.state()) <= TOL64


@pytest.mark.parametrize("kn_out", inputs.PRESSURE_1601x16["kn_out"])
def test_fp64_pressure_channel_1601x16_1000_steps(clb, oracle_mod, kn_out):
    c = inputs.PRESSURE_1601x16
    ch, orc = pair(clb, oracle_mod, c["nx"], c["ny"], kn_out, "pressure", c["ratio"])
    ch.step(1000)
    orc.step(1000)
    assert per_pop_rel(ch.state(), orc.state()) <= TOL64


def test_fp64_pressure_channel_64x8_1000_steps(clb, oracle_mod):
    ch, orc = pair(clb, oracle_mod, 64, 8, 0.1, "pressure", 2.0)
    ch.step(1000)
    orc.step(1000)
    assert per_pop_rel(ch.state(), orc.state()) <= TOL64


@pytest.mark.parametrize("seed", inputs.SEEDS)
def test_fp64_random_states(clb, oracle_mod, seed):
    """Seeded perturbations (+-20 %) of the equilibrium exercise every term of
    the collision, the force included, and both drives."""
    r = inputs.rng(seed)
    drive = "pressure" if seed % 2 else "body_force"
    nx, ny = int(r.integers(5, 70)), int(r.integers(2, 12))
    kn = float(10 ** r.uniform(-2, 0.5))
    value = float(r.uniform(1.2, 2.5)) if drive == "pressure" else float(r.uniform(-1e-3, 1e-3))
    rb = float(r.uniform(0.3, 1.0))
    ch, orc = pair(clb, oracle_mod, nx, ny, kn, drive, value, r=rb)
    f0 = inputs.perturb(r, orc.state(), 0.2)
    ch.set_state(f0)
    orc.set_state(f0)
    ch.step(200)
    orc.step(200)
    assert per_pop_rel(ch.state(), orc.state()) <= TOL64


EDGE = [
    # (nx, ny, drive, vec, block_x)
    (1, 4, "body_force", 2, 32), (2, 1, "body_force", 1, 32), (3, 2, "body_force", 2, 64),
    (5, 3, "body_force", 1, 128), (33, 5, "body_force", 2, 32), (127, 4, "body_force", 2, 256),
    (129, 2, "body_force", 1, 32), (4, 3, "pressure", 2, 32), (5, 1, "pressure", 1, 32),
    (7, 2, "pressure", 2, 64), (131, 5, "pressure", 2, 32), (65, 6, "pressure", 1, 96),
]


@pytest.mark.parametrize("nx,ny,drive,vec,block_x", EDGE)
def test_fp64_edge_sizes_and_launch_shapes(clb, oracle_mod, nx, ny, drive, vec, block_x):
    value = 1.7 if drive == "pressure" else 3e-4
    ch, orc = pair(clb, oracle_mod, nx, ny, 0.3, drive, value, vec=vec, block_x=block_x)
    r = inputs.rng(nx * 100 + ny)
    f0 = inputs.perturb(r, orc.state(), 0.1)
    ch.set_state(f0)
    orc.set_state(f0)
    ch.step(150)
    orc.step(150)
    assert per_pop_rel(ch.state(), orc.state()) <= TOL64


def test_zero_steps_and_state_roundtrip(clb, oracle_mod):
    ch, orc = pair(clb, oracle_mod, 10, 4, 0.1, "body_force", 1e-4)
    f = inputs.perturb(inputs.rng(3), orc.state(), 0.1)
    ch.set_state(f)
    ch.step(0)
    np.testing.assert_array_equal(ch.state(), f)


def test_fp64_observables_match(clb, oracle_mod):
    for drive, value, nx, ny in (("pressure", 2.0, 160, 10), ("body_force", 1e-5, 6, 11)):
        ch, orc = pair(clb, oracle_mod, nx, ny, 0.15, drive, value)
        ch.step(700)
        orc.step(700)
        for col in (-1, 0, nx // 3):
            g = ch.observables(col)
            o = orc.observables(col)
            # absolute floors on each quantity's physical scale: u_y and the
            # pressure deviation are identically zero in the periodic channel
            vel = np.abs(o["ux_prof"]).max()
            floors = dict(ux_prof=vel, uy_prof=vel, p_centre=1.0, dp_nonlin=1.0, m_of_x=np.abs(o["m_of_x"]).max())
            for key, scale in floors.items():
                np.testing.assert_allclose(g[key], o[key], rtol=1e-10, atol=1e-12 * scale, err_msg=key)
            for key in ("mass_flow", "q_norm", "u_slip", "total_mass", "ux_max"):
                assert g[key] == pytest.approx(o[key], rel=1e-10, abs=1e-18), key
        assert g["step"] == 700


def test_residual_tracks_mass_flow(clb):
    ch = clb.Channel(4, 16, 0.1, drive="body_force", drive_value=1e-6, storage="fp64")
    assert ch.observables()["residual"] == -1.0
    ch.step(500)
    r1 = ch.observables()["residual"]
    ch.step(5000)
    r2 = ch.observables()["residual"]
    assert r1 > 0 and r2 < r1


# ------------------------------------------------------------- FP32 parity

def test_fp32_periodic_channel_4x32_1000_steps(clb, oracle_mod):
    c = inputs.PERIODIC_4x32
    ch, orc = pair(clb, oracle_mod, c["nx"], c["ny"], c["kn"], "body_force", c["gx"], storage="fp32s")
    ch.step(1000)
    orc.step(1000)
    so = orc.state()
    assert np.abs(ch.state() - so).max() <= tol32(1000) * dev_scale(so, oracle_mod, "body_force")
    assert ch.observables()["mass_flow"] == pytest.approx(orc.observables()["mass_flow"], rel=1e-5)


@pytest.mark.parametrize("kn_out", inputs.PRESSURE_1601x16["kn_out"])
def test_fp32_pressure_channel_1601x16_1000_steps(clb, oracle_mod, kn_out):
    c = inputs.PRESSURE_1601x16
    ch, orc = pair(clb, oracle_mod, c["nx"], c["ny"], kn_out, "pressure", c["ratio"], storage="fp32s")
    ch.step(1000)
    orc.step(1000)
    so = orc.state()
    g, o = ch.observables(), orc.observables()
    scale = dev_scale(so, oracle_mod, "pressure", c["ratio"])
    assert np.abs(ch.state() - so).max() <= tol32(1000) * scale
    assert g["mass_flow"] == pytest.approx(o["mass_flow"], rel=1e-5)
    # dp = (rho_c/3 - p_l)/p_out with p_out = 1/3: its error is the density error
    assert np.abs(g["dp_nonlin"] - o["dp_nonlin"]).max() <= rho_bound(1000, scale)


@pytest.mark.parametrize("nx,ny,drive,vec,block_x", EDGE)
def test_fp32_edge_sizes_and_launch_shapes(clb, oracle_mod, nx, ny, drive, vec, block_x):
    value = 1.7 if drive == "pressure" else 3e-4
    # the direct-load sweep at the given launch shapes, then the default engine
    launches = [dict(vec=v, block_x=block_x, pipeline=1) for v in sorted({vec, 4})] + [{}]
    for launch in launches:
        ch, orc = pair(clb, oracle_mod, nx, ny, 0.3, drive, value, storage="fp32s", **launch)
        r = inputs.rng(nx * 100 + ny)
        f0 = inputs.perturb(r, orc.state(), 0.1)
        ch.set_state(f0)
        orc.set_state(f0)
        ch.step(150)
        orc.step(150)
        so = orc.state()
        assert np.abs(ch.state() - so).max() <= tol32(150) * dev_scale(so, oracle_mod, drive, value)


@pytest.mark.parametrize("seed", inputs.SEEDS[:3])
def test_fp32_random_states(clb, oracle_mod, seed):
    r = inputs.rng(seed)
    drive = "pressure" if seed % 2 else "body_force"
    nx, ny = int(r.integers(5, 70)), int(r.integers(2, 12))
    kn = float(10 ** r.uniform(-2, 0.5))
    value = float(r.uniform(1.2, 2.5)) if drive == "pressure" else float(r.uniform(-1e-3, 1e-3))
    ch, orc = pair(clb, oracle_mod, nx, ny, kn, drive, value, storage="fp32s")
    f0 = inputs.perturb(r, orc.state(), 0.2)
    ch.set_state(f0)
    orc.set_state(f0)
    ch.step(200)
    orc.step(200)
    so = orc.state()
    scale = dev_scale(so, oracle_mod, drive, value)
    assert np.abs(ch.state() - so).max() <= tol32(200) * scale
    nodes = nx * ny
    assert abs(ch.observables()["total_mass"] - orc.observables()["total_mass"]) <= nodes * rho_bound(200, scale)


# ------------------------------------------------------------ 16-bit parity
#
# FP16 (x 2^14) and BF16 store the deviations with unit round-off 2^-11 and
# 2^-8; the collision runs in FP32.  Same error model as FP32 with that
# round-off: c * eps * sqrt(n) * max|d| per population, c = 4; the mass flow
# (a sum of six populations per node) within 6x that per node.

EPS16 = {"fp16s": 2.0**-11, "bf16s": 2.0**-8}


def tol16(storage, n):
    return 4 * EPS16[storage] * np.sqrt(max(n, 1))


@pytest.mark.parametrize("storage", ["fp16s", "bf16s"])
@pytest.mark.parametrize("kn_out", [0.0194, 0.2])
def test_16bit_pressure_channel_1601x16_1000_steps(clb, oracle_mod, storage, kn_out):
    c = inputs.PRESSURE_1601x16
    ch, orc = pair(clb, oracle_mod, c["nx"], c["ny"], kn_out, "pressure", c["ratio"], storage=storage)
    ch.step(1000)
    orc.step(1000)
    so = orc.state()
    scale = dev_scale(so, oracle_mod, "pressure", c["ratio"])
    err = np.abs(ch.state() - so).max()
    assert err <= tol16(storage, 1000) * scale
    g, o = ch.observables(), orc.observables()
    assert abs(g["mass_flow"] - o["mass_flow"]) <= 6 * c["ny"] * tol16(storage, 1000) * scale


@pytest.mark.parametrize("storage", ["fp16s", "bf16s"])
@pytest.mark.parametrize("nx,ny,drive,vec", [(5, 3, "body_force", 4), (37, 4, "body_force", 8),
                                             (4, 2, "pressure", 4), (131, 5, "pressure", 8)])
def test_16bit_edge_sizes(clb, oracle_mod, storage, nx, ny, drive, vec):
    value = 1.7 if drive == "pressure" else 3e-4
    for launch in (dict(vec=vec, block_x=32, pipeline=1), {}):
        ch, orc = pair(clb, oracle_mod, nx, ny, 0.3, drive, value, storage=storage, **launch)
        f0 = inputs.perturb(inputs.rng(nx + ny), orc.state(), 0.1)
        ch.set_state(f0)
        orc.set_state(f0)
        ch.step(100)
        orc.step(100)
        so = orc.state()
        # the initial state itself is rounded to 16 bits: one more rounding step
        assert np.abs(ch.state() - so).max() <= tol16(storage, 101) * dev_scale(so, oracle_mod, drive, value)


# ------------------------------------------- centreline Knudsen number (Sec. 3.2)

def centre_pair(clb, oracle_mod, nx, ny, kn, value, storage):
    ch = clb.Channel(nx, ny, kn, drive="pressure", drive_value=value, storage=storage, kn_mode=1)
    orc = oracle_mod.OracleSim(oracle_mod.OracleParams(nx=nx, ny=ny, pressure=True, kn=kn, rho_in=value,
                                                       kn_mode=1))
    return ch, orc


@pytest.mark.parametrize("kn_out", [0.0194, 0.2])
def test_fp64_centreline_kn_1601x16_1000_steps(clb, oracle_mod, kn_out):
    ch, orc = centre_pair(clb, oracle_mod, 1601, 16, kn_out, 2.0, "fp64")
    ch.step(1000)
    orc.step(1000)
    assert per_pop_rel(ch.state(), orc.state()) <= TOL64


@pytest.mark.parametrize("nx,ny,storage", [(37, 5, "fp64"), (130, 6, "fp64"), (37, 5, "fp32s"), (130, 6, "fp32s")])
def test_centreline_kn_random_states(clb, oracle_mod, nx, ny, storage):
    ch, orc = centre_pair(clb, oracle_mod, nx, ny, 0.15, 1.6, storage)
    f0 = inputs.perturb(inputs.rng(nx + ny), orc.state(), 0.1)
    ch.set_state(f0)
    orc.set_state(f0)
    ch.step(300)
    orc.step(300)
    so = orc.state()
    if storage == "fp64":
        assert per_pop_rel(ch.state(), so) <= TOL64
    else:
        assert np.abs(ch.state() - so).max() <= tol32(300) * dev_scale(so, oracle_mod, "pressure", 1.6)
