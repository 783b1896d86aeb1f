"""What Sec. 3.2 reports about the steady long channel, on the oracle.

Kept apart from the pin files that the mutation tests run (test_oracle_algebra,
test_oracle_flow, test_oracle_gradient): the test here runs two channels to
steady state, about 20 s of oracle time in all.
"""
import numpy as np


def _steady_pressure_channel(oracle_mod, kn_out, nx=801, ny=8, ratio=2.0, tol=1e-7):
    """The Sec. 3.2 channel (L/H = 100, sigma = 1, centreline Knudsen
    number) stepped in chunks of 1000 until the mean mass flow changes by
    less than `tol` over a chunk."""
    p = oracle_mod.OracleParams(nx=nx, ny=ny, pressure=True, kn=kn_out, rho_in=ratio, rho_out=1.0, kn_mode=1)
    s = oracle_mod.OracleSim(p)
    prev = s.observables()["mass_flow"]
    for _ in range(300):
        s.step(1000, 0)
        m = s.observables()["mass_flow"]
        if abs(m - prev) < tol * abs(m):
            return s
        prev = m
    raise AssertionError(f"no steady state at Kn_out = {kn_out}")


def test_long_channel_observations_of_sec_3_2(oracle_mod):
    """What Sec. 3.2 reports for the long channel at p_in/p_out = 2 (Fig. 4-6),
    on an 801 x 8 channel of the same L/H = 100:
    * the centreline pressure lies above the straight line (delta p > 0);
    * delta p shrinks from Kn_out = 0.194 to Kn_out = 0.388;
    * at Kn_out = 0.194 the wall slip velocity grows along the channel;
    * the spanwise velocity is far smaller than the streamwise one and points
      from the centreline towards each wall as the gas moves downstream."""
    ny = 8
    dp_max = {}
    for kn_out in (0.194, 0.388):
        s = _steady_pressure_channel(oracle_mod, kn_out)
        o = s.observables()
        dp = o["dp_nonlin"]
        assert np.all(dp[1:-1] > 0), kn_out
        dp_max[kn_out] = dp.max()
        if kn_out == 0.194:
            _, ux, uy = s.macro()
            inner = slice(5, ux.shape[1] - 5)
            slip = 0.5 * ((1.5 * ux[0] - 0.5 * ux[1]) + (1.5 * ux[-1] - 0.5 * ux[-2]))
            assert np.all(np.diff(slip[inner]) > 0)
            assert np.abs(uy).max() < 0.01 * ux[:, -1].max()
            assert np.all(uy[: ny // 2, inner] < 0) and np.all(uy[ny // 2 :, inner] > 0)
    assert dp_max[0.388] < dp_max[0.194], dp_max
