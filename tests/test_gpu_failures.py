"""Failure detection, exercised without faulting the GPU: a non-finite field
is reported as CLB_ENUMERIC, a refused allocation as CLB_ENOMEM, and an
expired bounded wait in the TMA-staged sweeps (inputs withheld on purpose by
the testing option) as CLB_ETIMEOUT, after which the context still works and
a two-step channel, its counters cleared, runs on correctly."""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def clb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1603_01955_gb300.clb as clb

    return clb


def test_non_finite_field_reported(clb):
    ch = clb.Channel(40, 6, 0.2, drive="pressure", drive_value=1.5, storage="fp32s")
    f = ch.state()
    f[3, 2, 17] = np.nan
    ch.set_state(f)
    ch.step(5)
    o = ch.observables(check=False)
    assert o["status"] == clb.CLB_ENUMERIC
    assert b"non-finite" in clb.lib.clb_last_error()


def test_refused_allocation_reported(clb):
    with pytest.raises(clb.CLBError) as err:
        clb.Channel(4000, 64, 0.1, drive="pressure", drive_value=2.0, storage="fp32s",
                    alloc_hook=lambda nbytes: nbytes < (1 << 20))
    assert err.value.status == clb.CLB_ENOMEM


def test_expired_wait_reported_and_context_survives(clb, oracle_mod):
    ch = clb.Channel(3000, 12, 0.1, drive="pressure", drive_value=2.0, storage="fp32s", pipeline=2,
                     test_withhold_tile=3)
    ch.step(1)
    with pytest.raises(clb.CLBError) as err:
        ch.sync()
    assert err.value.status == clb.CLB_ETIMEOUT
    ch.close()
    # the context is still usable: a normal run matches the oracle
    ok = clb.Channel(60, 5, 0.2, drive="pressure", drive_value=1.5, storage="fp64", pipeline=1)
    orc = oracle_mod.OracleSim(oracle_mod.OracleParams(nx=60, ny=5, pressure=True, kn=0.2, rho_in=1.5))
    f0 = inputs.perturb(inputs.rng(9), orc.state(), 0.05)
    ok.set_state(f0)
    orc.set_state(f0)
    ok.step(50)
    orc.step(50)
    want = orc.state()
    assert (np.abs(ok.state() - want) / np.abs(want)).max() <= 1e-12
    ok.sync()
