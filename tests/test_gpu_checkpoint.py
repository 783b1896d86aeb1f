"""Checkpoint and resume (clb_save / clb_load): a channel saved after n1
steps and loaded into a new simulation continues bit for bit like the
original, for every storage, both drives, the centreline Knudsen mode and
every sweep engine (the stored populations and the centreline densities are
saved raw).  Damaged or foreign files are refused with CLB_EIO."""
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


CASES = [
    # (storage, drive, kn_mode, pipeline of the saved run, pipeline of the resumed run)
    ("fp64", "pressure", 0, 0, 0),
    ("fp32s", "pressure", 0, 0, 1),
    ("fp32s", "body_force", 0, 2, 3),
    ("fp16s", "pressure", 0, 0, 0),
    ("bf16s", "body_force", 0, 4, 2),
    ("fp32s", "pressure", 1, 0, 0),
    ("fp64", "pressure", 1, 0, 0),
]


@pytest.mark.parametrize("storage,drive,kn_mode,p_save,p_load", CASES)
def test_resume_is_bit_identical(clb, tmp_path, storage, drive, kn_mode, p_save, p_load):
    nx, ny = 301, 13
    value = 1.9 if drive == "pressure" else 3e-5
    kw = dict(drive=drive, drive_value=value, storage=storage, kn_mode=kn_mode)
    a = clb.Channel(nx, ny, 0.15, pipeline=p_save, **kw)
    a.set_state(inputs.perturb(inputs.rng(17), a.state(), 0.05))
    a.step(37)
    a.observables()  # starts the residual history
    path = tmp_path / "run.ckpt"
    a.save(path)
    a.step(55)
    want = a.state()
    want_obs = a.observables()
    b = clb.Channel.load(path, pipeline=p_load)
    info = b.info()
    assert (info["nx"], info["ny"], info["step"], info["kn_mode"]) == (nx, ny, 37, kn_mode)
    b.step(55)
    np.testing.assert_array_equal(b.state(), want)
    got_obs = b.observables()
    for key in ("mass_flow", "total_mass", "residual", "step"):
        assert got_obs[key] == want_obs[key], key
    a.close()
    b.close()


def test_damaged_files_are_refused(clb, tmp_path):
    ch = clb.Channel(40, 6, 0.2, drive="pressure", drive_value=1.5, storage="fp32s")
    ch.step(3)
    good = tmp_path / "good.ckpt"
    ch.save(good)
    raw = good.read_bytes()
    cases = {
        "truncated": raw[:-100],
        "flipped_payload_byte": raw[:500] + bytes([raw[500] ^ 0x40]) + raw[501:],
        "bad_magic": b"XLBCKPT1" + raw[8:],
        "header_only": raw[:176],
        "empty": b"",
    }
    for name, data in cases.items():
        p = tmp_path / f"{name}.ckpt"
        p.write_bytes(data)
        with pytest.raises(clb.CLBError) as err:
            clb.Channel.load(p)
        assert err.value.status == clb.CLB_EIO, name
    with pytest.raises(clb.CLBError) as err:
        clb.Channel.load(tmp_path / "missing.ckpt")
    assert err.value.status == clb.CLB_EIO
    with pytest.raises(clb.CLBError) as err:
        ch.save(tmp_path / "no_such_dir" / "x.ckpt")
    assert err.value.status == clb.CLB_EIO
    ch.close()
