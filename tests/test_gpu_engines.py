"""The TMA-staged sweep (pipelines 2 to 4, its three tile shapes, tiles
claimed in whatever order the blocks reach them) against the direct-load
sweep (pipeline 1): node for node the same arithmetic, so the states must
agree bit for bit, on random perturbed states, ragged sizes (tiles of 1024
and 512 columns, rows of one node, channels shorter than one tile), odd and
even step counts, both drives and every non-FP64 storage.  The direct sweep
itself is checked against the oracle in test_gpu_parity.py."""
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


SHAPES = [(5, 3, "body_force"), (513, 1, "body_force"), (1030, 7, "body_force"), (4, 2, "pressure"),
          (600, 4, "pressure"), (1601, 16, "pressure")]
PIPELINES = (2, 3, 4)


@pytest.mark.parametrize("storage", ["fp32s", "fp16s", "bf16s"])
@pytest.mark.parametrize("nx,ny,drive", SHAPES)
def test_tma_pipelines_bitwise_equal_direct(clb, oracle_mod, storage, nx, ny, drive):
    value = 1.8 if drive == "pressure" else 2e-4
    ref = clb.Channel(nx, ny, 0.2, drive=drive, drive_value=value, storage=storage, pipeline=1)
    f0 = inputs.perturb(inputs.rng(nx * 7 + ny), ref.state(), 0.05)
    ref.set_state(f0)
    ref.step(57)
    want = ref.state()
    for pipeline in PIPELINES:
        ch = clb.Channel(nx, ny, 0.2, drive=drive, drive_value=value, storage=storage, pipeline=pipeline)
        ch.set_state(f0)
        ch.step(57)
        np.testing.assert_array_equal(ch.state(), want, err_msg=f"pipeline {pipeline}")
        ch.sync()
        ch.close()


def test_tma_full_size_bitwise_equal_direct(clb):
    c = inputs.PRESSURE_25601x256
    states = []
    for pipeline in (1, 2, 0, 3):
        ch = clb.Channel(c["nx"], c["ny"], c["kn_out"], drive="pressure", drive_value=c["ratio"], storage="fp32s",
                         pipeline=pipeline)
        ch.step(25)
        ch.sync()
        states.append(ch.state())
        ch.close()
    for k in range(1, len(states)):
        np.testing.assert_array_equal(states[0], states[k])


@pytest.mark.parametrize("storage", ["fp32s", "bf16s"])
@pytest.mark.parametrize("nx,ny,drive", [(300, 70, "pressure"), (2100, 33, "body_force"), (77, 17, "pressure")])
def test_tma_many_launches(clb, storage, nx, ny, drive):
    """Many consecutive TMA-staged launches taken in uneven chunks (the tile
    order alternates from launch to launch): bit-identical to the direct sweep
    after 400 steps."""
    value = 1.8 if drive == "pressure" else 2e-4
    ref = clb.Channel(nx, ny, 0.2, drive=drive, drive_value=value, storage=storage, pipeline=1)
    f0 = inputs.perturb(inputs.rng(nx + 3 * ny), ref.state(), 0.05)
    ref.set_state(f0)
    ref.step(400)
    for pipeline in PIPELINES:
        ch = clb.Channel(nx, ny, 0.2, drive=drive, drive_value=value, storage=storage, pipeline=pipeline)
        ch.set_state(f0)
        for n in (1, 2, 97, 100, 200):
            ch.step(n)
        ch.sync()
        np.testing.assert_array_equal(ch.state(), ref.state(), err_msg=f"pipeline {pipeline}")
        ch.close()


@pytest.mark.parametrize("storage,kn_mode,want", [("fp64", 0, 1), ("fp32s", 0, 2), ("fp16s", 0, 3),
                                                  ("bf16s", 0, 3), ("fp32s", 1, 1)])
def test_default_engine(clb, storage, kn_mode, want):
    """TMA shapes for channels of 2^20 nodes and more, the direct sweep below."""
    ch = clb.Channel(4097, 256, 0.2, drive="pressure", drive_value=1.5, storage=storage, kn_mode=kn_mode)
    assert ch.info()["pipeline"] == want
    ch.close()
    small = clb.Channel(4095, 256, 0.2, drive="pressure", drive_value=1.5, storage=storage, kn_mode=kn_mode)
    assert small.info()["pipeline"] == 1
    small.close()


@pytest.mark.parametrize("storage,nx,ny,want", [("fp32s", 1601, 16, 1), ("fp32s", 767, 256, 1),
                                                ("fp32s", 769, 256, 4), ("fp64", 1601, 16, 1),
                                                ("fp64", 4097, 256, 1), ("fp16s", 1601, 16, 4)])
def test_default_nodes_per_thread(clb, storage, nx, ny, want):
    """The direct sweep's default nodes per thread: one for FP32 channels below
    196,608 nodes and for FP64, four otherwise."""
    ch = clb.Channel(nx, ny, 0.2, drive="pressure", drive_value=1.5, storage=storage)
    assert ch.info()["vec"] == want
    ch.close()
