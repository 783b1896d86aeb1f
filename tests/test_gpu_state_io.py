"""clb_set_state / clb_get_state with pinned host arrays (read and written by
the conversion kernels directly, walking the FP64 array in its memory order)
and with ordinary pageable arrays (staged through a device buffer, walked row
by row) give the same bits, for every storage and both drives (the periodic
channel also fills its halo columns on the way in), on shapes from one node to
states of several grid strides (each thread of the flat walk then steps more
than once, across row ends, and with nx wider than a stride)."""
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


@pytest.mark.parametrize("storage", ["fp64", "fp32s", "fp16s", "bf16s"])
@pytest.mark.parametrize("drive,value", [("pressure", 1.7), ("body_force", 3e-5)])
@pytest.mark.parametrize("nx,ny", [(777, 13), (4, 1), (4097, 64), (400001, 2)])
def test_pinned_and_pageable_state_io_agree(clb, storage, drive, value, nx, ny):
    import torch

    ch = clb.Channel(nx, ny, 0.2, drive=drive, drive_value=value, storage=storage)
    f0 = inputs.perturb(inputs.rng(nx + ny), ch.state(), 0.05)
    pin_in = torch.empty((9, ny, nx), dtype=torch.float64, pin_memory=True)
    pin_in.numpy()[...] = f0
    pin_out = torch.zeros((9, ny, nx), dtype=torch.float64, pin_memory=True)

    ch.set_state(f0)  # pageable in
    ch.step(7)
    want = ch.state()  # pageable out

    clb.clb_set_state(ch.sim, pin_in.data_ptr())  # pinned in
    ch.step(7)
    clb.clb_get_state(ch.sim, pin_out.data_ptr())  # pinned out
    np.testing.assert_array_equal(pin_out.numpy(), want)
    np.testing.assert_array_equal(ch.state(), want)
    ch.close()
