"""CUDA-graph replay of clb_step (clb_opts.graph_steps): chunks of sweeps
captured once per buffer parity and replayed give bit for bit the populations
of the same sweeps launched one by one, whatever the chunking of the steps,
for both drives, the centreline Knudsen mode and the sweep engines."""
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


def make(clb, storage, drive, kn_mode, pipeline, graph_steps):
    import ctypes as C

    import torch

    o = clb.clb_opts_default()
    o.storage = clb.STORAGE[storage]
    o.kn_mode = kn_mode
    o.pipeline = pipeline
    o.graph_steps = graph_steps
    stream = torch.cuda.Stream()
    o.stream = C.c_void_p(stream.cuda_stream)
    value = 1.8 if drive == "pressure" else 2e-4
    return clb.clb_create(801, 12, 0.2, 2.0, -1.0, clb.DRIVE[drive], value, o), stream


@pytest.mark.parametrize("storage,drive,kn_mode,pipeline", [("fp32s", "pressure", 0, 0), ("fp32s", "body_force", 0, 1),
                                                          ("fp16s", "pressure", 0, 0), ("fp64", "pressure", 0, 0),
                                                          ("fp32s", "pressure", 1, 0), ("fp16s", "pressure", 0, 3),
                                                          ("fp32s", "body_force", 0, 2)])
def test_replayed_chunks_equal_single_launches(clb, storage, drive, kn_mode, pipeline):
    f0 = None
    states = []
    for graph_steps in (-1, 8, 6):
        sim, stream = make(clb, storage, drive, kn_mode, pipeline, graph_steps)
        if f0 is None:
            f0 = np.empty((9, 12, 801))
            clb.clb_get_state(sim, f0.ctypes.data)
            f0 = inputs.perturb(inputs.rng(5), f0, 0.05)
        clb.clb_set_state(sim, f0.ctypes.data)
        for n in (3, 8, 17, 1, 40, 2):
            clb.clb_step(sim, n)
        clb.clb_sync(sim)
        out = np.empty_like(f0)
        clb.clb_get_state(sim, out.ctypes.data)
        assert clb.clb_info(sim).step == 71
        states.append(out)
        clb.clb_destroy(sim)
    np.testing.assert_array_equal(states[0], states[1])
    np.testing.assert_array_equal(states[0], states[2])
