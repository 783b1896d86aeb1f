"""Degenerate and out-of-range inputs of the entry points: each is refused
with CLB_EINVAL (and the library stays usable), or is a well-defined no-op."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def clb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1603_01955_gb300.clb as clb

    return clb


def test_zero_steps_is_a_no_op(clb):
    ch = clb.Channel(33, 5, 0.2, drive="pressure", drive_value=1.5, storage="fp32s")
    before = ch.state()
    ch.step(0)
    np.testing.assert_array_equal(ch.state(), before)
    assert ch.info()["step"] == 0
    ch.close()


def test_q_of_a_channel_without_force_is_refused(clb):
    """Q = J / (3 G ny^2 sqrt(1/6)) is undefined for G = 0."""
    fg = clb.FlowGradient(2, 4, 0.3, 2.0, 0.8, 0.0, 10, storage="fp64")
    with pytest.raises(clb.CLBError) as err:
        fg.q_norm
    assert err.value.status == clb.CLB_EINVAL
    with pytest.raises(clb.CLBError) as err:
        fg.q_grad()
    assert err.value.status == clb.CLB_EINVAL
    # dJ/d(r, a, G) is defined: with no force the flow stays zero
    J = fg.J
    g = fg.grad()
    fg.close()
    assert J == 0.0
    assert np.isfinite(g).all()


@pytest.mark.parametrize("npt,packed", [(3, 0), (0, 1), (16, 0)])
def test_bad_batch_schedule_is_refused(clb, npt, packed):
    b = clb.Batch([4, 4], [16, 8], [0.1, 1.0], g=1e-6, storage="fp32s", block_x=64)
    before = b.schedule()
    with pytest.raises(clb.CLBError) as err:
        b.set_schedule(npt, packed)
    assert err.value.status == clb.CLB_EINVAL
    assert b.schedule() == before  # the schedule in use is kept
    b.step(3)
    assert b.info()["step"] == 3
    b.close()


def test_batch_schedule_too_wide_is_refused(clb):
    """A block takes at most 512 threads: a 512-node channel fits at one node
    per thread, an 800-node one needs two."""
    b = clb.Batch([4], [128], [0.5], g=1e-6, storage="fp32s")
    b.set_schedule(1, 0)
    assert b.schedule()["threads_per_block"] == 512
    b.close()
    b = clb.Batch([4, 4], [200, 8], [0.5, 0.1], g=1e-6, storage="fp32s")
    with pytest.raises(clb.CLBError) as err:
        b.set_schedule(1, 0)
    assert err.value.status == clb.CLB_EINVAL
    b.set_schedule(2, 1)  # 416 threads for the wide channel; the 32 of the other do not fit beside it
    assert b.schedule() == {"threads_per_block": 416, "nodes_per_thread": 2, "blocks": 2, "packed": 1}
    b.close()


@pytest.mark.parametrize("kw", [dict(nx=0, ny=4), dict(nx=3, ny=0), dict(nx=3, ny=4, kn=0.0),
                                dict(nx=3, ny=4, r=1.5), dict(nx=3, ny=4, drive="pressure", drive_value=2.0)])
def test_bad_channel_is_refused(clb, kw):
    args = dict(nx=3, ny=4, kn=0.2, r=-1.0, drive="body_force", drive_value=1e-5)
    args.update(kw)
    with pytest.raises(clb.CLBError) as err:
        clb.Channel(args.pop("nx"), args.pop("ny"), args.pop("kn"), **args)
    assert err.value.status == clb.CLB_EINVAL
