"""Out-of-bounds writes and repeatability, without compute-sanitizer: every
device allocation of the library goes through allocator hooks that surround
it with guard zones holding a fixed byte pattern.  After runs of every sweep
engine, storage and drive on ragged sizes, no guard byte may have changed.
The same run repeated gives bit-identical populations."""
import ctypes as C

import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu

GUARD = 4096
PATTERN = 0x5A


@pytest.fixture(scope="module")
def clb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1603_01955_gb300.clb as clb

    return clb


class GuardedAllocator:
    def __init__(self, clb, torch):
        self.torch = torch
        self.live = {}
        self.freed = []

        def _alloc(n, ctx):
            t = torch.full((int(n) + 2 * GUARD,), PATTERN, dtype=torch.uint8, device="cuda")
            torch.cuda.synchronize()
            ptr = t.data_ptr() + GUARD
            self.live[ptr] = (t, int(n))
            return ptr

        def _free(p, ctx):
            self.freed.append(self.live.pop(int(p)))

        self.hooks = (clb.ALLOC_FN(_alloc), clb.FREE_FN(_free))

    def damaged(self):
        self.torch.cuda.synchronize()
        bad = []
        for t, n in list(self.live.values()) + self.freed:
            head, tail = t[:GUARD], t[GUARD + n:]
            if bool((head != PATTERN).any()) or bool((tail != PATTERN).any()):
                bad.append(n)
        return bad


def run(clb, alloc, stream, nx, ny, drive, storage, pipeline, kn_mode, f0, steps):
    o = clb.clb_opts_default()
    o.storage = clb.STORAGE[storage]
    o.pipeline = pipeline
    o.kn_mode = kn_mode
    o.stream = C.c_void_p(stream.cuda_stream)
    o.alloc, o.free = alloc.hooks
    value = 1.7 if drive == "pressure" else 2e-4
    sim = clb.clb_create(nx, ny, 0.2, 2.0, -1.0, clb.DRIVE[drive], value, o)
    clb.clb_set_state(sim, f0.ctypes.data)
    clb.clb_step(sim, steps)
    clb.clb_sync(sim)
    s = clb.clb_scalars()
    clb.clb_observables(sim, -1, s, None, None, None, None, None)
    out = np.empty_like(f0)
    clb.clb_get_state(sim, out.ctypes.data)
    clb.clb_destroy(sim)
    return out


CASES = [
    # (storage, pipelines, kn_mode)
    ("fp64", (1,), 0),
    ("fp32s", (1, 2, 3), 0),
    ("fp16s", (1, 3, 2), 0),
    ("bf16s", (4, 3), 0),
    ("fp32s", (1,), 1),
]


@pytest.mark.parametrize("nx,ny,drive", [(1030, 7, "body_force"), (5, 3, "body_force"), (777, 34, "pressure"),
                                         (4, 2, "pressure")])
@pytest.mark.parametrize("storage,pipelines,kn_mode", CASES)
def test_guard_zones_intact_and_runs_repeat(clb, nx, ny, drive, storage, pipelines, kn_mode):
    import torch

    if kn_mode and drive != "pressure":
        pytest.skip("the centreline Knudsen number belongs to the pressure channel")
    stream = torch.cuda.Stream()
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    f0 = inputs.perturb(inputs.rng(nx + ny), np.broadcast_to(w, (9, ny, nx)).copy(), 0.05)
    for pipeline in pipelines:
        alloc = GuardedAllocator(clb, torch)
        first = run(clb, alloc, stream, nx, ny, drive, storage, pipeline, kn_mode, f0, 33)
        again = run(clb, alloc, stream, nx, ny, drive, storage, pipeline, kn_mode, f0, 33)
        assert alloc.damaged() == [], f"pipeline {pipeline}: guard zone written"
        np.testing.assert_array_equal(first, again, err_msg=f"pipeline {pipeline}")
