"""Python binding of the C ABI in ``include/clb.h`` (ctypes; marshalling only).

The functions ``clb_create``, ``clb_step``, ``clb_observables``,
``clb_get_state``, ``clb_set_state``, ``clb_info``, ``clb_sync`` and
``clb_destroy`` have the names and arguments of the C entry points; every step
of the computation runs in the CUDA library.  ``Channel`` wraps one simulation
with PyTorch supplying the device memory (its caching allocator) and the stream
(the current stream of the device).

There is no fallback: if ``libclb_gb300.so`` is missing or cannot be loaded,
importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

CLB_OK, CLB_EINVAL, CLB_ENOMEM, CLB_ECUDA, CLB_ENUMERIC, CLB_ETIMEOUT, CLB_EIO = range(7)
CLB_DRIVE_BODY_FORCE, CLB_DRIVE_PRESSURE = 0, 1
CLB_FP64, CLB_FP32_SHIFTED, CLB_FP16_SCALED, CLB_BF16_SCALED = 0, 1, 2, 3

STORAGE = {"fp64": CLB_FP64, "fp32s": CLB_FP32_SHIFTED, "fp16s": CLB_FP16_SCALED, "bf16s": CLB_BF16_SCALED}
DRIVE = {"body_force": CLB_DRIVE_BODY_FORCE, "pressure": CLB_DRIVE_PRESSURE}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class clb_opts(C.Structure):
    _fields_ = [
        ("b2", C.c_double), ("sigma", C.c_double), ("s3", C.c_double), ("s8", C.c_double),
        ("rho_out", C.c_double), ("storage", C.c_int), ("vec", C.c_int), ("block_x", C.c_int),
        ("stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", C.c_void_p),
        ("pipeline", C.c_int), ("kn_mode", C.c_int), ("test_withhold_tile", C.c_int), ("graph_steps", C.c_int),
    ]


class clb_scalars(C.Structure):
    _fields_ = [
        ("mass_flow", C.c_double), ("q_norm", C.c_double), ("u_slip", C.c_double),
        ("residual", C.c_double), ("total_mass", C.c_double), ("ux_max", C.c_double),
        ("step", C.c_int64),
    ]


class clb_info_t(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("pitch", C.c_int), ("storage", C.c_int),
        ("vec", C.c_int), ("block_x", C.c_int), ("drive", C.c_int),
        ("bytes_per_node", C.c_double), ("sv", C.c_double), ("sq", C.c_double), ("r", C.c_double),
        ("kn", C.c_double), ("a", C.c_double), ("g", C.c_double), ("rho_in", C.c_double),
        ("rho_out", C.c_double), ("step", C.c_int64), ("stream", C.c_void_p),
        ("pipeline", C.c_int), ("kn_mode", C.c_int),
    ]


class CLBError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"clb status {status}: {msg}")
        self.status = status


def _load():
    path = _build.LIB
    if _build.stale():
        # compile in place when nvcc is at hand; otherwise fail loudly below
        try:
            _build.build_library()
        except Exception as e:  # noqa: BLE001
            raise ImportError(f"CUDA library {path} is missing or stale and could not be built: {e}") from e
    if not os.path.exists(path):
        raise ImportError(f"CUDA library {path} not found; run __graft_entry__.build()")
    lib = C.CDLL(path)
    P = C.c_void_p
    D = C.POINTER(C.c_double)
    lib.clb_opts_default.argtypes = [C.POINTER(clb_opts)]
    lib.clb_opts_default.restype = None
    lib.clb_create.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_int, C.c_double,
                               C.POINTER(clb_opts), C.POINTER(P)]
    lib.clb_step.argtypes = [P, C.c_int64]
    lib.clb_observables.argtypes = [P, C.c_int, C.POINTER(clb_scalars), D, D, D, D, D]
    lib.clb_get_state.argtypes = [P, P]
    lib.clb_set_state.argtypes = [P, P]
    lib.clb_info.argtypes = [P, C.POINTER(clb_info_t)]
    lib.clb_sync.argtypes = [P]
    lib.clb_destroy.argtypes = [P]
    lib.clb_last_error.argtypes = []
    lib.clb_last_error.restype = C.c_char_p
    lib.clb_save.argtypes = [P, C.c_char_p]
    lib.clb_load.argtypes = [C.c_char_p, C.POINTER(clb_opts), C.POINTER(P)]
    lib.clb_observables_noalloc.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                            C.c_double, C.c_int, P, C.POINTER(clb_scalars), D, D, D, D, D]
    I = C.POINTER(C.c_int)
    lib.clb_batch_create.argtypes = [C.c_int, I, I, D, C.c_double, C.c_double, C.c_double, C.POINTER(clb_opts),
                                     C.POINTER(P)]
    lib.clb_batch_step.argtypes = [P, C.c_int64]
    lib.clb_batch_tune.argtypes = [P, I]
    lib.clb_batch_set_schedule.argtypes = [P, C.c_int, C.c_int]
    lib.clb_batch_schedule.argtypes = [P, I, I, I, I]
    lib.clb_batch_observables.argtypes = [P, C.POINTER(clb_scalars)]
    lib.clb_batch_get_state.argtypes = [P, C.c_int, P]
    lib.clb_batch_set_state.argtypes = [P, C.c_int, P]
    lib.clb_batch_info.argtypes = [P, I, C.POINTER(C.c_int64), C.POINTER(P)]
    lib.clb_batch_destroy.argtypes = [P]
    lib.clb_adjoint_forward.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                        C.c_int64, C.c_int, C.POINTER(clb_opts), C.POINTER(P), D]
    lib.clb_adjoint_backward.argtypes = [P, C.c_double, D]
    lib.clb_adjoint_q.argtypes = [P, D]
    lib.clb_adjoint_q_backward.argtypes = [P, C.c_double, D]
    lib.clb_adjoint_destroy.argtypes = [P]
    lib.clb_peak_fma.argtypes = [C.c_int, P, D]
    for name in ("clb_create", "clb_step", "clb_observables", "clb_get_state", "clb_set_state",
                 "clb_info", "clb_sync", "clb_destroy", "clb_save", "clb_load", "clb_observables_noalloc",
                 "clb_batch_create",
                 "clb_batch_step", "clb_batch_tune", "clb_batch_set_schedule", "clb_batch_schedule",
                 "clb_batch_observables", "clb_batch_get_state",
                 "clb_batch_set_state", "clb_batch_info", "clb_batch_destroy", "clb_adjoint_forward",
                 "clb_adjoint_backward", "clb_adjoint_q", "clb_adjoint_q_backward", "clb_adjoint_destroy",
                 "clb_peak_fma"):
        getattr(lib, name).restype = C.c_int
    return lib


lib = _load()
LIB_PATH = _build.LIB


def _check(st):
    if st != CLB_OK:
        raise CLBError(st, lib.clb_last_error().decode(errors="replace"))
    return st


def _dptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


# ------------------------------------------------------------ C-ABI mirror

def clb_opts_default() -> clb_opts:
    o = clb_opts()
    lib.clb_opts_default(C.byref(o))
    return o


def clb_create(nx, ny, kn, a, r, drive, drive_value, opts: clb_opts | None = None):
    h = C.c_void_p()
    _check(lib.clb_create(int(nx), int(ny), float(kn), float(a), float(r), int(drive), float(drive_value),
                          C.byref(opts) if opts is not None else None, C.byref(h)))
    return h


def clb_step(sim, n):
    return _check(lib.clb_step(sim, int(n)))


def clb_observables(sim, profile_col, s, ux_prof, uy_prof, p_centre, dp_nonlin, m_of_x, check=True):
    st = lib.clb_observables(sim, int(profile_col), C.byref(s) if s is not None else None, _dptr(ux_prof),
                             _dptr(uy_prof), _dptr(p_centre), _dptr(dp_nonlin), _dptr(m_of_x))
    return _check(st) if check else st


def clb_observables_noalloc(f_dev_ptr, nx, ny, drive, g, rho_in, rho_out, kn, profile_col, stream_ptr, s,
                            ux_prof, uy_prof, p_centre, dp_nonlin, m_of_x, check=True):
    """Observables of a caller-owned FP64 device array [9][ny][nx]; allocates nothing."""
    st = lib.clb_observables_noalloc(C.c_void_p(f_dev_ptr), int(nx), int(ny), int(drive), float(g), float(rho_in),
                                     float(rho_out), float(kn), int(profile_col), C.c_void_p(stream_ptr),
                                     C.byref(s) if s is not None else None, _dptr(ux_prof), _dptr(uy_prof),
                                     _dptr(p_centre), _dptr(dp_nonlin), _dptr(m_of_x))
    return _check(st) if check else st


def clb_peak_fma(storage, stream_ptr=None) -> float:
    """Measured fused multiply-add throughput (TFLOP/s) in FP32 (CLB_FP32_SHIFTED) or FP64."""
    out = C.c_double()
    _check(lib.clb_peak_fma(int(storage), C.c_void_p(stream_ptr) if stream_ptr else None, C.byref(out)))
    return out.value


def clb_get_state(sim, host_ptr):
    return _check(lib.clb_get_state(sim, C.c_void_p(host_ptr)))


def clb_set_state(sim, host_ptr):
    return _check(lib.clb_set_state(sim, C.c_void_p(host_ptr)))


def clb_info(sim) -> clb_info_t:
    i = clb_info_t()
    _check(lib.clb_info(sim, C.byref(i)))
    return i


def clb_sync(sim):
    return _check(lib.clb_sync(sim))


def clb_destroy(sim):
    return _check(lib.clb_destroy(sim))


def clb_save(sim, path):
    return _check(lib.clb_save(sim, os.fsencode(path)))


def clb_load(path, opts: clb_opts | None = None):
    h = C.c_void_p()
    _check(lib.clb_load(os.fsencode(path), C.byref(opts) if opts is not None else None, C.byref(h)))
    return h


# ------------------------------------------------------------ convenience

class Channel:
    """One channel on the current CUDA device.

    drive='body_force': periodic in x, ``drive_value`` = G (lattice acceleration).
    drive='pressure': inlet/outlet, ``drive_value`` = p_in/p_out, ``kn`` = Kn_out.
    ``r`` < 0 takes r_b from Eq. 21 with ``sigma``.
    All work runs on ``self.stream`` (the given non-default torch stream, or a
    new one); time it with events recorded on that stream.
    """

    def __init__(self, nx, ny, kn, a=2.0, r=-1.0, drive="body_force", drive_value=0.0, storage="fp32s",
                 vec=0, block_x=0, b2=0.55, sigma=1.0, s3=1.1, s8=1.2, rho_out=1.0, stream=None,
                 torch_allocator=True, pipeline=0, kn_mode=0, test_withhold_tile=-1, alloc_hook=None, graph_steps=0):
        import torch

        self.nx, self.ny = int(nx), int(ny)
        o = self._runtime_opts(stream, vec, block_x, pipeline, torch_allocator, alloc_hook, graph_steps)
        o.b2, o.sigma, o.s3, o.s8, o.rho_out = b2, sigma, s3, s8, rho_out
        o.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        o.kn_mode = int(kn_mode)
        o.test_withhold_tile = int(test_withhold_tile)
        d = DRIVE[drive] if isinstance(drive, str) else int(drive)
        self.sim = clb_create(nx, ny, kn, a, r, d, drive_value, o)

    def _runtime_opts(self, stream, vec, block_x, pipeline, torch_allocator, alloc_hook, graph_steps=0) -> clb_opts:
        """Options that do not define the problem: stream, engine, allocator, graph replay."""
        import torch

        dev = torch.cuda.current_device()
        # a stream of its own by default; the legacy default stream (handle 0)
        # cannot be handed over, because NULL asks the library for its own stream
        if stream is None or stream.cuda_stream == 0:
            stream = torch.cuda.Stream(dev)
        self._stream = stream
        o = clb_opts_default()
        o.vec, o.block_x = int(vec), int(block_x)
        o.pipeline = int(pipeline)
        o.graph_steps = int(graph_steps)
        o.stream = C.c_void_p(self._stream.cuda_stream)
        if torch_allocator:
            s = self._stream

            def _alloc(n, ctx):
                if alloc_hook is not None and not alloc_hook(int(n)):
                    return None  # the caller's hook refuses this allocation
                try:
                    return torch.cuda.caching_allocator_alloc(int(n), dev, s)
                except Exception:  # noqa: BLE001 - reported to the library as NULL
                    return None

            def _free(p, ctx):
                torch.cuda.caching_allocator_delete(int(p))

            self._hooks = (ALLOC_FN(_alloc), FREE_FN(_free))
            o.alloc, o.free = self._hooks
        return o

    def save(self, path) -> None:
        """Checkpoint the channel to a file (clb_save)."""
        clb_save(self.sim, path)

    @classmethod
    def load(cls, path, stream=None, vec=0, block_x=0, pipeline=0, torch_allocator=True, alloc_hook=None,
             graph_steps=0):
        """A channel resumed from a checkpoint file (clb_load); the problem
        comes from the file, the engine and stream from the arguments."""
        ch = cls.__new__(cls)
        o = ch._runtime_opts(stream, vec, block_x, pipeline, torch_allocator, alloc_hook, graph_steps)
        ch.sim = clb_load(path, o)
        i = clb_info(ch.sim)
        ch.nx, ch.ny = i.nx, i.ny
        return ch

    def close(self):
        if getattr(self, "sim", None):
            clb_destroy(self.sim)
            self.sim = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def stream(self):
        return self._stream

    def step(self, n=1):
        clb_step(self.sim, n)

    def sync(self):
        clb_sync(self.sim)

    def info(self) -> dict:
        i = clb_info(self.sim)
        return {k: getattr(i, k) for k, _ in clb_info_t._fields_ if k != "stream"}

    def state(self) -> np.ndarray:
        f = np.empty((9, self.ny, self.nx), np.float64)
        clb_get_state(self.sim, f.ctypes.data)
        return f

    def set_state(self, f) -> None:
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(9, self.ny, self.nx)
        clb_set_state(self.sim, f.ctypes.data)

    def observables(self, profile_col=-1, check=True) -> dict:
        s = clb_scalars()
        # the library writes every element of every output (np.empty: no page-zeroing pass)
        ux = np.empty(self.ny)
        uy = np.empty(self.ny)
        pc = np.empty(self.nx)
        dp = np.empty(self.nx)
        mx = np.empty(self.nx)
        st = clb_observables(self.sim, profile_col, s, ux, uy, pc, dp, mx, check=check)
        out = {k: getattr(s, k) for k, _ in clb_scalars._fields_}
        out.update(ux_prof=ux, uy_prof=uy, p_centre=pc, dp_nonlin=dp, m_of_x=mx, status=st)
        return out


# ------------------------------------------------------------ batched sweep

def clb_batch_create(nx, ny, kn, a, r, g, opts: clb_opts | None = None):
    n = len(kn)
    ax = (C.c_int * n)(*[int(v) for v in nx])
    ay = (C.c_int * n)(*[int(v) for v in ny])
    ak = (C.c_double * n)(*[float(v) for v in kn])
    h = C.c_void_p()
    _check(lib.clb_batch_create(n, ax, ay, ak, float(a), float(r), float(g),
                                C.byref(opts) if opts is not None else None, C.byref(h)))
    return h


def clb_batch_step(b, n):
    return _check(lib.clb_batch_step(b, int(n)))


def clb_batch_tune(b):
    blk = C.c_int()
    _check(lib.clb_batch_tune(b, C.byref(blk)))
    return blk.value


def clb_batch_set_schedule(b, nodes_per_thread, packed):
    return _check(lib.clb_batch_set_schedule(b, int(nodes_per_thread), int(packed)))


def clb_batch_schedule(b):
    v = [C.c_int() for _ in range(4)]
    _check(lib.clb_batch_schedule(b, *[C.byref(x) for x in v]))
    return dict(zip(("threads_per_block", "nodes_per_thread", "blocks", "packed"), (x.value for x in v)))


def clb_batch_observables(b, n):
    s = (clb_scalars * n)()
    _check(lib.clb_batch_observables(b, s))
    return s


def clb_batch_get_state(b, k, host_ptr):
    return _check(lib.clb_batch_get_state(b, int(k), C.c_void_p(host_ptr)))


def clb_batch_set_state(b, k, host_ptr):
    return _check(lib.clb_batch_set_state(b, int(k), C.c_void_p(host_ptr)))


def clb_batch_info(b):
    blk = C.c_int()
    step = C.c_int64()
    st = C.c_void_p()
    _check(lib.clb_batch_info(b, C.byref(blk), C.byref(step), C.byref(st)))
    return blk.value, step.value, st.value


def clb_batch_destroy(b):
    return _check(lib.clb_batch_destroy(b))


class Batch:
    """Many periodic body-force channels (the Knudsen sweep of Sec. 3.1) in one
    persistent launch per chunk of steps, on its own torch stream."""

    def __init__(self, nx, ny, kn, a=2.0, r=-1.0, g=1e-6, storage="fp32s", block_x=0, b2=0.55, sigma=1.0,
                 s3=1.1, s8=1.2, rho_out=1.0, stream=None, torch_allocator=True):
        import torch

        self.nx, self.ny, self.kn = list(nx), list(ny), list(kn)
        self.n = len(self.kn)
        dev = torch.cuda.current_device()
        if stream is None or stream.cuda_stream == 0:
            stream = torch.cuda.Stream(dev)
        self._stream = stream
        o = clb_opts_default()
        o.b2, o.sigma, o.s3, o.s8, o.rho_out = b2, sigma, s3, s8, rho_out
        o.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        o.block_x = int(block_x)
        o.stream = C.c_void_p(stream.cuda_stream)
        if torch_allocator:
            def _alloc(nbytes, ctx):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)
                except Exception:  # noqa: BLE001 - reported to the library as NULL
                    return None

            def _free(p, ctx):
                torch.cuda.caching_allocator_delete(int(p))

            self._hooks = (ALLOC_FN(_alloc), FREE_FN(_free))
            o.alloc, o.free = self._hooks
        self.b = clb_batch_create(self.nx, self.ny, self.kn, a, r, g, o)

    @property
    def stream(self):
        return self._stream

    def close(self):
        if getattr(self, "b", None):
            clb_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def step(self, n=1):
        clb_batch_step(self.b, n)

    def tune(self):
        return clb_batch_tune(self.b)

    def set_schedule(self, nodes_per_thread, packed):
        clb_batch_set_schedule(self.b, nodes_per_thread, packed)

    def schedule(self):
        return clb_batch_schedule(self.b)

    def info(self):
        blk, step, _ = clb_batch_info(self.b)
        return {"block_x": blk, "step": step}

    def observables(self):
        s = clb_batch_observables(self.b, self.n)
        return [{k: getattr(x, k) for k, _ in clb_scalars._fields_} for x in s]

    def state(self, k):
        f = np.empty((9, self.ny[k], self.nx[k]), np.float64)
        clb_batch_get_state(self.b, k, f.ctypes.data)
        return f

    def set_state(self, k, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(9, self.ny[k], self.nx[k])
        clb_batch_set_state(self.b, k, f.ctypes.data)


# ------------------------------------------------------------ adjoint

def clb_adjoint_forward(nx, ny, kn, a, r, g, nsteps, checkpoint_every=0, opts: clb_opts | None = None):
    h = C.c_void_p()
    J = C.c_double()
    _check(lib.clb_adjoint_forward(int(nx), int(ny), float(kn), float(a), float(r), float(g), int(nsteps),
                                   int(checkpoint_every), C.byref(opts) if opts is not None else None,
                                   C.byref(h), C.byref(J)))
    return h, J.value


def clb_adjoint_backward(h, seed=1.0):
    grad = (C.c_double * 3)()
    _check(lib.clb_adjoint_backward(h, float(seed), grad))
    return list(grad)


def clb_adjoint_q(h):
    q = C.c_double()
    _check(lib.clb_adjoint_q(h, C.byref(q)))
    return q.value


def clb_adjoint_q_backward(h, seed=1.0):
    grad = (C.c_double * 3)()
    _check(lib.clb_adjoint_q_backward(h, float(seed), grad))
    return list(grad)


def clb_adjoint_destroy(h):
    return _check(lib.clb_adjoint_destroy(h))


class FlowGradient:
    """J = mean_x sum_y u_x of a periodic body-force channel after nsteps, and
    its adjoint gradient with respect to (r_b, a, G); the normalised flow rate
    Q of Sec. 3.1 and its gradient come from the library as well."""

    def __init__(self, nx, ny, kn, a, r, g, nsteps, storage="fp32s", checkpoint_every=0, b2=0.55, sigma=1.0,
                 s3=1.1, s8=1.2, rho_out=1.0, stream=None, pipeline=0):
        import torch

        dev = torch.cuda.current_device()
        if stream is None or stream.cuda_stream == 0:
            stream = torch.cuda.Stream(dev)
        self._stream = stream
        o = clb_opts_default()
        o.b2, o.sigma, o.s3, o.s8, o.rho_out = b2, sigma, s3, s8, rho_out
        o.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        o.stream = C.c_void_p(stream.cuda_stream)
        o.pipeline = int(pipeline)  # 1: one launch per step instead of one block per pass

        def _alloc(nbytes, ctx):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)
            except Exception:  # noqa: BLE001 - reported to the library as NULL
                return None

        def _free(p, ctx):
            torch.cuda.caching_allocator_delete(int(p))

        self._hooks = (ALLOC_FN(_alloc), FREE_FN(_free))
        o.alloc, o.free = self._hooks
        self.h, self.J = clb_adjoint_forward(nx, ny, kn, a, r, g, nsteps, checkpoint_every, o)

    def grad(self, seed=1.0):
        """seed * dJ/d(r_b, a, G)."""
        return clb_adjoint_backward(self.h, seed)

    @property
    def q_norm(self):
        """Q after the forward pass (clb_adjoint_q)."""
        return clb_adjoint_q(self.h)

    def q_grad(self, seed=1.0):
        """seed * dQ/d(r_b, a, G) (clb_adjoint_q_backward)."""
        return clb_adjoint_q_backward(self.h, seed)

    def close(self):
        if getattr(self, "h", None):
            clb_adjoint_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


def _flow_rate_function():
    import torch

    class FlowRate(torch.autograd.Function):
        """Q(r_b, a, G) of a periodic channel (Sec. 3.1) as a differentiable
        torch op: the forward pass runs the channel with checkpoints, the
        backward pass runs the hand-written adjoint kernels."""

        @staticmethod
        def forward(ctx, r, a, g, cfg):
            fg = FlowGradient(cfg["nx"], cfg["ny"], cfg["kn"], float(a), float(r), float(g), cfg["nsteps"],
                              storage=cfg.get("storage", "fp32s"), checkpoint_every=cfg.get("checkpoint_every", 0))
            ctx.fg = fg
            return torch.tensor(fg.q_norm, dtype=torch.float64)

        @staticmethod
        def backward(ctx, gout):
            fg = ctx.fg
            grads = fg.q_grad(float(gout))
            fg.close()
            return tuple(torch.tensor(v, dtype=torch.float64) for v in grads) + (None,)

    return FlowRate


def flow_rate(r, a, g, cfg):
    """Differentiable normalised flow rate Q (see FlowRate); r, a, g are
    0-dim float64 tensors, cfg = dict(nx, ny, kn, nsteps[, storage,
    checkpoint_every])."""
    return _flow_rate_function().apply(r, a, g, cfg)
