"""ctypes wrapper of the FP64 CPU oracle (``clb_oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).  The shared library is
compiled from the C source by :func:`build_oracle` with
``-O2 -ffp-contract=off -fopenmp`` so that no fused multiply-add changes the
oracle's rounding.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# Directory holding the C source and the libraries built from it.  The
# mutation tests point CLB_ORACLE_DIR at a copy with one planted mistake.
_DIR = os.environ.get("CLB_ORACLE_DIR", _HERE)
_SRC = os.path.join(_DIR, "clb_oracle.c")
_LIB = os.path.join(_DIR, "liboracle_clb.so")
_LIB_CS = os.path.join(_DIR, "liboracle_clb_cs.so")  # complex-step build

_lib = None
_lib_cs = None


def _fresh(lib):
    return os.path.exists(lib) and os.path.getmtime(lib) >= max(os.path.getmtime(_SRC),
                                                               os.path.getmtime(_SRC[:-1] + "h"))


def build_oracle(force: bool = False) -> str:
    """Compile the oracle shared libraries in place (the FP64 oracle and its
    complex-step build); returns the FP64 one's path."""
    for lib, extra in ((_LIB, []), (_LIB_CS, ["-DORACLE_COMPLEX"])):
        if not force and _fresh(lib):
            continue
        tmp = lib + ".tmp%d" % os.getpid()
        cmd = [
            "gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", *extra,
            "-o", tmp, _SRC, "-lm",
        ]
        subprocess.run(cmd, check=True)
        os.replace(tmp, lib)
    return _LIB


class _Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("pressure", C.c_int),
        ("kn", C.c_double), ("a", C.c_double), ("r", C.c_double), ("b2", C.c_double),
        ("s3", C.c_double), ("s8", C.c_double), ("gx", C.c_double), ("gy", C.c_double),
        ("rho_in", C.c_double), ("rho_out", C.c_double),
        ("sv_override", C.c_double), ("sq_override", C.c_double),
        ("same_node_bsr", C.c_int),
        ("r_im", C.c_double), ("a_im", C.c_double), ("gx_im", C.c_double),
        ("kn_mode", C.c_int),
    ]


@dataclass
class OracleParams:
    """Problem statement of one channel (defaults: the paper's Sec. 3 values)."""

    nx: int
    ny: int
    pressure: bool = False
    kn: float = 0.1
    a: float = 2.0
    r: float | None = None  # None: Eq. 21 from sigma
    sigma: float = 1.0
    b2: float = 0.55
    s3: float = 1.1
    s8: float = 1.2
    gx: float = 0.0
    gy: float = 0.0
    rho_in: float = 1.0
    rho_out: float = 1.0
    sv_override: float = 0.0
    sq_override: float = 0.0
    same_node_bsr: bool = False
    r_im: float = 0.0  # imaginary parts, read by the complex-step build only
    a_im: float = 0.0
    gx_im: float = 0.0
    kn_mode: int = 0  # pressure mode: 0 node pressure, 1 centreline pressure of the previous step

    def c(self) -> _Params:
        r = self.r if self.r is not None else r_from_sigma(self.sigma)
        return _Params(
            self.nx, self.ny, int(self.pressure), self.kn, self.a, r, self.b2, self.s3, self.s8,
            self.gx, self.gy, self.rho_in, self.rho_out, self.sv_override, self.sq_override,
            int(self.same_node_bsr), self.r_im, self.a_im, self.gx_im, int(self.kn_mode),
        )


def load():
    global _lib
    if _lib is not None:
        return _lib
    build_oracle()
    lib = C.CDLL(_LIB)
    D = C.POINTER(C.c_double)
    I = C.POINTER(C.c_int)
    lib.oracle_lattice.argtypes = [I, I]
    lib.oracle_tmat.argtypes = [D]
    lib.oracle_tinv.argtypes = [D]
    lib.oracle_kmat.argtypes = [D]
    lib.oracle_feq.argtypes = [C.c_double, C.c_double, C.c_double, D]
    lib.oracle_rates_kn.argtypes = [C.c_double, C.c_int, C.c_double, C.c_double, D, D]
    lib.oracle_r_from_sigma.argtypes = [C.c_double]
    lib.oracle_r_from_sigma.restype = C.c_double
    lib.oracle_collide.argtypes = [D, C.c_double, C.c_double, D, D, D, D]
    lib.oracle_create.argtypes = [C.POINTER(_Params)]
    lib.oracle_create.restype = C.c_void_p
    lib.oracle_destroy.argtypes = [C.c_void_p]
    lib.oracle_get_state.argtypes = [C.c_void_p, D]
    lib.oracle_set_state.argtypes = [C.c_void_p, D]
    lib.oracle_step.argtypes = [C.c_void_p, C.c_int64, C.c_int]
    lib.oracle_step.restype = C.c_int64
    lib.oracle_threads_used.restype = C.c_int
    lib.oracle_prestate.argtypes = [C.c_void_p, D]
    lib.oracle_step_nodes.argtypes = [C.POINTER(_Params), D, C.c_int, I, I, D]
    lib.oracle_observables.argtypes = [C.c_void_p, C.c_int, D, D, D, D, D, D]
    lib.oracle_macro.argtypes = [C.c_void_p, D, D, D]
    _lib = lib
    return lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def lattice():
    ex = np.zeros(9, np.int32)
    ey = np.zeros(9, np.int32)
    load().oracle_lattice(_ip(ex), _ip(ey))
    return ex, ey


def _mat(fn):
    m = np.zeros(81)
    fn(_dp(m))
    return m.reshape(9, 9)


def tmat():
    return _mat(load().oracle_tmat)


def tinv():
    return _mat(load().oracle_tinv)


def kmat():
    return _mat(load().oracle_kmat)


def feq(rho, ux, uy):
    out = np.zeros(9)
    load().oracle_feq(rho, ux, uy, _dp(out))
    return out


def rates_kn(kn_local, ny, a=2.0, b2=0.55):
    sv = C.c_double()
    sq = C.c_double()
    load().oracle_rates_kn(kn_local, ny, a, b2, C.byref(sv), C.byref(sq))
    return sv.value, sq.value


def r_from_sigma(sigma):
    return load().oracle_r_from_sigma(sigma)


def collide(fbar, Fx, Fy, s):
    """One-node collision; returns (f~, g^, S)."""
    fb = np.ascontiguousarray(fbar, dtype=np.float64)
    sv = np.ascontiguousarray(s, dtype=np.float64)
    out = np.zeros(9)
    g = np.zeros(9)
    S = np.zeros(9)
    load().oracle_collide(_dp(fb), Fx, Fy, _dp(sv), _dp(out), _dp(g), _dp(S))
    return out, g, S


def threads_used():
    return load().oracle_threads_used()


def step_nodes(params: OracleParams, f_prev, xs, ys):
    f = np.ascontiguousarray(f_prev, dtype=np.float64)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    out = np.zeros((len(xs), 9))
    p = params.c()
    load().oracle_step_nodes(C.byref(p), _dp(f), len(xs), _ip(xs), _ip(ys), _dp(out))
    return out


class OracleSim:
    """A channel advanced by the oracle; state is the post-collision f~, [9][ny][nx]."""

    def __init__(self, params: OracleParams):
        self.params = params
        self._p = params.c()
        lib = load()
        self._h = lib.oracle_create(C.byref(self._p))
        if not self._h:
            raise ValueError("oracle_create rejected the parameters")
        self.steps = 0

    def close(self):
        if self._h:
            load().oracle_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (9, self.params.ny, self.params.nx)

    def state(self):
        f = np.zeros(self.shape)
        load().oracle_get_state(self._h, _dp(f))
        return f

    def set_state(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.shape)
        load().oracle_set_state(self._h, _dp(f))

    def step(self, n: int, threads: int = 0):
        load().oracle_step(self._h, int(n), int(threads))
        self.steps += int(n)

    def prestate(self):
        f = np.zeros(self.shape)
        load().oracle_prestate(self._h, _dp(f))
        return f

    def macro(self):
        ny, nx = self.params.ny, self.params.nx
        rho = np.zeros((ny, nx))
        ux = np.zeros((ny, nx))
        uy = np.zeros((ny, nx))
        load().oracle_macro(self._h, _dp(rho), _dp(ux), _dp(uy))
        return rho, ux, uy

    def observables(self, profile_col: int = -1):
        ny, nx = self.params.ny, self.params.nx
        scal = np.zeros(5)
        uxp = np.zeros(ny)
        uyp = np.zeros(ny)
        pc = np.zeros(nx)
        dp = np.zeros(nx)
        mx = np.zeros(nx)
        load().oracle_observables(self._h, profile_col, _dp(scal), _dp(uxp), _dp(uyp), _dp(pc), _dp(dp), _dp(mx))
        return dict(
            mass_flow=scal[0], q_norm=scal[1], u_slip=scal[2], total_mass=scal[3], ux_max=scal[4],
            ux_prof=uxp, uy_prof=uyp, p_centre=pc, dp_nonlin=dp, m_of_x=mx,
        )



# ------------------------------------------------------ complex-step gradient

def load_cs():
    """The complex-step build: every real_t is a (re, im) pair of doubles."""
    global _lib_cs
    if _lib_cs is not None:
        return _lib_cs
    build_oracle()
    lib = C.CDLL(_LIB_CS)
    P = C.c_void_p
    lib.oracle_create.argtypes = [C.POINTER(_Params)]
    lib.oracle_create.restype = P
    lib.oracle_destroy.argtypes = [P]
    lib.oracle_step.argtypes = [P, C.c_int64, C.c_int]
    lib.oracle_step.restype = C.c_int64
    lib.oracle_macro.argtypes = [P, P, P, P]
    lib.oracle_get_state.argtypes = [P, P]
    _lib_cs = lib
    return lib


def flow_sum_cs(params: OracleParams, nsteps: int, threads: int = 1):
    """J = mean over x of sum_y u_x after nsteps (complex-step build): returns
    the complex J and the complex state; Im parts carry the perturbation."""
    lib = load_cs()
    p = params.c()
    h = lib.oracle_create(C.byref(p))
    if not h:
        raise ValueError("oracle_create rejected the parameters")
    try:
        lib.oracle_step(h, int(nsteps), int(threads))
        ny, nx = params.ny, params.nx
        ux = np.zeros((ny, nx), np.complex128)
        lib.oracle_macro(h, None, ux.ctypes.data, None)
        return ux.sum() / nx
    finally:
        lib.oracle_destroy(h)


def gradient_cs(params: OracleParams, nsteps: int, h: float = 1e-30, threads: int = 1):
    """Exact derivatives of J = mean_x sum_y u_x after nsteps with respect to
    r, a and G (gx), by complex-step differentiation: J(theta + i h) has
    imaginary part h dJ/dtheta + O(h^3).  Returns (J, {"r", "a", "g"})."""
    from dataclasses import replace

    if params.r is None:
        params = replace(params, r=r_from_sigma(params.sigma))
    out = {}
    J = None
    for name, field in (("r", "r_im"), ("a", "a_im"), ("g", "gx_im")):
        Jc = flow_sum_cs(replace(params, **{field: h}), nsteps, threads)
        out[name] = Jc.imag / h
        J = Jc.real
    return J, out
