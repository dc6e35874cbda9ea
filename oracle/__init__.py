"""FP64 CPU oracle of the coupled MRT lattice Boltzmann update (test infrastructure).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  It is a
ctypes wrapper around ``oracle.c`` (plain C, FP64), which restates the paper's
algorithm literally (moment-space MRT with explicit matrices, literal
strain-rate double sum, push streaming).  It shares no code with the CUDA
library in ``paper_2011_15073_gb300``.

Parity status: every function of ``oracle.c`` is pinned by a CPU test
(``tests/test_oracle_*.py``) against what the paper and the mathematics fix;
the pins are listed in the block comments of ``oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` beside it (gcc, -O2, OpenMP).

    ``-ffp-contract=off`` keeps x86-64 and aarch64 results bit-identical."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-std=c11", "-Wall",
           "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Lattice(ctypes.Structure):
    """Mirror of ``orc_lattice`` (lattice-unit parameters of one run)."""

    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("n", ctypes.c_double), ("nu_ref", ctypes.c_double),
        ("gamma_scale", ctypes.c_double), ("gamma1", ctypes.c_double),
        ("gamma2", ctypes.c_double), ("clamp_mode", ctypes.c_int),
        ("K", ctypes.c_double), ("eps", ctypes.c_double),
        ("Feps", ctypes.c_double), ("gbeta", ctypes.c_double),
        ("Tm", ctypes.c_double), ("Gx", ctypes.c_double),
        ("tauT", ctypes.c_double), ("s", ctypes.c_double * 9),
        ("s_e", ctypes.c_double), ("s_p", ctypes.c_double),
        ("periodic_x", ctypes.c_int), ("T_hot", ctypes.c_double),
        ("T_cold", ctypes.c_double), ("L", ctypes.c_double),
        ("tau0", ctypes.c_double), ("rho0", ctypes.c_double),
        ("T0", ctypes.c_double), ("tau_iters", ctypes.c_int),
    ]

    def copy(self) -> "Lattice":
        out = Lattice()
        ctypes.memmove(ctypes.byref(out), ctypes.byref(self), ctypes.sizeof(Lattice))
        return out


_D = ctypes.POINTER(ctypes.c_double)


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_D)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.orc_map_params.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 6 + [
                ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.POINTER(Lattice)]
            L.orc_map_params.restype = ctypes.c_int
            L.orc_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(Lattice)]
            L.orc_create.restype = ctypes.c_int
            L.orc_destroy.argtypes = [ctypes.c_void_p]
            L.orc_destroy.restype = None
            L.orc_get_lattice.argtypes = [ctypes.c_void_p, ctypes.POINTER(Lattice)]
            L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
            L.orc_step.restype = ctypes.c_int
            L.orc_get_state.argtypes = [ctypes.c_void_p, _D, _D, _D]
            L.orc_set_state.argtypes = [ctypes.c_void_p, _D, _D, _D]
            L.orc_fields.argtypes = [ctypes.c_void_p] + [_D] * 6
            L.orc_nusselt.argtypes = [ctypes.c_void_p, _D, _D, _D]
            L.orc_set_darcy_field.argtypes = [ctypes.c_void_p, _D]
            L.orc_set_darcy_field.restype = None
            L.orc_matrices.argtypes = [_D] * 4
            L.orc_meq.argtypes = [ctypes.c_double] * 4 + [_D]
            L.orc_feq.argtypes = [ctypes.c_double] * 4 + [_D]
            L.orc_forcing_vel.argtypes = [ctypes.c_double] * 6 + [_D]
            L.orc_collide_node.argtypes = [ctypes.POINTER(Lattice), _D, _D, ctypes.c_double,
                                           _D, _D, _D, _D]
            L.orc_phi.argtypes = [ctypes.POINTER(Lattice), _D, _D, ctypes.c_double, _D]
            L.orc_phi.restype = ctypes.c_double
            L.orc_implicit_tau.argtypes = [ctypes.POINTER(Lattice), _D, _D]
            L.orc_implicit_tau.restype = ctypes.c_double
            _lib = L
    return _lib


def map_params(nx, ny, n, Da, Ra, Pr, porosity=0.6, Ma=0.1, porous_model=1,
               clamp_mode=0, s_e=1.5, s_p=1.5, tau_iters=0) -> Lattice:
    """Lattice-unit parameters of the cavity problem (see ``orc_map_params``);
    tau_iters > 0 selects the node-local implicit tau with that many Newton steps."""
    lat = Lattice()
    rc = lib().orc_map_params(nx, ny, n, Da, Ra, Pr, porosity, Ma, porous_model,
                              clamp_mode, s_e, s_p, ctypes.byref(lat))
    if rc != 0 or tau_iters < 0:
        raise ValueError("invalid cavity parameters")
    lat.tau_iters = int(tau_iters)
    return lat


def matrices():
    M = np.zeros(81); Mi = np.zeros(81); N = np.zeros(25); Ni = np.zeros(25)
    lib().orc_matrices(_ptr(M), _ptr(Mi), _ptr(N), _ptr(Ni))
    return M.reshape(9, 9), Mi.reshape(9, 9), N.reshape(5, 5), Ni.reshape(5, 5)


def meq(rho, ux, uy, eps):
    out = np.zeros(9)
    lib().orc_meq(rho, ux, uy, eps, _ptr(out))
    return out


def feq(rho, ux, uy, eps):
    out = np.zeros(9)
    lib().orc_feq(rho, ux, uy, eps, _ptr(out))
    return out


def forcing_vel(rho, ux, uy, Fx, Fy, eps):
    out = np.zeros(9)
    lib().orc_forcing_vel(rho, ux, uy, Fx, Fy, eps, _ptr(out))
    return out


def collide_node(lat: Lattice, f, g, tau_prev):
    """Single-node collision: returns (f*, g*, tau_new, |gamma|)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    fo = np.zeros(9); go = np.zeros(5)
    tn = ctypes.c_double(); gm = ctypes.c_double()
    lib().orc_collide_node(ctypes.byref(lat), _ptr(f), _ptr(g), float(tau_prev),
                           _ptr(fo), _ptr(go), ctypes.byref(tn), ctypes.byref(gm))
    return fo, go, tn.value, gm.value


def phi(lat: Lattice, f, g, tau):
    """The implicit-tau map of one node: (Phi(tau), Newton factor J)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    J = ctypes.c_double()
    v = lib().orc_phi(ctypes.byref(lat), _ptr(f), _ptr(g), float(tau), ctypes.byref(J))
    return v, J.value


def implicit_tau(lat: Lattice, f, g):
    """lat.tau_iters Newton steps toward the node's implicit tau."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    return lib().orc_implicit_tau(ctypes.byref(lat), _ptr(f), _ptr(g))


class Cavity:
    """One oracle run: state f[9][ny][nx], g[5][ny][nx], tau[ny][nx] (FP64)."""

    def __init__(self, lat: Lattice):
        self.lat = lat.copy()
        self.nx, self.ny = lat.nx, lat.ny
        h = ctypes.c_void_p()
        rc = lib().orc_create(ctypes.byref(h), ctypes.byref(self.lat))
        if rc != 0:
            raise MemoryError("orc_create failed")
        self._h = h

    @classmethod
    def from_params(cls, nx, ny, n, Da, Ra, Pr, **kw) -> "Cavity":
        return cls(map_params(nx, ny, n, Da, Ra, Pr, **kw))

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, k: int):
        lib().orc_step(self._h, int(k))

    def get_state(self):
        nn = self.nx * self.ny
        f = np.zeros((9, self.ny, self.nx)); g = np.zeros((5, self.ny, self.nx))
        tau = np.zeros((self.ny, self.nx))
        lib().orc_get_state(self._h, _ptr(f), _ptr(g), _ptr(tau))
        assert f.size == 9 * nn
        return f, g, tau

    def set_state(self, f, g, tau):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        tau = np.ascontiguousarray(tau, dtype=np.float64)
        assert f.shape == (9, self.ny, self.nx) and g.shape == (5, self.ny, self.nx)
        assert tau.shape == (self.ny, self.nx)
        lib().orc_set_state(self._h, _ptr(f), _ptr(g), _ptr(tau))

    def fields(self):
        """Streamed fields: dict of rho, ux, uy, T, nu, gamma, each [ny][nx]."""
        out = {k: np.zeros((self.ny, self.nx)) for k in ("rho", "ux", "uy", "T", "nu", "gamma")}
        lib().orc_fields(self._h, *[_ptr(out[k]) for k in ("rho", "ux", "uy", "T", "nu", "gamma")])
        return out

    def set_darcy_field(self, Da):
        """Per-node Darcy numbers [ny][nx] (None: uniform K again)."""
        if Da is None:
            lib().orc_set_darcy_field(self._h, None)
            return
        Da = np.ascontiguousarray(Da, dtype=np.float64)
        assert Da.shape == (self.ny, self.nx)
        self._Da = Da
        lib().orc_set_darcy_field(self._h, _ptr(Da))

    def nusselt(self):
        """(hot-wall average Nu, cold-wall average Nu, hot-wall local Nu[ny])."""
        h = ctypes.c_double(); c = ctypes.c_double(); loc = np.zeros(self.ny)
        lib().orc_nusselt(self._h, ctypes.byref(h), ctypes.byref(c), _ptr(loc))
        return h.value, c.value, loc
