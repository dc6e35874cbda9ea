"""Thin ctypes binding of ``include/lbm.h`` (argument marshalling only).

Every function here has the name of the C call it wraps, without the
``lbm_`` prefix.  All computation happens in ``libmrtlbm.so``; if the library
is missing or cannot be loaded, :func:`lib` raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

F64, F32, BF16D, F16D, F32D, F16S, BF16S = 0, 1, 2, 3, 4, 5, 6
PREC_NAMES = {"f64": F64, "f32": F32, "bf16d": BF16D, "f16d": F16D, "f32d": F32D, "f16s": F16S, "bf16s": BF16S}
STORE_DTYPE = {F64: np.float64, F32: np.float32, BF16D: np.uint16, F16D: np.float16, F32D: np.float32,
               F16S: np.float16, BF16S: np.uint16}
TAU_DTYPE = {F64: np.float64, F32: np.float32, BF16D: np.float32, F16D: np.float32, F32D: np.float32,
             F16S: np.float32, BF16S: np.float32}

ERRORS = {0: "LBM_OK", -1: "LBM_ERR_ARG", -2: "LBM_ERR_UNSTABLE", -3: "LBM_ERR_NONFINITE",
          -4: "LBM_ERR_CUDA", -5: "LBM_ERR_OOM", -6: "LBM_ERR_TIMEOUT", -7: "LBM_ERR_UNSUPPORTED",
          -8: "LBM_ERR_SIZE"}
NOALLOC_MAX_ROWS = 16384


class LBMError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = f"{what}: {ERRORS.get(code, code)}"
        if code == -4 or code == -5:
            msg += f" ({lib().lbm_last_cuda_error().decode()})"
        super().__init__(msg)


class Opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("Ma", ctypes.c_double), ("clamp_mode", ctypes.c_int),
                ("porous_model", ctypes.c_int), ("s_e", ctypes.c_double), ("s_p", ctypes.c_double),
                ("resid_interval", ctypes.c_int), ("layout", ctypes.c_int),
                ("cuda_stream", ctypes.c_void_p), ("device", ctypes.c_int),
                ("stag_floor", ctypes.c_double), ("tau_iters", ctypes.c_int), ("staging", ctypes.c_int),
                ("graph_steps", ctypes.c_int), ("seed", ctypes.c_uint64)]


class Lattice(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("n", ctypes.c_double),
                ("nu_ref", ctypes.c_double), ("gamma_scale", ctypes.c_double),
                ("gamma1", ctypes.c_double), ("gamma2", ctypes.c_double),
                ("clamp_mode", ctypes.c_int), ("K", ctypes.c_double), ("eps", ctypes.c_double),
                ("Feps", ctypes.c_double), ("gbeta", ctypes.c_double), ("Tm", ctypes.c_double),
                ("tauT", ctypes.c_double), ("s_e", ctypes.c_double), ("s_p", ctypes.c_double),
                ("T_hot", ctypes.c_double), ("T_cold", ctypes.c_double), ("L", ctypes.c_double),
                ("tau0", ctypes.c_double), ("prec", ctypes.c_int), ("pitch", ctypes.c_int64)]


_D = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p
_lock = threading.Lock()
_lib = None

# (name, restype, argtypes) of every entry point declared in include/lbm.h
SIGNATURES = [
    ("lbm_default_opts", None, [ctypes.POINTER(Opts)]),
    ("lbm_init", ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                ctypes.POINTER(Opts)]),
    ("lbm_destroy", None, [_VP]),
    ("lbm_get_lattice", ctypes.c_int, [_VP, ctypes.POINTER(Lattice)]),
    ("lbm_set_darcy_field", ctypes.c_int, [_VP, _D]),
    ("lbm_step", ctypes.c_int, [_VP, ctypes.c_int64]),
    ("lbm_synchronize", ctypes.c_int, [_VP]),
    ("lbm_fields", ctypes.c_int, [_VP, _D, _D, _D, _D, _D]),
    ("lbm_nusselt", ctypes.c_int, [_VP, _D, _D, _D]),
    ("lbm_residual", ctypes.c_int, [_VP, _D]),
    ("lbm_run_to_steady", ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_int64,
                                         ctypes.POINTER(ctypes.c_int64), _D,
                                         ctypes.POINTER(ctypes.c_int)]),
    ("lbm_state_bytes", ctypes.c_size_t, [_VP]),
    ("lbm_get_state", ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    ("lbm_set_state", ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    ("lbm_get_state_f64", ctypes.c_int, [_VP, _D, _D, _D]),
    ("lbm_set_state_f64", ctypes.c_int, [_VP, _D, _D, _D]),
    ("lbm_batch_create", ctypes.c_int, [ctypes.POINTER(_VP), _VP, ctypes.c_int, ctypes.POINTER(Opts)]),
    ("lbm_batch_destroy", None, [_VP]),
    ("lbm_batch_get_case", ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(_VP)]),
    ("lbm_batch_step", ctypes.c_int, [_VP, ctypes.c_int64]),
    ("lbm_batch_run_to_steady", ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_int64, ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_int64), _D,
                                               ctypes.POINTER(ctypes.c_int)]),
    ("lbm_batch_nusselt", ctypes.c_int, [_VP, _D, _D]),
    ("lbm_batch_tune", ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    ("lbm_adjoint_nu", ctypes.c_int, [_VP, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D, _D]),
    ("lbm_residual_noalloc", ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP]),
    ("lbm_batch_set_plan", ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    ("lbm_batch_get_plan", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int)]),
    ("lbm_batch_set_wait_budget", ctypes.c_int, [_VP, ctypes.c_int64]),
    ("lbm_init_slab", ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.POINTER(Opts)]),
    ("lbm_slab_rows", ctypes.c_int, [_VP] + [ctypes.POINTER(ctypes.c_int)] * 4),
    ("lbm_halo_bytes", ctypes.c_size_t, [_VP]),
    ("lbm_halo_pack", ctypes.c_int, [_VP, _VP, _VP]),
    ("lbm_halo_unpack", ctypes.c_int, [_VP, _VP, _VP]),
    ("lbm_nusselt_sums", ctypes.c_int, [_VP, _D, _D]),
    ("lbm_residual_sums", ctypes.c_int, [_VP, _D]),
    ("lbm_checkpoint_bytes", ctypes.c_size_t, [_VP]),
    ("lbm_checkpoint_save", ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    ("lbm_checkpoint_load", ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    ("lbm_debug_padding_canary", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_ulonglong)]),
    ("lbm_debug_sr_pairs", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _VP, _VP, _VP, ctypes.c_size_t]),
    ("lbm_bench_fma_peak", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D]),
    ("lbm_strerror", ctypes.c_char_p, [ctypes.c_int]),
    ("lbm_last_cuda_error", ctypes.c_char_p, []),
]


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load ``libmrtlbm.so`` (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            if not _build.up_to_date():
                _build.build()
            L = ctypes.CDLL(_build.LIB)
            for name, res, args in SIGNATURES:
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_D)


def _check(rc: int, what: str):
    if rc != 0:
        raise LBMError(rc, what)


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)   # torch.cuda.Stream


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().lbm_default_opts(ctypes.byref(o))
    names = {f[0] for f in Opts._fields_}
    for k, v in kw.items():
        if k not in names:
            raise TypeError(f"unknown lbm_opts field {k!r}")
        if k == "prec" and isinstance(v, str):
            v = PREC_NAMES[v]
        if k == "cuda_stream":
            v = _stream_handle(v)
        setattr(o, k, v)
    return o


def init(nx, ny, n, Da, Ra, Pr, porosity=0.6, **opts):
    """Create a cavity run; returns an opaque context handle (int)."""
    h = _VP()
    o = default_opts(**opts)
    _check(lib().lbm_init(ctypes.byref(h), nx, ny, n, Da, Ra, Pr, porosity, ctypes.byref(o)), "lbm_init")
    return h.value


def destroy(ctx):
    lib().lbm_destroy(ctx)


def get_lattice(ctx) -> Lattice:
    L = Lattice()
    _check(lib().lbm_get_lattice(ctx, ctypes.byref(L)), "lbm_get_lattice")
    return L


def set_darcy_field(ctx, Da):
    """Per-node Darcy numbers [ny][nx] (None: back to the uniform Da)."""
    if Da is None:
        _check(lib().lbm_set_darcy_field(ctx, None), "lbm_set_darcy_field")
        return
    Da = np.ascontiguousarray(Da, dtype=np.float64)
    _check(lib().lbm_set_darcy_field(ctx, _ptr(Da)), "lbm_set_darcy_field")


def step(ctx, k: int):
    _check(lib().lbm_step(ctx, int(k)), "lbm_step")


def synchronize(ctx):
    _check(lib().lbm_synchronize(ctx), "lbm_synchronize")


def fields(ctx, nx, ny):
    """Streamed fields as a dict of [ny][nx] float64 arrays (rho, ux, uy, T, nu)."""
    out = {k: np.empty((ny, nx)) for k in ("rho", "ux", "uy", "T", "nu")}
    _check(lib().lbm_fields(ctx, *[_ptr(out[k]) for k in ("rho", "ux", "uy", "T", "nu")]), "lbm_fields")
    return out


def nusselt(ctx, ny=None):
    """(hot-wall average Nu, cold-wall average Nu, local hot-wall Nu or None)."""
    h = ctypes.c_double(); c = ctypes.c_double()
    loc = np.empty(ny) if ny else None
    _check(lib().lbm_nusselt(ctx, ctypes.byref(h), ctypes.byref(c), _ptr(loc)), "lbm_nusselt")
    return h.value, c.value, loc


def residual(ctx) -> float:
    r = ctypes.c_double()
    _check(lib().lbm_residual(ctx, ctypes.byref(r)), "lbm_residual")
    return r.value


def residual_noalloc(ctx, d_snapshot: int, first: bool, d_result: int):
    """Allocation-free residual: device pointers in, results left on the device."""
    _check(lib().lbm_residual_noalloc(ctx, d_snapshot, 1 if first else 0, d_result), "lbm_residual_noalloc")


def adjoint_nu(ctx, nx, ny, steps: int, ckpt_every: int = 500, from_rest: bool = True):
    """(J, dJ/dDa[ny][nx], dJ/dn, dJ/dRa, peak device bytes) by the discrete adjoint."""
    J = ctypes.c_double(); dn = ctypes.c_double(); dRa = ctypes.c_double(); pk = ctypes.c_double()
    dDa = np.empty((ny, nx))
    _check(lib().lbm_adjoint_nu(ctx, int(steps), int(ckpt_every), 1 if from_rest else 0, ctypes.byref(J),
                                _ptr(dDa), ctypes.byref(dn), ctypes.byref(dRa), ctypes.byref(pk)),
           "lbm_adjoint_nu")
    return J.value, dDa, dn.value, dRa.value, pk.value


def run_to_steady(ctx, tol: float, max_steps: int):
    """Returns (steps_done, residual, reason) with reason 0 tol, 1 stagnated, 2 max_steps."""
    s = ctypes.c_int64(); r = ctypes.c_double(); why = ctypes.c_int()
    _check(lib().lbm_run_to_steady(ctx, tol, int(max_steps), ctypes.byref(s), ctypes.byref(r),
                                   ctypes.byref(why)), "lbm_run_to_steady")
    return s.value, r.value, why.value


def state_bytes(ctx) -> int:
    return int(lib().lbm_state_bytes(ctx))


def get_state(ctx, host):
    """Copy the native state into ``host`` (numpy array or torch CPU tensor)."""
    ptr = host.ctypes.data if isinstance(host, np.ndarray) else host.data_ptr()
    nbytes = host.nbytes if isinstance(host, np.ndarray) else host.numel() * host.element_size()
    _check(lib().lbm_get_state(ctx, ptr, nbytes), "lbm_get_state")


def set_state(ctx, host):
    ptr = host.ctypes.data if isinstance(host, np.ndarray) else host.data_ptr()
    nbytes = host.nbytes if isinstance(host, np.ndarray) else host.numel() * host.element_size()
    _check(lib().lbm_set_state(ctx, ptr, nbytes), "lbm_set_state")


def get_state_f64(ctx, nx, ny):
    f = np.empty((9, ny, nx)); g = np.empty((5, ny, nx)); tau = np.empty((ny, nx))
    _check(lib().lbm_get_state_f64(ctx, _ptr(f), _ptr(g), _ptr(tau)), "lbm_get_state_f64")
    return f, g, tau


def set_state_f64(ctx, f=None, g=None, tau=None):
    conv = [None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in (f, g, tau)]
    _check(lib().lbm_set_state_f64(ctx, *[_ptr(a) for a in conv]), "lbm_set_state_f64")


def checkpoint_save(ctx) -> bytes:
    """The run's checkpoint blob (header + native state)."""
    nb = int(lib().lbm_checkpoint_bytes(ctx))
    buf = (ctypes.c_char * nb)()
    _check(lib().lbm_checkpoint_save(ctx, ctypes.cast(buf, _VP), nb), "lbm_checkpoint_save")
    return bytes(buf)


def checkpoint_load(ctx, blob: bytes):
    buf = ctypes.create_string_buffer(bytes(blob), len(blob))
    _check(lib().lbm_checkpoint_load(ctx, ctypes.cast(buf, _VP), len(blob)), "lbm_checkpoint_load")


def init_slab(nx, ny, y0, y1, n, Da, Ra, Pr, porosity=0.6, **opts):
    """Create the row slab [y0, y1) of an nx x ny cavity; returns a context handle."""
    h = _VP()
    o = default_opts(**opts)
    _check(lib().lbm_init_slab(ctypes.byref(h), nx, ny, y0, y1, n, Da, Ra, Pr, porosity, ctypes.byref(o)),
           "lbm_init_slab")
    return h.value


def slab_rows(ctx):
    """(y0, row_lo, row_hi, ny_local) of a context."""
    v = [ctypes.c_int() for _ in range(4)]
    _check(lib().lbm_slab_rows(ctx, *[ctypes.byref(x) for x in v]), "lbm_slab_rows")
    return tuple(x.value for x in v)


def halo_bytes(ctx) -> int:
    return int(lib().lbm_halo_bytes(ctx))


def halo_pack(ctx, d_lo, d_hi):
    _check(lib().lbm_halo_pack(ctx, d_lo, d_hi), "lbm_halo_pack")


def halo_unpack(ctx, d_lo, d_hi):
    _check(lib().lbm_halo_unpack(ctx, d_lo, d_hi), "lbm_halo_unpack")


def nusselt_sums(ctx):
    h = ctypes.c_double()
    c = ctypes.c_double()
    _check(lib().lbm_nusselt_sums(ctx, ctypes.byref(h), ctypes.byref(c)), "lbm_nusselt_sums")
    return h.value, c.value


def residual_sums(ctx):
    s = np.zeros(7)
    _check(lib().lbm_residual_sums(ctx, _ptr(s)), "lbm_residual_sums")
    return s


def debug_padding_canary(ctx) -> int:
    """Nonzero bytes in the pitch padding of the state planes (lbm_debug.h): 0 unless a kernel wrote outside the rows."""
    n = ctypes.c_ulonglong()
    _check(lib().lbm_debug_padding_canary(ctx, ctypes.byref(n)), "lbm_debug_padding_canary")
    return n.value


def debug_sr_pairs(fmt: str, x, r, device: int = 0):
    """The 16-bit storages' stochastic rounding of value pairs (lbm_debug.h):
    fmt 'f16' or 'bf16'; x: 2n float32 values (pair i = x[2i] low, x[2i+1]
    high), r: n uint32 random words -> 2n uint16 codes."""
    k = {"f16": 0, "bf16": 1}[fmt]
    x = np.ascontiguousarray(x, dtype=np.float32)
    r = np.ascontiguousarray(r, dtype=np.uint32)
    if x.size != 2 * r.size:
        raise ValueError("x must hold two values per random word")
    out = np.empty(x.size, dtype=np.uint16)
    _check(lib().lbm_debug_sr_pairs(device, k, x.ctypes.data, r.ctypes.data, out.ctypes.data, r.size),
           "lbm_debug_sr_pairs")
    return out


def bench_fma_peak(kind: str, device: int = -1, reps: int = 20):
    """Measured FMA throughput (lbm_bench.h): kind 'f64', 'f32' or 'f32x2'
    -> (thread-level FMAs per second, instructions per second)."""
    k = {"f64": 0, "f32": 1, "f32x2": 2}[kind]
    f = ctypes.c_double()
    i = ctypes.c_double()
    _check(lib().lbm_bench_fma_peak(k, device, reps, ctypes.byref(f), ctypes.byref(i)), "lbm_bench_fma_peak")
    return f.value, i.value


def strerror(code: int) -> str:
    return lib().lbm_strerror(code).decode()


class Case(ctypes.Structure):
    """Mirror of ``lbm_case``."""
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("n", ctypes.c_double),
                ("Da", ctypes.c_double), ("Ra", ctypes.c_double), ("Pr", ctypes.c_double),
                ("porosity", ctypes.c_double)]


class Batch:
    """Owning wrapper of an ``lbm_batch`` (a sweep of independent cavities)."""

    def __init__(self, cases, **opts):
        arr = (Case * len(cases))(*[Case(c["nx"], c["ny"], c["n"], c["Da"], c["Ra"], c["Pr"],
                                         c.get("porosity", 0.6)) for c in cases])
        self.cases = list(cases)
        self.n = len(cases)
        o = default_opts(**opts)
        h = _VP()
        _check(lib().lbm_batch_create(ctypes.byref(h), ctypes.cast(arr, _VP), self.n, ctypes.byref(o)),
               "lbm_batch_create")
        self.h = h.value

    def close(self):
        if getattr(self, "h", None):
            lib().lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def case_ctx(self, i):
        c = _VP()
        _check(lib().lbm_batch_get_case(self.h, i, ctypes.byref(c)), "lbm_batch_get_case")
        return c.value

    def step(self, k):
        _check(lib().lbm_batch_step(self.h, int(k)), "lbm_batch_step")

    def run_to_steady(self, tol, max_steps, graph_mode=1):
        steps = (ctypes.c_int64 * self.n)(); res = np.empty(self.n); why = (ctypes.c_int * self.n)()
        _check(lib().lbm_batch_run_to_steady(self.h, tol, int(max_steps), graph_mode, steps, _ptr(res), why),
               "lbm_batch_run_to_steady")
        return list(steps), res, list(why)

    def nusselt(self):
        hot = np.empty(self.n); cold = np.empty(self.n)
        _check(lib().lbm_batch_nusselt(self.h, _ptr(hot), _ptr(cold)), "lbm_batch_nusselt")
        return hot, cold

    def tune(self, steps=200):
        t = ctypes.c_int()
        _check(lib().lbm_batch_tune(self.h, int(steps), ctypes.byref(t)), "lbm_batch_tune")
        return t.value

    def set_plan(self, mode, threads=128, blocks_per_sm=8):
        """mode 'per_step' / 'persistent' (or 0 / 1)."""
        m = {"per_step": 0, "persistent": 1}.get(mode, mode)
        _check(lib().lbm_batch_set_plan(self.h, int(m), int(threads), int(blocks_per_sm)), "lbm_batch_set_plan")

    def plan(self):
        m, t, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().lbm_batch_get_plan(self.h, ctypes.byref(m), ctypes.byref(t), ctypes.byref(b)),
               "lbm_batch_get_plan")
        return {"mode": ("per_step", "persistent")[m.value], "threads": t.value, "blocks_per_sm": b.value}

    def set_wait_budget(self, cycles):
        _check(lib().lbm_batch_set_wait_budget(self.h, int(cycles)), "lbm_batch_set_wait_budget")


class Cavity:
    """Owning wrapper of one context with the calls above as methods."""

    def __init__(self, nx, ny, n, Da, Ra, Pr, porosity=0.6, **opts):
        self.nx, self.ny = nx, ny
        self.prec = PREC_NAMES.get(opts.get("prec"), opts.get("prec", F64))
        self.ctx = init(nx, ny, n, Da, Ra, Pr, porosity, **opts)

    def close(self):
        if getattr(self, "ctx", None):
            destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def lattice(self):
        return get_lattice(self.ctx)

    def set_darcy_field(self, Da):
        set_darcy_field(self.ctx, Da)

    def adjoint_nu(self, steps, ckpt_every=500, from_rest=True):
        return adjoint_nu(self.ctx, self.nx, self.ny, steps, ckpt_every, from_rest)

    def step(self, k):
        step(self.ctx, k)

    def synchronize(self):
        synchronize(self.ctx)

    def fields(self):
        return fields(self.ctx, self.nx, self.ny)

    def nusselt(self, local=False):
        return nusselt(self.ctx, self.ny if local else None)

    def residual(self):
        return residual(self.ctx)

    def run_to_steady(self, tol, max_steps):
        return run_to_steady(self.ctx, tol, max_steps)

    def get_state_f64(self):
        return get_state_f64(self.ctx, self.nx, self.ny)

    def set_state_f64(self, f=None, g=None, tau=None):
        set_state_f64(self.ctx, f, g, tau)

    def state_bytes(self):
        return state_bytes(self.ctx)

    def checkpoint(self) -> bytes:
        return checkpoint_save(self.ctx)

    def restore(self, blob: bytes):
        checkpoint_load(self.ctx, blob)

    def get_state(self, host):
        get_state(self.ctx, host)

    def set_state(self, host):
        set_state(self.ctx, host)
