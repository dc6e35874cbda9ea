"""Host-side checks of the C-ABI library that need no GPU: it loads, it exports
every entry point ``include/lbm.h`` declares, and argument validation rejects
bad input before any CUDA call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names.update(re.findall(r"\b(lbm_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def L():
    from paper_2011_15073_gb300 import lbm
    return lbm.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("lbm_init", "lbm_step", "lbm_fields", "lbm_nusselt", "lbm_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(L):
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2011_15073_gb300 import lbm
    bound = {name for name, _, _ in lbm.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_default_opts(L):
    from paper_2011_15073_gb300 import lbm
    o = lbm.default_opts()
    assert (o.prec, o.Ma, o.clamp_mode, o.porous_model, o.s_e, o.s_p, o.resid_interval, o.layout) == \
        (0, 0.1, 0, 1, 1.5, 1.5, 1000, 0)
    assert not o.cuda_stream and o.device == -1 and o.stag_floor == -1.0
    assert o.tau_iters == 0 and o.staging == 0 and o.graph_steps == 0


@pytest.mark.parametrize("args,code", [
    ((1, 8, 0.6, 1e-2, 1e5, 6.2, 0.6), -1),      # nx < 2
    ((8, 1, 0.6, 1e-2, 1e5, 6.2, 0.6), -1),      # ny < 2
    ((8, 65536, 0.6, 1e-2, 1e5, 6.2, 0.6), -1),  # ny above the launch-grid limit
    ((8, 8, 0.0, 1e-2, 1e5, 6.2, 0.6), -1),      # n <= 0
    ((8, 8, 0.6, -1.0, 1e5, 6.2, 0.6), -1),      # Da <= 0
    ((8, 8, 0.6, 1e-2, 0.0, 6.2, 0.6), -1),      # Ra <= 0
    ((8, 8, 0.6, 1e-2, 1e5, float("nan"), 0.6), -1),
    ((8, 8, 0.6, 1e-2, 1e5, 6.2, 1.5), -1),      # porosity > 1
    ((8, 8, 0.6, 1e-2, 1e5, 6.2, 0.0), -1),      # porosity <= 0
    ((8, 8, 1.0, 1e-2, 1e5, 1e-12, 0.6), -2),    # tau0 -> 1/2: unstable
])
def test_init_rejects_bad_arguments(L, args, code):
    from paper_2011_15073_gb300 import lbm
    h = ctypes.c_void_p(123)
    o = lbm.default_opts()
    rc = L.lbm_init(ctypes.byref(h), *args, ctypes.byref(o))
    assert rc == code and h.value is None


@pytest.mark.parametrize("field,value,code", [
    ("prec", 7, -1), ("prec", -1, -1), ("Ma", 0.0, -1), ("clamp_mode", 2, -1), ("porous_model", 3, -1),
    ("s_e", 2.5, -1), ("s_p", 0.0, -1), ("resid_interval", 0, -1), ("layout", 2, -7),
    ("device", -2, -1), ("tau_iters", -1, -1), ("tau_iters", 17, -1),
    ("staging", -1, -1), ("staging", 2, -7), ("staging", 3, -7), ("staging", 4, -1), ("graph_steps", -2, -1),
    # (the default storage is F64: neither the staged nor the four-node kernel is built for it)
])
def test_init_rejects_bad_options(L, field, value, code):
    from paper_2011_15073_gb300 import lbm
    h = ctypes.c_void_p()
    o = lbm.default_opts()
    setattr(o, field, value)
    assert L.lbm_init(ctypes.byref(h), 8, 8, 0.6, 1e-2, 1e5, 6.2, 0.6, ctypes.byref(o)) == code


@pytest.mark.parametrize("prec,tau_iters", [(0, 0), (1, 0), (4, 0), (4, 2), (1, 1)])
def test_four_node_mode_is_refused_where_not_built(L, prec, tau_iters):
    """staging = 3 (four nodes per thread) exists for the 16-bit storages
    (2, 3, 5, 6) only."""
    from paper_2011_15073_gb300 import lbm
    h = ctypes.c_void_p()
    o = lbm.default_opts()
    o.prec, o.staging, o.tau_iters = prec, 3, tau_iters
    assert L.lbm_init(ctypes.byref(h), 8, 8, 0.6, 1e-2, 1e5, 6.2, 0.6, ctypes.byref(o)) == -7


def test_darcy_field_rejects_bad_values(L):
    import numpy as np
    from paper_2011_15073_gb300 import lbm
    bad = np.full(4, -1.0)
    assert L.lbm_set_darcy_field(None, bad.ctypes.data_as(lbm._D)) == -1


def test_null_context_is_rejected(L):
    assert L.lbm_step(None, 1) == -1
    assert L.lbm_nusselt(None, None, None, None) == -1
    assert L.lbm_state_bytes(None) == 0
    L.lbm_destroy(None)


def test_strerror_names_codes(L):
    from paper_2011_15073_gb300 import lbm
    for code, name in lbm.ERRORS.items():
        assert lbm.strerror(code).startswith(name)


def test_binding_rejects_unknown_option():
    from paper_2011_15073_gb300 import lbm
    with pytest.raises(TypeError):
        lbm.default_opts(tau_iter=2)


def test_header_struct_matches_binding():
    """lbm_opts in include/lbm.h and the ctypes mirror list the same fields
    in the same order."""
    import re
    from paper_2011_15073_gb300 import lbm
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    body = src[src.index("typedef struct {\n    int prec;"):src.index("} lbm_opts;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = re.findall(r"\b(?:int|double|uint64_t|void\s*\*)\s*\**\s*(\w+(?:\s*,\s*\w+)*)\s*;",
                       body.split("{", 1)[1])
    flat = [n.strip() for grp in names for n in grp.split(",")]
    assert flat == [f[0] for f in lbm.Opts._fields_]


@pytest.mark.parametrize("opts", [dict(layout=1), dict(prec=5, layout=1)])
def test_batch_refuses_what_is_not_built(L, opts):
    """The batched sweep is not built for the in-place layout (checked
    before any device work)."""
    from paper_2011_15073_gb300 import lbm
    o = lbm.default_opts(resid_interval=1000, **opts)
    case = lbm.Case(16, 16, 0.6, 1e-2, 1e5, 6.2, 0.6)
    h = ctypes.c_void_p()
    assert L.lbm_batch_create(ctypes.byref(h), ctypes.byref(case), 1, ctypes.byref(o)) == -7
    assert h.value is None


def test_graphs_refused_for_stochastic_storages_in_place(L):
    """Step graphs of the stochastic-rounding storages are built for the
    two-buffer layout only (their seeds come from the device there)."""
    from paper_2011_15073_gb300 import lbm
    for prec in ("f16s", "bf16s"):
        o = lbm.default_opts(prec=prec, graph_steps=16, layout=1)
        h = ctypes.c_void_p()
        assert L.lbm_init(ctypes.byref(h), 8, 8, 0.6, 1e-2, 1e5, 6.2, 0.6, ctypes.byref(o)) == -7


def test_fma_probe_rejects_bad_arguments():
    """lbm_bench_fma_peak validates its arguments before touching a device."""
    import ctypes
    from paper_2011_15073_gb300 import lbm
    out = ctypes.c_double()
    assert lbm.lib().lbm_bench_fma_peak(3, -1, 5, ctypes.byref(out), None) == -1
    assert lbm.lib().lbm_bench_fma_peak(0, -1, 0, ctypes.byref(out), None) == -1
    assert lbm.lib().lbm_bench_fma_peak(0, -1, 5, None, None) == -1


def test_sr_pairs_check_rejects_bad_arguments():
    """lbm_debug_sr_pairs validates its arguments (and does nothing for zero
    pairs) before touching a device."""
    import numpy as np
    from paper_2011_15073_gb300 import lbm
    L = lbm.lib()
    x, r, o = np.zeros(2, np.float32), np.zeros(1, np.uint32), np.zeros(2, np.uint16)
    assert L.lbm_debug_sr_pairs(0, 2, x.ctypes.data, r.ctypes.data, o.ctypes.data, 1) == -1
    assert L.lbm_debug_sr_pairs(0, 0, None, r.ctypes.data, o.ctypes.data, 1) == -1
    assert L.lbm_debug_sr_pairs(0, 1, x.ctypes.data, r.ctypes.data, None, 1) == -1
    assert L.lbm_debug_sr_pairs(0, 0, x.ctypes.data, r.ctypes.data, o.ctypes.data, 0) == 0
    with __import__("pytest").raises(ValueError):
        lbm.debug_sr_pairs("f16", np.zeros(3, np.float32), np.zeros(1, np.uint32))


def test_slab_and_batch_calls_validate_arguments_before_the_device():
    """Slab creation, slab queries, halo and partial-sum calls and the batch
    plan calls reject bad arguments with LBM_ERR_ARG before any CUDA call."""
    import ctypes
    from paper_2011_15073_gb300 import lbm
    lib = lbm.lib()
    h = ctypes.c_void_p()
    o = lbm.default_opts()
    for (ny, y0, y1) in [(1, 0, 1), (40, -1, 10), (40, 10, 41), (40, 20, 20), (40, 30, 20)]:
        assert lib.lbm_init_slab(ctypes.byref(h), 32, ny, y0, y1, 0.6, 1e-2, 1e5, 6.2, 0.6, ctypes.byref(o)) == -1
        assert h.value is None
    o.layout = 1   # the in-place layout has no slab form
    assert lib.lbm_init_slab(ctypes.byref(h), 32, 40, 0, 20, 0.6, 1e-2, 1e5, 6.2, 0.6, ctypes.byref(o)) == -7
    assert lib.lbm_slab_rows(None, None, None, None, None) == -1
    assert lib.lbm_halo_bytes(None) == 0
    assert lib.lbm_halo_pack(None, None, None) == -1
    assert lib.lbm_halo_unpack(None, None, None) == -1
    assert lib.lbm_nusselt_sums(None, None, None) == -1
    assert lib.lbm_residual_sums(None, None) == -1
    assert lib.lbm_batch_set_plan(None, 0, 128, 8) == -1
    assert lib.lbm_batch_get_plan(None, None, None, None) == -1
    assert lib.lbm_batch_set_wait_budget(None, 100) == -1


def test_checkpoint_calls_validate_arguments():
    from paper_2011_15073_gb300 import lbm
    lib = lbm.lib()
    assert lib.lbm_checkpoint_bytes(None) == 0
    assert lib.lbm_checkpoint_save(None, None, 0) == -1
    assert lib.lbm_checkpoint_load(None, None, 0) == -1
