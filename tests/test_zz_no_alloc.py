"""The allocation-free residual against the ordinary one.

``lbm_residual_noalloc`` serves callers that cannot call cudaMalloc where they
check convergence: host loops that must not block on an allocation (cudaMalloc
and cudaFree can synchronise the device), and applications whose device
memory all belongs to their own pool allocator.  They pass device buffers they
already own; the library's only scratch is a fixed array inside it.  The
result must match ``lbm_residual`` call after call.  This file is collected
last so that a run stopping at its first failure has run every other test.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


# (storage, per-node Darcy field, implicit tau steps): the residual kernel
# reads the state through the same pull and velocity solve as the step, so
# each storage form, the field and the implicit tau take their own path
VARIANTS = [("f64", False, 0), ("f32", False, 0), ("bf16d", False, 0), ("f16s", False, 0),
            ("f32", True, 2), ("f64", True, 4)]


@pytest.mark.parametrize("prec,field,tau_iters", VARIANTS)
def test_noalloc_residual_matches_lbm_residual(prec, field, tau_iters):
    torch = pytest.importorskip("torch")
    import oracle
    from paper_2011_15073_gb300 import inputs, lbm

    nx, ny = 96, 80
    case = dict(n=0.6, Da=1e-2, Ra=1e5, Pr=6.2, porosity=0.6)
    rest = oracle.Cavity.from_params(nx, ny, case["n"], case["Da"], case["Ra"], case["Pr"],
                                     porosity=case["porosity"])
    state = inputs.perturbed_state(rest.get_state(), seed=21)
    snap = torch.empty(3 * nx * ny, dtype=torch.float64, device="cuda:0")
    out = torch.empty(4, dtype=torch.float64, device="cuda:0")
    with lbm.Cavity(nx, ny, prec=prec, device=0, tau_iters=tau_iters, **case) as cav:
        if field:
            cav.set_darcy_field(inputs.darcy_field(31, nx, ny))
        cav.set_state_f64(*state)
        assert math.isinf(cav.residual())
        lbm.residual_noalloc(cav.ctx, snap.data_ptr(), True, out.data_ptr())
        cav.synchronize()
        assert np.all(np.isinf(out.cpu().numpy()[:3]))
        for _ in range(2):   # two calls in a row
            cav.step(50)
            expect = cav.residual()
            lbm.residual_noalloc(cav.ctx, snap.data_ptr(), False, out.data_ptr())
            cav.synchronize()
            got = out.cpu().numpy()
            assert got[3] == 0.0
            assert max(got[:3]) == pytest.approx(expect, rel=1e-12, abs=0)
            assert expect > 0


def test_noalloc_residual_refuses_grids_beyond_its_scratch():
    pytest.importorskip("torch")
    import torch
    from paper_2011_15073_gb300 import lbm

    ny = lbm.NOALLOC_MAX_ROWS + 1
    snap = torch.empty(3 * 2 * ny, dtype=torch.float64, device="cuda:0")
    out = torch.zeros(4, dtype=torch.float64, device="cuda:0")
    with lbm.Cavity(2, ny, n=1.0, Da=1e-1, Ra=1e3, Pr=6.2, porosity=0.6, prec="f32", device=0) as cav:
        with pytest.raises(lbm.LBMError) as e:
            lbm.residual_noalloc(cav.ctx, snap.data_ptr(), True, out.data_ptr())
        assert e.value.code == -8
    assert torch.count_nonzero(out).item() == 0
