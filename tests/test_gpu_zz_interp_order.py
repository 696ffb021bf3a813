"""GPU parity of the 6- and 8-point interpolation of the coarse correction
(heat3d_config.interp = 6, 8) against the oracle: MLSDC with both fine
stencils (same iterations and V-cycles, result to 1e-11), two-node levels
(the one-pass point-wise kernel), fixed-count PFASST, and PFASST on 8 slices
of the paper's step size iterated to the 1e-10 residual, where the 8-point
stencil wraps around the 7-point coarse lines."""
import numpy as np
import pytest

from paper_1307_7867_gb300 import inputs
from tests import test_gpu_parity as base

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

H = base.H
rel = base.rel


@pytest.mark.parametrize("interp", [6, 8])
@pytest.mark.parametrize("order", [4, 19])
def test_run_mlsdc_midpoint_rules(H, oracle, order, interp):
    base.test_run_mlsdc_cubic_correction_interpolation(H, oracle, order, interp=interp)


def test_mlsdc_two_nodes_8_point(H, oracle):
    base.test_mlsdc_cubic_two_nodes(H, oracle, interp=8)


def test_pfasst_fixed_iterations_8_point(H, oracle):
    base.test_pfasst_cubic_interpolation_fixed_iterations(H, oracle, interp=8)


def test_pfasst_at_the_paper_step_with_8_point_interpolation(H, oracle):
    """8 slices of the paper's dt = 0.1875 (15^3 / 7^3, where the 8-point
    stencil wraps around the 7-point coarse lines), iterated to the 1e-10
    residual: the oracle's iteration count and result."""
    fine, coarse = (15, 4, 5), (7, 2, 3)
    P = 8
    cfg = H.make_config(fine, coarse, dt=0.1875, T=P * 0.1875, sweeps_fine=1, slices=P, iters=30,
                        tol_sdc=1e-10, mg_tol=1e-12, interp=8)
    ctx = H.Context(cfg)
    u0 = inputs.sine_mode(15)
    uT = np.empty_like(u0)
    rc, st = H.pfasst_run(ctx, u0, uT)
    ref, orc, ost = oracle.pfasst_run(fine, coarse, oracle.Prob(mg_tol=1e-12, interp=8), 0.1875, P,
                                      P, u0, nsweeps_fine=1, max_iters=30, tol=1e-10)
    assert orc == oracle.OK and ost["residual"] <= 1e-10
    assert st["iters"] == ost["iters"] and st["residual"] <= 1e-10
    assert rel(uT, ref) <= 1e-11
