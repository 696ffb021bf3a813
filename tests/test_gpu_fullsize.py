"""GPU checks at the benchmark's full sizes (255^3 / 127^3 and 511^3 / 255^3),
in the launch configuration bench.py times (CUDA graphs, autotuned shapes).

Elementwise against the oracle where the oracle finishes in seconds (the
operator at 255^3 and 511^3, one V(2,1) cycle at 255^3); otherwise through
properties that hold at any size: the error against the closed-form solution
of Eqs. 3-4, the collocation residual, and the fact that a sine-mode initial
value stays a multiple of that mode.
"""
import numpy as np
import pytest

from paper_1307_7867_gb300 import inputs
from tests import independent as ind

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NU = 0.1


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1307_7867_gb300 import build, heat3d
    build.build()
    heat3d.load()
    return heat3d


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("N,order", [(255, 4), (255, 19), (511, 4)])
def test_fullsize_operator(H, oracle, N, order):
    ctx = H.Context(H.make_config((N, order, 3), nu=NU))
    u = inputs.random_field(N, seed=31)
    out = torch.empty(N, N, N, dtype=torch.float64, device="cuda")
    H.heat3d_apply_laplacian(ctx, 0, torch.from_numpy(u).cuda(), out)
    torch.cuda.synchronize()
    assert rel(out.cpu().numpy(), NU * oracle.laplacian(u, order)) <= 1e-12


@pytest.mark.parametrize("order", [4, 19])
def test_fullsize_vcycle_255(H, oracle, order):
    """One V(2,1) cycle of the first fine substep of the 255^3 workload (wide
    or compact stencil, c = dt nu tau_1), with graphs and autotuned shapes,
    equals the oracle's cycle."""
    N = 255
    c = (1 / 64) * NU * 0.17267316464601143
    cfg = H.make_config((N, order, 5), use_graphs=1, autotune=1)
    ctx = H.Context(cfg, stream=torch.cuda.Stream())
    b = inputs.smooth_random_field(N, seed=32, kmax=8)
    u0 = inputs.random_field(N, seed=33, scale=1e-3)
    u = torch.from_numpy(u0.copy()).cuda()
    H.mg_vcycle(ctx, 0, c, torch.from_numpy(b).cuda(), u, 1, -1.0)
    torch.cuda.synchronize()
    ref, _, _, _ = oracle.mg_solve(u0, b, order, c, tol=-1.0, max_cycles=1)
    assert rel(u.cpu().numpy(), ref) <= 1e-11


def _mode_error(uT, t, lam):
    """Relative error against a(t) Phi, and the part of uT that is not a
    multiple of Phi (relative)."""
    N = uT.shape[0]
    phi = inputs.sine_mode(N)
    a = ind.semidiscrete_amplitude(lam, t, NU, 1.0)
    err = np.abs(uT - a * phi).max() / abs(a)
    coef = np.sum(uT * phi) / np.sum(phi * phi)
    impurity = np.abs(uT - coef * phi).max() / abs(coef)
    return err, impurity


@pytest.mark.parametrize("order", [4, 19])
def test_fullsize_mlsdc_step_properties(H, order):
    """One step of the 255^3 / 127^3 MLSDC workload (dt = 1/64, residual 1e-10)
    in FP64 and mixed precision: the result is a multiple of the initial sine
    mode up to the solver tolerances (1e-9; interpolation and multigrid add
    other modes only at that level), within 1e-10 of the PDE solution (the spatial error of
    either fourth-order stencil at h = 1/256 is ~6e-11), and the two precisions
    agree to 1e-9."""
    outs = []
    for prec in (H.FP64, H.MIXED):
        cfg = H.make_config((255, order, 5), (127, 2, 3), dt=1 / 64, T=1 / 64, sweeps_fine=2,
                            iters=20, tol_sdc=1e-10, mg_tol=1e-11, precision=prec,
                            inner=2 if prec == H.MIXED else 1, use_graphs=1, autotune=1)
        ctx = H.Context(cfg, stream=torch.cuda.Stream())
        u0 = torch.from_numpy(inputs.sine_mode(255)).cuda()
        uT = torch.empty_like(u0)
        rc, st = H.pfasst_run(ctx, u0, uT)
        assert st["residual"] <= 1e-10 and st["notconv"] == 0
        outs.append(uT.cpu().numpy())
        ctx.close()
    err, impurity = _mode_error(outs[0], 1 / 64, -3 * NU * np.pi**2)
    assert err <= 1e-10 and impurity <= 1e-9
    assert rel(outs[1], outs[0]) <= 1e-9


def test_fullsize_511_mixed_step(H):
    """One step of the 511^3 / 255^3 mixed-precision workload (dt = 1/32):
    residual 1e-10, a multiple of the sine mode, within 1e-10 of the PDE
    solution."""
    cfg = H.make_config((511, 4, 5), (255, 2, 3), dt=1 / 32, T=1 / 32, sweeps_fine=2, iters=20,
                        tol_sdc=1e-10, mg_tol=1e-11, precision=H.MIXED, inner=2, use_graphs=1,
                        autotune=1)
    ctx = H.Context(cfg, stream=torch.cuda.Stream())
    u0 = torch.from_numpy(inputs.sine_mode(511)).cuda()
    uT = torch.empty_like(u0)
    rc, st = H.pfasst_run(ctx, u0, uT)
    assert st["residual"] <= 1e-10 and st["notconv"] == 0
    err, impurity = _mode_error(uT.cpu().numpy(), 1 / 32, -3 * NU * np.pi**2)
    assert err <= 1e-10 and impurity <= 1e-9


@pytest.mark.parametrize("order", [4, 19])
def test_max_size_operator_on_sine_modes(H, order):
    """The largest grid the library accepts (N = 1023, 1.07e9 points, 8.6 GB
    per field): the operator applied to sine modes equals the mode times its
    closed-form symbol, to the rounding of the stencil sums (fields made and
    compared on the device)."""
    N = 1023
    ctx = H.Context(H.make_config((N, order, 2), nu=1.0, autotune=0))
    h = 1.0 / (N + 1)
    x = torch.arange(1, N + 1, device="cuda", dtype=torch.float64) * h
    out = torch.empty(N, N, N, dtype=torch.float64, device="cuda")
    for k in ((1, 1, 1), (3, 5, 7)):
        sx, sy, sz = (torch.sin(kk * np.pi * x) for kk in k)
        u = sz[:, None, None] * sy[None, :, None] * sx[None, None, :]
        H.heat3d_apply_laplacian(ctx, 0, u, out)
        if order == 4:
            lam = sum(ind.eig_1d(N, 4, kk) for kk in k)
        else:
            lam = ind.compact_eigs(N, k)[0]
        err = (out - lam * u).abs().max().item()
        # rounding of the neighbour sums: coefficients up to ~8 / h^2
        assert err <= 50 * 1e-14 / h**2, (k, err, lam)
        del u
    torch.cuda.synchronize()
