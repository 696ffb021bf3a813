"""GPU parity of the compact (Mehrstellen) fine stencil against the FP64 oracle.

The 19-point operator L, the weighting matrix W, multigrid on W - c L, SDC in
the weighted form and the FAS restriction's W^{-1} (Sec. 1, Sec. 1.2).  FP64
to 1e-11 relative max-norm with equal V-cycle and iteration counts where
tolerances decide them; mixed precision to 1e-9; sizes with ragged tiles.
"""
import numpy as np
import pytest

from paper_1307_7867_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("N", [1, 3, 7, 31, 63, 127])
def test_compact_operator(H, oracle, N):
    cfg = H.make_config((N, H.COMPACT, 3), nu=0.1)
    ctx = H.Context(cfg)
    u = inputs.random_field(N, seed=200 + N)
    out = torch.empty(N, N, N, dtype=torch.float64, device="cuda")
    H.heat3d_apply_laplacian(ctx, 0, dev(u), out)
    assert rel(host(out), 0.1 * oracle.laplacian(u, oracle.COMPACT)) <= 1e-12


@pytest.mark.parametrize("N,ch2,cycles", [(1, 3.0, 1), (3, 3.0, 2), (15, 20.0, 3), (63, 17.0, 2),
                                          (127, 5.0, 1), (31, 0.0, 3)])
def test_compact_mg_fixed_cycles(H, oracle, N, ch2, cycles):
    """V(2,1) cycles on W - c L (c = 0: the weighting matrix) equal the oracle's."""
    c = ch2 / (N + 1) ** 2
    ctx = H.Context(H.make_config((N, H.COMPACT, 3)))
    b = inputs.random_field(N, seed=1)
    u0 = inputs.random_field(N, seed=2, scale=0.1)
    u = dev(u0)
    H.mg_vcycle(ctx, 0, c, dev(b), u, cycles, -1.0)
    ref, rc, cyc, res = oracle.mg_solve(u0, b, oracle.COMPACT, c, tol=-1.0, max_cycles=cycles)
    assert rel(host(u), ref) <= 1e-11


def test_compact_mg_tolerance_and_mixed(H, oracle):
    N = 63
    c = 17.0 / (N + 1) ** 2
    b = inputs.random_field(N, seed=3)
    ctx = H.Context(H.make_config((N, H.COMPACT, 3)))
    u = dev(np.zeros_like(b))
    rc, st = H.mg_vcycle(ctx, 0, c, dev(b), u, 50, 1e-12)
    ref, orc, ocyc, _ = oracle.mg_solve(np.zeros_like(b), b, oracle.COMPACT, c, tol=1e-12,
                                        max_cycles=50)
    assert st["vcycles"] == ocyc and rel(host(u), ref) <= 1e-11
    ctxm = H.Context(H.make_config((N, H.COMPACT, 3), precision=H.MIXED))
    um = dev(np.zeros_like(b))
    H.mg_vcycle(ctxm, 0, c, dev(b), um, 60, 1e-12)
    assert rel(host(um), ref) <= 1e-9


PROB = dict(nu=0.1, forcing=1, kappa=1.0, mg_tol=1e-12, mg_max=50)


@pytest.mark.parametrize("N,M", [(31, 3), (63, 5)])
def test_compact_sdc_sweep(H, oracle, N, M):
    """Two weighted-form sweeps node by node, and the weighted residual."""
    cfg = H.make_config((N, H.COMPACT, M), dt=1.0 / 16, mg_tol=1e-12)
    ctx = H.Context(cfg)
    u0 = inputs.smooth_random_field(N, seed=5, kmax=6)
    t0 = 0.25
    H.heat3d_set_state(ctx, 0, 0, t0, u0)
    prob = oracle.Prob(**PROB)
    U, F = oracle.spread(N, oracle.COMPACT, M, prob, u0)
    for sweep in range(2):
        H.sdc_sweep(ctx, 0, 0, 1)
        U, F, rc, st = oracle.sdc_sweep(N, oracle.COMPACT, M, prob, t0, 1.0 / 16, U, F)
        out = np.empty((N, N, N))
        for m in range(M):
            H.heat3d_get_node(ctx, 0, 0, m, out)
            assert rel(out, U[m]) <= 1e-11, (sweep, m)
    r = H.heat3d_sdc_residual(ctx, 0, 0)
    ro = oracle.sdc_residual(N, oracle.COMPACT, M, prob, t0, 1.0 / 16, U, F)
    assert abs(r - ro) <= 1e-11 * max(1.0, ro) + 1e-14


def test_compact_fas_restrict_coarse_sweep_interpolate(H, oracle):
    """Restriction with the W-solve, FAS-corrected coarse sweep and interpolation."""
    fine, coarse = (31, 19, 5), (15, 2, 3)
    dt, t0 = 1.0 / 16, 0.5
    ctx = H.Context(H.make_config((31, H.COMPACT, 5), (15, 2, 3), dt=dt, mg_tol=1e-12))
    prob = oracle.Prob(**PROB)
    u0 = inputs.smooth_random_field(31, seed=7, kmax=6)
    H.heat3d_set_state(ctx, 0, 0, t0, u0)
    H.heat3d_set_state(ctx, 1, 0, t0, np.zeros((15, 15, 15)))
    H.sdc_sweep(ctx, 0, 0, 1)
    UF, FF = oracle.spread(*fine, prob, u0)
    UF, FF, _, _ = oracle.sdc_sweep(*fine, prob, t0, dt, UF, FF)
    H.heat3d_fas_restrict(ctx, 0, 1)
    UG, FG, UGr, tQ = oracle.fas_restrict(fine, coarse, prob, t0, dt, UF, FF)
    og = np.empty((15, 15, 15))
    for m in range(3):
        H.heat3d_get_node(ctx, 1, 0, m, og)
        assert rel(og, UG[m]) <= 1e-14
    rg = H.heat3d_sdc_residual(ctx, 1, 0)
    assert abs(rg - oracle.sdc_residual(*coarse, prob, t0, dt, UG, FG, tQ)) <= 1e-12
    H.sdc_sweep(ctx, 1, 0, 1)
    UG2, FG2, _, _ = oracle.sdc_sweep(*coarse, prob, t0, dt, UG, FG, tQ)
    for m in range(3):
        H.heat3d_get_node(ctx, 1, 0, m, og)
        assert rel(og, UG2[m]) <= 1e-11
    H.heat3d_fas_interpolate(ctx, 0, 1)
    UF2, FF2 = oracle.fas_interpolate(fine, coarse, prob, UG2, UGr, UF)
    of = np.empty((31, 31, 31))
    for j in range(5):
        H.heat3d_get_node(ctx, 0, 0, j, of)
        assert rel(of, UF2[j]) <= 1e-11


def test_compact_run_mlsdc(H, oracle):
    """MLSDC, compact fine / 7-point coarse level, to residual 1e-10: same
    iterations and V-cycles (substep solves and W-solves) as the oracle."""
    fine, coarse = (31, 19, 5), (15, 2, 3)
    cfg = H.make_config((31, H.COMPACT, 5), coarse, dt=1 / 64, T=2 / 64, sweeps_fine=2, iters=20,
                        tol_sdc=1e-10, mg_tol=1e-11)
    ctx = H.Context(cfg)
    u0 = inputs.smooth_random_field(31, seed=8, kmax=5)
    uT = np.empty_like(u0)
    rc, st = H.pfasst_run(ctx, u0, uT)
    ref, orc, ost = oracle.mlsdc_run(fine, coarse, oracle.Prob(mg_tol=1e-11), 1 / 64, 2, u0,
                                     nsweeps_fine=2, max_iters=20, tol=1e-10)
    assert st["iters"] == ost["iters"] and st["vcycles"] == ost["vcycles"]
    assert rel(uT, ref) <= 1e-11


def test_compact_pfasst_fixed_iterations(H, oracle):
    fine, coarse = (15, 19, 5), (7, 2, 3)
    P, K = 4, 3
    cfg = H.make_config((15, H.COMPACT, 5), coarse, dt=1 / 16, T=P / 16, sweeps_fine=1, slices=P,
                        iters=K, tol_sdc=-1.0, mg_tol=1e-12)
    ctx = H.Context(cfg)
    u0 = inputs.smooth_random_field(15, seed=9, kmax=4)
    uT = np.empty_like(u0)
    H.pfasst_run(ctx, u0, uT)
    ref, _, _ = oracle.pfasst_run(fine, coarse, oracle.Prob(mg_tol=1e-12), 1 / 16, P, P, u0,
                                  nsweeps_fine=1, max_iters=K)
    assert rel(uT, ref) <= 1e-11


def test_compact_mixed_precision_matches_fp64_oracle(H, oracle):
    fine, coarse = (31, 19, 5), (15, 2, 3)
    cfg = H.make_config((31, H.COMPACT, 5), coarse, dt=1 / 32, T=2 / 32, precision=H.MIXED,
                        mg_tol=1e-11, inner=2)
    ctx = H.Context(cfg)
    u0 = inputs.sine_mode(31)
    uT = np.empty_like(u0)
    H.pfasst_run(ctx, u0, uT)
    ref, _, _ = oracle.mlsdc_run(fine, coarse, oracle.Prob(mg_tol=1e-11), 1 / 32, 2, u0,
                                 nsweeps_fine=2, max_iters=20, tol=1e-10)
    assert rel(uT, ref) <= 1e-9


SHAPES = [(1, 4), (2, 8), (3, 16), (4, 4), (5, 8), (6, 16), (7, 8), (10, 64), (15, 8), (19, -1)]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_compact_every_launch_shape_is_bitwise_identical(H, precision, monkeypatch):
    """Forced launch shapes (the FP32 four-point tiles fall back to the 32-wide
    tile for the compact stencil) give the default shapes' result bitwise."""
    prec = H.FP64 if precision == "fp64" else H.MIXED

    def run():
        cfg = H.make_config((127, H.COMPACT, 3), (63, 2, 3), dt=1 / 32, T=2 / 32, sweeps_fine=1,
                            slices=2, iters=2, tol_sdc=-1.0, mg_tol=1e-10, precision=prec,
                            autotune=0, inner=2 if prec == H.MIXED else 1)
        ctx = H.Context(cfg, stream=torch.cuda.Stream())
        u0 = inputs.smooth_random_field(127, seed=11, kmax=6)
        uT = np.empty_like(u0)
        rc, st = H.pfasst_run(ctx, u0, uT)
        ctx.close()
        return uT, st["vcycles"]

    monkeypatch.delenv("HEAT3D_SHAPE", raising=False)
    ref, vref = run()
    for kind, zc in SHAPES:
        monkeypatch.setenv("HEAT3D_SHAPE", f"{kind},{zc}")
        uT, v = run()
        assert np.array_equal(uT, ref) and v == vref, (kind, zc)
    monkeypatch.delenv("HEAT3D_SHAPE")
