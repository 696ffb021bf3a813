"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances: FP64 path 1e-11 relative max-norm (element by element); mixed
precision 1e-9 of the FP64 oracle after refinement.  Sizes span several
32 x 4 thread tiles with ragged tails (N = 63, 127 against tile widths of 32
and chunks of 16 planes) and include the one-unknown grid (N = 1).
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


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("N", [1, 3, 7, 31, 63, 127])
def test_laplacian(H, oracle, order, N):
    cfg = H.make_config((N, order, 3), nu=0.1)
    ctx = H.Context(cfg)
    u = inputs.random_field(N, seed=100 + N)
    out = torch.empty(N, N, N, dtype=torch.float64, device="cuda")
    H.heat3d_apply_laplacian(ctx, 0, dev(u), out)
    ref = 0.1 * oracle.laplacian(u, order)
    assert rel(host(out), ref) <= 1e-12


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("N,c,cycles", [(1, 0.3, 1), (3, 0.05, 2), (15, 0.01, 3), (63, 0.002, 2),
                                        (127, 0.0005, 1)])
def test_mg_fixed_cycles_fp64(H, oracle, order, N, c, cycles):
    """V(2,1) cycles in FP64 equal the oracle's cycles (fixed count)."""
    cfg = H.make_config((N, order, 3))
    ctx = H.Context(cfg)
    b = inputs.random_field(N, seed=1)
    u0 = inputs.random_field(N, seed=2, scale=0.1)
    u = dev(u0)
    H.mg_vcycle(ctx, 0, c, dev(b), u, cycles, -1.0)
    ref, rc, cyc, res = oracle.mg_solve(u0, b, order, c, tol=-1.0, max_cycles=cycles)
    assert rel(host(u), ref) <= 1e-11


@pytest.mark.parametrize("order", [2, 4])
def test_mg_tolerance_and_notconv(H, oracle, order):
    N, c = 31, 0.01
    cfg = H.make_config((N, order, 3))
    ctx = H.Context(cfg)
    b = inputs.random_field(N, seed=3)
    u = dev(np.zeros_like(b))
    rc, st = H.mg_vcycle(ctx, 0, c, dev(b), u, 50, 1e-12)
    ref, orc, ocyc, ores = oracle.mg_solve(np.zeros_like(b), b, order, c, tol=1e-12, max_cycles=50)
    assert st["vcycles"] == ocyc
    assert rel(host(u), ref) <= 1e-11
    assert st["mg_residual"] <= 1e-12
    u2 = dev(np.zeros_like(b))
    rc, st = H.mg_vcycle(ctx, 0, c, dev(b), u2, 2, 1e-14, allow_notconv=True)
    assert rc == H.ENOTCONV and st["notconv"] == 1


@pytest.mark.parametrize("order", [2, 4])
def test_mg_mixed_precision_refinement(H, oracle, order):
    """FP32 V-cycles inside FP64 residual refinement reach the FP64 solution to 1e-9."""
    N, c = 63, 0.002
    cfg = H.make_config((N, order, 3), precision=H.MIXED)
    ctx = H.Context(cfg)
    b = inputs.random_field(N, seed=4)
    u = dev(np.zeros_like(b))
    rc, st = H.mg_vcycle(ctx, 0, c, dev(b), u, 60, 1e-12)
    ref, _, ocyc, _ = oracle.mg_solve(np.zeros_like(b), b, order, c, tol=1e-13, max_cycles=80)
    assert rel(host(u), ref) <= 1e-9
    assert st["vcycles"] <= ocyc + 3


PROB = dict(nu=0.1, forcing=1, kappa=1.0, mg_tol=1e-12, mg_max=50)


@pytest.mark.parametrize("N,order,M", [(31, 2, 3), (15, 4, 5), (63, 4, 5)])
def test_sdc_sweep(H, oracle, N, order, M):
    """One sweep from a spread initial value, then a second one, node by node."""
    cfg = H.make_config((N, order, M), dt=1.0 / 16, mg_tol=1e-12)
    ctx = H.Context(cfg)
    u0 = inputs.smooth_random_field(N, seed=5, kmax=6)
    t0 = 0.25
    H.heat3d_set_state(ctx, 0, 0, t0, u0)
    prob = oracle.Prob(**PROB)
    U, F = oracle.spread(N, order, M, prob, u0)
    for sweep in range(2):
        H.sdc_sweep(ctx, 0, 0, 1)
        U, F, rc, st = oracle.sdc_sweep(N, order, M, prob, t0, 1.0 / 16, U, F)
        out = np.empty((N, N, N))
        for m in range(M):
            H.heat3d_get_node(ctx, 0, 0, m, out)
            assert rel(out, U[m]) <= 1e-11, (sweep, m)
    r = H.heat3d_sdc_residual(ctx, 0, 0)
    ro = oracle.sdc_residual(N, order, M, prob, t0, 1.0 / 16, U, F)
    assert abs(r - ro) <= 1e-11 * max(1.0, ro) + 1e-14


def test_sdc_batched_items_match_single(H, oracle):
    """Three items swept in one batch equal each item swept alone (masks are per item)."""
    N, order, M = 31, 4, 5
    cfg = H.make_config((N, order, M), dt=1.0 / 32, batch=3, mg_tol=1e-11)
    ctx = H.Context(cfg)
    us = [inputs.smooth_random_field(N, seed=s, kmax=5) * (1 + s) for s in range(3)]
    for i, u in enumerate(us):
        H.heat3d_set_state(ctx, 0, i, 0.1 * i, u)
    H.sdc_sweep(ctx, 0, 0, 3)
    got = []
    for i in range(3):
        o = np.empty((N, N, N))
        H.heat3d_get_node(ctx, 0, i, M - 1, o)
        got.append(o)
    for i, u in enumerate(us):
        H.heat3d_set_state(ctx, 0, 0, 0.1 * i, u)
        H.sdc_sweep(ctx, 0, 0, 1)
        o = np.empty((N, N, N))
        H.heat3d_get_node(ctx, 0, 0, M - 1, o)
        assert np.array_equal(o, got[i])


def test_fas_restrict_coarse_sweep_interpolate(H, oracle):
    fine, coarse = (31, 4, 5), (15, 2, 3)
    dt, t0 = 1.0 / 16, 0.5
    cfg = H.make_config(fine, coarse, dt=dt, mg_tol=1e-12)
    ctx = H.Context(cfg)
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


def test_run_config1_sdc(H, oracle):
    """Plain serial SDC at the 31^3 / 7-point / 3-node / dt = 1/8 / 4-sweep setup, T = 1."""
    N = 31
    cfg = H.make_config((N, 2, 3), dt=0.125, T=1.0, sweeps_fine=4, tol_sdc=-1.0, mg_tol=1e-10)
    ctx = H.Context(cfg)
    u0 = inputs.sine_mode(N)
    uT = np.empty_like(u0)
    rc, st = H.pfasst_run(ctx, u0, uT)
    ref, orc, ost = oracle.sdc_run(N, 2, 3, oracle.Prob(mg_tol=1e-10), 0.125, 8, 4, u0)
    assert rel(uT, ref) <= 1e-11
    assert st["sweeps"] == ost["sweeps"] and st["vcycles"] == ost["vcycles"]


def test_run_mlsdc_small(H, oracle):
    fine, coarse = (31, 4, 5), (15, 2, 3)
    cfg = H.make_config(fine, coarse, dt=1 / 64, T=2 / 64, sweeps_fine=2, iters=20, tol_sdc=1e-10,
                        mg_tol=1e-11)
    ctx = H.Context(cfg)
    u0 = inputs.sine_mode(31)
    uT = np.empty_like(u0)
    rc, st = H.pfasst_run(ctx, u0, uT)
    ref, orc, ost = oracle.mlsdc_run(fine, coarse, oracle.Prob(mg_tol=1e-11), 1 / 64, 2, u0,
                                     nsweeps_fine=2, max_iters=20, tol=1e-10)
    assert st["iters"] == ost["iters"]
    assert rel(uT, ref) <= 1e-11


@pytest.mark.parametrize("mg_rel", [0.01, 0.1])
def test_run_mlsdc_adaptive_inner_tolerance(H, oracle, mg_rel):
    """Per-item solver tolerance max(mg_tol, mg_rel x incoming collocation
    residual), on both levels: same iterations and V-cycles as the oracle."""
    fine, coarse = (31, 4, 5), (15, 2, 3)
    cfg = H.make_config(fine, coarse, dt=1 / 64, T=2 / 64, sweeps_fine=2, iters=20, tol_sdc=1e-10,
                        mg_tol=1e-12, mg_rel=mg_rel)
    ctx = H.Context(cfg)
    u0 = inputs.smooth_random_field(31, seed=4, kmax=5)
    uT = np.empty_like(u0)
    rc, st = H.pfasst_run(ctx, u0, uT)
    ref, orc, ost = oracle.mlsdc_run(fine, coarse, oracle.Prob(mg_tol=1e-12, mg_rel=mg_rel), 1 / 64,
                                     2, u0, nsweeps_fine=2, max_iters=20, tol=1e-10)
    assert st["iters"] == ost["iters"] and st["vcycles"] == ost["vcycles"]
    assert rel(uT, ref) <= 1e-11


def test_adaptive_inner_tolerance_mixed_and_batched(H, oracle):
    """Mixed precision with the adaptive tolerance, PFASST with two slices in
    one batch, iterated to residual 1e-11: the result matches the converged
    FP64 oracle to 1e-9."""
    fine, coarse = (31, 4, 5), (15, 2, 3)
    cfg = H.make_config(fine, coarse, dt=1 / 32, T=2 / 32, sweeps_fine=1, slices=2, iters=40,
                        tol_sdc=1e-11, mg_tol=1e-12, mg_rel=0.05, precision=H.MIXED, inner=2)
    ctx = H.Context(cfg)
    u0 = inputs.sine_mode(31)
    uT = np.empty_like(u0)
    rc, st = H.pfasst_run(ctx, u0, uT)
    ref, _, ost = oracle.pfasst_run(fine, coarse, oracle.Prob(mg_tol=1e-12, mg_rel=0.05), 1 / 32,
                                    2, 2, u0, nsweeps_fine=1, max_iters=40, tol=1e-11)
    assert st["residual"] <= 1e-11 and ost["residual"] <= 1e-11
    assert rel(uT, ref) <= 1e-9


def test_adaptive_tolerance_rejects_bad_rel(H):
    for bad in (-0.1, 1.0, float("nan")):
        cfg = H.make_config((15, 2, 3), dt=1 / 8, T=1 / 8, mg_rel=bad)
        with pytest.raises(H.Heat3DError):
            H.Context(cfg)
    with pytest.raises(H.Heat3DError):
        H.Context(H.make_config((15, 2, 3), dt=1 / 8, T=1 / 8, interp=3))
    with pytest.raises(H.Heat3DError):  # the compact stencil is for the fine level only
        H.Context(H.make_config((15, 4, 5), (7, H.COMPACT, 3), dt=1 / 8, T=1 / 8))


@pytest.mark.parametrize("order", [4, 19])
def test_run_mlsdc_cubic_correction_interpolation(H, oracle, order, interp=4):
    """interp = 4 (cubic interpolation of the coarse correction): same
    iterations and V-cycles as the oracle, result to 1e-11."""
    fine, coarse = (31, order, 5), (15, 2, 3)
    cfg = H.make_config(fine, coarse, dt=1 / 64, T=2 / 64, sweeps_fine=2, iters=20, tol_sdc=1e-10,
                        mg_tol=1e-11, interp=interp)
    ctx = H.Context(cfg)
    u0 = inputs.smooth_random_field(31, seed=12, kmax=5)
    uT = np.empty_like(u0)
    rc, st = H.pfasst_run(ctx, u0, uT)
    ref, orc, ost = oracle.mlsdc_run(fine, coarse, oracle.Prob(mg_tol=1e-11, interp=interp), 1 / 64,
                                     2, u0, nsweeps_fine=2, max_iters=20, tol=1e-10)
    assert st["iters"] == ost["iters"] and st["vcycles"] == ost["vcycles"]
    assert rel(uT, ref) <= 1e-11


def test_mlsdc_cubic_two_nodes(H, oracle, interp=4):
    """Two-node levels (M = 2): the cubic interpolation runs as the one-pass
    point-wise kernel (no spare integral fields for the separable passes)."""
    fine, coarse = (31, 4, 2), (15, 2, 2)
    cfg = H.make_config(fine, coarse, dt=1 / 64, T=2 / 64, sweeps_fine=2, iters=20, tol_sdc=1e-10,
                        mg_tol=1e-11, interp=interp)
    ctx = H.Context(cfg)
    u0 = inputs.smooth_random_field(31, seed=25, kmax=5)
    uT = np.empty_like(u0)
    rc, st = H.pfasst_run(ctx, u0, uT)
    ref, orc, ost = oracle.mlsdc_run(fine, coarse, oracle.Prob(mg_tol=1e-11, interp=interp), 1 / 64,
                                     2, u0, nsweeps_fine=2, max_iters=20, tol=1e-10)
    assert st["iters"] == ost["iters"] and st["vcycles"] == ost["vcycles"]
    assert rel(uT, ref) <= 1e-11


def test_pfasst_cubic_interpolation_fixed_iterations(H, oracle, interp=4):
    fine, coarse = (31, 4, 5), (15, 2, 3)
    P, K = 4, 3
    cfg = H.make_config(fine, coarse, dt=1 / 8, T=P / 8, sweeps_fine=1, slices=P, iters=K,
                        tol_sdc=-1.0, mg_tol=1e-12, interp=interp)
    ctx = H.Context(cfg)
    u0 = inputs.smooth_random_field(31, seed=13, kmax=4)
    uT = np.empty_like(u0)
    H.pfasst_run(ctx, u0, uT)
    ref, _, _ = oracle.pfasst_run(fine, coarse, oracle.Prob(mg_tol=1e-12, interp=interp), 1 / 8, P,
                                  P, u0, nsweeps_fine=1, max_iters=K)
    assert rel(uT, ref) <= 1e-11


@pytest.mark.parametrize("P,K", [(4, 3), (8, 2)])
def test_run_pfasst_small(H, oracle, P, K):
    fine, coarse = (15, 4, 5), (7, 2, 3)
    cfg = H.make_config(fine, coarse, dt=1 / 16, T=P / 16, sweeps_fine=1, slices=P, iters=K,
                        tol_sdc=-1.0, mg_tol=1e-12)
    ctx = H.Context(cfg)
    u0 = inputs.smooth_random_field(15, seed=9, kmax=4)
    uT = np.empty_like(u0)
    H.pfasst_run(ctx, u0, uT)
    ref, _, _ = oracle.pfasst_run(fine, coarse, oracle.Prob(mg_tol=1e-12), 1 / 16, P, P, u0,
                                  nsweeps_fine=1, max_iters=K)
    assert rel(uT, ref) <= 1e-11


def test_run_mixed_precision_matches_fp64_oracle(H, oracle):
    fine, coarse = (31, 4, 5), (15, 2, 3)
    cfg = H.make_config(fine, coarse, dt=1 / 32, T=2 / 32, precision=H.MIXED, mg_tol=1e-11)
    ctx = H.Context(cfg)
    u0 = inputs.sine_mode(31)
    uT = np.empty_like(u0)
    H.pfasst_run(ctx, u0, uT)
    ref, _, _ = oracle.mlsdc_run(fine, coarse, oracle.Prob(mg_tol=1e-11), 1 / 32, 2, u0,
                                 nsweeps_fine=2, max_iters=20, tol=1e-10)
    assert rel(uT, ref) <= 1e-9


def test_adaptive_fp32_cycles_per_refinement_match_fp64_oracle(H, oracle):
    """Mixed precision with the number of FP32 V-cycles per FP64 residual
    chosen per refinement step (inner = 0, graph replay, launch sequence):
    the MLSDC result stays within 1e-9 of the FP64 oracle at the same
    residual threshold, with no more V-cycles than 3 per step would take."""
    fine, coarse = (31, 4, 5), (15, 2, 3)
    outs = {}
    for inner in (0, 3):
        cfg = H.make_config(fine, coarse, dt=1 / 32, T=2 / 32, precision=H.MIXED, mg_tol=1e-11,
                            inner=inner, use_graphs=1, persistent=0)
        ctx = H.Context(cfg, stream=torch.cuda.Stream())
        u0 = inputs.sine_mode(31)
        uT = np.empty_like(u0)
        rc, st = H.pfasst_run(ctx, u0, uT)
        outs[inner] = (uT, st)
        ctx.close()
    ref, _, _ = oracle.mlsdc_run(fine, coarse, oracle.Prob(mg_tol=1e-11), 1 / 32, 2, inputs.sine_mode(31),
                                 nsweeps_fine=2, max_iters=20, tol=1e-10)
    uT, st = outs[0]
    assert rel(uT, ref) <= 1e-9
    assert st["residual"] <= 1e-10
    assert st["vcycles"] <= outs[3][1]["vcycles"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graphs_and_autotune_change_nothing(H, oracle, precision):
    """V-cycles replayed from CUDA graphs (private stream), autotuned launch
    shapes, the fused coarse-level kernel and the persistent solve kernel give
    bitwise the same MLSDC result as plain launches with the default shapes;
    the FP64 run also matches the oracle."""
    fine, coarse = (31, 4, 5), (15, 2, 3)
    prec = H.FP64 if precision == "fp64" else H.MIXED
    outs = []
    for graphs, tune, fuse, pers in ((0, 0, 0, 0), (1, 1, 1, 0), (1, 0, 0, 0), (0, 1, 1, 0),
                                     (1, 1, 1, -1)):
        cfg = H.make_config(fine, coarse, dt=1 / 32, T=2 / 32, precision=prec, mg_tol=1e-11,
                            use_graphs=graphs, autotune=tune, fuse_coarse=fuse, persistent=pers)
        ctx = H.Context(cfg, stream=torch.cuda.Stream())
        u0 = inputs.sine_mode(31)
        uT = np.empty_like(u0)
        rc, st = H.pfasst_run(ctx, u0, uT)
        outs.append((uT, st["vcycles"]))
    for uT, v in outs[1:]:
        assert np.array_equal(uT, outs[0][0]) and v == outs[0][1]
    if precision == "fp64":
        ref, _, _ = oracle.mlsdc_run(fine, coarse, oracle.Prob(mg_tol=1e-11), 1 / 32, 2,
                                     inputs.sine_mode(31), nsweeps_fine=2, max_iters=20, tol=1e-10)
        assert rel(outs[1][0], ref) <= 1e-11


SHAPES = [(1, 4), (2, 8), (3, 16), (4, 4), (5, 8), (6, 16), (7, 8), (8, 2), (9, 16), (10, 64),
          (11, 16), (12, 4), (13, 32), (14, 8), (15, 1), (15, 12), (16, 3), (16, 24), (17, 7),
          (17, 64), (18, 5), (18, 16), (15, -1), (19, 1), (19, 12), (20, 3), (20, -1), (21, 7),
          (21, 64), (22, 5), (22, -2), (23, 1), (23, -1), (24, 3), (24, 37), (25, 2), (25, 16),
          (26, 7), (26, -2)]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_every_launch_shape_is_bitwise_identical(H, oracle, precision, monkeypatch):
    """Every stencil launch shape (z-march, the 32-wide tiles, the FP32
    four-points-per-thread tiles, with the z neighbours in shared memory or
    in registers, planes loaded by cp.async or by TMA, with block barriers
    or as a producer/consumer pipeline; chunk lengths below,
    at and above the register kernel's ring period, and wave-fitted) forced
    on all grids with N >= 16 gives
    bitwise the result of the default shapes: PFASST with two slices batched
    (items in one launch), fine 127^3 (a ragged last x group of 3 points)."""
    fine, coarse = (127, 4, 3), (63, 2, 3)
    prec = H.FP64 if precision == "fp64" else H.MIXED

    def run():
        cfg = H.make_config(fine, coarse, dt=1 / 32, T=2 / 32, sweeps_fine=1, slices=2, iters=2,
                            tol_sdc=-1.0, mg_tol=1e-10, precision=prec, autotune=0,
                            inner=2 if prec == H.MIXED else 1)
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


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_every_fusion_depth_is_bitwise_identical(H, precision, monkeypatch):
    """The coarse levels fused into one kernel down from N <= 15, 7, 3 or not
    at all give bitwise the same MLSDC result and V-cycles."""
    prec = H.FP64 if precision == "fp64" else H.MIXED
    outs = []
    for fm in (15, 7, 3, 0):
        monkeypatch.setenv("HEAT3D_FUSE_MAX", str(fm))
        cfg = H.make_config((63, 4, 5), (31, 2, 3), dt=1 / 32, T=2 / 32, precision=prec,
                            mg_tol=1e-11, use_graphs=1, inner=2 if prec == H.MIXED else 1,
                            persistent=0)
        ctx = H.Context(cfg, stream=torch.cuda.Stream())
        u0 = inputs.smooth_random_field(63, seed=23, kmax=5)
        uT = np.empty_like(u0)
        rc, st = H.pfasst_run(ctx, u0, uT)
        outs.append((uT, st["vcycles"]))
    monkeypatch.delenv("HEAT3D_FUSE_MAX")
    for uT, v in outs[1:]:
        assert np.array_equal(uT, outs[0][0]) and v == outs[0][1]


def test_tune_file_records_and_reuses_shapes(H, monkeypatch, tmp_path):
    """HEAT3D_TUNE_FILE: the first context times its shapes and records one
    line per SDC level; a second context takes them from the file (no timing)
    and gives bitwise the same result."""
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("HEAT3D_TUNE_FILE", str(path))
    outs = []
    for _ in range(2):
        cfg = H.make_config((63, 4, 5), (31, 2, 3), dt=1 / 32, T=2 / 32, mg_tol=1e-11, use_graphs=1)
        ctx = H.Context(cfg, stream=torch.cuda.Stream())
        u0 = inputs.smooth_random_field(63, seed=24, kmax=5)
        uT = np.empty_like(u0)
        rc, st = H.pfasst_run(ctx, u0, uT)
        outs.append((uT, st["vcycles"]))
        ctx.close()
    lines = path.read_text().strip().splitlines()
    assert len(lines) == 2  # one per level, written once
    assert [int(x) for x in lines[0].split()[:4]] == [8, 4, 63, 1]
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]
    monkeypatch.delenv("HEAT3D_TUNE_FILE")


def test_chunked_device_stop_rule_matches_host_loop(H, oracle):
    """With graphs the stop rule runs on the device and the host waits once per
    chunk of cycles (4 on grids below 127): identical cycles and results to
    the host-checked loop, for tolerance, fixed-count and cycle-cap solves and
    for MLSDC with several items (PFASST slices)."""
    N, c = 31, 0.01
    b = inputs.random_field(N, seed=21)
    outs = {}
    for graphs in (0, 1):
        ctx = H.Context(H.make_config((N, 4, 3), use_graphs=graphs, persistent=0),
                        stream=torch.cuda.Stream())
        u = dev(np.zeros_like(b))
        rc, st = H.mg_vcycle(ctx, 0, c, dev(b), u, 50, 1e-12)
        uf = dev(np.zeros_like(b))
        H.mg_vcycle(ctx, 0, c, dev(b), uf, 3, -1.0)
        un = dev(np.zeros_like(b))
        rcn, stn = H.mg_vcycle(ctx, 0, c, dev(b), un, 2, 1e-14, allow_notconv=True)
        outs[graphs] = (host(u), st["vcycles"], host(uf), rcn, stn["notconv"], host(un))
    g0, g1 = outs[0], outs[1]
    assert np.array_equal(g0[0], g1[0]) and g0[1] == g1[1]
    assert np.array_equal(g0[2], g1[2]) and np.array_equal(g0[5], g1[5])
    assert g1[3] == H.ENOTCONV and g1[4] == 1
    ref, _, ocyc, _ = oracle.mg_solve(np.zeros_like(b), b, 4, c, tol=1e-12, max_cycles=50)
    assert g1[1] == ocyc
    res = []
    for graphs in (0, 1):
        cfg = H.make_config((31, 4, 5), (15, 2, 3), dt=1 / 16, T=4 / 16, sweeps_fine=1, slices=4,
                            iters=3, tol_sdc=-1.0, mg_tol=1e-11, use_graphs=graphs, persistent=0)
        ctx = H.Context(cfg, stream=torch.cuda.Stream())
        u0 = inputs.smooth_random_field(31, seed=22, kmax=4)
        uT = np.empty_like(u0)
        rc, st = H.pfasst_run(ctx, u0, uT)
        res.append((uT, st["vcycles"]))
    assert np.array_equal(res[0][0], res[1][0]) and res[0][1] == res[1][1]


def test_graph_replay_counts_launches_and_profile(H):
    """Launch counter and the kernel profile include graph replays."""
    N = 63
    cfg = H.make_config((N, 4, 5), dt=1 / 16, T=1 / 16, sweeps_fine=1, tol_sdc=-1.0,
                        use_graphs=1)
    ctx = H.Context(cfg, stream=torch.cuda.Stream())
    u0 = inputs.sine_mode(N)
    uT = np.empty_like(u0)
    H.pfasst_run(ctx, u0, uT)  # captures the graphs
    H.heat3d_profile(ctx, H.PROF_JACOBI_FINE)
    n0 = H.heat3d_kernel_launches()
    rc, st = H.pfasst_run(ctx, u0, uT)
    n1 = H.heat3d_kernel_launches()
    prof = H.heat3d_profile_read(ctx)
    assert n1 - n0 > 10 * st["vcycles"]
    assert prof["launches"] == 2 * st["vcycles"] and prof["ms"] > 0


def test_fp64_probe_reports_a_plausible_rate(H):
    """The FP64 FMA probe (the FP64 stencils' roofline denominator) returns a
    rate between 1e10 and 1e13 FMAs per second, repeatably within 10 %."""
    a = H.heat3d_fp64_probe()
    b = H.heat3d_fp64_probe()
    assert 1e10 < a < 1e13 and abs(a - b) <= 0.1 * max(a, b)
