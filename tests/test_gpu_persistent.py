"""The persistent solve kernel (heat3d_config.persistent): each multigrid
solve of a small grid as one cooperative launch.  It must give bitwise the
solution, V-cycle counts and return codes of the launch sequence (plain
launches and graph replays) for every stop mode (tolerance, fixed count,
cycle cap, NaN), both precisions, both stencils, several items per launch,
other smoothing schedules and inner cycles; FP64 results also match the
oracle.  The bounded grid barrier gives up and reports HEAT3D_ETIMEOUT when a
block stays away, and the device stays usable.
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


def solves(H, N, order, prec, persistent, graphs, nu1=2, nu2=1, inner=1):
    """Tolerance, fixed-count and capped solves of one context."""
    c = 0.2 / (N + 1) ** 2 * 4
    ctx = H.Context(H.make_config((N, order, 3), precision=prec, use_graphs=graphs, nu1=nu1,
                                  nu2=nu2, inner=inner, persistent=persistent),
                    stream=torch.cuda.Stream())
    b = inputs.random_field(N, seed=40 + N)
    u0 = inputs.random_field(N, seed=41 + N, scale=0.1)
    tol = 1e-12 if prec == H.FP64 else 1e-10
    out = []
    u = dev(u0)
    rc, st = H.mg_vcycle(ctx, 0, c, dev(b), u, 50, tol, allow_notconv=True)  # weak V(1,0) may cap
    out.append((host(u), rc, st["vcycles"], st["mg_residual"]))
    u = dev(u0)
    rc, st = H.mg_vcycle(ctx, 0, c, dev(b), u, 3, -1.0)
    out.append((host(u), rc, st["vcycles"], st["mg_residual"]))
    u = dev(np.zeros_like(u0))
    rc, st = H.mg_vcycle(ctx, 0, c, dev(b), u, 2, 1e-15, allow_notconv=True)
    out.append((host(u), rc, st["vcycles"], st["notconv"]))
    ctx.close()
    return out


@pytest.mark.parametrize("N,order,precision", [(15, 2, "fp64"), (31, 2, "fp64"), (31, 4, "fp64"),
                                               (31, 4, "mixed"), (63, 4, "fp64"),
                                               (63, 2, "mixed")])
def test_solve_is_bitwise_the_launch_sequence(H, N, order, precision):
    prec = H.FP64 if precision == "fp64" else H.MIXED
    inner = 2 if prec == H.MIXED else 1
    ref = solves(H, N, order, prec, 0, 0, inner=inner)
    for graphs in (0, 1):
        got = solves(H, N, order, prec, 1, graphs, inner=inner)
        for (ug, rcg, vg, xg), (ur, rcr, vr, xr) in zip(got, ref):
            assert np.array_equal(ug, ur) and rcg == rcr and vg == vr and xg == xr
    assert ref[2][1] == H.ENOTCONV and ref[1][2] == 3 * inner


@pytest.mark.parametrize("nu1,nu2,inner", [(1, 0, 1), (3, 2, 2), (1, 1, 3)])
def test_other_smoothing_schedules(H, nu1, nu2, inner):
    """nu2 = 0 (the separate update step), longer schedules and warm inner cycles."""
    for prec in (H.FP64, H.MIXED):
        ref = solves(H, 31, 4, prec, 0, 1, nu1=nu1, nu2=nu2, inner=inner)
        got = solves(H, 31, 4, prec, 1, 0, nu1=nu1, nu2=nu2, inner=inner)
        for (ug, rcg, vg, xg), (ur, rcr, vr, xr) in zip(got, ref):
            assert np.array_equal(ug, ur) and rcg == rcr and vg == vr and xg == xr


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_mlsdc_and_batched_pfasst(H, oracle, precision):
    """MLSDC 31^3/15^3 (both levels persistent by default) and PFASST with four
    slices batched (four items per launch): the launch sequence's results;
    FP64 MLSDC also matches the oracle to 1e-11."""
    prec = H.FP64 if precision == "fp64" else H.MIXED
    inner = 2 if prec == H.MIXED else 1
    fine, coarse = (31, 4, 5), (15, 2, 3)
    u0 = inputs.smooth_random_field(31, seed=31, kmax=5)
    outs = []
    for persistent in (-1, 0):
        cfg = H.make_config(fine, coarse, dt=1 / 32, T=2 / 32, precision=prec, mg_tol=1e-11,
                            inner=inner, use_graphs=1, persistent=persistent)
        ctx = H.Context(cfg, stream=torch.cuda.Stream())
        uT = np.empty_like(u0)
        rc, st = H.pfasst_run(ctx, u0, uT)
        cfg = H.make_config(fine, coarse, dt=1 / 16, T=4 / 16, sweeps_fine=1, slices=4, iters=3,
                            tol_sdc=-1.0, precision=prec, mg_tol=1e-11, inner=inner, use_graphs=1,
                            persistent=persistent)
        ctx2 = H.Context(cfg, stream=torch.cuda.Stream())
        uP = np.empty_like(u0)
        rc2, st2 = H.pfasst_run(ctx2, u0, uP)
        outs.append((uT, st["vcycles"], uP, st2["vcycles"]))
    (a, va, p, vp), (b, vb, q, vq) = outs
    assert np.array_equal(a, b) and va == vb
    assert np.array_equal(p, q) and vp == vq
    if prec == H.FP64:
        ref, _, _ = oracle.mlsdc_run(fine, coarse, oracle.Prob(mg_tol=1e-11), 1 / 32, 2, u0,
                                     nsweeps_fine=2, max_iters=20, tol=1e-10)
        assert rel(a, ref) <= 1e-11


def test_one_launch_per_solve(H):
    """A persistent solve is one kernel launch whatever its cycle count."""
    N, c = 31, 0.004
    b = inputs.random_field(N, seed=50)
    counts = {}
    for persistent in (1, 0):
        ctx = H.Context(H.make_config((N, 2, 3), persistent=persistent), stream=torch.cuda.Stream())
        u = dev(np.zeros_like(b))
        H.mg_vcycle(ctx, 0, c, dev(b), u, 50, 1e-12)  # warm-up
        u = dev(np.zeros_like(b))
        n0 = H.heat3d_kernel_launches()
        rc, st = H.mg_vcycle(ctx, 0, c, dev(b), u, 50, 1e-12)
        counts[persistent] = (H.heat3d_kernel_launches() - n0, st["vcycles"])
        ctx.close()
    (n1, v1), (n0_, v0) = counts[1], counts[0]
    assert v1 == v0 and v1 >= 5
    assert n1 <= 4  # layout copies around the solve + the solve itself
    assert n0_ >= 6 * v0


def test_nan_reported(H):
    N = 31
    ctx = H.Context(H.make_config((N, 4, 3), persistent=1), stream=torch.cuda.Stream())
    b = inputs.random_field(N, seed=51)
    b[5, 6, 7] = np.nan
    u = dev(np.zeros_like(b))
    with pytest.raises(H.Heat3DError) as e:
        H.mg_vcycle(ctx, 0, 0.01, dev(b), u, 50, 1e-12)
    assert e.value.code == H.ENAN
    b[5, 6, 7] = 0.0  # the context goes on working
    u = dev(np.zeros_like(b))
    rc, st = H.mg_vcycle(ctx, 0, 0.01, dev(b), u, 50, 1e-12)
    assert rc == H.OK and st["mg_residual"] <= 1e-12


def test_bounded_barrier_times_out_and_device_stays_usable(H):
    s = torch.cuda.Stream()
    assert H.heat3d_selftest_barrier(-1, s) == H.OK
    assert H.heat3d_selftest_barrier(2, s) == H.ETIMEOUT
    assert H.heat3d_selftest_barrier(-1, s) == H.OK
    x = torch.ones(1000, device="cuda")
    assert float(x.sum()) == 1000.0


def test_bounded_mbarrier_wait_times_out_and_device_stays_usable(H):
    """The bounded mbarrier wait of the FP32 stencils' TMA plane loader: a
    barrier that nothing completes makes every waiting thread give up after
    about a second; the call reports HEAT3D_ETIMEOUT and the device, and a
    mixed-precision solve, keep working."""
    import time
    s = torch.cuda.Stream()
    assert H.heat3d_selftest_mbarrier(1, s) == H.OK
    t0 = time.perf_counter()
    assert H.heat3d_selftest_mbarrier(0, s) == H.ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    assert H.heat3d_selftest_mbarrier(1, s) == H.OK
    N = 63
    ctx = H.Context(H.make_config((N, 4, 3), precision=H.MIXED))
    b = inputs.random_field(N, seed=52)
    u = torch.zeros(N, N, N, dtype=torch.float64, device="cuda")
    rc, st = H.mg_vcycle(ctx, 0, 0.01, torch.from_numpy(b).cuda(), u, 50, 1e-12)
    assert rc == H.OK and st["mg_residual"] <= 1e-12
