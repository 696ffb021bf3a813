"""Serving loop (continuous batching): every result equals the oracle's serial
SDC run of that request, and equals the same request served alone (results do
not depend on what else is in the batch)."""
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


def make_server(H, precision, pool_gb=2.0, max_active=4, sweeps=4):
    pool = torch.empty(int(pool_gb * 2**30), dtype=torch.uint8, device="cuda")
    return H.Server(pool, max_active=max_active, sweeps=sweeps, precision=precision,
                    mg_tol=1e-12), pool


def requests(n=6):
    rs = inputs.request_stream(n, rate=0.0, seed=1307, sizes=(15, 31), horizons=(0.125, 0.25),
                               dt=1.0 / 32)
    return rs


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_served_results_match_oracle_and_solo_runs(H, oracle, precision):
    prec = H.FP64 if precision == "fp64" else H.MIXED
    tol = 1e-11 if precision == "fp64" else 1e-9
    srv, pool = make_server(H, prec)
    reqs = requests()
    tickets = [srv.submit(r) for r in reqs]
    mixed = [srv.wait(t) for t in tickets]
    for r, (u, st) in zip(reqs, mixed):
        u0 = r.initial_value()
        ref, rc, _ = oracle.sdc_run(r.N, 2, 3, oracle.Prob(nu=r.nu, forcing=0, mg_tol=1e-12), r.dt,
                                    int(round(r.T / r.dt)), 4, u0)
        # relative to the initial value: the solutions decay by orders of magnitude while
        # the solver tolerances are absolute
        assert np.abs(u - ref).max() <= tol * np.abs(u0).max(), r
    p50, p99, n = srv.latency()
    assert n == len(reqs) and 0 < p50 <= p99
    srv.close()
    for r, (u, st) in zip(reqs[:3], mixed[:3]):
        solo, pool2 = make_server(H, prec)
        us, _ = solo.wait(solo.submit(r))
        solo.close()
        assert np.array_equal(us, u)


def test_admission_waits_for_memory_and_rejects_impossible(H):
    """A pool that holds one N=31 group at a time still completes requests of
    two sizes (groups are released and re-admitted); a request that can never
    fit is refused with HEAT3D_ENOMEM."""
    pool_bytes = H.group_bytes_estimate(31, max_active=2)
    pool = torch.empty(int(pool_bytes * 1.05), dtype=torch.uint8, device="cuda")
    srv = H.Server(pool, max_active=2, sweeps=2, precision=H.FP64, mg_tol=1e-11)
    reqs = inputs.request_stream(4, rate=0.0, seed=7, sizes=(15, 31), horizons=(0.125,),
                                 dt=1.0 / 16)
    outs = [srv.wait(srv.submit(r))[0] for r in reqs]
    assert all(np.isfinite(o).all() for o in outs)
    big = inputs.request_stream(1, rate=0.0, seed=8, sizes=(255,), horizons=(0.125,))[0]
    with pytest.raises(H.Heat3DError) as e:
        srv.submit(big)
    assert e.value.code == H.ENOMEM
    srv.close()


def served_exact(r, nsweeps=4):
    """The semi-discrete solution the served request must reach: every sine mode
    of the initial value times R(nu lam_k dt)^n, R the scalar 3-node SDC step
    factor with exact solves."""
    from tests import independent as ind
    n = int(round(r.T / r.dt))
    u = np.zeros((r.N,) * 3)
    for k1, k2, k3, a in r.modes:
        z = r.nu * ind.lap7_eig(r.N, (k1, k2, k3)) * r.dt
        u += a * ind.sdc_step_factor(z, 3, nsweeps) ** n * inputs.sine_mode(r.N, k1, k2, k3)
    return u


def test_serving_real_sizes_with_arrivals_in_flight(H):
    """Grid sizes of the serving workload (63^3, 127^3, 255^3), mixed precision:
    small requests submitted while large ones are resident are admitted at
    once, run beside them (each grid size has its own stream) and finish
    first; every result equals the semi-discrete solution of its request to
    1e-9 of its initial value, and equals the same request served alone."""
    import time
    srv, pool = make_server(H, H.MIXED, pool_gb=24.0, max_active=4, sweeps=4)
    big = inputs.request_stream(3, rate=0.0, seed=2024, sizes=(127,), horizons=(1.0,),
                                dt=1.0 / 32)
    big += inputs.request_stream(1, rate=0.0, seed=2025, sizes=(255,), horizons=(0.25,),
                                 dt=1.0 / 32)
    small = inputs.request_stream(3, rate=0.0, seed=2026, sizes=(63,), horizons=(0.25,),
                                  dt=1.0 / 32)
    t_sub, tickets = [], []
    for r in big:
        t_sub.append(time.perf_counter())
        tickets.append(srv.submit(r))
    time.sleep(0.05)
    assert not all(srv.poll(t) for t in tickets), "the first requests finished too early"
    for r in small:
        t_sub.append(time.perf_counter())
        tickets.append(srv.submit(r))
    outs = [srv.wait(t) for t in tickets]
    done = [ts + st["seconds"] for ts, (u, st) in zip(t_sub, outs)]
    assert max(done[len(big):]) < max(done[:len(big)])
    for r, (u, st) in zip(big + small, outs):
        u0 = r.initial_value()
        assert np.abs(u - served_exact(r)).max() <= 1e-9 * np.abs(u0).max(), (r.N, r.T)
    srv.close()
    for r, (u, _) in zip(small[:1] + big[3:], outs[len(big):len(big) + 1] + outs[3:4]):
        solo, pool2 = make_server(H, H.MIXED, pool_gb=8.0, max_active=4, sweeps=4)
        us, _ = solo.wait(solo.submit(r))
        solo.close()
        assert np.array_equal(us, u)
