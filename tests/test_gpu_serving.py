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
