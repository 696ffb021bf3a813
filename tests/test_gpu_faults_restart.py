"""Failure detection without any GPU fault (bad arguments, NaN inputs, the
multigrid cycle cap) and restart equivalence: integrating [0, 2 dt] equals
integrating [0, dt], keeping u(dt) on the host, and restarting from it."""
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


@pytest.mark.parametrize("levels", [1, 2])
def test_restart_from_saved_state_is_bitwise_identical(H, levels):
    fine, coarse = (31, 4, 5), ((15, 2, 3) if levels == 2 else None)
    cfg = H.make_config(fine, coarse, dt=1 / 32, T=2 / 32, sweeps_fine=2 if levels == 2 else 4,
                        tol_sdc=1e-10 if levels == 2 else -1.0, mg_tol=1e-11)
    ctx = H.Context(cfg)
    u0 = inputs.smooth_random_field(31, seed=12, kmax=5)
    full = np.empty_like(u0)
    H.pfasst_run(ctx, u0, full)
    half = np.empty_like(u0)
    H.heat3d_set_interval(ctx, 0.0, 1 / 32)
    H.pfasst_run(ctx, u0, half)
    again = np.empty_like(u0)
    H.heat3d_set_interval(ctx, 1 / 32, 1 / 32)
    H.pfasst_run(ctx, half, again)
    assert np.array_equal(again, full)


def test_nan_input_is_reported_not_propagated_silently(H):
    N = 15
    ctx = H.Context(H.make_config((N, 2, 3), dt=1 / 16, T=1 / 16, sweeps_fine=2, tol_sdc=-1.0))
    u0 = inputs.sine_mode(N)
    u0[3, 4, 5] = np.nan
    uT = np.empty_like(u0)
    with pytest.raises(H.Heat3DError) as e:
        H.pfasst_run(ctx, u0, uT)
    assert e.value.code == H.ENAN
    # the context stays usable after the error
    ok = np.empty_like(u0)
    H.pfasst_run(ctx, inputs.sine_mode(N), ok)
    assert np.isfinite(ok).all()


def test_bad_configurations_are_rejected(H):
    for kwargs in (dict(fine=(30, 2, 3)), dict(fine=(31, 3, 3)), dict(fine=(31, 2, 7)),
                   dict(fine=(31, 2, 3), coarse=(7, 2, 3)), dict(fine=(31, 4, 5), coarse=(15, 2, 4))):
        fine = kwargs.pop("fine")
        coarse = kwargs.pop("coarse", None)
        cfg = H.make_config(fine, coarse)
        with pytest.raises(H.Heat3DError) as e:
            H.Context(cfg)
        assert e.value.code == H.EINVAL
    ctx = H.Context(H.make_config((15, 2, 3), dt=1 / 16, T=0.1))
    with pytest.raises(H.Heat3DError) as e:  # T is not a multiple of dt
        H.pfasst_run(ctx, inputs.sine_mode(15), np.empty((15, 15, 15)))
    assert e.value.code == H.EINVAL


def test_cycle_cap_surfaces_as_not_converged_in_a_sweep(H):
    N = 31
    cfg = H.make_config((N, 4, 5), dt=1 / 8, mg_tol=1e-15, max_cycles=2)
    ctx = H.Context(cfg)
    H.heat3d_set_state(ctx, 0, 0, 0.0, inputs.smooth_random_field(N, seed=3, kmax=6))
    rc, st = H.sdc_sweep(ctx, 0, 0, 1, allow_notconv=True)
    assert rc == H.ENOTCONV and st["notconv"] >= 1
