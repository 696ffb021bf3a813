"""Pins of the oracle's PFASST iterates at a fixed iteration count (CPU only).

Sec. 1.1 describes PFASST as MLSDC sweeps on every time slice with a serial
coarse pass that hands each slice's new coarse end value to the next slice,
and the fine end values sent forward after the sweeps.  The order of the
steps inside an iteration is the reading stated at ``or_pfasst_run``:
fine sweeps, restriction + tau, the serial coarse pass, interpolation of the
correction, then the forward pass of the fine end values.

Two independent routes fix the iterates:
  * On one sine mode with both levels on the same mesh (coarsening in nodes
    and stencil order only), every field is one amplitude and every operator
    a number, so the whole schedule reduces to a scalar recursion written
    out in numpy (``independent.scalar_pfasst``).  The oracle must match it
    slice by slice after K = 1, 2, 3 iterations, and the planted readings a
    reader might take instead (forward pass before the interpolation, the
    coarse chain started from the previous pass's end values, the start
    value's coarse change dropped from the correction) must all miss it.
  * Causality: nothing flows backwards in time, so the first slice after K
    iterations is the first step of MLSDC after K iterations, and the first
    Q slices of a P-slice run are a Q-slice run.
"""
import numpy as np
import pytest

from paper_1307_7867_gb300 import inputs
from tests import independent as ind

NU, KAPPA = 0.1, 1.0


def _lam(N, order):
    """nu times the eigenvalue of the 3-D stencil on the (1,1,1) sine mode."""
    return NU * 3.0 * float(ind.eig_1d(N, order, 1))


def _oracle_slices(oracle, N, P, K, dt, nsweeps_fine, mg_tol):
    prob = oracle.Prob(nu=NU, forcing=1, kappa=KAPPA, mg_tol=mg_tol, mg_max=200)
    u0 = inputs.sine_mode(N)
    _, rc, st = oracle.pfasst_run((N, 4, 5), (N, 2, 3), prob, dt, P, P, u0,
                                  nsweeps_fine=nsweeps_fine, max_iters=K)
    assert rc == oracle.OK
    # amplitude of the mode at every node of every slice, and what is left outside it
    phi = inputs.sine_mode(N)
    U = st["slice_nodes"]
    amp = np.einsum("pmzyx,zyx->pm", U, phi) / (phi * phi).sum()
    rest = float(np.abs(U - amp[:, :, None, None, None] * phi).max())
    return amp, rest, st


@pytest.mark.parametrize("N,mg_tol,tol", [(1, 1e-14, 2e-14), (7, 1e-15, 1e-12)])
@pytest.mark.parametrize("K", [1, 2, 3])
@pytest.mark.parametrize("nsweeps_fine", [1, 2])
def test_pfasst_iterates_equal_scalar_schedule(oracle, N, mg_tol, tol, K, nsweeps_fine):
    """Oracle PFASST (fine wide stencil M=5, coarse 7-point M=3, same mesh) on
    the (1,1,1) mode equals the scalar schedule after K iterations, at every
    node of every slice."""
    P, dt = 4, 0.1875
    amp, rest, _ = _oracle_slices(oracle, N, P, K, dt, nsweeps_fine, mg_tol)
    _, ref, _ = ind.scalar_pfasst(_lam(N, 4), _lam(N, 2), 5, 3, dt, P, K, 1.0, NU, KAPPA,
                                  nsweeps_fine=nsweeps_fine)
    assert rest <= tol  # the mode is an eigenvector of every step
    assert np.abs(amp - ref).max() <= tol * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("variant", ["forward_first", "stale_coarse_u0", "no_start_correction"])
def test_other_schedule_readings_are_told_apart(oracle, variant):
    """Each planted reading changes the iterates by far more than the
    tolerance of the comparison above, so that comparison pins the order."""
    P, dt = 4, 0.1875
    lf, lg = _lam(1, 4), _lam(1, 2)
    for K in (1, 2, 3):
        amp, _, _ = _oracle_slices(oracle, 1, P, K, dt, 1, 1e-14)
        _, good, _ = ind.scalar_pfasst(lf, lg, 5, 3, dt, P, K, 1.0, NU, KAPPA)
        _, bad, _ = ind.scalar_pfasst(lf, lg, 5, 3, dt, P, K, 1.0, NU, KAPPA, variant=variant)
        assert np.abs(amp - good).max() <= 2e-14
        assert np.abs(bad - good).max() >= 1e-6, (variant, K)


def test_scalar_schedule_converges_to_serial_collocation():
    """The scalar recursion itself, iterated to convergence, gives slice by
    slice the serial fine collocation solution (closed form: dense M x M solve
    per step), so the recursion is PFASST and not some other iteration."""
    P, dt = 4, 0.1875
    lf, lg = _lam(1, 4), _lam(1, 2)
    ends, nodes, res = ind.scalar_pfasst(lf, lg, 5, 3, dt, P, 60, 1.0, NU, KAPPA)
    a, serial = 1.0, []
    for p in range(P):
        a = ind.scalar_collocation(lf, a, p * dt, dt, NU, KAPPA)(5)[-1]
        serial.append(a)
    assert res.max() <= 1e-13
    assert np.abs(ends - np.array(serial)).max() <= 1e-13


@pytest.mark.parametrize("K", [1, 3])
def test_first_slice_is_first_mlsdc_step(oracle, K):
    """With real spatial coarsening (15^3 / 7^3) and a non-eigen initial value:
    slice 0 of PFASST after K iterations is the first step of MLSDC after K
    iterations with the same predictor, bit for bit."""
    fine, coarse = (15, 4, 5), (7, 2, 3)
    prob = oracle.Prob(nu=NU, forcing=1, kappa=KAPPA, mg_tol=1e-12, mg_max=100, interp=8)
    u0 = inputs.smooth_random_field(15, seed=11, kmax=4)
    dt = 1 / 8
    _, rc, st = oracle.pfasst_run(fine, coarse, prob, dt, 4, 4, u0, max_iters=K)
    one, rc2, _ = oracle.mlsdc_run(fine, coarse, prob, dt, 1, u0, nsweeps_fine=1,
                                   max_iters=K, tol=-1.0)
    assert rc == rc2 == oracle.OK
    assert np.array_equal(st["slice_nodes"][0, -1], one)


def test_slices_do_not_depend_on_later_slices(oracle):
    """The first 2 slices of a 4-slice run equal a 2-slice run (no backward flow)."""
    fine, coarse = (7, 4, 5), (3, 2, 3)
    prob = oracle.Prob(nu=NU, forcing=1, kappa=KAPPA, mg_tol=1e-12, mg_max=100)
    u0 = inputs.smooth_random_field(7, seed=12, kmax=3)
    _, _, s4 = oracle.pfasst_run(fine, coarse, prob, 1 / 8, 4, 4, u0, max_iters=3)
    _, _, s2 = oracle.pfasst_run(fine, coarse, prob, 1 / 8, 2, 2, u0, max_iters=3)
    assert np.array_equal(s4["slice_nodes"][:2], s2["slice_nodes"])
