"""Pins of the oracle's spatial operators and multigrid (CPU only).

Paper: Sec. 1 (method of lines; 2nd- and 4th-order Laplacians) and Sec. 1.2
(multigrid solve of the implicit systems, coarsest grid of one unknown).
"""
import numpy as np
import pytest

from paper_1307_7867_gb300 import inputs
from tests import independent as ind

pytestmark = pytest.mark.filterwarnings("ignore")


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("N,k", [(7, (1, 1, 1)), (12, (2, 5, 3)), (31, (1, 3, 7)), (1, (1, 1, 1)),
                                 (2, (2, 1, 2))])
def test_laplacian_sine_eigenmodes(oracle, order, N, k):
    """Delta_h sin(k.pi x) = sum_axes lambda(k_a) sin(k.pi x), exact to rounding."""
    u = inputs.sine_mode(N, *k)
    lam = sum(ind.eig_1d(N, order, ka) for ka in k)
    out = oracle.laplacian(u, order)
    assert np.abs(out - lam * u).max() <= 1e-12 * abs(lam) * max(1.0, np.abs(u).max()) * 10


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("N", [1, 2, 3, 5, 7])
def test_operator_equals_spectral_matrix(oracle, order, N):
    """A u for random u equals the Kronecker-sum matrix built from the sine basis,
    which pins every row, including the boundary rows and the wide stencil's
    odd-reflection ghosts."""
    c = 0.37
    A = ind.A_dense(N, order, c)
    u = inputs.random_field(N, seed=11 + N)
    out = oracle.apply_A(u, order, c)
    ref = (A @ u.reshape(-1)).reshape(u.shape)
    assert np.abs(out - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("N", [1, 3, 7])
def test_mg_solve_matches_dense_solve(oracle, order, N):
    """Multigrid iterated to 1e-14 equals a dense LU solve of (I - c Delta_h) u = b."""
    c = 0.05
    A = ind.A_dense(N, order, c)
    b = inputs.random_field(N, seed=5)
    u, rc, cyc, res = oracle.mg_solve(np.zeros_like(b), b, order, c, tol=1e-14, max_cycles=200)
    assert rc == oracle.OK and res <= 1e-14
    ref = np.linalg.solve(A, b.reshape(-1)).reshape(b.shape)
    assert np.abs(u - ref).max() <= 1e-13
    if N == 1:
        assert cyc == 1  # one exact solve on the one-unknown grid


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("N,c", [(15, 0.05), (31, 0.00625), (31, 1.0)])
def test_mg_contraction(oracle, order, N, c):
    """The max-norm residual drops at every V(2,1) cycle by a factor <= 0.5
    (damped Jacobi V(2,1); measured factors are 0.2-0.4)."""
    b = inputs.random_field(N, seed=3)
    u = np.zeros_like(b)
    prev = np.abs(oracle.residual(u, b, order, c)).max()
    for _ in range(6):
        u = oracle.vcycle(u, b, order, c)
        r = np.abs(oracle.residual(u, b, order, c)).max()
        assert r <= 0.5 * prev
        prev = r


def test_mg_cycle_cap_reports_not_converged(oracle):
    b = inputs.random_field(15, seed=1)
    u, rc, cyc, res = oracle.mg_solve(np.zeros_like(b), b, 2, 0.1, tol=1e-14, max_cycles=2)
    assert rc == oracle.ENOTCONV and cyc == 2 and res > 1e-14
    u2, rc2, cyc2, _ = oracle.mg_solve(np.zeros_like(b), b, 2, 0.1, tol=-1.0, max_cycles=3)
    assert rc2 == oracle.OK and cyc2 == 3


@pytest.mark.parametrize("order", [2, 4])
def test_jacobi_on_eigenmode_and_fixed_point(oracle, order):
    """One damped-Jacobi sweep multiplies a sine mode (b = 0) by
    1 - omega (1 - c lambda)/D, and leaves the exact solution unchanged."""
    N, c = 9, 0.02
    h = 1.0 / (N + 1)
    k = (2, 3, 1)
    u = inputs.sine_mode(N, *k)
    lam = sum(ind.eig_1d(N, order, ka) for ka in k)
    omega, D = (6 / 7, 1 + 6 * c / h**2) if order == 2 else (9 / 11, 1 + 7.5 * c / h**2)
    out = oracle.jacobi(u, np.zeros_like(u), order, c)
    assert np.abs(out - (1 - omega * (1 - c * lam) / D) * u).max() <= 1e-13
    A = ind.A_dense(5, order, c)
    b = inputs.random_field(5, seed=2)
    ustar = np.linalg.solve(A, b.reshape(-1)).reshape(b.shape)
    assert np.abs(oracle.jacobi(ustar, b, order, c) - ustar).max() <= 1e-13


def test_full_weighting_properties(oracle):
    """Full weighting keeps constants, is 1/8 times the adjoint of trilinear
    prolongation, and the prolongation equals per-axis piecewise-linear
    interpolation (numpy.interp) of the coarse values with zero boundary."""
    Nc = 7
    Nf = 2 * Nc + 1
    ones = np.ones((Nf, Nf, Nf))
    assert np.abs(oracle.restrict_fw(ones) - 1.0).max() == 0.0
    r = inputs.random_field(Nf, seed=8)
    e = inputs.random_field(Nc, seed=9)
    lhs = np.sum(oracle.restrict_fw(r) * e)
    rhs = np.sum(r * oracle.prolong_add(e, np.zeros((Nf, Nf, Nf)))) / 8.0
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # tensor-product piecewise-linear interpolation through numpy.interp
    xc = np.arange(0, Nc + 2) / (Nc + 1)
    xf = np.arange(1, Nf + 1) / (Nf + 1)
    ep = np.pad(e, 1)  # zero boundary values
    t = np.apply_along_axis(lambda v: np.interp(xf, xc, v), 2, ep)
    t = np.apply_along_axis(lambda v: np.interp(xf, xc, v), 1, t)
    t = np.apply_along_axis(lambda v: np.interp(xf, xc, v), 0, t)
    ref = t  # shape (Nf, Nf, Nf): interpolated from the padded coarse grid
    out = oracle.prolong_add(e, np.zeros((Nf, Nf, Nf)))
    assert np.abs(out - ref).max() <= 1e-14
