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


# --------------------------------------------------------------------------
# compact (Mehrstellen) fine stencil: W u' = nu L u + W f (Sec. 1, Sec. 1.2)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("N,k", [(7, (1, 1, 1)), (12, (2, 5, 3)), (1, (1, 1, 1)), (2, (2, 1, 2)),
                                 (15, (15, 1, 8))])
def test_compact_sine_eigenmodes(oracle, N, k):
    """L and W multiply each sine mode by their symbols (faces 2, edges 1 for L;
    centre 6, faces 1 for 12 W), exact to rounding; the mode (N, ..) checks the
    boundary rows."""
    u = inputs.sine_mode(N, *k)
    lamL, lamW = ind.compact_eigs(N, k)
    assert np.abs(oracle.laplacian(u, oracle.COMPACT) - lamL * u).max() <= 1e-12 * abs(lamL) * 10
    assert np.abs(oracle.weight(u, oracle.COMPACT) - lamW * u).max() <= 1e-14


def test_compact_is_fourth_order_consistent(oracle):
    """W^{-1} L on the (1,1,1) mode approximates -3 pi^2 with error O(h^4)."""
    errs = []
    for N in (7, 15, 31):
        lamL, lamW = ind.compact_eigs(N, (1, 1, 1))
        errs.append(abs(lamL / lamW + 3 * np.pi**2))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 4.0) <= 0.1), rates


@pytest.mark.parametrize("N", [1, 2, 3, 5])
def test_compact_operator_equals_spectral_matrix(oracle, N):
    """(W - c L) u for random u equals the sine-basis matrix: every row,
    including edges and corners of the cube."""
    c = 0.37 / (N + 1) ** 2
    A = ind.compact_A_dense(N, c)
    u = inputs.random_field(N, seed=21 + N)
    ref = (A @ u.reshape(-1)).reshape(u.shape)
    out = oracle.apply_A(u, oracle.COMPACT, c)
    assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("N,ch2", [(1, 3.0), (3, 3.0), (7, 3.0), (7, 0.2)])
def test_compact_mg_matches_dense_solve(oracle, N, ch2):
    """Multigrid on W - c L iterated to 1e-14 equals a dense solve."""
    c = ch2 / (N + 1) ** 2
    A = ind.compact_A_dense(N, c)
    b = inputs.random_field(N, seed=6)
    u, rc, cyc, res = oracle.mg_solve(np.zeros_like(b), b, oracle.COMPACT, c, tol=1e-14,
                                      max_cycles=300)
    assert rc == oracle.OK and res <= 1e-14
    ref = np.linalg.solve(A, b.reshape(-1)).reshape(b.shape)
    assert np.abs(u - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


def test_compact_weight_solve(oracle):
    """The weighting-matrix inversion (multigrid with c = 0) on a smooth
    right-hand side reaches the dense W^{-1} b."""
    N = 15
    b = inputs.smooth_random_field(N, seed=2, kmax=4)
    u, rc, cyc, res = oracle.mg_solve(b.copy(), b, oracle.COMPACT, 0.0, tol=1e-13, max_cycles=200)
    assert rc == oracle.OK
    x = np.zeros_like(b)
    for kz in range(1, 5):
        for ky in range(1, 5):
            for kx in range(1, 5):
                m = inputs.sine_mode(N, kx, ky, kz)
                coef = np.sum(b * m) / np.sum(m * m)
                x += coef / ind.compact_eigs(N, (kx, ky, kz))[1] * m
    assert np.abs(u - x).max() <= 1e-11


@pytest.mark.parametrize("N,ch2", [(15, 20.0), (31, 20.0), (31, 1.0)])
def test_compact_mg_contraction(oracle, N, ch2):
    """V(2,1) with omega = 12/11 contracts the compact system's residual by
    at least 0.5 per cycle (diffusion-dominated and balanced c h^-2)."""
    c = ch2 / (N + 1) ** 2
    b = inputs.random_field(N, seed=3)
    u = np.zeros_like(b)
    prev = np.abs(oracle.residual(u, b, oracle.COMPACT, c)).max()
    for _ in range(5):
        u = oracle.vcycle(u, b, oracle.COMPACT, c)
        r = np.abs(oracle.residual(u, b, oracle.COMPACT, c)).max()
        assert r <= 0.5 * prev
        prev = r


# --------------------------------------------------------------------------
# cubic interpolation of the FAS correction (option interp = 4)
# --------------------------------------------------------------------------

def test_cubic_interpolation_properties(oracle):
    """Even fine points take the coarse values; away from the boundary the
    tensor-product 4-point rule reproduces any cubic polynomial exactly
    (numpy polynomial evaluation); on sin(pi x) (odd about both ends, as the
    odd reflection assumes) the error falls like h^4."""
    Nc = 7
    Nf = 2 * Nc + 1
    xc = np.arange(1, Nc + 1) / (Nc + 1)
    xf = np.arange(1, Nf + 1) / (Nf + 1)
    pc = [0.3, -1.2, 0.7, 2.0]  # a cubic, coefficients low -> high
    px = lambda x: np.polynomial.polynomial.polyval(x, pc)
    py = lambda x: np.polynomial.polynomial.polyval(x, [1.0, 0.5, -0.25, 0.125])
    e = px(xc)[None, None, :] * py(xc)[None, :, None] * px(xc)[:, None, None]
    out = oracle.prolong_add_cubic(e, np.zeros((Nf, Nf, Nf)))
    ref = px(xf)[None, None, :] * py(xf)[None, :, None] * px(xf)[:, None, None]
    inner = slice(3, Nf - 3)  # 4-point stencils that stay inside the coarse grid
    assert np.abs(out[inner, inner, inner] - ref[inner, inner, inner]).max() <= 1e-13
    assert np.array_equal(out[1::2, 1::2, 1::2], e)
    errs = []
    for nc in (7, 15, 31):
        nf = 2 * nc + 1
        ec = inputs.sine_mode(nc)
        errs.append(np.abs(oracle.prolong_add_cubic(ec, np.zeros((nf, nf, nf))) -
                           inputs.sine_mode(nf)).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 3.7), (errs, rates)


# --------------------------------------------------------------------------
# 6- and 8-point midpoint rules for the FAS correction (options interp = 6, 8)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("npts", [6, 8])
def test_higher_order_midpoint_rules(oracle, npts):
    """Even fine points take the coarse values; away from the boundary the
    tensor-product npts-point rule reproduces polynomials of degree npts - 1
    exactly (numpy polynomial evaluation); on sin(pi x) the error falls like
    h^npts; the 4-point member of the family is the cubic rule."""
    Nc = 15
    Nf = 2 * Nc + 1
    xc = np.arange(1, Nc + 1) / (Nc + 1)
    xf = np.arange(1, Nf + 1) / (Nf + 1)
    rng = np.random.default_rng(npts)
    pc = rng.standard_normal(npts)  # degree npts - 1, coefficients low -> high
    px = lambda x: np.polynomial.polynomial.polyval(x, pc)
    py = lambda x: np.polynomial.polynomial.polyval(x, pc[::-1])
    e = px(xc)[None, None, :] * py(xc)[None, :, None] * px(xc)[:, None, None]
    out = oracle.prolong_add_lagrange(e, np.zeros((Nf, Nf, Nf)), npts)
    ref = px(xf)[None, None, :] * py(xf)[None, :, None] * px(xf)[:, None, None]
    inner = slice(npts - 1, Nf - npts + 1)  # stencils that stay inside the coarse grid
    assert np.abs(out[inner, inner, inner] - ref[inner, inner, inner]).max() <= 1e-11 * np.abs(ref).max()
    assert np.array_equal(out[1::2, 1::2, 1::2], e)
    errs = []
    for nc in (7, 15, 31):
        nf = 2 * nc + 1
        errs.append(np.abs(oracle.prolong_add_lagrange(inputs.sine_mode(nc), np.zeros((nf, nf, nf)),
                                                       npts) - inputs.sine_mode(nf)).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > npts - 0.3), (errs, rates)
    e4 = inputs.random_field(7, seed=9)
    assert np.array_equal(oracle.prolong_add_lagrange(e4, np.zeros((15, 15, 15)), 4),
                          oracle.prolong_add_cubic(e4, np.zeros((15, 15, 15))))


def test_midpoint_rule_odd_extension_on_small_grids(oracle):
    """On 1- and 3-point coarse lines the 6- and 8-point stencils reach past
    both boundaries, on the 1-point line more than once.  With the odd
    extension about both ends (the symmetry of every sine mode) the error on
    sin(pi x) still falls with every order step (a zero extension makes it
    grow from 4 to 8 points on the 3-point line)."""
    for nc, factor in ((1, 1.8), (3, 5.0)):
        nf = 2 * nc + 1
        errs = [np.abs(oracle.prolong_add_lagrange(inputs.sine_mode(nc), np.zeros((nf, nf, nf)), n)
                       - inputs.sine_mode(nf)).max() for n in (4, 6, 8)]
        assert errs[0] > factor * errs[1] and errs[1] > factor * errs[2], (nc, errs)
    assert errs[2] <= 5e-4
