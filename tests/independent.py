"""Independent constructions used to pin the oracle (not the oracle itself).

Each helper reaches a quantity by a different route from the oracle's code:
spectral (sine-basis) matrices instead of stencil loops, numpy polynomial
integration instead of Lagrange-coefficient expansion, closed-form ODE
solutions instead of time stepping.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import polynomial as P


def eig_1d(N: int, order: int, k):
    """Eigenvalue of the 1-D second-difference operator on sin(k pi x), h = 1/(N+1).

    order 2: (2 cos(theta) - 2) / h^2;  order 4 (wide, odd reflection):
    (-2 cos(2 theta) + 32 cos(theta) - 30) / (12 h^2), theta = k pi h.
    """
    h = 1.0 / (N + 1)
    th = np.asarray(k, dtype=np.float64) * np.pi * h
    if order == 2:
        return (2.0 * np.cos(th) - 2.0) / h**2
    return (-2.0 * np.cos(2 * th) + 32.0 * np.cos(th) - 30.0) / (12.0 * h**2)


def dst_basis(N: int):
    """Orthonormal sine basis: column k-1 is sqrt(2h) sin(k pi x_i)."""
    h = 1.0 / (N + 1)
    i = np.arange(1, N + 1)
    return np.sqrt(2.0 * h) * np.sin(np.outer(i, i) * np.pi * h)


def lap_1d_dense(N: int, order: int):
    """The 1-D operator as V diag(lambda) V^T (exact: sines are its eigenvectors)."""
    V = dst_basis(N)
    lam = eig_1d(N, order, np.arange(1, N + 1))
    return V @ np.diag(lam) @ V.T


def A_dense(N: int, order: int, c: float):
    """I - c (L (x) I (x) I + I (x) L (x) I + I (x) I (x) L) on the z,y,x-ordered vector."""
    L = lap_1d_dense(N, order)
    I = np.eye(N)
    lap = np.kron(np.kron(L, I), I) + np.kron(np.kron(I, L), I) + np.kron(np.kron(I, I), L)
    return np.eye(N**3) - c * lap


def compact_eigs(N: int, k):
    """Eigenvalues of the compact scheme on sin(k1 pi x) sin(k2 pi y) sin(k3 pi z),
    from its symbol with c_a = cos(k_a pi h): the 19-point operator gives
    (-24 + 4 (c1 + c2 + c3) + 4 (c1 c2 + c1 c3 + c2 c3)) / (6 h^2) (faces weigh
    2, edges 1), the weighting matrix (3 + c1 + c2 + c3) / 6.  Returns (lam_L, lam_W)."""
    h = 1.0 / (N + 1)
    c = [np.cos(np.asarray(ka, dtype=np.float64) * np.pi * h) for ka in k]
    s1 = c[0] + c[1] + c[2]
    s2 = c[0] * c[1] + c[0] * c[2] + c[1] * c[2]
    return (-24.0 + 4.0 * s1 + 4.0 * s2) / (6.0 * h * h), (3.0 + s1) / 6.0


def compact_A_dense(N: int, c: float):
    """W - c L of the compact scheme as V diag(lam_W - c lam_L) V^T over the 3-D
    sine basis (sines are its eigenvectors)."""
    V1 = dst_basis(N)
    V = np.kron(np.kron(V1, V1), V1)
    k = np.arange(1, N + 1)
    K3, K2, K1 = np.meshgrid(k, k, k, indexing="ij")  # z, y, x order of the vector
    lamL, lamW = compact_eigs(N, (K1.reshape(-1), K2.reshape(-1), K3.reshape(-1)))
    return V @ np.diag(lamW - c * lamL) @ V.T


def gl_nodes_legendre(M: int):
    """Gauss-Lobatto nodes on [0,1]: ends plus roots of P'_{M-1} (numpy legendre)."""
    from numpy.polynomial import legendre as Lg
    c = np.zeros(M)
    c[M - 1] = 1.0
    r = np.sort(np.real(Lg.legroots(Lg.legder(c))))
    x = np.concatenate([[-1.0], r, [1.0]])
    return 0.5 * (x + 1.0)


def qmatrix_numpy(tau):
    """Q[m][j] = int_0^{tau_m} l_j(s) ds via numpy polyfit of the Lagrange data."""
    M = len(tau)
    Q = np.zeros((M, M))
    for j in range(M):
        y = np.zeros(M)
        y[j] = 1.0
        coef = np.polyfit(tau, y, M - 1)[::-1]  # low -> high
        integ = P.polyint(coef)
        for m in range(M):
            Q[m, j] = P.polyval(tau[m], integ)
    return Q


def forcing_g(t, nu, kappa):
    return -(np.sin(t) - kappa * nu * np.pi**2 * np.cos(t))


def scalar_collocation(lam, a0, t0, dt, nu, kappa, forcing=True):
    """Solve the M=5 or M=3 collocation system of a' = lam a + g(t) exactly.

    a_m = a0 + dt sum_j Q[m][j] (lam a_j + g(t_j)), a dense (M x M) linear solve.
    Returns a function M -> node values."""
    def solve(M):
        tau = gl_nodes_legendre(M)
        Q = qmatrix_numpy(tau)
        g = forcing_g(t0 + dt * tau, nu, kappa) if forcing else np.zeros(M)
        A = np.eye(M) - dt * lam * Q
        rhs = a0 * np.ones(M) + dt * Q @ g
        return np.linalg.solve(A, rhs)
    return solve


def semidiscrete_amplitude(lam, t, nu, kappa, a0=1.0):
    """Exact solution of a' = lam a + g(t), g = -(sin t - kappa nu pi^2 cos t), a(0) = a0.

    With c = -lam, d = kappa nu pi^2: a = A cos t + B sin t + (a0 - A) e^{-c t},
    A = (1 + c d)/(1 + c^2), B = (d - c)/(1 + c^2)."""
    c = -lam
    d = kappa * nu * np.pi**2
    A = (1.0 + c * d) / (1.0 + c * c)
    B = (d - c) / (1.0 + c * c)
    return A * np.cos(t) + B * np.sin(t) + (a0 - A) * np.exp(-c * t)


def lagrange_basis_value(tau, m, s):
    """l_m(s) on the nodes tau, from the product formula."""
    v = 1.0
    for i, ti in enumerate(tau):
        if i != m:
            v *= (s - ti) / (tau[m] - ti)
    return v


def scalar_pfasst(lamF, lamG, MF, MG, dt, P, K, a0, nu, kappa, nsweeps_fine=1,
                  nsweeps_coarse=1, predictor=True, variant=None):
    """Two-level PFASST on one sine mode with both levels on the same mesh
    (coarsening in nodes and stencil order only), so that every field is one
    amplitude and every operator a number: f^I = lam a on each level
    (lamF, lamG = nu times the fine and coarse stencils' eigenvalue on the
    mode), f^E = g(t) (Eq. 3), and the implicit substep is a division.

    Written from Sec. 1.1: the IMEX-Euler sweep
        a_{m+1} = a_m + dt_m (f^I(a_{m+1}) - f^I(a^k_{m+1})) + dt sum_j S_mj f(a^k_j) [+ tau_{m+1} - tau_m],
    the FAS correction tau_m = R(dt Q^F f^F)_{m} - dt Q^G f^G(R a^F)_m in
    cumulative form (spatial restriction = identity here), the correction
    interpolated by Lagrange polynomials in time through the coarse nodes, and
    the PFASST iteration: fine sweeps on every slice, restriction, the coarse
    sweeps slice after slice with each slice starting from the coarse end
    value its predecessor computed in this pass, interpolation, then the fine
    end values forwarded to the next slice's start.  The block starts from the
    initial value spread to every node of every slice, and a predictor pass
    (the same without fine sweeps) runs first.

    variant plants a schedule a reader might take instead (to check that a
    comparison tells them apart): "forward_first" forwards the fine end values
    before the interpolation; "stale_coarse_u0" starts each slice's coarse
    sweep from its predecessor's coarse end value of the previous pass;
    "no_start_correction" leaves the coarse change of the start value out of
    the interpolated correction.

    Returns (end values per slice, fine node values per slice, residual per
    slice) after K iterations."""
    tF, tG = gl_nodes_legendre(MF), gl_nodes_legendre(MG)
    QF, QG = qmatrix_numpy(tF), qmatrix_numpy(tG)
    SF, SG = np.diff(QF, axis=0), np.diff(QG, axis=0)
    jmap = [int(np.argmin(np.abs(tF - t))) for t in tG]
    assert np.allclose(tF[jmap], tG)
    ell = np.array([[lagrange_basis_value(tG, m, s) for m in range(MG)] for s in tF])

    def g(t):
        return forcing_g(t, nu, kappa)

    def sweep(a, lam, tau, S, t0, tauQ=None):
        a = a.copy()
        fold = lam * a + g(t0 + dt * tau)
        for m in range(len(tau) - 1):
            dtm = dt * (tau[m + 1] - tau[m])
            rhs = a[m] - dtm * lam * a[m + 1] + dt * (S[m] @ fold)
            if tauQ is not None:
                rhs += tauQ[m + 1] - tauQ[m]
            a[m + 1] = rhs / (1.0 - dtm * lam)
        return a

    def residual(a, lam, tau, Q, t0):
        f = lam * a + g(t0 + dt * tau)
        return np.abs(a[0] + dt * (Q @ f) - a)[1:].max()

    aF = np.full((P, MF), float(a0))
    aG = np.zeros((P, MG))
    prev_end = np.zeros(P)  # coarse end values of the previous pass
    res = np.zeros(P)
    for it in range(-1, K):
        if it < 0 and not predictor:
            continue
        if it >= 0:
            for p in range(P):
                for _ in range(nsweeps_fine):
                    aF[p] = sweep(aF[p], lamF, tF, SF, p * dt)
        aGr = aF[:, jmap].copy()
        tauQ = np.zeros((P, MG))
        for p in range(P):
            t0 = p * dt
            fF = lamF * aF[p] + g(t0 + dt * tF)
            fG = lamG * aGr[p] + g(t0 + dt * tG)
            tauQ[p] = dt * (QF[jmap] @ fF) - dt * (QG @ fG)
        aG = aGr.copy()
        for p in range(P):
            if p > 0:
                aG[p, 0] = prev_end[p - 1] if variant == "stale_coarse_u0" and it >= 0 else aG[p - 1, MG - 1]
            for _ in range(nsweeps_coarse):
                aG[p] = sweep(aG[p], lamG, tG, SG, p * dt, tauQ[p])
        prev_end = aG[:, MG - 1].copy()
        delta = aG - aGr
        if variant == "no_start_correction":
            delta[:, 0] = 0.0
        if variant == "forward_first":
            for p in range(P - 1, 0, -1):
                aF[p, 0] = aF[p - 1, MF - 1]
        aF = aF + delta @ ell.T
        if variant != "forward_first":
            for p in range(P - 1, 0, -1):
                aF[p, 0] = aF[p - 1, MF - 1]
        if it >= 0:
            res = np.array([residual(aF[p], lamF, tF, QF, p * dt) for p in range(P)])
    return aF[:, MF - 1].copy(), aF, res


def sdc_step_factor(z, M, nsweeps):
    """R(z): the factor by which one step of M-node Gauss-Lobatto SDC (initial
    value spread to every node, nsweeps implicit-Euler sweeps, exact solves,
    no forcing) multiplies a mode of a' = lam a, with z = lam dt (Sec. 1.1,
    the sweep equation in scalar form, step length 1)."""
    tau = gl_nodes_legendre(M)
    S = np.diff(qmatrix_numpy(tau), axis=0)
    a = np.ones(M, dtype=np.complex128 if np.iscomplexobj(z) else np.float64)
    for _ in range(nsweeps):
        f = z * a
        new = a.copy()
        for m in range(M - 1):
            dtm = tau[m + 1] - tau[m]
            new[m + 1] = (new[m] - dtm * f[m + 1] + S[m] @ f) / (1.0 - dtm * z)
        a = new
    return a[-1]


def lap7_eig(N, k):
    """Eigenvalue of the 7-point Laplacian on sin(k1 pi x) sin(k2 pi y) sin(k3 pi z)."""
    return float(sum(eig_1d(N, 2, ka) for ka in k))
