"""ctypes wrapper of the FP64 CPU oracle (``heat3d_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use this module; the product library never
imports, links or calls it.  It shares no code with the CUDA path.

Arrays are numpy float64, C order ``[z][y][x]`` of the N^3 interior values,
x fastest, h = 1/(N+1) and zero Dirichlet boundary values (Sec. 1, Eqs. 1-2).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "heat3d_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_heat3d.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_heat3d_omp.so")

OK, EINVAL, ENOMEM, ENOTCONV = 0, -1, -2, -3
COMPACT = 19  # order code of the compact (Mehrstellen) 19-point stencil


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle with gcc: -O2, no FMA contraction, no fast-math.
    omp=True builds the OpenMP variant (same source, per-point loops spread
    over the host cores; bitwise the same results), used only for timing."""
    out = _LIB_OMP if omp else _LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
                               *(["-fopenmp"] if omp else []), "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


class Level(C.Structure):
    _fields_ = [("N", C.c_int), ("order", C.c_int), ("M", C.c_int)]


class Problem(C.Structure):
    _fields_ = [("nu", C.c_double), ("forcing", C.c_int), ("kappa", C.c_double),
                ("mg_tol", C.c_double), ("mg_max", C.c_int), ("nu1", C.c_int), ("nu2", C.c_int),
                ("mg_rel", C.c_double), ("interp", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("vcycles", C.c_long), ("solves", C.c_long), ("sweeps", C.c_long),
                ("iters", C.c_long), ("residual", C.c_double), ("notconv", C.c_int),
                ("vcycle_points", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class MlsdcOpts(C.Structure):
    _fields_ = [("nsweeps_fine", C.c_int), ("nsweeps_coarse", C.c_int), ("max_iters", C.c_int),
                ("tol", C.c_double), ("predictor", C.c_int)]


_libs = {}
_use_omp = False
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


class openmp:
    """Context manager: the wrappers below call the OpenMP build inside it."""

    def __enter__(self):
        global _use_omp
        self.prev, _use_omp = _use_omp, True
        return self

    def __exit__(self, *exc):
        global _use_omp
        _use_omp = self.prev


def lib():
    L = _libs.get(_use_omp)
    if L is None:
        L = _load(_use_omp)
        _libs[_use_omp] = L
    return L


def _load(omp):
    L = C.CDLL(build(omp=omp))
    P, I, D = C.POINTER, C.c_int, C.c_double
    L.or_laplacian.argtypes = [I, I, _dp, _dp]
    L.or_weight.argtypes = [I, I, _dp, _dp]
    L.or_apply_A.argtypes = [I, I, D, _dp, _dp]
    L.or_residual.argtypes = [I, I, D, _dp, _dp, _dp]
    L.or_jacobi.argtypes = [I, I, D, _dp, _dp, _dp]
    L.or_restrict_fw.argtypes = [I, _dp, _dp]
    L.or_prolong_add.argtypes = [I, _dp, _dp]
    L.or_prolong_add_cubic.argtypes = [I, _dp, _dp]
    L.or_prolong_add_lagrange.argtypes = [I, I, _dp, _dp]
    L.or_vcycle.argtypes = [I, I, D, _dp, _dp, I, I]
    L.or_mg_solve.argtypes = [I, I, D, _dp, _dp, D, I, I, I, P(I), P(D)]
    L.or_mg_solve.restype = I
    L.or_gl_nodes.argtypes = [I, _dp]
    L.or_qmatrix.argtypes = [I, _dp]
    L.or_smatrix.argtypes = [I, _dp]
    L.or_phi.argtypes = [I, _dp]
    L.or_maxabs.argtypes = [C.c_size_t, _dp]
    L.or_maxabs.restype = D
    L.or_eval_F_all.argtypes = [P(Level), P(Problem), _dp, _dp]
    L.or_spread.argtypes = [P(Level), P(Problem), _dp, _dp, _dp]
    L.or_sdc_sweep.argtypes = [P(Level), P(Problem), D, D, _dp, _dp, C.c_void_p, P(Stats)]
    L.or_sdc_sweep.restype = I
    L.or_sdc_residual.argtypes = [P(Level), P(Problem), D, D, _dp, _dp, C.c_void_p]
    L.or_sdc_residual.restype = D
    L.or_sdc_run.argtypes = [P(Level), P(Problem), D, I, I, D, _dp, _dp, P(Stats)]
    L.or_sdc_run.restype = I
    L.or_fas_restrict.argtypes = [P(Level), P(Level), P(Problem), D, D, _dp, _dp, _dp, _dp,
                                  _dp, _dp]
    L.or_fas_restrict.restype = I
    L.or_fas_interpolate.argtypes = [P(Level), P(Level), P(Problem), _dp, _dp, _dp, _dp]
    L.or_fas_interpolate.restype = I
    L.or_mlsdc_run.argtypes = [P(Level), P(Level), P(Problem), D, I, P(MlsdcOpts), _dp, _dp,
                               P(Stats)]
    L.or_mlsdc_run.restype = I
    L.or_pfasst_run.argtypes = [P(Level), P(Level), P(Problem), D, I, I, P(MlsdcOpts), _dp,
                                _dp, C.c_void_p, C.c_void_p, P(Stats)]
    L.or_pfasst_run.restype = I
    return L


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# --------------------------------------------------------------------------
# spatial operators and multigrid (Sec. 1 method of lines; Sec. 1.2)
# --------------------------------------------------------------------------

def laplacian(u, order):
    u = _c(u)
    out = np.empty_like(u)
    lib().or_laplacian(u.shape[0], order, u, out)
    return out


def weight(u, order):
    """W u: the compact scheme's weighting matrix (the identity for orders 2 and 4)."""
    u = _c(u)
    out = np.empty_like(u)
    lib().or_weight(u.shape[0], order, u, out)
    return out


def apply_A(u, order, c):
    u = _c(u)
    out = np.empty_like(u)
    lib().or_apply_A(u.shape[0], order, c, u, out)
    return out


def residual(u, b, order, c):
    u, b = _c(u), _c(b)
    out = np.empty_like(u)
    lib().or_residual(u.shape[0], order, c, u, b, out)
    return out


def jacobi(u, b, order, c):
    u, b = _c(u), _c(b)
    out = np.empty_like(u)
    lib().or_jacobi(u.shape[0], order, c, u, b, out)
    return out


def restrict_fw(r):
    r = _c(r)
    nc = (r.shape[0] - 1) // 2
    out = np.empty((nc, nc, nc))
    lib().or_restrict_fw(r.shape[0], r, out)
    return out


def prolong_add(e, uf):
    e = _c(e)
    uf = _c(uf).copy()
    lib().or_prolong_add(e.shape[0], e, uf)
    return uf


def prolong_add_cubic(e, uf):
    """uf += tensor-product cubic (4-point) interpolation of e (FAS correction, interp = 4)."""
    e = _c(e)
    uf = _c(uf).copy()
    lib().or_prolong_add_cubic(e.shape[0], e, uf)
    return uf


def prolong_add_lagrange(e, uf, npts):
    """uf += tensor-product npts-point midpoint interpolation of e (npts = 4, 6, 8;
    FAS correction with interp = npts)."""
    e = _c(e)
    uf = _c(uf).copy()
    lib().or_prolong_add_lagrange(e.shape[0], int(npts), e, uf)
    return uf


def vcycle(u, b, order, c, nu1=2, nu2=1):
    u = _c(u).copy()
    b = _c(b)
    lib().or_vcycle(u.shape[0], order, c, u, b, nu1, nu2)
    return u


def mg_solve(u, b, order, c, tol=1e-10, max_cycles=50, nu1=2, nu2=1):
    """Returns (u, status, cycles, final max|b - A u|)."""
    u = _c(u).copy()
    b = _c(b)
    cyc = C.c_int(0)
    res = C.c_double(0.0)
    rc = lib().or_mg_solve(u.shape[0], order, c, u, b, tol, max_cycles, nu1, nu2,
                           C.byref(cyc), C.byref(res))
    return u, rc, cyc.value, res.value


# --------------------------------------------------------------------------
# collocation (Sec. 1.1)
# --------------------------------------------------------------------------

def gl_nodes(M):
    t = np.empty(M)
    if lib().or_gl_nodes(M, t) != OK:
        raise ValueError(M)
    return t


def qmatrix(M):
    q = np.empty(M * M)
    lib().or_qmatrix(M, q)
    return q.reshape(M, M)


def smatrix(M):
    s = np.empty(M * M)
    lib().or_smatrix(M, s)
    return s.reshape(M, M)[: M - 1]


def phi(N):
    out = np.empty((N, N, N))
    lib().or_phi(N, out)
    return out


# --------------------------------------------------------------------------
# SDC / MLSDC / PFASST
# --------------------------------------------------------------------------

@dataclass
class Prob:
    nu: float = 0.1
    forcing: int = 1
    kappa: float = 1.0
    mg_tol: float = 1e-10
    mg_max: int = 50
    nu1: int = 2
    nu2: int = 1
    mg_rel: float = 0.0
    interp: int = 2

    def c(self):
        return Problem(self.nu, self.forcing, self.kappa, self.mg_tol, self.mg_max, self.nu1,
                       self.nu2, self.mg_rel, self.interp)


def spread(N, order, M, prob: Prob, u0):
    lv = Level(N, order, M)
    U = np.empty((M, N, N, N))
    F = np.empty((M, N, N, N))
    lib().or_spread(C.byref(lv), C.byref(prob.c()), _c(u0), U, F)
    return U, F


def eval_F_all(N, order, M, prob: Prob, U):
    lv = Level(N, order, M)
    F = np.empty_like(U)
    lib().or_eval_F_all(C.byref(lv), C.byref(prob.c()), _c(U), F)
    return F


def sdc_sweep(N, order, M, prob: Prob, t0, dt, U, F, tauQ=None):
    """One sweep; returns (U, F, status, stats) with fresh arrays."""
    lv = Level(N, order, M)
    U = _c(U).copy()
    F = _c(F).copy()
    tq = None if tauQ is None else _c(tauQ)
    st = Stats()
    rc = lib().or_sdc_sweep(C.byref(lv), C.byref(prob.c()), t0, dt, U, F, _ptr(tq), C.byref(st))
    return U, F, rc, st.as_dict()


def sdc_residual(N, order, M, prob: Prob, t0, dt, U, F, tauQ=None):
    lv = Level(N, order, M)
    tq = None if tauQ is None else _c(tauQ)
    return lib().or_sdc_residual(C.byref(lv), C.byref(prob.c()), t0, dt, _c(U), _c(F), _ptr(tq))


def sdc_run(N, order, M, prob: Prob, dt, nsteps, nsweeps, u0, tol=-1.0):
    lv = Level(N, order, M)
    uT = np.empty((N, N, N))
    st = Stats()
    rc = lib().or_sdc_run(C.byref(lv), C.byref(prob.c()), dt, nsteps, nsweeps, tol, _c(u0), uT,
                          C.byref(st))
    return uT, rc, st.as_dict()


def fas_restrict(fine, coarse, prob: Prob, t0, dt, UF, FF):
    """fine, coarse: (N, order, M).  Returns (UG, FG, UGr, tauQ)."""
    lf, lg = Level(*fine), Level(*coarse)
    NG, MG = coarse[0], coarse[2]
    UG = np.empty((MG, NG, NG, NG))
    FG, UGr, tQ = np.empty_like(UG), np.empty_like(UG), np.empty_like(UG)
    rc = lib().or_fas_restrict(C.byref(lf), C.byref(lg), C.byref(prob.c()), t0, dt, _c(UF),
                               _c(FF), UG, FG, UGr, tQ)
    if rc != OK:
        raise ValueError(rc)
    return UG, FG, UGr, tQ


def fas_interpolate(fine, coarse, prob: Prob, UG, UGr, UF):
    lf, lg = Level(*fine), Level(*coarse)
    UF = _c(UF).copy()
    FF = np.empty_like(UF)
    rc = lib().or_fas_interpolate(C.byref(lf), C.byref(lg), C.byref(prob.c()), _c(UG), _c(UGr),
                                  UF, FF)
    if rc != OK:
        raise ValueError(rc)
    return UF, FF


def mlsdc_run(fine, coarse, prob: Prob, dt, nsteps, u0, nsweeps_fine=2, nsweeps_coarse=1,
              max_iters=20, tol=1e-10, predictor=1):
    lf, lg = Level(*fine), Level(*coarse)
    N = fine[0]
    uT = np.empty((N, N, N))
    st = Stats()
    o = MlsdcOpts(nsweeps_fine, nsweeps_coarse, max_iters, tol, predictor)
    rc = lib().or_mlsdc_run(C.byref(lf), C.byref(lg), C.byref(prob.c()), dt, nsteps, C.byref(o),
                            _c(u0), uT, C.byref(st))
    return uT, rc, st.as_dict()


def pfasst_run(fine, coarse, prob: Prob, dt, nsteps, nslices, u0, nsweeps_fine=1,
               nsweeps_coarse=1, max_iters=5, tol=-1.0, predictor=1):
    lf, lg = Level(*fine), Level(*coarse)
    N = fine[0]
    uT = np.empty((N, N, N))
    sres = np.zeros(nslices)
    snodes = np.zeros((nslices, fine[2], N, N, N))
    st = Stats()
    o = MlsdcOpts(nsweeps_fine, nsweeps_coarse, max_iters, tol, predictor)
    rc = lib().or_pfasst_run(C.byref(lf), C.byref(lg), C.byref(prob.c()), dt, nsteps, nslices,
                             C.byref(o), _c(u0), uT, _ptr(sres), _ptr(snodes), C.byref(st))
    d = st.as_dict()
    d["slice_residuals"] = sres
    d["slice_nodes"] = snodes  # fine node values of every slice of the last block
    d["slice_end"] = snodes[:, -1]
    return uT, rc, d
