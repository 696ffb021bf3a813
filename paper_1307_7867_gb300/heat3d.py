"""Thin ctypes binding of libheat3d.so (the C ABI declared in include/heat3d.h).

Functions carry the ABI's names and only marshal arguments: every step of the
solver runs in the library's CUDA kernels.  PyTorch provides device memory
(the context workspace, device arrays) and the CUDA stream.  There is no CPU
fallback: if the library is missing or no GPU is present, loading fails.

Arrays: dense ``[z][y][x]`` float64 of the N^3 interior values, either CUDA
tensors (device) or numpy arrays / CPU tensors (host); see the header for
which arguments accept which.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libheat3d.so")

OK, EINVAL, ENOMEM, ENOTCONV, ENAN, ETIMEOUT, ECUDA, ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
PROF_OFF, PROF_JACOBI_FINE, PROF_RESID64_FINE, PROF_JACOBI_FINE_STORE = 0, 1, 2, 3
FP64, MIXED = 0, 1
FORCING_NONE, FORCING_PAPER_LITERAL, FORCING_EXACT = 0, 1, 2
COMPACT = 19  # heat3d_level.order of the compact 19-point (Mehrstellen) fine stencil

ABI_FUNCTIONS = [
    "heat3d_config_default", "heat3d_workspace_size", "heat3d_init", "heat3d_bind_workspace",
    "heat3d_destroy", "heat3d_last_error", "heat3d_set_stream", "heat3d_apply_laplacian",
    "mg_vcycle", "heat3d_set_state", "heat3d_get_node", "heat3d_set_node", "sdc_sweep",
    "heat3d_sdc_residual", "heat3d_fas_restrict", "heat3d_fas_interpolate", "pfasst_run",
    "heat3d_set_interval", "heat3d_kernel_launches", "heat3d_profile", "heat3d_profile_read",
    "heat3d_selftest_barrier", "heat3d_selftest_mbarrier", "heat3d_fp64_probe", "mg_vcycle_noalloc",
    "mg_vcycle_noalloc_last_error",
    "heat3d_server_create", "heat3d_submit", "heat3d_poll", "heat3d_wait",
    "heat3d_server_latency", "heat3d_server_destroy", "heat3d_server_last_error",
]


class Heat3DError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"heat3d error {code}: {msg}")
        self.code = code


class Level(C.Structure):
    _fields_ = [("N", C.c_int), ("order", C.c_int), ("M", C.c_int)]


class MG(C.Structure):
    _fields_ = [("nu1", C.c_int), ("nu2", C.c_int), ("max_cycles", C.c_int), ("tol", C.c_double),
                ("inner", C.c_int), ("rel", C.c_double)]


class Config(C.Structure):
    _fields_ = [("nu", C.c_double), ("T", C.c_double), ("dt", C.c_double), ("nlevels", C.c_int),
                ("levels", Level * 2), ("sweeps_fine", C.c_int), ("sweeps_coarse", C.c_int),
                ("slices", C.c_int), ("iters", C.c_int), ("tol_sdc", C.c_double),
                ("predictor", C.c_int), ("mg", MG), ("precision", C.c_int), ("forcing", C.c_int),
                ("batch", C.c_int), ("device", C.c_int), ("stream", C.c_void_p),
                ("use_graphs", C.c_int), ("autotune", C.c_int), ("fuse_coarse", C.c_int),
                ("interp", C.c_int), ("persistent", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("vcycles", C.c_longlong), ("solves", C.c_longlong), ("sweeps", C.c_longlong),
                ("iters", C.c_longlong), ("steps", C.c_longlong), ("notconv", C.c_int),
                ("residual", C.c_double), ("mg_residual", C.c_double), ("seconds", C.c_double),
                ("bytes", C.c_double), ("vcycles_level", C.c_longlong * 2)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["vcycles_level"] = list(self.vcycles_level)
        return d


class ServerConfig(C.Structure):
    _fields_ = [("device", C.c_int), ("pool", C.c_void_p), ("pool_bytes", C.c_size_t),
                ("max_active", C.c_int), ("sweeps", C.c_int), ("precision", C.c_int),
                ("mg", MG)]


class Request(C.Structure):
    _fields_ = [("N", C.c_int), ("nu", C.c_double), ("T", C.c_double), ("dt", C.c_double),
                ("nmodes", C.c_int), ("k", (C.c_int * 3) * 8), ("amp", C.c_double * 8)]


_lib = None


def open_library(path: str = LIB_PATH):
    """dlopens the library at `path`; raises if it is missing (no CPU fallback exists)."""
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run __graft_entry__.build() (no CPU fallback exists)")
    return C.CDLL(path)


def load():
    """Loads libheat3d.so once and declares the ABI's argument types."""
    global _lib
    if _lib is not None:
        return _lib
    L = open_library(LIB_PATH)
    P, I, D, V = C.POINTER, C.c_int, C.c_double, C.c_void_p
    L.heat3d_config_default.argtypes = [P(Config)]
    L.heat3d_config_default.restype = None
    L.heat3d_workspace_size.argtypes = [P(Config), P(C.c_size_t)]
    L.heat3d_init.argtypes = [P(Config), P(V)]
    L.heat3d_bind_workspace.argtypes = [V, V, C.c_size_t]
    L.heat3d_destroy.argtypes = [V]
    L.heat3d_last_error.argtypes = [V]
    L.heat3d_last_error.restype = C.c_char_p
    L.heat3d_set_stream.argtypes = [V, V]
    L.heat3d_apply_laplacian.argtypes = [V, I, V, V]
    L.mg_vcycle.argtypes = [V, I, D, V, V, I, D, P(Stats)]
    L.heat3d_set_state.argtypes = [V, I, I, D, V]
    L.heat3d_get_node.argtypes = [V, I, I, I, V]
    L.heat3d_set_node.argtypes = [V, I, I, I, V]
    L.sdc_sweep.argtypes = [V, I, I, I, P(Stats)]
    L.heat3d_sdc_residual.argtypes = [V, I, I, P(D)]
    L.heat3d_fas_restrict.argtypes = [V, I, I]
    L.heat3d_fas_interpolate.argtypes = [V, I, I]
    L.pfasst_run.argtypes = [V, V, V, P(Stats)]
    L.heat3d_set_interval.argtypes = [V, D, D]
    L.heat3d_kernel_launches.argtypes = []
    L.heat3d_kernel_launches.restype = C.c_longlong
    L.heat3d_profile.argtypes = [V, I]
    L.heat3d_profile_read.argtypes = [V, P(D), P(C.c_longlong), P(D), P(D), P(D)]
    L.heat3d_selftest_barrier.argtypes = [V, I]
    L.heat3d_fp64_probe.argtypes = [V, P(D)]
    L.heat3d_selftest_mbarrier.argtypes = [V, I]
    L.mg_vcycle_noalloc.argtypes = [I, I, I, D, V, V, I, D, V, P(Stats)]
    L.mg_vcycle_noalloc_last_error.argtypes = []
    L.mg_vcycle_noalloc_last_error.restype = C.c_char_p
    if hasattr(L, "heat3d_server_create"):
        L.heat3d_server_create.argtypes = [P(ServerConfig), P(V)]
        L.heat3d_submit.argtypes = [V, P(Request), P(C.c_uint64)]
        L.heat3d_poll.argtypes = [V, C.c_uint64, P(I)]
        L.heat3d_wait.argtypes = [V, C.c_uint64, V, P(Stats)]
        L.heat3d_server_latency.argtypes = [V, P(D), P(D), P(C.c_longlong)]
        L.heat3d_server_destroy.argtypes = [V]
        L.heat3d_server_last_error.argtypes = [V]
        L.heat3d_server_last_error.restype = C.c_char_p
    _lib = L
    return L


def _ptr(a):
    """Device or host address of a float64 array-like (torch tensor or numpy)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        import torch
        assert a.dtype == torch.float64 and a.is_contiguous(), "need a contiguous float64 tensor"
        return C.c_void_p(a.data_ptr())
    assert isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous
    return C.c_void_p(a.ctypes.data)


def _check(rc, ctx=None, allow=()):
    if rc == OK or rc in allow:
        return rc
    msg = load().heat3d_last_error(ctx).decode() if ctx else ""
    raise Heat3DError(rc, msg)


def heat3d_config_default() -> Config:
    cfg = Config()
    load().heat3d_config_default(C.byref(cfg))
    return cfg


def heat3d_workspace_size(cfg: Config) -> int:
    n = C.c_size_t(0)
    _check(load().heat3d_workspace_size(C.byref(cfg), C.byref(n)))
    return n.value


class Context:
    """A heat3d context with a torch-allocated workspace bound to it."""

    def __init__(self, cfg: Config, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("heat3d needs a CUDA device (no CPU fallback)")
        L = load()
        self.cfg = cfg
        dev = torch.device("cuda", cfg.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        cfg.stream = C.c_void_p(self.stream.cuda_stream)
        h = C.c_void_p()
        _check(L.heat3d_init(C.byref(cfg), C.byref(h)))
        self.h = h
        nbytes = heat3d_workspace_size(cfg)
        self.workspace = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=dev)
        _check(L.heat3d_bind_workspace(h, C.c_void_p(self.workspace.data_ptr()), nbytes), h)

    def close(self):
        if getattr(self, "h", None):
            load().heat3d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return load().heat3d_last_error(self.h).decode()


def heat3d_apply_laplacian(ctx: Context, level, u, out):
    return _check(load().heat3d_apply_laplacian(ctx.h, level, _ptr(u), _ptr(out)), ctx.h)


def mg_vcycle(ctx: Context, level, c, rhs, u, max_cycles, tol, allow_notconv=False):
    st = Stats()
    rc = load().mg_vcycle(ctx.h, level, float(c), _ptr(rhs), _ptr(u), int(max_cycles), float(tol),
                          C.byref(st))
    _check(rc, ctx.h, allow=(ENOTCONV,) if allow_notconv else ())
    return rc, st.as_dict()


def heat3d_set_state(ctx: Context, level, item, t0, u0):
    return _check(load().heat3d_set_state(ctx.h, level, item, float(t0), _ptr(u0)), ctx.h)


def heat3d_get_node(ctx: Context, level, item, node, out):
    return _check(load().heat3d_get_node(ctx.h, level, item, node, _ptr(out)), ctx.h)


def heat3d_set_node(ctx: Context, level, item, node, arr):
    return _check(load().heat3d_set_node(ctx.h, level, item, node, _ptr(arr)), ctx.h)


def sdc_sweep(ctx: Context, level, batch_begin, batch_count, allow_notconv=False):
    st = Stats()
    rc = load().sdc_sweep(ctx.h, level, batch_begin, batch_count, C.byref(st))
    _check(rc, ctx.h, allow=(ENOTCONV,) if allow_notconv else ())
    return rc, st.as_dict()


def heat3d_sdc_residual(ctx: Context, level, item) -> float:
    r = C.c_double(0.0)
    _check(load().heat3d_sdc_residual(ctx.h, level, item, C.byref(r)), ctx.h)
    return r.value


def heat3d_fas_restrict(ctx: Context, begin, count):
    return _check(load().heat3d_fas_restrict(ctx.h, begin, count), ctx.h)


def heat3d_fas_interpolate(ctx: Context, begin, count):
    return _check(load().heat3d_fas_interpolate(ctx.h, begin, count), ctx.h)


def pfasst_run(ctx: Context, u0, uT, allow_notconv=False):
    st = Stats()
    rc = load().pfasst_run(ctx.h, _ptr(u0), _ptr(uT), C.byref(st))
    _check(rc, ctx.h, allow=(ENOTCONV,) if allow_notconv else ())
    return rc, st.as_dict()


def make_config(fine, coarse=None, *, nu=0.1, T=1.0, dt=1.0 / 64, sweeps_fine=2, sweeps_coarse=1,
                slices=1, iters=20, tol_sdc=1e-10, predictor=1, nu1=2, nu2=1, max_cycles=50,
                mg_tol=1e-10, precision=FP64, forcing=FORCING_PAPER_LITERAL, batch=1, device=0,
                use_graphs=0, autotune=1, inner=1, fuse_coarse=1, mg_rel=0.0, interp=2,
                persistent=-1) -> Config:
    """fine, coarse: (N, order, M) tuples; coarse None gives single-level SDC."""
    cfg = heat3d_config_default()
    cfg.nu, cfg.T, cfg.dt = nu, T, dt
    cfg.nlevels = 1 if coarse is None else 2
    cfg.levels[0] = Level(*fine)
    if coarse is not None:
        cfg.levels[1] = Level(*coarse)
    cfg.sweeps_fine, cfg.sweeps_coarse = sweeps_fine, sweeps_coarse
    cfg.slices, cfg.iters, cfg.tol_sdc, cfg.predictor = slices, iters, tol_sdc, predictor
    cfg.mg = MG(nu1, nu2, max_cycles, mg_tol, inner, mg_rel)
    cfg.precision, cfg.forcing, cfg.batch, cfg.device = precision, forcing, batch, device
    cfg.use_graphs = use_graphs
    cfg.autotune = autotune
    cfg.fuse_coarse = fuse_coarse
    cfg.interp = interp
    cfg.persistent = persistent
    return cfg


def heat3d_set_interval(ctx: Context, t0, T):
    return _check(load().heat3d_set_interval(ctx.h, float(t0), float(T)), ctx.h)


def heat3d_kernel_launches() -> int:
    return int(load().heat3d_kernel_launches())


def heat3d_profile(ctx: Context, kernel_class):
    return _check(load().heat3d_profile(ctx.h, int(kernel_class)), ctx.h)


def heat3d_profile_read(ctx: Context) -> dict:
    ms, b, dp, fl = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    n = C.c_longlong()
    _check(load().heat3d_profile_read(ctx.h, C.byref(ms), C.byref(n), C.byref(b), C.byref(dp),
                                      C.byref(fl)), ctx.h)
    return {"ms": ms.value, "launches": n.value, "bytes": b.value, "dp_ops": dp.value,
            "flops": fl.value}


def heat3d_fp64_probe(stream=None) -> float:
    """FP64 FMAs per second of the current device (heat3d_fp64_probe)."""
    sp = None if stream is None else C.c_void_p(stream.cuda_stream)
    v = C.c_double(0.0)
    rc = load().heat3d_fp64_probe(sp, C.byref(v))
    if rc != OK:
        raise Heat3DError(rc, "FP64 probe failed")
    return v.value


def heat3d_selftest_mbarrier(arrive, stream=None) -> int:
    """Bounded mbarrier wait self-test: OK if the barrier completes, ETIMEOUT if not."""
    sp = None if stream is None else C.c_void_p(stream.cuda_stream)
    return load().heat3d_selftest_mbarrier(sp, int(arrive))


def heat3d_selftest_barrier(absent_block, stream=None) -> int:
    """Return code of the bounded grid-barrier self-test (OK, or ETIMEOUT when
    block `absent_block` of the four stays away)."""
    sp = C.c_void_p(stream.cuda_stream) if stream is not None else None
    return load().heat3d_selftest_barrier(sp, int(absent_block))


def mg_vcycle_noalloc(N, order, precision, c, rhs, u, max_cycles, tol, stream=None,
                      allow_notconv=False):
    """mg_vcycle without device allocation (static scratch inside the library, N <= 63)."""
    for name, a in (("rhs", rhs), ("u", u)):
        n = a.numel() if hasattr(a, "numel") else np.asarray(a).size
        if n != int(N) ** 3:
            raise ValueError(f"{name} holds {n} values, not N^3 = {int(N) ** 3}")
    st = Stats()
    sp = None
    if stream is not None:
        sp = C.c_void_p(stream.cuda_stream)
    rc = load().mg_vcycle_noalloc(int(N), int(order), int(precision), float(c), _ptr(rhs), _ptr(u),
                                  int(max_cycles), float(tol), sp, C.byref(st))
    if rc != OK and not (allow_notconv and rc == ENOTCONV):
        raise Heat3DError(rc, load().mg_vcycle_noalloc_last_error().decode())
    return rc, st.as_dict()


class Server:
    """Continuous-batching server (heat3d_server_*) over a torch-allocated pool."""

    def __init__(self, pool, max_active=8, sweeps=4, precision=FP64, mg_tol=1e-10,
                 max_cycles=50, nu1=2, nu2=1, inner=1, device=0, mg_rel=0.0):
        self.pool = pool  # keep the memory alive
        cfg = ServerConfig()
        cfg.device = device
        cfg.pool = C.c_void_p(pool.data_ptr())
        cfg.pool_bytes = pool.numel() * pool.element_size()
        cfg.max_active, cfg.sweeps, cfg.precision = max_active, sweeps, precision
        cfg.mg = MG(nu1, nu2, max_cycles, mg_tol, inner, mg_rel)
        h = C.c_void_p()
        rc = load().heat3d_server_create(C.byref(cfg), C.byref(h))
        if rc != OK:
            raise Heat3DError(rc, "server creation failed")
        self.h = h
        self._sizes = {}

    def _err(self, rc):
        raise Heat3DError(rc, load().heat3d_server_last_error(self.h).decode())

    def submit(self, req) -> int:
        """req: paper_1307_7867_gb300.inputs.Request (or anything with N, nu, T, dt, modes)."""
        r = Request()
        r.N, r.nu, r.T, r.dt = req.N, req.nu, req.T, req.dt
        r.nmodes = len(req.modes)
        for m, (k1, k2, k3, a) in enumerate(req.modes):
            r.k[m][0], r.k[m][1], r.k[m][2] = k1, k2, k3
            r.amp[m] = a
        t = C.c_uint64()
        rc = load().heat3d_submit(self.h, C.byref(r), C.byref(t))
        if rc != OK:
            self._err(rc)
        self._sizes[t.value] = req.N
        return t.value

    def poll(self, ticket) -> bool:
        d = C.c_int(0)
        rc = load().heat3d_poll(self.h, C.c_uint64(ticket), C.byref(d))
        if rc != OK:
            self._err(rc)
        return bool(d.value)

    def wait(self, ticket, out=None):
        """Blocks until done; returns (u(T) as a dense N^3 array, stats dict).  `out` may
        be a preallocated numpy array or CUDA tensor of N^3 float64."""
        st = Stats()
        N = self._sizes.pop(ticket, None)
        if out is None:
            if N is None:
                raise Heat3DError(EINVAL, "unknown ticket")
            out = np.empty((N, N, N))
        rc = load().heat3d_wait(self.h, C.c_uint64(ticket), _ptr(out), C.byref(st))
        if rc not in (OK, ENOTCONV):
            self._err(rc)
        return out, st.as_dict()

    def latency(self):
        p50, p99 = C.c_double(), C.c_double()
        n = C.c_longlong()
        load().heat3d_server_latency(self.h, C.byref(p50), C.byref(p99), C.byref(n))
        return p50.value, p99.value, n.value

    def close(self):
        if getattr(self, "h", None):
            load().heat3d_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def group_bytes_estimate(N, max_active=1, precision=FP64):
    """Pool bytes one grid-size group of the server needs (workspace + state)."""
    cfg = make_config((N, 2, 3), precision=precision, batch=max_active)
    n = heat3d_workspace_size(cfg)
    px = (N + 3) // 4 * 4
    fs = (px * N * N + 63) // 64 * 64
    return n + fs * 8 * max_active + 8 * (3 * N * 8 + 8) + 1024
