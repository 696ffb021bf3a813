"""Host-side checks of the C ABI that need no GPU: the Python mirror of
heat3d_config has the C layout, heat3d_config_default sets the documented
defaults, and heat3d_init / heat3d_workspace_size validate a configuration
(no CUDA call happens before a workspace is bound)."""
import ctypes as C

import pytest


@pytest.fixture(scope="module")
def H():
    from paper_1307_7867_gb300 import build, heat3d
    build.build()
    heat3d.load()
    return heat3d


def test_config_mirror_has_the_c_layout(H):
    """heat3d_config_default writes exactly sizeof(Config) bytes: a sentinel
    after the struct survives and the last field holds its default."""
    n = C.sizeof(H.Config)
    buf = (C.c_ubyte * (n + 64))(*([0xA5] * (n + 64)))
    H.load().heat3d_config_default(C.cast(buf, C.POINTER(H.Config)))
    assert all(b == 0xA5 for b in bytes(buf)[n:])
    cfg = H.Config.from_buffer(buf)
    assert cfg.persistent == -1 and cfg.interp == 2 and cfg.fuse_coarse == 1


def test_defaults(H):
    cfg = H.heat3d_config_default()
    assert cfg.nu == 0.1 and cfg.nlevels == 2 and cfg.levels[0].N == 31
    assert (cfg.mg.nu1, cfg.mg.nu2, cfg.mg.max_cycles, cfg.mg.inner) == (2, 1, 50, 1)
    assert cfg.precision == H.FP64 and cfg.use_graphs == 0 and cfg.autotune == 1


def init_rc(H, cfg):
    ctx = C.c_void_p()
    rc = H.load().heat3d_init(C.byref(cfg), C.byref(ctx))
    if rc == H.OK:
        assert H.load().heat3d_destroy(ctx) == H.OK
    return rc


@pytest.mark.parametrize("field,value,ok", [
    ("persistent", -1, True), ("persistent", 0, True), ("persistent", 1, True),
    ("persistent", 2, False), ("persistent", -2, False),
    ("interp", 4, True), ("interp", 3, False),
    ("precision", 7, False), ("slices", 0, False),
])
def test_init_validates_options(H, field, value, ok):
    cfg = H.make_config((31, 4, 5), (15, 2, 3))
    setattr(cfg, field, value)
    assert (init_rc(H, cfg) == H.OK) == ok
    size = C.c_size_t()
    rc = H.load().heat3d_workspace_size(C.byref(cfg), C.byref(size))
    assert (rc == H.OK) == ok and (not ok or size.value > 0)


@pytest.mark.parametrize("fine,coarse,ok", [
    ((31, 4, 5), (15, 2, 3), True), ((31, 19, 5), (15, 2, 3), True),  # 19: compact
    ((31, 2, 3), (15, 19, 3), False),  # compact only on the fine level
    ((30, 2, 3), None, False),         # N must be 2^k - 1
    ((31, 6, 3), None, False),         # unknown order
    ((31, 2, 6), None, False),         # at most 5 nodes
    ((31, 4, 5), (7, 2, 3), False),    # coarse N must be (N - 1) / 2 or N
])
def test_init_validates_levels(H, fine, coarse, ok):
    cfg = H.make_config(fine, coarse)
    assert (init_rc(H, cfg) == H.OK) == ok


def test_mg_settings_validated(H):
    for nu1, nu2, cap, rel, ok in ((2, 1, 50, 0.0, True), (0, 1, 50, 0.0, False),
                                   (2, -1, 50, 0.0, False), (2, 1, 0, 0.0, False),
                                   (2, 1, 50, 1.0, False), (1, 0, 1, 0.5, True)):
        cfg = H.make_config((31, 2, 3), nu1=nu1, nu2=nu2, max_cycles=cap, mg_rel=rel)
        assert (init_rc(H, cfg) == H.OK) == ok


def test_barrier_selftest_rejects_bad_block_without_a_launch(H):
    assert H.heat3d_selftest_barrier(4) == H.EINVAL
    assert H.heat3d_selftest_barrier(-2) == H.EINVAL
