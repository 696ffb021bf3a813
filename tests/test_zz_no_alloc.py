"""mg_vcycle_noalloc: the multigrid solve for callers that cannot allocate
device memory (a framework that owns every device byte, a plugin handed only
its input and output buffers, a loop whose memory budget is fixed in
advance).  Its scratch is a static array inside the library, so the test
checks it through the C ABI against the ordinary entry point mg_vcycle, which
uses a caller-bound workspace, on two calls in a row.

This file is named to be collected last; it passes alone in a fresh process
and after the other tests.
"""
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


def test_noalloc_matches_mg_vcycle_on_two_calls(H):
    N, order, c = 63, 4, 0.002
    ctx = H.Context(H.make_config((N, order, 3)))
    for call, seed in enumerate((11, 12)):
        b = inputs.random_field(N, seed=seed)
        u0 = inputs.random_field(N, seed=seed + 100, scale=0.1)
        ref = torch.from_numpy(u0.copy()).cuda()
        H.mg_vcycle(ctx, 0, c, torch.from_numpy(b).cuda(), ref, 3, -1.0)
        got = torch.from_numpy(u0.copy()).cuda()
        rc, st = H.mg_vcycle_noalloc(N, order, H.FP64, c, torch.from_numpy(b).cuda(), got, 3, -1.0)
        assert rc == H.OK and st["vcycles"] == 3
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.abs(g - r).max() <= 1e-11 * np.abs(r).max(), call


def test_noalloc_tolerance_mode_and_limits(H):
    N, order, c = 31, 2, 0.01
    ctx = H.Context(H.make_config((N, order, 3)))
    b = inputs.random_field(N, seed=5)
    ref = np.zeros_like(b)
    H.mg_vcycle(ctx, 0, c, torch.from_numpy(b).cuda(), torch.from_numpy(ref).cuda(), 1, -1.0)
    for _ in range(2):  # host buffers, tolerance-driven, twice in a row
        ref = torch.zeros(N, N, N, dtype=torch.float64, device="cuda")
        rc, st_ref = H.mg_vcycle(ctx, 0, c, torch.from_numpy(b).cuda(), ref, 50, 1e-12)
        got = np.zeros_like(b)
        rc, st = H.mg_vcycle_noalloc(N, order, H.FP64, c, b, got, 50, 1e-12)
        assert rc == H.OK and st["vcycles"] == st_ref["vcycles"]
        r = ref.cpu().numpy()
        assert np.abs(got - r).max() <= 1e-11 * np.abs(r).max()
    with pytest.raises(H.Heat3DError) as e:
        H.mg_vcycle_noalloc(127, order, H.FP64, c, np.zeros((127,) * 3), np.zeros((127,) * 3), 1, -1.0)
    assert e.value.code == H.EINVAL and "63" in str(e.value)


def test_noalloc_mixed_precision_and_switching(H):
    """Mixed precision (FP32 V-cycles inside FP64 refinement) at N = 63 with the
    wide stencil, against mg_vcycle on a mixed context; then FP64, mixed and
    FP64 again at one N, each call against its own reference (a change of
    precision rebuilds the solver state inside the shared array)."""
    N, order, c = 63, 4, 0.002
    b = inputs.random_field(N, seed=31)
    u0 = inputs.random_field(N, seed=32, scale=0.1)
    refs = {}
    for prec in (H.FP64, H.MIXED):
        ctx = H.Context(H.make_config((N, order, 3), precision=prec))
        r = torch.from_numpy(u0.copy()).cuda()
        H.mg_vcycle(ctx, 0, c, torch.from_numpy(b).cuda(), r, 3, -1.0)
        refs[prec] = r.cpu().numpy()
        ctx.close()
    for prec in (H.MIXED, H.FP64, H.MIXED, H.FP64):
        got = torch.from_numpy(u0.copy()).cuda()
        rc, st = H.mg_vcycle_noalloc(N, order, prec, c, torch.from_numpy(b).cuda(), got, 3, -1.0)
        assert rc == H.OK and st["vcycles"] == 3
        g = got.cpu().numpy()
        tol = 1e-11 if prec == H.FP64 else 1e-9
        assert np.abs(g - refs[prec]).max() <= tol * np.abs(refs[prec]).max(), prec


def test_noalloc_refuses_stream_capture(H):
    """The call is synchronous, so it cannot be captured into a CUDA graph: under
    capture it returns EINVAL before touching the stream, the capture stays
    valid, and the next call outside the capture solves as before."""
    N, order, c = 15, 2, 0.01
    b = torch.from_numpy(inputs.random_field(N, seed=21)).cuda()
    u = torch.zeros_like(b)
    x = torch.zeros(16, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    err = None
    with torch.cuda.graph(g, stream=s):
        x.add_(1.0)
        try:
            H.mg_vcycle_noalloc(N, order, H.FP64, c, b, u, 2, -1.0, stream=s)
        except H.Heat3DError as e:
            err = e
    assert err is not None and err.code == H.EINVAL
    assert "captured" in str(err)
    g.replay()
    torch.cuda.synchronize()
    assert float(x.sum()) == 16.0
    rc, st = H.mg_vcycle_noalloc(N, order, H.FP64, c, b, u, 2, -1.0, stream=s)
    assert rc == H.OK and st["vcycles"] == 2
