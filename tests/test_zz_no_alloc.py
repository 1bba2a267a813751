"""The allocation-free depth -> points entry point, called through the C ABI.

It serves callers that cannot allocate device memory when they need the result (a tracking
loop with a hard deadline, an application whose own pool owns the device, code that may not
allocate after initialisation).  Its scratch is a fixed array inside the library, shared by
all calls, so two calls in a row must each match the allocating entry point exactly (the
second call must not see anything left over from the first).  Collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from synth import Intrinsics, add_depth_noise, circle_poses, make_room, raycast_depth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_12550_b300 as g
    return g


def _image(seed, W, H, holes):
    intr = Intrinsics(W, H, 0.5 * W, 0.5 * W, (W - 1) / 2, (H - 1) / 2)
    scene = make_room(seed)
    rng = np.random.default_rng(seed)
    P = circle_poses(rng, scene, 1)[0]
    d = add_depth_noise(raycast_depth(scene, P, intr), rng, 1e-3, dropout=holes)
    d[rng.random(d.shape) < holes] = np.nan
    return intr, d


def _noalloc_via_abi(g, depth, intr, stride, cap, with_z=True, with_total=True):
    """Direct ctypes call of gsicp_depth_to_points_noalloc with caller-owned buffers; z and the
    unclamped count are passed as NULL when not wanted."""
    pts = torch.full((cap, 3), np.nan, device="cuda", dtype=torch.float32)
    z = torch.full((cap,), np.nan, device="cuda", dtype=torch.float32) if with_z else None
    n = torch.full((1,), -1, device="cuda", dtype=torch.int32)
    total = torch.full((1,), -1, device="cuda", dtype=torch.int32) if with_total else None
    H, W = depth.shape
    fi = (C.c_float * 4)(*[float(v) for v in intr])
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = (lambda t: C.c_void_p(t.data_ptr()) if t is not None else None)
    st = g.lib.gsicp_depth_to_points_noalloc(ptr(depth), W, H, fi, stride, 0.1, 10.0, ptr(pts), ptr(z), cap,
                                             ptr(n), ptr(total), stream)
    assert st == 0, g.gsicp_last_error()
    torch.cuda.synchronize()
    k = int(n.item())
    return (pts[:k].cpu().numpy(), z[:k].cpu().numpy() if with_z else None, k,
            int(total.item()) if with_total else None)


def test_noalloc_matches_allocating_entry_point_on_two_calls(g):
    """Three calls in a row share the library's array: a 1200 x 680 frame, a larger sample grid
    (640 x 480 at stride 1), then a smaller one again (320 x 240 at stride 2) with the capacity
    below the number of valid samples, the order in which counts or offsets left over from a
    larger call would show.  Each call equals the allocating entry point bit for bit (the a1 bar)."""
    ctx = g.Context()
    cases = [(_image(3, 1200, 680, 0.0), 2, None), (_image(4, 640, 480, 0.05), 1, None),
             (_image(6, 320, 240, 0.1), 2, 5000)]
    for (intr, depth), stride, cap in cases:
        d = torch.from_numpy(depth).cuda()
        H, W = depth.shape
        full = ((W + stride - 1) // stride) * ((H + stride - 1) // stride)
        pts_ref, z_ref = g.gsicp_depth_to_points(ctx, d, intr.as_array(), stride, 0.1, 10.0)
        n_ref = pts_ref.shape[0]
        cap = full if cap is None else cap
        pts, z, k, total = _noalloc_via_abi(g, d, intr.as_array(), stride, cap)
        assert total == n_ref and k == min(cap, n_ref)
        if cap < n_ref:
            assert k == cap  # clamped: the first cap points in row-major order
        np.testing.assert_array_equal(pts, pts_ref[:k].cpu().numpy())
        np.testing.assert_array_equal(z, z_ref[:k].cpu().numpy())
    ctx.close()


def test_noalloc_null_depths_and_total(g):
    """z and the unclamped count are optional (NULL): the points still equal the allocating path's."""
    ctx = g.Context()
    intr, depth = _image(7, 640, 480, 0.02)
    d = torch.from_numpy(depth).cuda()
    pts_ref, _ = g.gsicp_depth_to_points(ctx, d, intr.as_array(), 2, 0.1, 10.0)
    pts, z, k, total = _noalloc_via_abi(g, d, intr.as_array(), 2, 320 * 240, with_z=False, with_total=False)
    assert z is None and total is None and k == pts_ref.shape[0]
    np.testing.assert_array_equal(pts, pts_ref.cpu().numpy())
    ctx.close()


def test_noalloc_allocates_nothing(g):
    """Once the library's module is loaded in this context (the first call, which also looks up
    the array's address), further calls of any admissible size leave the device's free memory and
    torch's allocator exactly as they were: no device allocation happens inside them."""
    intr, depth = _image(8, 640, 480, 0.0)
    d = torch.from_numpy(depth).cuda()
    cap = 640 * 480
    pts = torch.empty((cap, 3), device="cuda", dtype=torch.float32)
    z = torch.empty((cap,), device="cuda", dtype=torch.float32)
    n = torch.zeros((1,), device="cuda", dtype=torch.int32)
    total = torch.zeros((1,), device="cuda", dtype=torch.int32)
    g.gsicp_depth_to_points_noalloc(d, intr.as_array(), 2, 0.1, 10.0, pts, z, n, total)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for stride in (1, 2, 3, 1):
        g.gsicp_depth_to_points_noalloc(d, intr.as_array(), stride, 0.1, 10.0, pts, z, n, total)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert int(total.item()) == int(np.sum(np.isfinite(depth) & (depth >= 0.1) & (depth <= 10.0)))


def test_noalloc_capacity_and_size_limit(g):
    intr, depth = _image(5, 320, 240, 0.0)
    d = torch.from_numpy(depth).cuda()
    pts, z, k, total = _noalloc_via_abi(g, d, intr.as_array(), 1, 1000)
    assert k == 1000 and total == int(np.isfinite(depth).sum())
    big = torch.zeros((4097, 1025), device="cuda", dtype=torch.float32)  # 4197425 samples > 2^22
    n = torch.zeros((1,), device="cuda", dtype=torch.int32)
    pts = torch.empty((16, 3), device="cuda", dtype=torch.float32)
    with pytest.raises(g.GsicpError) as e:
        g.gsicp_depth_to_points_noalloc(big, [500, 500, 512, 2048], 1, 0.1, 10.0, pts, None, n)
    assert e.value.status == g.ERR_INVALID_ARG and "4194304" in g.gsicp_last_error()


def test_noalloc_invalid_arguments_set_a_message(g):
    """Every rejected argument returns GSICP_ERR_INVALID_ARG with its own message (not one left
    over from an earlier call)."""
    d = torch.ones((12, 16), device="cuda", dtype=torch.float32)
    pts = torch.empty((16, 3), device="cuda", dtype=torch.float32)
    n = torch.zeros((1,), device="cuda", dtype=torch.int32)
    fi = (C.c_float * 4)(10.0, 10.0, 7.5, 5.5)
    f0 = (C.c_float * 4)(0.0, 10.0, 7.5, 5.5)
    P = (lambda t: C.c_void_p(t.data_ptr()))
    cases = [((None, 16, 12, fi, 1, P(pts), 16, P(n)), "NULL"),
             ((P(d), 0, 12, fi, 1, P(pts), 16, P(n)), "positive"),
             ((P(d), 16, 12, fi, 0, P(pts), 16, P(n)), "positive"),
             ((P(d), 16, 12, fi, 1, P(pts), -1, P(n)), "cap"),
             ((P(d), 16, 12, f0, 1, P(pts), 16, P(n)), "focal"),
             ((P(d), 16, 12, fi, 1, P(pts), 16, None), "NULL")]
    for (dp, W, H, intr, stride, pp, cap, npt), word in cases:
        st = g.lib.gsicp_depth_to_points_noalloc(dp, W, H, intr, stride, 0.1, 10.0, pp, None, cap, npt, None, None)
        assert st == g.ERR_INVALID_ARG and word in g.gsicp_last_error(), (W, H, stride, cap, g.gsicp_last_error())
