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


def _noalloc_via_abi(g, depth, intr, stride, cap):
    """Direct ctypes call of gsicp_depth_to_points_noalloc with caller-owned buffers."""
    pts = torch.empty((cap, 3), device="cuda", dtype=torch.float32)
    z = torch.empty((cap,), device="cuda", dtype=torch.float32)
    n = torch.full((1,), -1, device="cuda", dtype=torch.int32)
    total = torch.full((1,), -1, device="cuda", dtype=torch.int32)
    H, W = depth.shape
    fi = (C.c_float * 4)(*[float(v) for v in intr])
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = g.lib.gsicp_depth_to_points_noalloc(C.c_void_p(depth.data_ptr()), W, H, fi, stride, 0.1, 10.0,
                                             C.c_void_p(pts.data_ptr()), C.c_void_p(z.data_ptr()), cap,
                                             C.c_void_p(n.data_ptr()), C.c_void_p(total.data_ptr()), stream)
    assert st == 0, g.gsicp_last_error()
    torch.cuda.synchronize()
    k = int(n.item())
    return pts[:k].cpu().numpy(), z[:k].cpu().numpy(), k, int(total.item())


def test_noalloc_matches_allocating_entry_point_on_two_calls(g):
    ctx = g.Context()
    cases = [(_image(3, 1200, 680, 0.0), 2), (_image(4, 640, 480, 0.05), 1)]
    for (intr, depth), stride in cases:  # two calls in a row, different sizes and hole patterns
        d = torch.from_numpy(depth).cuda()
        H, W = depth.shape
        cap = ((W + stride - 1) // stride) * ((H + stride - 1) // stride)
        pts_ref, z_ref = g.gsicp_depth_to_points(ctx, d, intr.as_array(), stride, 0.1, 10.0)
        pts, z, k, total = _noalloc_via_abi(g, d, intr.as_array(), stride, cap)
        assert k == total == pts_ref.shape[0]
        np.testing.assert_array_equal(pts, pts_ref.cpu().numpy())  # the a1 parity bar is bit-exact
        np.testing.assert_array_equal(z, z_ref.cpu().numpy())
    ctx.close()


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
