"""The batch autotuner's host logic on CPU: every candidate index shape is built and timed, its
maps are released, the fastest wins (ties to the earlier candidate), and a keyed result is reused."""
import pytest

from paper_2403_12550_b300 import RegParams
from paper_2403_12550_b300 import autotune as at


class _Map:
    live = 0

    def __init__(self, shape):
        self.shape = shape
        _Map.live += 1

    def close(self):
        _Map.live -= 1


@pytest.fixture()
def fake_maps(monkeypatch):
    built = []

    def build(ctx, t, c, bucket, cell):
        built.append((bucket, cell))
        return _Map((bucket, cell))
    monkeypatch.setattr(at, "gsicp_build_map_index", build)
    monkeypatch.setattr(at.torch.cuda, "get_device_name", lambda *a: "fake")
    at._CACHE.clear()
    yield built
    at._CACHE.clear()


def test_fastest_shape_wins_and_maps_are_released(fake_maps):
    ms = {(16, 0.012): 3.0, (8, 0.012): 2.5, (32, 0.012): 4.0, (16, 0.008): 2.5, (16, 0.005): 2.7, (8, 0.008): 9.0}
    seen = []

    def timer(ctx, srcs, scovs, maps, T0s, params, reps):
        assert len(maps) == 2 and reps == 3 and _Map.live == 2
        seen.append(maps[0].shape)
        return ms[maps[0].shape]
    r = at.tune_index_params(None, [0, 1], [0, 1], ["t0", "t1"], ["c0", "c1"], None, RegParams(), timer=timer)
    assert seen == list(at.CANDIDATES) and len(fake_maps) == 2 * len(at.CANDIDATES)
    assert (r["bucket"], r["cell"]) == (8, 0.012)  # 2.5 ms, first of the two tied
    assert r["ms"] == ms and _Map.live == 0


def test_keyed_result_is_reused(fake_maps):
    calls = []

    def timer(*a):
        calls.append(1)
        return 1.0
    r1 = at.tune_index_params(None, [0], [0], ["t"], ["c"], None, RegParams(), key="w", timer=timer)
    r2 = at.tune_index_params(None, [0], [0], ["t"], ["c"], None, RegParams(), key="w", timer=timer)
    assert r1 is r2 and len(calls) == len(at.CANDIDATES)


def test_maps_are_released_when_timing_fails(fake_maps):
    def timer(*a):
        raise RuntimeError("batch failed")
    with pytest.raises(RuntimeError):
        at.tune_index_params(None, [0], [0], ["t"], ["c"], None, RegParams(), timer=timer)
    assert _Map.live == 0


def test_frame_tuner_covers_shapes_then_coop_and_keeps_the_fastest(fake_maps, monkeypatch):
    coop_set, block_set = [], []
    monkeypatch.setattr(at, "gsicp_ctx_set_coop_walks", lambda ctx, c: coop_set.append(c))
    monkeypatch.setattr(at, "gsicp_ctx_set_gn_block", lambda ctx, b: block_set.append(b))
    shape_ms = {s: 5.0 + i for i, s in enumerate(at.FRAME_CANDIDATES)}
    shape_ms[at.FRAME_CANDIDATES[3]] = 1.0
    shape_ms[at.FRAME_CANDIDATES[5]] = 1.0   # tie: the earlier candidate wins
    coop_ms = {4: 2.0, 2: 1.5, 8: 1.5, 0: 3.0}
    block_ms = {256: 1.2, 128: 1.1, 384: 1.1}
    seen = []

    def timer(ctx, depth, intr, stride, z_min, z_max, cp, m, T0, params, reps):
        assert _Map.live == 1
        seen.append((m.shape, coop_set[-1] if coop_set else None))
        if block_set:
            return block_ms[block_set[-1]]
        return coop_ms[coop_set[-1]] if coop_set else shape_ms[m.shape]
    r = at.tune_frame(None, "d", [1, 1, 0, 0], 2, 0.1, 10.0, None, "means", "covs", None, RegParams(), timer=timer)
    best = at.FRAME_CANDIDATES[3]
    assert [s for s, _ in seen[:len(at.FRAME_CANDIDATES)]] == list(at.FRAME_CANDIDATES)
    assert (r["bucket"], r["cell"]) == best and r["ms"] == shape_ms
    # the threshold is timed on the chosen shape, every candidate once, and the fastest is left set
    nc, nb = len(at.COOP_CANDIDATES), len(at.BLOCK_CANDIDATES)
    assert [s for s, _ in seen[len(at.FRAME_CANDIDATES):]] == [best] * (nc + nb)
    assert coop_set[:nc] == list(at.COOP_CANDIDATES)
    assert r["coop"] == 2 and coop_set[-1] == 2 and r["coop_ms"] == coop_ms
    # then the block size, on the same shape and with the chosen threshold; ties to the earlier
    assert block_set[:nb] == list(at.BLOCK_CANDIDATES) and r["block_ms"] == block_ms
    assert r["block"] == 128 and block_set[-1] == 128
    assert _Map.live == 0


def test_frame_tuner_keyed_result_sets_its_threshold_again(fake_maps, monkeypatch):
    coop_set, block_set = [], []
    monkeypatch.setattr(at, "gsicp_ctx_set_coop_walks", lambda ctx, c: coop_set.append(c))
    monkeypatch.setattr(at, "gsicp_ctx_set_gn_block", lambda ctx, b: block_set.append(b))
    calls = []

    def timer(*a):
        calls.append(1)
        return 1.0
    r1 = at.tune_frame(None, "d", [1, 1, 0, 0], 2, 0.1, 10.0, None, "m", "c", None, RegParams(), key="f", timer=timer)
    n = len(calls)
    r2 = at.tune_frame(None, "d", [1, 1, 0, 0], 2, 0.1, 10.0, None, "m", "c", None, RegParams(), key="f", timer=timer)
    assert r1 is r2 and len(calls) == n == len(at.FRAME_CANDIDATES) + len(at.COOP_CANDIDATES) + \
        len(at.BLOCK_CANDIDATES)
    assert coop_set[-1] == r1["coop"] and block_set[-1] == r1["block"]


def test_frame_tuner_releases_maps_when_timing_fails(fake_maps, monkeypatch):
    monkeypatch.setattr(at, "gsicp_ctx_set_coop_walks", lambda ctx, c: None)
    monkeypatch.setattr(at, "gsicp_ctx_set_gn_block", lambda ctx, b: None)

    def timer(*a):
        raise RuntimeError("frame failed")
    with pytest.raises(RuntimeError):
        at.tune_frame(None, "d", [1, 1, 0, 0], 2, 0.1, 10.0, None, "m", "c", None, RegParams(), timer=timer)
    assert _Map.live == 0
