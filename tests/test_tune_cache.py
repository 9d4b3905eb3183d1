"""The walker tuner's JSON cache (host logic, no GPU): a miss tunes and stores the shape under a key of
(device, graph size class, weight format, walk length); a hit applies the stored shape without tuning;
a graph of another size class, another device or another length misses."""
import json
import types

import paper_2504_10233_gb300 as B


class FakeGraph:
    """The four calls the cache makes, recorded: config, state_sizes, autotune, set_walk_config."""

    def __init__(self, n, m, max_bits=21, shape=(4, 16, 0, 0)):
        self.n, self.m, self.max_bits, self.shape = n, m, max_bits, shape
        self.tuned, self.applied = 0, []

    def config(self):
        return types.SimpleNamespace(max_bits=self.max_bits, bias_format=0, radix_base=0)

    def state_sizes(self):
        return {"m": self.m}

    def autotune(self, starts, length, stream=None):
        self.tuned += 1
        lanes, wpb, bps, regv = self.shape
        return types.SimpleNamespace(lanes_per_walker=lanes, warps_per_block=wpb, blocks_per_sm=bps, reg_variant=regv)

    def set_walk_config(self, lanes, wpb, bps=0, regv=0):
        self.applied.append((lanes, wpb, bps, regv))


def test_miss_tunes_and_stores_then_hit_applies(tmp_path):
    path = str(tmp_path / "tune.json")
    g1 = FakeGraph(1 << 20, 1 << 24, shape=(1, 16, 0, 0))
    r1 = B.cached_walk_tune(g1, None, 80, path, "GB300")
    assert r1["cached"] is False and g1.tuned == 1 and g1.applied == []
    data = json.load(open(path))
    key = B.walk_tune_key(g1, 80, "GB300")
    assert data["entries"][key] == {"lanes_per_walker": 1, "warps_per_block": 16, "blocks_per_sm": 0,
                                    "reg_variant": 0}
    # the same size class (within a factor of two) hits: the stored shape is applied, nothing is timed
    g2 = FakeGraph((1 << 20) - 5, (1 << 24) - 100, shape=(32, 4, 0, 1))
    r2 = B.cached_walk_tune(g2, None, 80, path, "GB300")
    assert r2["cached"] is True and g2.tuned == 0 and g2.applied == [(1, 16, 0, 0)]


def test_other_class_device_or_length_misses(tmp_path):
    path = str(tmp_path / "tune.json")
    B.cached_walk_tune(FakeGraph(1 << 20, 1 << 24), None, 80, path, "GB300")
    for g, length, dev in ((FakeGraph(1 << 22, 1 << 26), 80, "GB300"), (FakeGraph(1 << 20, 1 << 24), 40, "GB300"),
                           (FakeGraph(1 << 20, 1 << 24), 80, "other"), (FakeGraph(1 << 20, 1 << 24, max_bits=31), 80,
                                                                        "GB300")):
        r = B.cached_walk_tune(g, None, length, path, dev)
        assert r["cached"] is False and g.tuned == 1
    assert len(json.load(open(path))["entries"]) == 5
