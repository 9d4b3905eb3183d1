"""The byte models behind bench.py's roofline figures, on hand-counted toy states (no GPU).

Exports are built by hand in the layout bingo_export_state returns: per vertex its degree, edges in
order (destination, bias, edge id), and [n][32] counts and kinds (BINGO_KIND_*: 0 empty, 1 dense,
2 one-element, 3 sparse, 4 regular).
"""
import numpy as np

import bench

EMPTY, DENSE, ONE, SPARSE, REGULAR = range(5)


def _export(deg, dst, bias, eid, n):
    return {"deg": np.array(deg, np.uint32), "dst": np.array(dst, np.uint32), "bias": np.array(bias, np.uint32),
            "eid": np.array(eid, np.uint64), "kind": np.zeros((n, 32), np.uint8), "cnt": np.zeros((n, 32), np.uint32)}


def test_update_bytes_hand_count():
    # before: 0->1 (bias 5 = bits 0, 2), 0->2 (bias 3); 1->0 (bias 1); groups of vertex 0: bit 0 regular,
    # bit 2 one-element
    ex0 = _export([2, 1, 0], [1, 2, 0], [5, 3, 1], [0, 1, 2], 3)
    ex0["kind"][0, 0], ex0["kind"][0, 2] = REGULAR, ONE
    ex1 = _export([2, 1, 0], [2, 2, 0], [3, 6, 1], [1, 3, 2], 3)
    ex1["kind"][0, 0], ex1["kind"][0, 1], ex1["kind"][0, 2] = REGULAR, ONE, DENSE
    ex1["cnt"][0, 0], ex1["cnt"][0, 1], ex1["cnt"][0, 2] = 1, 1, 1
    rec = np.array([[0, 2, 6, 0],    # insert 0->2, bias 6: bit 1 one-element after, bit 2 dense: no list entry
                    [0, 1, 0, 1],    # delete 0->1: found, bias 5; bit 0 was regular (a list), bit 2 one-element
                    [2, 0, 0, 1],    # delete 2->0: no such edge
                    [1, 0, 9, 2]],   # bias change 1->0: an insertion (bits 0, 3: no list) and a found deletion
                   np.uint32)
    records = 16 * 4
    sort = 64 * (2 + 3)              # two insertions, three deletions
    inserts = 32 * 2                 # adjacency slots; no set bit lands in a list group
    deletes = 96 * 2 + 128 * 1       # two found; one set bit in a list group (bit 0 of vertex 0)
    lines = 2 * 32 * 1               # vertex 0: K_v = 3, one sector; vertices 1 and 2 have no groups after
    assert bench.update_bytes(ex0, ex1, rec) == records + sort + inserts + deletes + lines


def test_update_bytes_earliest_copy_decides_the_removed_bias():
    # two copies of 0->1: edge id 4 (bias 2, bit 1 in a list) and edge id 7 (bias 1, bit 0 not a list)
    ex0 = _export([2], [1, 1], [1, 2], [7, 4], 1)
    ex0["kind"][0, 1] = SPARSE
    ex1 = _export([1], [1], [1], [7], 1)
    ex1["cnt"][0, 0] = 1
    rec = np.array([[0, 1, 0, 1]], np.uint32)
    assert bench.update_bytes(ex0, ex1, rec) == 16 + 64 + 96 + 128 + 2 * 32


def test_walk_bytes_per_vertex_and_sum():
    # vertex 0: d = 4, group 0 dense with 2 members (W = 2), group 2 regular with 1 member (W = 4),
    # group 3 sparse with 1 member (W = 8); vertex 1: no edges
    ex = _export([4, 0], [1, 1, 1, 1], [1, 1, 4, 8], [0, 1, 2, 3], 2)
    ex["cnt"][0, 0], ex["cnt"][0, 2], ex["cnt"][0, 3] = 2, 1, 1
    ex["kind"][0, 0], ex["kind"][0, 2], ex["kind"][0, 3] = DENSE, REGULAR, SPARSE
    per = bench.expected_bytes_per_vertex(ex)
    # header 32 + count line 32 (K_v = 4) + path 4; picks weighted 2/14, 4/14, 8/14:
    # dense 32 * d/|G| = 64, regular 64, sparse 96
    want = 32 + 32 + 4 + (2 * 64 + 4 * 64 + 8 * 96) / 14
    assert np.isclose(per[0], want) and per[1] == 0
    paths = np.array([[0, 1, 0xFFFFFFFF], [0, 1, 0xFFFFFFFF], [1, 0xFFFFFFFF, 0xFFFFFFFF]], np.uint32)
    plen = np.array([2, 2, 1], np.uint32)
    assert np.isclose(bench.walk_bytes(per, paths, plen), 2 * want)


def test_cpu_baseline_leg_reports_a_bounded_sample():
    """The oracle timing of the bench line on a small graph: a positive rate in steps/s, the threads
    used, and a description of the sample it timed."""
    import workloads as W

    wl = W.make_workload("c1")
    cb = bench.cpu_baseline(wl.graph, wl.batches[0], wl.length, 77, target_s=0.2)
    assert cb["kind"] == "oracle" and cb["unit"] == "steps/s" and cb["value"] > 0 and cb["cores"] >= 1
    assert "DeepWalk walkers x 80" in cb["sample"]


def test_update_bytes_on_exported_rows_equals_whole_export():
    """The same batch counted from exports of only the touched vertices (rows in id order) gives the
    bytes of the whole export."""
    ex0 = _export([2, 1, 0], [1, 2, 0], [5, 3, 1], [0, 1, 2], 3)
    ex0["kind"][0, 0], ex0["kind"][0, 2] = REGULAR, ONE
    ex1 = _export([2, 1, 0], [2, 2, 0], [3, 6, 1], [1, 3, 2], 3)
    ex1["kind"][0, 0], ex1["kind"][0, 1], ex1["kind"][0, 2] = REGULAR, ONE, DENSE
    ex1["cnt"][0, 0], ex1["cnt"][0, 1], ex1["cnt"][0, 2] = 1, 1, 1
    rec = np.array([[0, 2, 6, 0], [0, 1, 0, 1], [2, 0, 0, 1], [1, 0, 9, 2]], np.uint32)
    whole = bench.update_bytes(ex0, ex1, rec)

    def rows(ex, ids):
        deg = ex["deg"].astype(np.int64)
        off = np.concatenate([[0], np.cumsum(deg)])
        sel = np.concatenate([np.arange(off[v], off[v + 1]) for v in ids]).astype(np.int64)
        return {"deg": ex["deg"][ids], "dst": ex["dst"][sel], "bias": ex["bias"][sel], "eid": ex["eid"][sel],
                "kind": ex["kind"][ids], "cnt": ex["cnt"][ids]}

    ids = np.array([0, 1, 2])
    assert bench.update_bytes(rows(ex0, ids), rows(ex1, ids), rec, ids=ids) == whole


def test_sampled_steps_are_uniform_over_the_launch_steps():
    plen = np.array([1, 3, 2, 0, 5], np.uint32)  # steps per walker: 0, 2, 1, 0, 4 (7 in all)
    w, t, tot = bench.sample_steps(plen, 70000, 3)
    assert tot == 7
    assert ((t >= 0) & (t < plen[w].astype(np.int64) - 1)).all()
    freq = np.bincount(w * 8 + t, minlength=64) / 70000
    for walker, steps in enumerate([0, 2, 1, 0, 4]):
        for step in range(steps):
            assert abs(freq[walker * 8 + step] - 1 / 7) < 0.01


def test_bytes_parts_and_node2vec_step():
    ex = _export([4, 0], [1, 1, 1, 1], [1, 1, 4, 8], [0, 1, 2, 3], 2)
    ex["cnt"][0, 0], ex["cnt"][0, 2], ex["cnt"][0, 3] = 2, 1, 1
    ex["kind"][0, 0], ex["kind"][0, 2], ex["kind"][0, 3] = DENSE, REGULAR, SPARSE
    per = bench.expected_bytes_per_vertex(ex)
    fixed, pick = bench.expected_bytes_parts(ex)
    assert np.allclose(fixed + pick + 4.0, per[:1].tolist() + [4.0]) and fixed[1] == 0 and pick[1] == 0
    assert fixed[0] == 32 + 32
    # always accepted, never probed: the first-order model
    assert np.isclose(bench.node2vec_step_bytes(fixed[0], pick[0], 1.0, 0.0), per[0])
    # half the candidates rejected, a probe on every second candidate
    assert np.isclose(bench.node2vec_step_bytes(64.0, 100.0, 0.5, 0.5), 64 + (100 + 32) * 2 + 4)
