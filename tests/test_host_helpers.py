"""Host-side helpers that need no GPU: the stored marker order, the launch-shape record of the
binding, and the bench's reading of the committed DRAM-traffic summary."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _morton10(P):
    q = np.floor(np.clip(P, 0.0, np.nextafter(1.0, 0.0)) * 1024.0).astype(np.uint64)
    key = np.zeros(q.shape[1], np.uint64)
    for b in range(10):
        for d in range(3):
            key |= ((q[d] >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + d)
    return key


def test_marker_morton_order_groups_bubbles_and_sorts_each():
    from paper_2605_20565_gb300 import synth
    rng = np.random.default_rng(4)
    P = rng.uniform(0, 1, (3, 3000))
    g = rng.integers(0, 7, 3000).astype(np.int32)
    perm = synth.marker_morton_order(P, g)
    assert np.array_equal(np.sort(perm), np.arange(3000))  # a permutation
    gs, ks = g[perm], _morton10(P[:, perm])
    assert np.all(np.diff(gs) >= 0)  # bubble by bubble
    for b in range(7):
        assert np.all(np.diff(ks[gs == b].astype(np.int64)) >= 0)  # Morton order inside each
    assert synth.marker_morton_order(np.zeros((3, 0)), np.zeros(0, np.int32)).size == 0


def test_order_markers_permutes_every_marker_array():
    from paper_2605_20565_gb300 import synth
    w = synth.tiny()
    before = (w.markers.copy(), w.forces.copy(), w.marker_group.copy())
    perm = synth.order_markers(w)
    assert np.array_equal(w.markers, before[0][:, perm])
    assert np.array_equal(w.forces, before[1][:, perm])
    assert np.array_equal(w.marker_group, before[2][perm])


def test_launch_record_round_trip():
    import paper_2605_20565_gb300 as ot
    d = dict(block=128, tile=2, blocks_per_sm=3, order_level=8, tri_tile=4, tri_blocks_per_sm=6, tri_records=-1)
    assert ot._Launch.of(d).as_dict() == d
    assert ot._Launch.of({}).as_dict() == {k: 0 for k in d}  # library defaults


def test_traffic_summary_is_read_only_for_its_own_capture():
    sys.path.insert(0, ROOT)
    import bench
    path = os.path.join(ROOT, "profiles", "particles_graph_many_bubbles_traffic.txt")
    fields = dict(line.split(":", 1) for line in open(path) if ":" in line and not line.startswith("#"))
    fields = {k.strip(): v.strip() for k, v in fields.items()}
    assert int(fields["bytes_per_replay"]) == int(fields["dram_bytes_read"]) + int(fields["dram_bytes_write"])
    wl, form, lvl = fields["workload"], fields["form"], int(fields["map_level"])
    mates = fields["level_mates"] == "table"
    # another workload, form, level map or level-mate form: no traffic
    assert bench.batch_traffic("single_bubble_l5-9", form, lvl, mates)[0] is None
    assert bench.batch_traffic(wl, "learned", lvl, mates)[0] is None
    assert bench.batch_traffic(wl, form, lvl + 1, mates)[0] is None
    assert bench.batch_traffic(wl, form, lvl, not mates)[0] is None
    value, source = bench.batch_traffic(wl, form, lvl, mates)
    if fields["kernel_sources_sha256"] == bench.kernel_sources_hash():
        assert value == int(fields["bytes_per_replay"]) and source.endswith("particles_graph_many_bubbles_traffic.txt")
    else:  # sources edited since the capture: reported as unknown, never stale
        assert value is None and "changed" in source
