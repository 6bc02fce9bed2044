"""Host-side work counts of bench.py against the oracle (CPU only).

The partial form's GTEPS counts, per source, the adjacency entries of the
vertices it expands (those closer than the distance D_s of its k-th
neighbour). bench.py derives that count from the kNN lists; here it must
equal the count the oracle's partial BFS keeps while it scans, on graphs
with ties, hubs, isolated vertices and components smaller than k + 1
(padded lists). The full form's count (edges of the source's component) is
checked against components found by the oracle's BFS."""
import numpy as np
import pytest

import bench
import oracle
import oracle_pins
from paper_2509_19703_gb300 import graphgen as gg


def graphs():
    gs = [g for g in oracle_pins.tiny_graphs() if g.n >= 2]
    gs += [gg.grid(17, 23), gg.path(90), gg.cycle(61), gg.star(40), gg.complete(12), gg.random_tree(500, 71),
           gg.barabasi_albert(800, 3, 72), gg.gnp(400, 0.01, 73),
           gg.disjoint_union([gg.star(5), gg.path(3), gg.path(1), gg.gnp(120, 0.05, 74), gg.complete(4)], "smallcomps")]
    return gs


@pytest.mark.parametrize("k", [1, 3, 15, 50])
@pytest.mark.parametrize("g", graphs(), ids=lambda g: g.name)
def test_partial_work_matches_the_oracle_scan(g, k):
    k = min(k, g.n - 1)
    idx, dist, work = oracle.knn_partial(g, k, return_work=True)
    entries, rows = bench.partial_work(g, idx, dist)
    assert np.array_equal(entries, work)
    # expanded rows: the source plus every listed vertex closer than D_s
    for s in range(0, g.n, max(1, g.n // 37)):
        d = oracle.bfs(g, s)
        reach = d >= 0
        listed_d = dist[s][idx[s] >= 0].astype(np.int64)
        D = listed_d[-1] if len(listed_d) == k else np.iinfo(np.int64).max
        assert rows[s] == int(np.count_nonzero(reach & (d < D)))


@pytest.mark.parametrize("g", graphs(), ids=lambda g: g.name)
def test_component_work_is_the_component_edge_count(g):
    per_src = bench.component_work(g)
    deg = np.diff(g.row_ptr)
    for s in range(0, g.n, max(1, g.n // 23)):
        comp = oracle.bfs(g, s) >= 0
        assert per_src[s] == int(deg[comp].sum()) // 2


def test_partial_work_accepts_int16_distances():
    g = gg.grid(9, 9)
    idx, dist, work = oracle.knn_partial(g, 15, return_work=True)
    entries, _ = bench.partial_work(g, idx, dist.view(np.int16))
    assert np.array_equal(entries, work)


def test_frontier_and_coo_byte_models():
    entries = np.array([4, 12, 0], dtype=np.int64)
    rows = np.array([1, 3, 1], dtype=np.int64)
    assert bench.frontier_alg_bytes(entries, rows, 15) == 8 * 5 + 4 * 16 + 6 * 15 * 3
    # each slot's id and weight read once, each entry's column and weight written once, row offsets
    assert bench.coo_alg_bytes(1000, 15, 24000) == 8 * 15000 + 8 * 24000 + 8 * 1000


def test_all_core_oracle_sample_covers_each_source_once():
    """The all-core CPU baseline splits one seeded source order over spawned
    processes in disjoint strides; with a budget large enough to finish, the
    processes together do every source of every graph."""
    graphs = [gg.grid(12, 12), gg.disjoint_union([gg.path(30), gg.star(9)], "pathstar")]
    works = [bench.component_work(g) for g in graphs]
    v, desc = bench.oracle_sample_all_cores(graphs, works, 60.0, 2)
    assert v > 0
    assert desc.startswith(f"{graphs[0].n} of {graphs[0].n} sources") and "2 processes" in desc
    assert f"{graphs[1].n} of {graphs[1].n} sources" in desc
