"""The level recurrences the MS-BFS kernel relies on, checked on the CPU
against plain BFS distances (no GPU): the frontier pull, the seen-set pull
and the accumulation of a hub's row from segments. These are properties of
BFS, not of the kernel; the GPU parity tests check the kernel itself.

Notation (one bit per (source, vertex) pair): S_d = pairs at distance <= d,
N_d = pairs at distance exactly d, A = adjacency.
  frontier pull: N_d = (A N_{d-1}) & ~S_{d-1},  S_d = S_{d-1} | N_d
  seen-set pull: S_d = S_{d-1} | ((A S_{d-1}) & ~S_{d-1}),  N_d = S_d & ~S_{d-1}
"""
import numpy as np
import pytest

from paper_2509_19703_gb300 import graphgen as gg


def bfs_dist(g):
    """Hop distances from every vertex (-1: unreachable), plain queue BFS."""
    n = g.n
    dist = np.full((n, n), -1, dtype=np.int64)
    for s in range(n):
        dist[s, s] = 0
        q = [s]
        head = 0
        while head < len(q):
            u = q[head]
            head += 1
            for e in range(g.row_ptr[u], g.row_ptr[u + 1]):
                v = g.col[e]
                if dist[s, v] < 0:
                    dist[s, v] = dist[s, u] + 1
                    q.append(v)
    return dist


def adjacency(g):
    a = np.zeros((g.n, g.n), dtype=bool)
    for u in range(g.n):
        a[u, g.col[g.row_ptr[u]:g.row_ptr[u + 1]]] = True
    return a


def graphs():
    return [gg.path(9), gg.grid(5, 7), gg.star(12), gg.barabasi_albert(60, 2, 3), gg.gnp(50, 0.08, 4),
            gg.random_tree(40, 5), gg.disjoint_union([gg.path(5), gg.star(6), gg.complete(4)], "mix")]


@pytest.mark.parametrize("g", graphs(), ids=lambda g: g.name)
def test_frontier_and_seen_set_pulls_give_the_bfs_levels(g):
    dist = bfs_dist(g)
    a = adjacency(g)
    # rows: vertices; columns: sources (the kernel's vertex-major bit rows)
    s_front = (dist.T == 0)
    n_front = s_front.copy()
    s_seen = s_front.copy()
    for d in range(1, g.n + 1):
        # frontier pull: a vertex is reached by the sources on a neighbour's frontier
        n_new = (a.astype(np.int64) @ n_front.astype(np.int64) > 0) & ~s_front
        s_front = s_front | n_new
        n_front = n_new
        # seen-set pull: by the sources that had reached a neighbour by level d - 1
        grown = s_seen | ((a.astype(np.int64) @ s_seen.astype(np.int64) > 0) & ~s_seen)
        new_seen = grown & ~s_seen
        s_seen = grown
        want = dist.T == d
        assert np.array_equal(n_front, want), (g.name, d)
        assert np.array_equal(new_seen, want), (g.name, d)
        assert np.array_equal(s_seen, s_front)
        if not want.any():
            break


@pytest.mark.parametrize("g", [gg.star(40), gg.barabasi_albert(80, 3, 7)], ids=lambda g: g.name)
def test_hub_row_from_segments_with_a_stale_subset_buffer(g):
    """A hub's S_d row built by ORing, segment by segment in any order, what
    each segment of its neighbour list finds (segment 0 also ORs S_{d-1})
    into a buffer that holds any subset of S_{d-1} equals S_d."""
    dist = bfs_dist(g)
    rng = np.random.default_rng(11)
    hub = int(np.argmax(np.diff(g.row_ptr)))
    nbrs = g.col[g.row_ptr[hub]:g.row_ptr[hub + 1]]
    for d in range(1, int(dist.max()) + 1):
        s_prev = (dist.T >= 0) & (dist.T <= d - 1)           # S_{d-1}, rows = vertices
        want = (dist.T[hub] >= 0) & (dist.T[hub] <= d)
        for trial in range(4):
            buf = s_prev[hub] & (rng.random(g.n) < 0.5)     # S_{d-3}: some subset of S_{d-1}
            segs = [nbrs[i:i + 3] for i in range(0, len(nbrs), 3)]
            order = rng.permutation(len(segs))
            for si in order:
                found = np.zeros(g.n, dtype=bool)
                for u in segs[si]:
                    found |= s_prev[u]
                found &= ~s_prev[hub]
                buf = buf | (found | (s_prev[hub] if si == 0 else False))
            assert np.array_equal(buf, want), (g.name, d, trial)
