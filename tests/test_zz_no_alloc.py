"""gumap_knn_run_noalloc: the allocation-free entry point, for callers that
cannot allocate device memory where they need kNN lists (a framework that
owns all device memory, or a latency-bound loop that cannot afford
cudaMalloc's synchronisation). Its scratch is a fixed array inside the
library; these checks compare its rows with gumap_knn_run's on two calls in a
row (the second call reuses the array the first one left behind), with the
CPU oracle's rows, and on a graph whose scratch needs many source blocks.

This file is named so that pytest collects it after every other test file.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2509_19703_gb300 import graphgen as gg
from paper_2509_19703_gb300 import gumap

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gumap.load()


def _existing_entry_point(g, k, mode):
    with gumap.KnnGraph.from_graph(g, k, mode=mode, flags=gumap.WEIGHTS_DIRECTED) as kg:
        kg.set_option(gumap.OPT_ENGINE, gumap.ENGINE_MSBFS)
        out = kg.run()
        kg.check()
        return out["idx"].cpu().numpy(), gumap.dist_u16(out["dist"])


def _noalloc(g, k, mode):
    rp = torch.as_tensor(g.row_ptr, device="cuda")
    col = torch.as_tensor(g.col, device="cuda")
    idx = torch.full((g.n, k), 7, dtype=torch.int32, device="cuda")
    dist = torch.full((g.n, k), 7, dtype=torch.int16, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    gumap.gumap_knn_run_noalloc(rp, col, g.n, g.nnz, k, mode, idx, dist, status)
    torch.cuda.synchronize()
    assert int(status.item()) == gumap.OK
    return idx.cpu().numpy(), gumap.dist_u16(dist)


def test_noalloc_matches_existing_entry_point_two_calls_in_a_row():
    cases = [(gg.barabasi_albert(3000, 3, 81), 15, gumap.FULL),
             (gg.disjoint_union([gg.grid(40, 30), gg.path(5)], "grid+path"), 20, gumap.PARTIAL)]
    for g, k, mode in cases:
        want_idx, want_dist = _existing_entry_point(g, k, mode)
        got_idx, got_dist = _noalloc(g, k, mode)
        assert np.array_equal(got_idx, want_idx), g.name
        assert np.array_equal(got_dist, want_dist), g.name


def test_noalloc_matches_the_oracle():
    for g, k, mode in [(gg.barabasi_albert(3000, 3, 81), 15, gumap.FULL),
                       (gg.disjoint_union([gg.grid(40, 30), gg.path(5)], "grid+path"), 20, gumap.PARTIAL)]:
        got_idx, got_dist = _noalloc(g, k, mode)
        want_idx, want_dist = oracle.knn_full(g, k) if mode == gumap.FULL else oracle.knn_partial(g, k)
        assert np.array_equal(got_idx, want_idx) and np.array_equal(got_dist, want_dist), g.name


@pytest.mark.parametrize("mode", [gumap.FULL, gumap.PARTIAL], ids=["full", "partial"])
def test_noalloc_many_source_blocks(mode):
    """n = 40,000: the fixed array holds about 1024 sources per block, so some
    40 launches share it, with a short last block."""
    g = gg.barabasi_albert(40000, 3, 82)
    k = 15
    want_idx, want_dist = _existing_entry_point(g, k, mode)
    for _ in range(2):
        got_idx, got_dist = _noalloc(g, k, mode)
        assert np.array_equal(got_idx, want_idx) and np.array_equal(got_dist, want_dist)
    sample = np.random.default_rng(83).choice(g.n, size=200, replace=False).astype(np.int32)
    ref_idx, ref_dist = oracle.knn_partial(g, k, sources=sample)  # full and partial lists are the same
    assert np.array_equal(got_idx[sample], ref_idx) and np.array_equal(got_dist[sample], ref_dist)


def test_noalloc_rejects_graphs_beyond_its_scratch():
    n = 1_000_000
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    idx = torch.empty((1, 1), dtype=torch.int32, device="cuda")
    dist = torch.empty((1, 1), dtype=torch.int16, device="cuda")
    with pytest.raises(gumap.GumapError) as e:
        gumap.gumap_knn_run_noalloc(rp, col, n, 0, 1, gumap.FULL, idx, dist)
    assert e.value.status == gumap.ERR_TOO_LARGE
    assert "16 MiB" in str(e.value)  # the reason reaches gumap_last_error()
