"""Batched engine (gumap_batch_create): many graphs in one persistent launch.

Each graph's rows must equal the oracle's (bit-exact indices/distances,
weights within 1e-5) and equal what a handle of that graph alone gives."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from gpu_helpers import W_TOL, assert_parity, oracle_ref
from paper_2509_19703_gb300 import graphgen as gg
from paper_2509_19703_gb300 import gumap

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gumap.load()


def run_batch(graphs, k, modes, coo=True, width=None, tune=False):
    kb, offs = gumap.KnnGraph.batch(graphs, k, modes)
    with kb:
        tuned = kb.autotune() if tune else None
        if width is not None:
            kb.set_option(gumap.OPT_BATCH_WIDTH, width)
        out = kb.run()
        rho, sigma = kb.rho_sigma()
        res = {}
        if coo:
            r, c, w = kb.coo()
            res["coo"] = (r.cpu().numpy(), c.cpu().numpy(), w.cpu().numpy().astype(np.float64))
        kb.check()
        torch.cuda.synchronize()
        res.update(idx=out["idx"].cpu().numpy(), dist=gumap.dist_u16(out["dist"]),
                   w=out["w"].cpu().numpy().astype(np.float64), rho=rho.cpu().numpy().astype(np.float64),
                   sigma=sigma.cpu().numpy().astype(np.float64), stats=kb.stats(), tuned=tuned)
    return res, offs


def small_mix(count, seed, n_hi=3000):
    items = gg.batch_mix(count=count, base_seed=seed, n_lo=10, n_hi=n_hi)
    return [it.graph for it in items], [gumap.FULL if it.mode == "full" else gumap.PARTIAL for it in items]


@pytest.mark.parametrize("k", [1, 15, 40])
def test_batch_matches_oracle_on_the_union(k):
    graphs, modes = small_mix(60, 91)
    graphs.append(gg.path(3))      # fewer than k + 1 vertices: padded rows
    modes.append(gumap.PARTIAL)
    res, _ = run_batch(graphs, k, modes)
    union = gg.disjoint_union(graphs)
    assert_parity(res, oracle_ref(union, k, "partial"), f"batch k={k}")
    assert res["stats"]["engine"] == gumap.ENGINE_BATCH
    assert res["stats"]["bfs_launches"] == 1


@pytest.mark.parametrize("width", [1, 4, 16, 64])
def test_batch_width_keeps_the_rows(width):
    """Units of at most `width` words (re-planned on the handle): same rows."""
    graphs, modes = small_mix(40, 95)
    res, _ = run_batch(graphs, 15, modes, width=width)
    assert_parity(res, oracle_ref(gg.disjoint_union(graphs), 15, "partial"), f"batch width {width}")


def test_batch_autotune_keeps_the_rows():
    graphs, modes = small_mix(40, 96)
    res, _ = run_batch(graphs, 15, modes, tune=True)
    assert res["tuned"]["batch_width"] in (8, 16, 32, 64) and res["tuned"]["candidates"] == 4
    assert_parity(res, oracle_ref(gg.disjoint_union(graphs), 15, "partial"), "tuned batch")


def test_batch_rows_equal_single_graph_handles():
    graphs = [gg.barabasi_albert(700, 3, 92), gg.grid(23, 17), gg.random_tree(500, 93), gg.gnp(400, 0.05, 94)]
    modes = [gumap.FULL, gumap.PARTIAL, gumap.FULL, gumap.PARTIAL]
    res, offs = run_batch(graphs, 15, modes, coo=False)
    for g, m, lo in zip(graphs, modes, offs[:-1]):
        with gumap.KnnGraph.from_graph(g, 15, mode=m) as kg:
            out = kg.run()
            kg.check()
            idx = out["idx"].cpu().numpy()
            sl = slice(int(lo), int(lo) + g.n)
            shifted = np.where(res["idx"][sl] >= 0, res["idx"][sl] - lo, -1)
            assert np.array_equal(shifted, idx), g.name
            assert np.array_equal(res["dist"][sl], gumap.dist_u16(out["dist"])), g.name
            assert np.array_equal(res["w"][sl], out["w"].cpu().numpy().astype(np.float64)), g.name


def test_batch_visited_in_global_slab():
    """A graph too large for three bitsets in shared memory keeps its visited
    bitset in the CTA's global slab."""
    graphs = [gg.barabasi_albert(19000, 2, 95), gg.grid(30, 30)]
    res, _ = run_batch(graphs, 15, [gumap.FULL, gumap.PARTIAL], coo=False)
    union = gg.disjoint_union(graphs)
    idx, dist = oracle.knn_partial(union, 15)
    rho, sigma, a = oracle.smooth_knn(dist)
    ref = dict(idx=idx, dist=dist, rho=rho, sigma=sigma, w=oracle.slot_union(idx, a))
    assert_parity(res, ref, "slab")


def test_batch_rejects_cross_graph_edges_and_oversized_graphs():
    g = gg.path(10)
    offs = np.array([0, 5, 10], dtype=np.int32)
    with pytest.raises(gumap.GumapError) as e:  # the path's edge (4, 5) crosses the two "graphs"
        gumap.gumap_batch_create(2, offs, g.row_ptr, g.col, g.nnz, 2, [gumap.FULL, gumap.FULL])
    assert e.value.status == gumap.ERR_INVALID_GRAPH
    big = gg.barabasi_albert(40000, 2, 96)
    with pytest.raises(gumap.GumapError) as e:
        gumap.KnnGraph.batch([big, gg.path(5)], 15, [gumap.FULL, gumap.FULL])
    assert e.value.status == gumap.ERR_TOO_LARGE


def test_config4_batch_of_2000_graphs():
    """2000 seeded graphs (n log-uniform in [100, 20000]; grid / BA 2..8 /
    G(n,p) mean degree 4..40 / random tree; full or partial), k = 15, one
    persistent launch; every row against the oracle."""
    items = gg.batch_mix(count=2000, base_seed=4)
    graphs = [it.graph for it in items]
    modes = [gumap.FULL if it.mode == "full" else gumap.PARTIAL for it in items]
    res, offs = run_batch(graphs, 15, modes, coo=False)
    union = gg.disjoint_union(graphs)
    idx, dist = oracle.knn_partial(union, 15)
    assert np.array_equal(res["idx"], idx)
    assert np.array_equal(res["dist"], dist)
    rho, sigma, a = oracle.smooth_knn(dist)
    w = oracle.slot_union(idx, a)
    err = float(np.max(np.abs(res["w"] - w)))
    assert err <= W_TOL, err
    print(f"config 4: {len(graphs)} graphs, {union.n} vertices, max |dw| = {err:.3g}")
