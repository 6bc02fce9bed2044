"""All-pairs hop-distance rows (gumap_knn_apsp: the matrix S of Algorithm 1,
C0) against the oracle's queue BFS: every row of every zoo graph, with
source blocks narrow enough to need several launches, explicit source lists,
sampled rows of the 20,000-vertex scale-free graph at full size, and the
argument errors."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import oracle_pins
from paper_2509_19703_gb300 import graphgen as gg
from paper_2509_19703_gb300 import gumap

pytestmark = pytest.mark.gpu

MSBFS = gumap.ENGINE_MSBFS


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gumap.load()


def zoo():
    gs = [g for g in oracle_pins.tiny_graphs() if g.n >= 2]
    gs += [gg.path(600), gg.cycle(101), gg.star(300), gg.complete(40), gg.grid(13, 29),
           gg.random_tree(2000, 51), gg.barabasi_albert(3000, 3, 52), gg.gnp(1500, 0.004, 53),
           gg.disjoint_union([gg.star(50), gg.path(7), gg.gnp(300, 0.03, 54), gg.path(1), gg.path(2)], "mixdis")]
    return gs


def u16(t):
    return t.cpu().numpy().view(np.uint16)


def apsp_gpu(g, k, sources=None, block_bits=None, options=(), repeat=1):
    with gumap.KnnGraph.from_graph(g, k, mode=gumap.FULL, flags=gumap.EMIT_APSP) as kg:
        kg.set_option(gumap.OPT_ENGINE, MSBFS)
        if block_bits is not None:
            kg.set_option(gumap.OPT_BLOCK_BITS, block_bits)
        for opt, val in options:
            kg.set_option(opt, val)
        src = None if sources is None else torch.as_tensor(np.asarray(sources, dtype=np.int32), device="cuda")
        for _ in range(repeat):  # the staged layout of a grid size is built on its second launch
            out = kg.apsp(src)
        kg.check()
        return u16(out["apsp"]), out["idx"].cpu().numpy(), gumap.dist_u16(out["dist"])


@pytest.mark.parametrize("g", zoo(), ids=lambda g: g.name)
def test_every_row_matches_the_oracle(g):
    k = min(15, g.n - 1)
    D = oracle.apsp(g)
    got, idx, dist = apsp_gpu(g, k, block_bits=128)  # several source blocks for n > 128
    if not np.array_equal(got, D):
        bad = np.argwhere(got != D)[:3]
        raise AssertionError(f"{g.name}: rows differ at {bad.tolist()}: gpu {got[tuple(bad.T)].tolist()} "
                             f"oracle {D[tuple(bad.T)].tolist()}")
    ridx, rdist = oracle.knn_full(g, k)
    assert np.array_equal(idx, ridx) and np.array_equal(dist, rdist), f"{g.name}: kNN lists differ"


@pytest.mark.parametrize("options", [(), ((gumap.OPT_STAGE, 0),), ((gumap.OPT_DIRECTION, gumap.DIRECTION_PUSH),)],
                         ids=["default", "unstaged", "push"])
def test_rows_on_every_build(options):
    g = gg.barabasi_albert(2500, 4, 61)
    got, _, _ = apsp_gpu(g, 15, options=options, repeat=2)
    assert np.array_equal(got, oracle.apsp(g))


def test_explicit_sources_with_duplicates():
    g = gg.disjoint_union([gg.grid(20, 30), gg.barabasi_albert(400, 2, 62)], "gridba")
    rng = np.random.default_rng(7)
    src = rng.integers(0, g.n, size=333).astype(np.int32)
    src[:5] = src[5]  # duplicates
    got, idx, dist = apsp_gpu(g, 15, sources=src, block_bits=128)
    assert np.array_equal(got, oracle.apsp(g)[src])
    ridx, rdist = oracle.knn_full(g, 15, src)
    assert np.array_equal(idx, ridx) and np.array_equal(dist, rdist)


def test_sampled_rows_at_the_scale_free_bench_size():
    """BA n = 20,000, m0 = 5 (the bench graph), all sources in the default
    configuration (800 MB of rows): 64 sampled rows against single BFS runs."""
    g = gg.config_ba20k()
    got, _, _ = apsp_gpu(g, 15)
    rng = np.random.default_rng(11)
    for s in rng.choice(g.n, size=64, replace=False):
        ref = oracle.bfs(g, int(s))
        ref = np.where(ref < 0, 0xFFFF, ref).astype(np.uint16)
        assert np.array_equal(got[s], ref), f"row {s} differs"


def test_flag_is_required_and_full_form_only():
    g = gg.grid(6, 6)
    with gumap.KnnGraph.from_graph(g, 5) as kg:
        with pytest.raises(gumap.GumapError) as e:
            kg.apsp()
        assert e.value.status == gumap.ERR_INVALID_ARG
    with pytest.raises(gumap.GumapError) as e:
        gumap.KnnGraph.from_graph(g, 5, mode=gumap.PARTIAL, flags=gumap.EMIT_APSP)
    assert e.value.status == gumap.ERR_INVALID_ARG
