"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Indices and distances must match bit for bit; weights within 1e-5 absolute
of the FP64 oracle; the COO structure exactly. Cases span several source
blocks with ragged tails, both BFS forms, every engine, k from 1 to 256, and
the degenerate graphs the method meets (isolated vertices, components
smaller than k, hubs, long paths)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import oracle_pins
from gpu_helpers import assert_parity, oracle_ref, run_gpu
from paper_2509_19703_gb300 import graphgen as gg
from paper_2509_19703_gb300 import gumap

pytestmark = pytest.mark.gpu

MSBFS, FRONTIER = gumap.ENGINE_MSBFS, gumap.ENGINE_FRONTIER


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


def ks_for(g):
    return sorted({k for k in (1, 7, 15, 50, 256) if k <= g.n - 1} | {min(g.n - 1, 256)})


CASES = [(g, k) for g in zoo() for k in ks_for(g)]


@pytest.mark.parametrize("g,k", CASES, ids=[f"{g.name}-k{k}" for g, k in CASES])
def test_zoo_full_msbfs(g, k):
    assert_parity(run_gpu(g, k, "full", engine=MSBFS), oracle_ref(g, k, "full"), f"{g.name} full k={k}")


@pytest.mark.parametrize("g,k", CASES, ids=[f"{g.name}-k{k}" for g, k in CASES])
def test_zoo_partial_both_engines(g, k):
    ref = oracle_ref(g, k, "partial")
    assert_parity(run_gpu(g, k, "partial", engine=FRONTIER), ref, f"{g.name} partial/frontier k={k}")
    assert_parity(run_gpu(g, k, "partial", engine=MSBFS), ref, f"{g.name} partial/msbfs k={k}")


@pytest.mark.parametrize("build", [gumap.FRONTIER_GROUP, gumap.FRONTIER_THREAD, gumap.FRONTIER_WARP],
                         ids=["group", "thread", "warp"])
@pytest.mark.parametrize("g,k", CASES, ids=[f"{g.name}-k{k}" for g, k in CASES])
def test_zoo_partial_frontier_builds(g, k, build):
    """Every merge build of the frontier engine (a group of lanes, one
    thread, one warp per source) gives the oracle's rows."""
    ref = oracle_ref(g, k, "partial")
    assert_parity(run_gpu(g, k, "partial", engine=FRONTIER, frontier_build=build), ref,
                  f"{g.name} partial/frontier build {build} k={k}")


@pytest.mark.parametrize("g,k", CASES, ids=[f"{g.name}-k{k}" for g, k in CASES])
def test_zoo_single_graph_on_the_batched_engine(g, k):
    """A single graph small enough for one CTA runs on the batched engine
    (shared-memory bitsets, __syncthreads levels) with the oracle's rows, in
    both forms and at several unit widths."""
    for mode in ("full", "partial"):
        ref = oracle_ref(g, k, mode)
        for width in (None, 2):
            res = run_gpu(g, k, mode, engine=gumap.ENGINE_BATCH, batch_width=width)
            assert_parity(res, ref, f"{g.name} {mode} k={k} batched engine width {width}")
            assert res["stats"]["engine"] == gumap.ENGINE_BATCH


def test_batched_engine_with_explicit_sources_uses_msbfs():
    g = gg.grid(20, 17)
    src = [5, 300, 5, 0, 339]
    ref = oracle_ref(g, 7, "full", sources=src, directed=True)
    res = run_gpu(g, 7, "full", engine=gumap.ENGINE_BATCH, sources=src, directed=True)
    assert_parity(res, ref, "explicit sources on the batched engine")
    assert res["stats"]["engine"] == gumap.ENGINE_MSBFS


@pytest.mark.parametrize("direction", [gumap.DIRECTION_PULL, gumap.DIRECTION_PUSH])
@pytest.mark.parametrize("g,k", CASES, ids=[f"{g.name}-k{k}" for g, k in CASES])
def test_zoo_forced_direction(g, k, direction):
    """Every level a pull, or every level from 2 on a push: same rows."""
    for mode in ("full", "partial"):
        ref = oracle_ref(g, k, mode)
        assert_parity(run_gpu(g, k, mode, engine=MSBFS, direction=direction, block_bits=256), ref,
                      f"{g.name} {mode} k={k} direction={direction}")


@pytest.mark.parametrize("build", [gumap.COO_RADIX, gumap.COO_ROWS], ids=["radix", "rows"])
@pytest.mark.parametrize("g,k", CASES, ids=[f"{g.name}-k{k}" for g, k in CASES])
def test_zoo_coo_builds(g, k, build):
    """Both builds of the union COO (radix-sorted (row, col) keys; rows
    counted, scanned, scattered and ranked by column) give the oracle's COO."""
    for mode in ("full", "partial"):
        ref = oracle_ref(g, k, mode)
        assert_parity(run_gpu(g, k, mode, coo_build=build), ref, f"{g.name} {mode} k={k} coo build {build}")


@pytest.mark.parametrize("g", [gg.star(3000), gg.barabasi_albert(20000, 5, 1)], ids=lambda g: g.name)
def test_long_rows_of_the_row_build(g):
    """Rows longer than one warp sorts (the star's centre: 2999 entries; the
    scale-free hubs) go through the shared-memory bitmap ranking."""
    ref = oracle_ref(g, 15, "partial")
    assert_parity(run_gpu(g, 15, "partial", coo_build=gumap.COO_ROWS), ref, f"{g.name} rows")


@pytest.mark.parametrize("width,ctas,stage", [(2, 3, 1), (4, 4, 1), (2, 4, 0), (4, 3, 0), (4, 3, 2)])
@pytest.mark.parametrize("g,k", CASES, ids=[f"{g.name}-k{k}" for g, k in CASES])
def test_zoo_kernel_builds(g, k, width, ctas, stage):
    """Every build of the kernel gives the same rows: pull items of 64 or 128
    bits, 3 or 4 CTAs per SM, rows staged in shared memory (1), read from the
    CSR (0), or the staged kernel's fallback reading its slice from global
    memory (2)."""
    ref = oracle_ref(g, k, "full")
    with gumap.KnnGraph.from_graph(g, k) as kg:
        kg.set_option(gumap.OPT_PULL_WIDTH, width)
        kg.set_option(gumap.OPT_CTAS_PER_SM, ctas)
        kg.set_option(gumap.OPT_STAGE, stage)
        kg.set_option(gumap.OPT_BLOCK_BITS, 384)
        kg.run()  # the staged layout of a grid size is built on its second launch
        kg.reset_stats()
        out = kg.run()
        r, c, w = kg.coo()
        kg.check()
        staged = kg.stats()["bfs_staged_launches"]
        res = dict(idx=out["idx"].cpu().numpy(), dist=gumap.dist_u16(out["dist"]),
                   w=out["w"].cpu().numpy().astype(np.float64), coo=(r.cpu().numpy(), c.cpu().numpy(),
                                                                      w.cpu().numpy().astype(np.float64)))
        rho, sigma = kg.rho_sigma()
        res.update(rho=rho.cpu().numpy().astype(np.float64), sigma=sigma.cpu().numpy().astype(np.float64))
    assert_parity(res, ref, f"{g.name} width {width} ctas {ctas} stage {stage} k={k}")
    if stage == 0:
        assert staged == 0
    elif g.n > 64:
        assert staged > 0


def test_direction_switches_on_a_long_grid():
    """Narrow source blocks on a long grid: the automatic rule runs push
    levels (sparse frontiers) and pull levels, with identical rows."""
    g = gg.grid(120, 80)
    ref = oracle_ref(g, 15, "full")
    res = run_gpu(g, 15, "full", engine=MSBFS, block_bits=256, direction=gumap.DIRECTION_AUTO)
    assert_parity(res, ref, "grid 120x80 auto")
    assert res["stats"]["bfs_push_levels"] > 0
    assert res["stats"]["bfs_level_sum"] > res["stats"]["bfs_push_levels"]


def test_config1_grid32_full():
    """32 x 32 grid, all 1024 sources, k = 15 (the small full-form case)."""
    g = gg.config_grid32()
    res = run_gpu(g, 15, "full")
    err = assert_parity(res, oracle_ref(g, 15, "full"), "grid32")
    assert res["stats"]["engine"] == MSBFS
    assert res["stats"]["levels_max"] == 62  # eccentricity of a corner of a 32 x 32 grid
    print(f"grid32 full k=15: max |dw| = {err:.3g}")


@pytest.mark.parametrize("bits", [128, 256, 384, 1024])
def test_block_tiling_ragged(bits):
    """Several source blocks with a ragged last block give the same rows."""
    g = gg.barabasi_albert(1000, 2, 61)
    ref = oracle_ref(g, 15, "full")
    assert_parity(run_gpu(g, 15, "full", engine=MSBFS, block_bits=bits), ref, f"bits={bits}")
    assert_parity(run_gpu(g, 15, "partial", engine=MSBFS, block_bits=bits), ref, f"partial bits={bits}")


@pytest.mark.parametrize("bits", [512, 4480])
@pytest.mark.parametrize("mode", ["full", "partial"])
@pytest.mark.parametrize("heavy", [0, 3, 1 << 30])
def test_heavy_threshold(heavy, mode, bits):
    """Heavy vertices as warp-wide items give the light pull's rows, with the
    rows read from the CSR (a grid size's first launch) and staged (later
    launches), in both forms, with 4 and with 35 groups of 128 source bits
    per row."""
    g = gg.disjoint_union([gg.barabasi_albert(1500, 3, 64), gg.star(200), gg.gnp(300, 0.05, 65)], "hv")
    ref = oracle_ref(g, 15, "full")
    with gumap.KnnGraph.from_graph(g, 15, mode=gumap.FULL if mode == "full" else gumap.PARTIAL) as kg:
        kg.set_option(gumap.OPT_ENGINE, MSBFS)
        kg.set_option(gumap.OPT_HEAVY_DEGREE, heavy)
        kg.set_option(gumap.OPT_BLOCK_BITS, bits)
        first = kg.run()
        kg.check()
        assert np.array_equal(first["idx"].cpu().numpy(), ref["idx"])
        kg.reset_stats()
        out = kg.run()
        if heavy == 3:
            assert kg.stats()["bfs_staged_launches"] > 0
        kg.check()
        assert np.array_equal(out["idx"].cpu().numpy(), ref["idx"])
        assert float(np.max(np.abs(out["w"].cpu().numpy() - ref["w"]))) <= 1e-5


@pytest.mark.parametrize("mode", ["full", "partial"])
def test_explicit_sources_with_duplicates(mode):
    g = gg.barabasi_albert(2000, 3, 62)
    rng = np.random.default_rng(63)
    src = rng.integers(0, g.n, size=777).astype(np.int32)
    src[10] = src[11] = src[12]
    ref = oracle_ref(g, 20, mode, sources=src, directed=True)
    engines = [MSBFS] if mode == "full" else [MSBFS, FRONTIER]
    for e in engines:
        res = run_gpu(g, 20, mode, engine=e, sources=src, directed=True)
        assert_parity(res, ref, f"{mode} engine={e}")


def _full_size_check(g, k, mode, engine, n_sample=150, seed=0):
    """All rows against the oracle's partial form (equal to the full form,
    a pinned invariant), plus sampled rows against the oracle's full BFS."""
    res = run_gpu(g, k, mode, engine=engine)
    ref = oracle_ref(g, k, "partial")
    err = assert_parity(res, ref, f"{g.name} {mode} k={k}")
    if mode == "full":
        rows = np.sort(np.random.default_rng(seed).choice(g.n, size=min(n_sample, g.n), replace=False))
        fi, fd = oracle.knn_full(g, k, sources=rows.astype(np.int32))
        assert np.array_equal(res["idx"][rows], fi) and np.array_equal(res["dist"][rows], fd)
    return res, err


@pytest.mark.parametrize("maker", [gg.config_ba20k, gg.config_er5k], ids=["ba20k", "er5k"])
def test_config2_full_all_sources(maker):
    g = maker()
    res, err = _full_size_check(g, 15, "full", None)
    assert res["stats"]["engine"] == MSBFS
    print(f"{g.name} full k=15: max |dw| = {err:.3g}, blocks = {res['stats']['n_blocks']}")


def test_hub_beyond_the_segment_limit():
    """The staged seen-set pull cuts a hub's row into at most 4096 segments,
    so a hub of more than 16 x 4096 neighbours gets segments longer than 16
    entries (this star's centre: 70,000 neighbours, segments of 18). Full
    form on the MS-BFS engine over several source blocks (the staged layout
    is used from the second block on); the centre's row and 40 sampled rows
    against the oracle's full BFS."""
    g = gg.star(70001)
    res = run_gpu(g, 15, "full", engine=MSBFS, coo=False)
    assert res["stats"]["bfs_staged_launches"] > 0
    rows = np.concatenate([[0], np.random.default_rng(5).choice(np.arange(1, g.n), size=40, replace=False)])
    rows = np.sort(rows).astype(np.int32)
    fi, fd = oracle.knn_full(g, 15, sources=rows)
    assert np.array_equal(res["idx"][rows], fi) and np.array_equal(res["dist"][rows], fd)


def test_config2_partial_msbfs_matches():
    g = gg.config_ba20k()
    _full_size_check(g, 15, "partial", MSBFS)


@pytest.mark.parametrize("k", [15, 50])
@pytest.mark.parametrize("maker", [gg.config_ba1m, gg.config_grid1m], ids=["ba1m", "grid1m"])
def test_config3_partial_all_sources(maker, k):
    g = maker()
    res = run_gpu(g, k, "partial", coo=(k == 15))
    idx, dist = oracle.knn_partial(g, k)
    rho, sigma, a = oracle.smooth_knn(dist)
    ref = dict(idx=idx, dist=dist, rho=rho, sigma=sigma, w=oracle.slot_union(idx, a))
    if k == 15:
        ref["coo"] = oracle.coo_union(idx, a)
    err = assert_parity(res, ref, f"{g.name} partial k={k}")
    assert res["stats"]["engine"] == FRONTIER
    print(f"{g.name} partial k={k}: max |dw| = {err:.3g}")


# ------------------------------------------------------------ edge cases

def test_n_src_zero_is_a_noop():
    g = gg.grid(5, 5)
    with gumap.KnnGraph.from_graph(g, 3, flags=gumap.WEIGHTS_DIRECTED) as kg:
        empty = torch.empty((0, 3), dtype=torch.int32, device="cuda")
        kg.run(sources=torch.empty(0, dtype=torch.int32, device="cuda"),
               out=dict(idx=empty, dist=empty.to(torch.int16), w=empty.float()))
        kg.check()


def test_union_with_explicit_sources_is_rejected():
    g = gg.grid(5, 5)
    with gumap.KnnGraph.from_graph(g, 3) as kg:
        with pytest.raises(gumap.GumapError) as e:
            kg.run(sources=torch.arange(4, dtype=torch.int32, device="cuda"))
        assert e.value.status == gumap.ERR_INVALID_ARG


def test_rows_are_staged_on_a_scale_free_graph():
    """A handle's first run reads the rows from the CSR; from its second run
    on the light rows are staged in shared memory (and the statistics say
    so); the rows match the oracle."""
    g = gg.barabasi_albert(4000, 4, 151)
    ref = oracle_ref(g, 15, "full")
    with gumap.KnnGraph.from_graph(g, 15) as kg:
        kg.run()
        kg.check()
        assert kg.stats()["bfs_staged_launches"] == 0  # a first launch reads the rows from the CSR
        kg.reset_stats()
        out = kg.run()
        rho, sigma = kg.rho_sigma()
        r, c, w = kg.coo()
        kg.check()
        assert kg.stats()["bfs_staged_launches"] > 0
        res = dict(idx=out["idx"].cpu().numpy(), dist=gumap.dist_u16(out["dist"]),
                   w=out["w"].cpu().numpy().astype(np.float64), rho=rho.cpu().numpy().astype(np.float64),
                   sigma=sigma.cpu().numpy().astype(np.float64),
                   coo=(r.cpu().numpy(), c.cpu().numpy(), w.cpu().numpy().astype(np.float64)))
    assert_parity(res, ref, "BA-4000 staged")


def test_bad_option_values_are_rejected():
    g = gg.grid(5, 5)
    with gumap.KnnGraph.from_graph(g, 3) as kg:
        for opt, val in ((gumap.OPT_CTAS_PER_SM, 5), (gumap.OPT_PULL_WIDTH, 3), (gumap.OPT_DIRECTION, 7),
                         (gumap.OPT_STAGE, 3), (gumap.OPT_COO_BUILD, 3)):
            with pytest.raises(gumap.GumapError) as e:
                kg.set_option(opt, val)
            assert e.value.status == gumap.ERR_INVALID_ARG


@pytest.mark.parametrize("bad", ["asym", "unsorted", "self", "dup", "range", "rowptr"])
@pytest.mark.parametrize("where", ["host", "device"])
def test_invalid_csr_rejected(bad, where):
    g = gg.grid(4, 4)
    rp, col = g.row_ptr.copy(), g.col.copy()
    if bad == "asym":
        col[0] = 5 if col[0] != 5 else 6  # (0, x) without (x, 0)
        col[: rp[1]] = np.sort(col[: rp[1]])
    elif bad == "unsorted":
        col[0], col[1] = col[1], col[0]
    elif bad == "self":
        col[0] = 0
    elif bad == "dup":
        col[1] = col[0]
    elif bad == "range":
        col[-1] = 99
    elif bad == "rowptr":
        rp[2] = rp[1] - 1  # a decreasing row pointer
    if where == "host":
        args = (rp, col)
        flags = 0
    else:
        args = (torch.as_tensor(rp, device="cuda"), torch.as_tensor(col, device="cuda"))
        flags = gumap.CSR_ON_DEVICE
    with pytest.raises(gumap.GumapError) as e:
        gumap.gumap_knn_create(args[0], args[1], g.n, g.nnz, 3, gumap.FULL, flags)
    assert e.value.status == gumap.ERR_INVALID_GRAPH


def test_device_csr_valid_path():
    g = gg.barabasi_albert(500, 3, 71)
    rp = torch.as_tensor(g.row_ptr, device="cuda")
    col = torch.as_tensor(g.col, device="cuda")
    h = gumap.gumap_knn_create(rp, col, g.n, g.nnz, 15, gumap.FULL, gumap.CSR_ON_DEVICE)
    try:
        idx = torch.empty((g.n, 15), dtype=torch.int32, device="cuda")
        dist = torch.empty((g.n, 15), dtype=torch.int16, device="cuda")
        w = torch.empty((g.n, 15), dtype=torch.float32, device="cuda")
        gumap.gumap_knn_run(h, None, g.n, idx, dist, w)
        gumap.gumap_knn_check(h)
        ref = oracle_ref(g, 15, "full", coo=False)
        assert np.array_equal(idx.cpu().numpy(), ref["idx"])
        assert float(np.max(np.abs(w.cpu().numpy() - ref["w"]))) <= 1e-5
    finally:
        gumap.gumap_knn_destroy(h)


def test_pooled_buffers_across_handles():
    """Handles destroyed and created again reuse pooled device buffers
    (holding the previous graph's data) and still give the oracle's rows."""
    gumap.gumap_pool_trim(-1)
    assert gumap.gumap_pool_cached_bytes() == 0
    graphs = [gg.barabasi_albert(2500, 3, 161), gg.grid(40, 60), gg.barabasi_albert(2500, 3, 162)]
    for g in graphs * 2:
        assert_parity(run_gpu(g, 15, "full"), oracle_ref(g, 15, "full"), g.name)
        assert gumap.gumap_pool_cached_bytes() > 0
    gumap.gumap_pool_trim(-1)
    assert gumap.gumap_pool_cached_bytes() == 0


def test_repeated_runs_are_identical():
    """The handle's scratch is reused across runs without leaking state."""
    g = gg.barabasi_albert(3000, 4, 72)
    with gumap.KnnGraph.from_graph(g, 15) as kg:
        a = kg.run()
        a = {k: v.clone() for k, v in a.items()}
        for _ in range(3):
            b = kg.run()
            kg.check()
            for key in a:
                assert torch.equal(a[key], b[key]), key
