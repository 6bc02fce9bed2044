"""Quality metrics of a drawing (Section 4.1.3) on the GPU against the CPU
oracle, through the C ABI: neighbourhood preservation (per-vertex counts
bit-exact; the sum within 1e-12 relative, as it adds the same exact
fractions in another order) and stress (d - |X_i - X_j| in FP64, the
division and square in FP32, about 3e-7 relative per term, summed in FP64:
rows and total within 1e-6 relative of the FP64 oracle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import oracle_pins
from paper_2509_19703_gb300 import graphgen as gg
from paper_2509_19703_gb300 import gumap

pytestmark = pytest.mark.gpu

STRESS_RTOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gumap.load()


def layouts(g, seed):
    rng = np.random.default_rng(seed)
    return {"normal": rng.standard_normal((g.n, 2)).astype(np.float32),
            "lattice": rng.integers(0, 4, size=(g.n, 2)).astype(np.float32),  # many ties: the id rule decides
            "dim3": (5.0 * rng.standard_normal((g.n, 3))).astype(np.float32)}


def zoo():
    gs = [g for g in oracle_pins.tiny_graphs() if g.n >= 2]
    gs += [gg.grid(13, 29), gg.barabasi_albert(1500, 3, 61), gg.random_tree(800, 62), gg.star(200),
           gg.complete(30), gg.gnp(600, 0.01, 63),
           gg.disjoint_union([gg.star(40), gg.path(7), gg.gnp(120, 0.05, 64), gg.path(1)], "mixq")]
    return gs


CASES = [(g, name) for g in zoo() for name in ("normal", "lattice", "dim3")]


def gpu_np(g, X, r):
    with gumap.KnnGraph.from_graph(g, 1, mode=gumap.FULL) as kg:
        c, inter, total = kg.quality_np(torch.as_tensor(X, device="cuda"), r)
        kg.check()
        return c.cpu().numpy(), inter.cpu().numpy(), float(total.item())


def gpu_stress(g, X):
    with gumap.KnnGraph.from_graph(g, 1, mode=gumap.PARTIAL) as kg:
        total, rows = kg.quality_stress(torch.as_tensor(X, device="cuda"))
        kg.check()
        return float(total.item()), rows.cpu().numpy()


@pytest.mark.parametrize("g,layout", CASES, ids=[f"{g.name}-{n}" for g, n in CASES])
def test_np_matches_oracle(g, layout):
    X = layouts(g, 7)[layout]
    for r in (1, 2, 3):
        c, inter, total = gpu_np(g, X, r)
        rc, ri, rt = oracle.np_metric(g, X, r)
        assert np.array_equal(c, rc), (g.name, layout, r)
        bad = np.flatnonzero(inter != ri)
        assert bad.size == 0, (g.name, layout, r, bad[:5].tolist(), inter[bad[:5]].tolist(), ri[bad[:5]].tolist())
        assert abs(total - rt) <= 1e-12 * max(1.0, rt), (total, rt)


@pytest.mark.parametrize("g,layout", CASES, ids=[f"{g.name}-{n}" for g, n in CASES])
def test_stress_matches_oracle(g, layout):
    X = layouts(g, 8)[layout]
    total, rows = gpu_stress(g, X)
    rt, rr = oracle.stress(g, X)
    np.testing.assert_allclose(rows, rr, rtol=STRESS_RTOL, atol=1e-12)
    assert abs(total - rt) <= STRESS_RTOL * max(rt, 1e-300), (total, rt)


def test_grid_on_its_coordinates_and_path_on_a_line():
    g = gg.grid(40, 25)
    X = np.array([[v % 40, v // 40] for v in range(g.n)], dtype=np.float32)
    c, inter, total = gpu_np(g, X, 2)
    assert np.array_equal(c, inter) and total == float(g.n)
    p = gg.path(300)
    total, rows = gpu_stress(p, np.array([[v, 0.0] for v in range(300)], dtype=np.float32))
    assert total == 0.0 and np.all(rows == 0.0)


@pytest.mark.parametrize("maker", [gg.config_ba20k, gg.config_er5k], ids=["ba20k", "er5k"])
def test_headline_graphs_sampled(maker):
    """At the headline graphs' sizes: every vertex on the GPU, a seeded sample
    of vertices (and of stress rows) on the oracle."""
    g = maker()
    X = np.random.default_rng(9).standard_normal((g.n, 2)).astype(np.float32)
    sample = np.random.default_rng(10).choice(g.n, size=40, replace=False).astype(np.int32)
    c, inter, _ = gpu_np(g, X, 2)
    rc, ri, _ = oracle.np_metric(g, X, 2, vertices=sample)
    assert np.array_equal(c[sample], rc) and np.array_equal(inter[sample], ri)
    _, rows = gpu_stress(g, X)
    _, rr = oracle.stress(g, X, vertices=sample)
    np.testing.assert_allclose(rows[sample], rr, rtol=STRESS_RTOL)


def test_bad_arguments_are_rejected():
    g = gg.path(10)
    with gumap.KnnGraph.from_graph(g, 2) as kg:
        X = torch.zeros((10, 9), dtype=torch.float32, device="cuda")
        with pytest.raises(gumap.GumapError) as e:
            kg.quality_np(X, 2)
        assert e.value.status == gumap.ERR_INVALID_ARG
        with pytest.raises(gumap.GumapError) as e:
            kg.quality_np(torch.zeros((10, 2), dtype=torch.float32, device="cuda"), 0)
        assert e.value.status == gumap.ERR_INVALID_ARG
        with pytest.raises(gumap.GumapError) as e:
            kg.quality_stress(X)
        assert e.value.status == gumap.ERR_INVALID_ARG
    kb, _ = gumap.KnnGraph.batch([gg.path(5), gg.path(6)], 2, [gumap.FULL, gumap.FULL])
    with kb:
        with pytest.raises(gumap.GumapError) as e:
            kb.quality_stress(torch.zeros((11, 2), dtype=torch.float32, device="cuda"))
        assert e.value.status == gumap.ERR_INVALID_ARG
