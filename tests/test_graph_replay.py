"""Runs replayed from a captured CUDA graph (GUMAP_OPT_GRAPH): the third run
with the same arguments on a non-default stream is captured and later runs
replay it; every run's rows (outputs cleared between runs) equal the
oracle's, on each engine, and any other call drops the graph."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_helpers import oracle_ref  # noqa: E402
from paper_2509_19703_gb300 import graphgen as gg  # noqa: E402
from paper_2509_19703_gb300 import gumap  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gumap.load()


CASES = [(gg.grid(32, 32), "full", gumap.ENGINE_BATCH), (gg.grid(32, 32), "full", gumap.ENGINE_MSBFS),
         (gg.barabasi_albert(3000, 3, 9), "partial", gumap.ENGINE_FRONTIER),
         (gg.barabasi_albert(3000, 3, 9), "partial", gumap.ENGINE_MSBFS)]


@pytest.mark.parametrize("g,mode,engine", CASES, ids=[f"{g.name}-{m}-e{e}" for g, m, e in CASES])
def test_replayed_runs_give_the_oracle_rows(g, mode, engine):
    ref = oracle_ref(g, 15, mode)
    s = torch.cuda.Stream()
    m = gumap.FULL if mode == "full" else gumap.PARTIAL
    with gumap.KnnGraph.from_graph(g, 15, mode=m) as kg:
        kg.set_option(gumap.OPT_ENGINE, engine)
        kg.set_option(gumap.OPT_GRAPH, 1)
        out = kg.alloc_outputs(g.n)
        for i in range(6):
            with torch.cuda.stream(s):
                for t in out.values():
                    t.zero_()
                kg.run(stream=s, out=out)
            s.synchronize()
            kg.check(stream=s)
            assert np.array_equal(out["idx"].cpu().numpy(), ref["idx"]), (g.name, i)
            assert np.array_equal(gumap.dist_u16(out["dist"]), ref["dist"]), (g.name, i)
            err = float(np.max(np.abs(out["w"].cpu().numpy().astype(np.float64) - ref["w"])))
            assert err <= 1e-5, (g.name, i, err)
        replays = kg.stats()["graph_replays"]
        if engine == gumap.ENGINE_MSBFS:
            # a cooperative launch in the capture may be refused: then every run was ordinary
            assert replays == 0 or replays >= 4, replays
            print(f"MS-BFS runs replayed from the graph: {replays}")
        else:
            assert replays >= 4, replays  # runs 3..6 came from the graph
        r, c, w = kg.coo()  # the replayed run's COO
        assert np.array_equal(r.cpu().numpy(), ref["coo"][0]) and np.array_equal(c.cpu().numpy(), ref["coo"][1])


def test_other_calls_drop_the_graph():
    g = gg.grid(16, 16)
    ref = oracle_ref(g, 15, "full")
    s = torch.cuda.Stream()
    with gumap.KnnGraph.from_graph(g, 15) as kg:
        kg.set_option(gumap.OPT_ENGINE, gumap.ENGINE_BATCH)
        kg.set_option(gumap.OPT_GRAPH, 1)
        out = kg.alloc_outputs(g.n)
        for _ in range(4):
            kg.run(stream=s, out=out)
        s.synchronize()
        before = kg.stats()["graph_replays"]
        assert before >= 2
        kg.set_option(gumap.OPT_ENGINE, gumap.ENGINE_MSBFS)  # drops the graph and the warm-up count
        kg.run(stream=s, out=out)
        s.synchronize()
        assert kg.stats()["graph_replays"] == before
        assert np.array_equal(out["idx"].cpu().numpy(), ref["idx"])
        other = kg.alloc_outputs(g.n)  # new outputs: a new key, warmed up again
        kg.run(stream=s, out=other)
        s.synchronize()
        assert kg.stats()["graph_replays"] == before
        assert np.array_equal(other["idx"].cpu().numpy(), ref["idx"])
