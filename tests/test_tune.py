"""Autotuner (gumap_knn_autotune): the chosen settings never change the
rows, the cache round-trips, and GUMAP_TUNE_CACHE applies cached settings
to a new handle of the same shape class."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_helpers import assert_parity, oracle_ref
from paper_2509_19703_gb300 import graphgen as gg
from paper_2509_19703_gb300 import gumap

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gumap.load()


def _rows(kg):
    out = kg.run()
    r, c, w = kg.coo()
    rho, sigma = kg.rho_sigma()
    kg.check()
    return dict(idx=out["idx"].cpu().numpy(), dist=gumap.dist_u16(out["dist"]),
                w=out["w"].cpu().numpy().astype(np.float64),
                coo=(r.cpu().numpy(), c.cpu().numpy(), w.cpu().numpy().astype(np.float64)),
                rho=rho.cpu().numpy().astype(np.float64), sigma=sigma.cpu().numpy().astype(np.float64))


@pytest.mark.parametrize("mode", ["full", "partial"])
def test_autotune_keeps_the_rows_and_caches(tmp_path, mode):
    g = gg.barabasi_albert(4000, 4, 151)
    m = gumap.FULL if mode == "full" else gumap.PARTIAL
    cache = str(tmp_path / "tune.jsonl")
    ref = oracle_ref(g, 15, mode)
    with gumap.KnnGraph.from_graph(g, 15, mode=m) as kg:
        res = kg.autotune(cache)
        assert res["from_cache"] == 0 and res["candidates"] >= 3
        assert res["best_ms"] <= res["default_ms"] * 1.5
        assert_parity(_rows(kg), ref, f"tuned {mode}")
    lines = [json.loads(x) for x in open(cache)]
    assert len(lines) == 1 and lines[0]["engine"] == res["engine"]
    with gumap.KnnGraph.from_graph(g, 15, mode=m) as kg:
        res2 = kg.autotune(cache)
        assert res2["from_cache"] == 1 and res2["engine"] == res["engine"]
        assert_parity(_rows(kg), ref, f"cached {mode}")


def test_environment_cache_applies_at_creation(tmp_path):
    """A new process with GUMAP_TUNE_CACHE set starts with the cached engine."""
    g = gg.barabasi_albert(3000, 3, 152)
    cache = tmp_path / "c.jsonl"
    with gumap.KnnGraph.from_graph(g, 15, mode=gumap.PARTIAL) as kg:
        kg.autotune(str(cache))
    want = json.loads(cache.read_text().splitlines()[0])["engine"]
    code = (
        "import sys; sys.path[:0] = [%r]\n"
        "from paper_2509_19703_gb300 import graphgen as gg, gumap\n"
        "g = gg.barabasi_albert(3000, 3, 152)\n"
        "kg = gumap.KnnGraph.from_graph(g, 15, mode=gumap.PARTIAL)\n"
        "kg.run(); kg.check(); print(kg.stats()['engine'])\n" % os.getcwd())
    env = dict(os.environ, GUMAP_TUNE_CACHE=str(cache))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=300)
    assert out.returncode == 0, out.stderr
    assert int(out.stdout.strip().splitlines()[-1]) == want
