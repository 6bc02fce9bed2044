"""Failure handling, tested without faulting a GPU.

GPU: a device-side wait that can never complete gives up after its limit and
reports GUMAP_ERR_TIMEOUT, and the context keeps working; a source id outside
the graph becomes a padded row and is reported by gumap_knn_check.
CPU: the replicated multi-rank bench step (gloo, world size 2) agrees on the
slowest rank's time, and a rank that dies before the collective makes the
other rank's collective fail within its timeout instead of hanging."""
import os
import time

import numpy as np
import pytest

from paper_2509_19703_gb300 import graphgen as gg


# ------------------------------------------------------------------ GPU

@pytest.mark.gpu
def test_bounded_wait_gives_up_and_context_survives():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_helpers import assert_parity, oracle_ref, run_gpu
    from paper_2509_19703_gb300 import gumap
    t0 = time.perf_counter()
    st = gumap.gumap_selftest_wait_timeout(0, 0.05)
    assert st == gumap.ERR_TIMEOUT, gumap.gumap_status_string(st)
    assert time.perf_counter() - t0 < 5.0
    g = gg.grid(12, 12)
    assert_parity(run_gpu(g, 15, "full"), oracle_ref(g, 15, "full"), "after timeout")


@pytest.mark.gpu
@pytest.mark.parametrize("engine", ["msbfs", "frontier"])
def test_out_of_range_source_is_reported(engine):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_2509_19703_gb300 import gumap
    g = gg.barabasi_albert(300, 3, 141)
    src = np.array([5, 17, g.n + 3, 42, -1], dtype=np.int32)
    mode = gumap.PARTIAL
    with gumap.KnnGraph.from_graph(g, 10, mode=mode, flags=gumap.WEIGHTS_DIRECTED) as kg:
        kg.set_option(gumap.OPT_ENGINE, gumap.ENGINE_MSBFS if engine == "msbfs" else gumap.ENGINE_FRONTIER)
        out = kg.run(sources=torch.as_tensor(src, device="cuda"))
        with pytest.raises(gumap.GumapError) as e:
            kg.check()
        assert e.value.status == gumap.ERR_INVALID_ARG
        idx = out["idx"].cpu().numpy()
        good = np.array([0, 1, 3])
        want, _ = oracle.knn_partial(g, 10, sources=src[good])
        assert np.array_equal(idx[good], want)
        assert np.all(idx[[2, 4]] == -1)
        kg.check()  # the status word was cleared by the first check


# ------------------------------------------------------------------ CPU, gloo

def _rank_main(rank, world, port, mode, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import datetime
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    try:
        if mode == "die" and rank == 1:
            raise SystemExit(3)  # leaves before the collective
        ms = bench.max_over_ranks(1.0 + rank, world)
        q.put((rank, "ok", ms, bench.job_value(1000, world, ms)))
    except SystemExit:
        raise
    except Exception as e:  # the collective failed on the surviving rank
        q.put((rank, "error", type(e).__name__, None))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def _spawn(mode):
    import multiprocessing as mp
    import socket
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, mode, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
            pytest.fail("a rank did not finish")
    out = []
    while not q.empty():
        out.append(q.get())
    return sorted(out), [p.exitcode for p in procs]


def test_replicas_agree_on_the_slowest_rank():
    res, codes = _spawn("ok")
    assert codes == [0, 0]
    assert [r[1] for r in res] == ["ok", "ok"]
    assert all(r[2] == 2.0 for r in res)              # max over ranks
    assert all(abs(r[3] - 2 * 1000 / 2e-3 / 1e9) < 1e-12 for r in res)  # both ranks' work / slowest time


def test_dead_rank_fails_the_collective_instead_of_hanging():
    res, codes = _spawn("die")
    assert codes[1] == 3
    assert res and res[0][0] == 0 and res[0][1] == "error"
