"""Request server (gumap_server_*): continuous batching under a device-memory
budget. Every result must be identical to the same graph computed alone by
a gumap_knn handle, whether it ran batched with others, alone, or was
admitted late because memory was short; and every result of the mixed
stream is checked against the CPU oracle (ids and distances exact, weights
within 1e-5)."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from gpu_helpers import W_TOL
from paper_2509_19703_gb300 import graphgen as gg
from paper_2509_19703_gb300 import gumap

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gumap.load()


def alone(g, k, mode):
    with gumap.KnnGraph.from_graph(g, k, mode=mode) as kg:
        out = kg.run()
        kg.check()
        return out["idx"].cpu().numpy(), gumap.dist_u16(out["dist"]), out["w"].cpu().numpy()


def read(s, rid, g, k):
    idx = torch.empty((g.n, k), dtype=torch.int32, device="cuda")
    dist = torch.empty((g.n, k), dtype=torch.int16, device="cuda")
    w = torch.empty((g.n, k), dtype=torch.float32, device="cuda")
    gumap.gumap_serve_read(s, rid, idx, dist, w)
    torch.cuda.synchronize()
    return idx.cpu().numpy(), gumap.dist_u16(dist), w.cpu().numpy()


def request_mix(count, seed):
    u = gg.uniform(seed, 3 * count).reshape(count, 3)
    out = []
    for i in range(count):
        n = int(np.exp(np.log(50) + u[i, 0] * (np.log(6000) - np.log(50))))
        kind = int(u[i, 1] * 3)
        g = (gg.barabasi_albert(max(n, 6), 3, seed * 1000 + i) if kind == 0 else
             gg.grid(max(2, int(np.sqrt(n))), max(2, int(np.sqrt(n)))) if kind == 1 else
             gg.gnp(n, min(1.0, 12.0 / n), seed * 1000 + i))
        k = 15 if u[i, 2] < 0.5 else 30
        mode = gumap.PARTIAL if (i % 10) < 7 else gumap.FULL
        out.append((g, min(k, g.n - 1), mode))
    return out


def check_all(s, reqs, against_oracle=False):
    for rid, (g, k, mode) in reqs:
        st, res = gumap.gumap_serve_wait(s, rid, 120.0)
        assert st == gumap.OK, (g.name, gumap.gumap_status_string(st))
        got = read(s, rid, g, k)
        want = alone(g, k, mode)
        for a, b, name in zip(got, want, ("idx", "dist", "w")):
            assert np.array_equal(a, b), (g.name, name, res["batch_graphs"], res["engine"])
        if against_oracle:
            # the two forms give the same rows (a pinned property of the oracle); the full
            # form's all-pairs BFS is used up to 6000 vertices, the partial one beyond
            form = "full" if mode == gumap.FULL and g.n <= 6000 else "partial"
            ref = oracle.knn_pipeline(g, k, form)
            assert np.array_equal(got[0], ref["idx"]) and np.array_equal(got[1], ref["dist"]), g.name
            err = float(np.max(np.abs(got[2].astype(np.float64) - ref["w"])))
            assert err <= W_TOL, (g.name, err)
        gumap.gumap_serve_release(s, rid)


def test_results_identical_alone_and_in_the_mix():
    mix = request_mix(48, 101)
    mix += [(gg.barabasi_albert(30000, 3, 102), 15, gumap.PARTIAL),   # too large to batch: frontier engine
            (gg.barabasi_albert(30000, 3, 103), 15, gumap.FULL)]      # too large to batch: MS-BFS engine
    s = gumap.gumap_server_create(0, 4 << 30)
    try:
        reqs = [(gumap.gumap_serve_submit(s, g.row_ptr, g.col, g.n, g.nnz, k, m), (g, k, m)) for g, k, m in mix]
        check_all(s, reqs, against_oracle=True)
        st = gumap.gumap_server_get_stats(s)
        assert st["completed"] == len(mix) and st["failed"] == 0
    finally:
        gumap.gumap_server_destroy(s)


def test_a_backlog_is_batched():
    """With one worker stream busy on a large full-form graph, the small
    requests that arrive meanwhile wait together and leave in few batched
    launches (how many arrive while a stream is busy is a matter of timing
    otherwise, so the test makes the backlog certain)."""
    big = (gg.barabasi_albert(60000, 4, 104), 15, gumap.FULL)
    small = request_mix(40, 105)
    s = gumap.gumap_server_create(0, 4 << 30, n_streams=1)
    try:
        reqs = [(gumap.gumap_serve_submit(s, g.row_ptr, g.col, g.n, g.nnz, k, m), (g, k, m))
                for g, k, m in [big] + small]
        check_all(s, reqs)
        st = gumap.gumap_server_get_stats(s)
        assert st["completed"] == 1 + len(small) and st["failed"] == 0
        assert st["launches"] < 1 + len(small) // 2, st  # the small requests were batched together
    finally:
        gumap.gumap_server_destroy(s)


def test_requests_arriving_while_others_run():
    s = gumap.gumap_server_create(0, 2 << 30, n_streams=2)
    try:
        reqs = []
        for wave in range(4):
            for g, k, m in request_mix(12, 110 + wave):
                reqs.append((gumap.gumap_serve_submit(s, g.row_ptr, g.col, g.n, g.nnz, k, m), (g, k, m)))
            time.sleep(0.002)
        check_all(s, reqs)
    finally:
        gumap.gumap_server_destroy(s)


def test_admission_under_a_small_budget():
    """A 48 MiB budget holds only a few launches at a time: the rest wait for
    releases, then run; a request larger than the budget is refused."""
    s = gumap.gumap_server_create(0, 48 << 20, n_streams=2, max_batch_graphs=4)
    try:
        mix = request_mix(30, 120)
        reqs = [(gumap.gumap_serve_submit(s, g.row_ptr, g.col, g.n, g.nnz, k, m), (g, k, m)) for g, k, m in mix]
        check_all(s, reqs)
        big = gg.grid(600, 600)
        with pytest.raises(gumap.GumapError) as e:
            gumap.gumap_serve_submit(s, big.row_ptr, big.col, big.n, big.nnz, 30, gumap.FULL)
        assert e.value.status == gumap.ERR_TOO_LARGE
        st = gumap.gumap_server_get_stats(s)
        assert st["arena_peak_bytes"] <= st["arena_bytes"]
    finally:
        gumap.gumap_server_destroy(s)


def test_release_and_unknown_requests():
    s = gumap.gumap_server_create(0, 256 << 20)
    try:
        g = gg.grid(20, 20)
        rid = gumap.gumap_serve_submit(s, g.row_ptr, g.col, g.n, g.nnz, 15, gumap.PARTIAL)
        st, _ = gumap.gumap_serve_wait(s, rid, 60.0)
        assert st == gumap.OK
        gumap.gumap_serve_release(s, rid)
        with pytest.raises(gumap.GumapError) as e:
            gumap.gumap_serve_release(s, rid)
        assert e.value.status == gumap.ERR_UNKNOWN_REQUEST
        with pytest.raises(gumap.GumapError) as e:
            gumap.gumap_serve_read(s, 987654, None, None, None)
        assert e.value.status == gumap.ERR_UNKNOWN_REQUEST
        bad = g.col.copy()
        bad[0] = 0  # self loop
        with pytest.raises(gumap.GumapError) as e:
            gumap.gumap_serve_submit(s, g.row_ptr, bad, g.n, g.nnz, 15, gumap.PARTIAL)
        assert e.value.status == gumap.ERR_INVALID_GRAPH
    finally:
        gumap.gumap_server_destroy(s)


def test_queue_full_returns_again():
    s = gumap.gumap_server_create(0, 1 << 30, n_streams=1, max_queue=2)
    try:
        heavy = gg.barabasi_albert(30000, 3, 130)
        small = gg.grid(10, 10)
        ids = [gumap.gumap_serve_submit(s, heavy.row_ptr, heavy.col, heavy.n, heavy.nnz, 15, gumap.FULL)]
        saw_again = False
        for _ in range(50):
            try:
                ids.append(gumap.gumap_serve_submit(s, small.row_ptr, small.col, small.n, small.nnz, 5,
                                                    gumap.PARTIAL))
            except gumap.GumapError as e:
                assert e.status == gumap.ERR_AGAIN
                saw_again = True
                break
        assert saw_again
        for rid in ids:
            st, _ = gumap.gumap_serve_wait(s, rid, 120.0)
            assert st == gumap.OK
            gumap.gumap_serve_release(s, rid)
    finally:
        gumap.gumap_server_destroy(s)
