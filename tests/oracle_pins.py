"""Pins for the CPU oracle: checks against what the paper and mathematics fix,
independent of the oracle's own code.

Each ``check_*`` takes an ``oracle.Oracle`` and raises AssertionError on a
mismatch. ``test_oracle_pins.py`` runs them on the real oracle;
``test_oracle_mutations.py`` runs them on copies of the oracle with planted
mistakes and requires every mistake to be caught.

Independent references used here:
  * Floyd-Warshall on a dense matrix (distances), a different algorithm from BFS;
  * closed-form hop distances on grids, paths, cycles, stars, complete graphs;
  * hand-derived kNN lists (tests/golden/closed_forms.json);
  * the calibration equation sum_j exp(-(d_j - rho)/sigma) = log2 k written as
    a polynomial in x = exp(-1/sigma) and solved by numpy.roots (companion
    matrix eigenvalues), not by bisection;
  * closed-form fuzzy-union weights on a star;
  * for the quality metrics of a drawing (Section 4.1.3): hand-derived
    values (tests/golden/quality_closed_forms.json), a grid drawn on its own
    integer coordinates (neighbourhood preservation 1 at every vertex), a path
    on a unit line and a star on the unit circle (stress in closed form), and
    brute force over the Floyd-Warshall matrix with numpy sorting.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

from paper_2509_19703_gb300 import graphgen as gg

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "closed_forms.json")
QUALITY_GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "quality_closed_forms.json")
INF16 = 0xFFFF


# --------------------------------------------------------------------------
# small graph zoo
# --------------------------------------------------------------------------

def tiny_graphs():
    """Seeded tiny graphs (n <= 64), connected and disconnected."""
    out = []
    for n, p, seed in [(1, 0.5, 1), (2, 1.0, 2), (5, 0.4, 3), (17, 0.15, 4), (40, 0.06, 5),
                       (64, 0.05, 6), (64, 0.2, 7), (33, 0.0, 8)]:
        out.append(gg.gnp(n, p, seed))
    out.append(gg.random_tree(50, 9))
    out.append(gg.barabasi_albert(60, 2, 10))
    out.append(gg.disjoint_union([gg.path(3), gg.cycle(7), gg.star(9), gg.grid(4, 5)], "mix"))
    out.append(gg.disjoint_union([gg.gnp(20, 0.2, 11), gg.complete(6), gg.path(1)], "mix2"))
    return out


def floyd_warshall(g) -> np.ndarray:
    n = g.n
    D = np.full((n, n), np.inf)
    if n:
        np.fill_diagonal(D, 0.0)
    for u in range(n):
        for e in range(g.row_ptr[u], g.row_ptr[u + 1]):
            D[u, g.col[e]] = 1.0
    for m in range(n):
        D = np.minimum(D, D[:, m:m + 1] + D[m:m + 1, :])
    return D


def brute_knn(D: np.ndarray, k: int):
    n = D.shape[0]
    idx = np.full((n, k), -1, dtype=np.int64)
    dist = np.full((n, k), INF16, dtype=np.int64)
    for s in range(n):
        cand = sorted((D[s, v], v) for v in range(n) if v != s and np.isfinite(D[s, v]))[:k]
        for t, (d, v) in enumerate(cand):
            idx[s, t] = v
            dist[s, t] = int(d)
    return idx, dist


# --------------------------------------------------------------------------
# distances and lists
# --------------------------------------------------------------------------

def check_apsp_floyd_warshall(orc):
    for g in tiny_graphs():
        D = floyd_warshall(g)
        A = orc.apsp(g).astype(np.float64)
        A[A == INF16] = np.inf
        assert np.array_equal(A, D), g.name


def check_knn_brute_force(orc):
    for g in tiny_graphs():
        if g.n < 2:
            continue
        D = floyd_warshall(g)
        for k in sorted({1, 3, 15, g.n - 1}):
            bi, bd = brute_knn(D, k)
            for fn in (orc.knn_full, orc.knn_partial):
                idx, dist = fn(g, k)
                assert np.array_equal(idx, bi), (g.name, k, fn.__name__)
                assert np.array_equal(dist.astype(np.int64), bd), (g.name, k, fn.__name__)


def check_closed_form_distances(orc):
    W, H = 6, 9
    D = orc.apsp(gg.grid(W, H)).astype(np.int64)
    r, c = np.divmod(np.arange(W * H), W)
    assert np.array_equal(D, np.abs(r[:, None] - r[None, :]) + np.abs(c[:, None] - c[None, :]))
    i = np.arange(13)
    assert np.array_equal(orc.apsp(gg.path(13)).astype(np.int64), np.abs(i[:, None] - i[None, :]))
    for n in (11, 12):
        i = np.arange(n)
        a = np.abs(i[:, None] - i[None, :])
        assert np.array_equal(orc.apsp(gg.cycle(n)).astype(np.int64), np.minimum(a, n - a))
    K = orc.apsp(gg.complete(9)).astype(np.int64)
    assert np.array_equal(K, 1 - np.eye(9, dtype=np.int64))
    S = orc.apsp(gg.star(10)).astype(np.int64)
    exp = np.full((10, 10), 2)
    exp[0, :] = 1
    exp[:, 0] = 1
    np.fill_diagonal(exp, 0)
    assert np.array_equal(S, exp)


def _golden_graph(case):
    kind = case["graph"]
    if kind == "grid":
        return gg.grid(case["W"], case["H"])
    return {"path": gg.path, "cycle": gg.cycle, "star": gg.star, "complete": gg.complete}[kind](case["n"])


def check_golden_lists(orc):
    with open(GOLDEN) as f:
        cases = json.load(f)["cases"]
    for case in cases:
        g = _golden_graph(case)
        v, k = case["vertex"], case["k"]
        for fn in (orc.knn_full, orc.knn_partial):
            idx, dist = fn(g, k, sources=np.array([v]))
            assert idx[0].tolist() == case["idx"], (case["why"], fn.__name__, idx[0].tolist())
            assert dist[0].astype(int).tolist() == case["dist"], (case["why"], fn.__name__)


def check_full_equals_partial(orc):
    graphs = [gg.barabasi_albert(400, 3, 21), gg.gnp(300, 0.02, 22), gg.random_tree(300, 23),
              gg.grid(17, 23), gg.disjoint_union([gg.gnp(100, 0.01, 24), gg.path(5)], "dis")]
    for g in graphs:
        for k in (1, 7, 15, 50):
            a = orc.knn_full(g, k)
            b = orc.knn_partial(g, k)
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), (g.name, k)


def check_partial_work(orc):
    """Edges scanned before the stopping level on a grid interior vertex:
    k=15 stops at D=3 after expanding 1+4+8 vertices of degree 4 (52);
    k=50 stops at D=5 after 1+4+8+12+16 vertices (164)."""
    W = 30
    g = gg.grid(W, W)
    v = 15 * W + 15
    for k, want in ((15, 52), (50, 164)):
        _, _, work = orc.knn_partial(g, k, sources=np.array([v]), return_work=True)
        assert int(work[0]) == want, (k, int(work[0]))
    # closed forms: path interior at k = 15 stops at D = 8 after 1 + 14
    # vertices of degree 2 (30), at k = 1 after the source alone (2); a star's
    # centre after itself (n - 1); a leaf after itself at k = 1 (1), after
    # itself and the centre at k >= 2 (1 + n - 1); K_n after the source
    # (n - 1); a component of fewer than k + 1 vertices is exhausted (2 m).
    cases = [(gg.path(100), 50, 15, 30), (gg.path(100), 50, 1, 2), (gg.star(40), 0, 15, 39),
             (gg.star(40), 7, 1, 1), (gg.star(40), 7, 15, 40), (gg.complete(20), 3, 15, 19),
             (gg.disjoint_union([gg.path(5), gg.complete(30)], "p5k30"), 2, 15, 8)]
    for g, v, k, want in cases:
        _, _, work = orc.knn_partial(g, k, sources=np.array([v]), return_work=True)
        assert int(work[0]) == want, (g.name, v, k, int(work[0]))
    # brute force from Floyd-Warshall distances: D_s is the k-th smallest
    # distance to another reachable vertex (infinite if fewer than k), and
    # the work is the degree sum over the vertices closer than D_s
    for g in tiny_graphs():
        if g.n < 2:
            continue
        D = floyd_warshall(g)
        deg = np.diff(g.row_ptr)
        for k in sorted({1, 3, min(15, g.n - 1)}):
            _, _, work = orc.knn_partial(g, k, return_work=True)
            for s_ in range(g.n):
                others = np.sort(D[s_][np.isfinite(D[s_]) & (np.arange(g.n) != s_)])
                Ds = others[k - 1] if len(others) >= k else np.inf
                want = int(deg[D[s_] < Ds].sum())
                assert int(work[s_]) == want, (g.name, k, s_, int(work[s_]), want)


# --------------------------------------------------------------------------
# rho, sigma, weights
# --------------------------------------------------------------------------

def _root_in_unit(coeffs_high_to_low):
    r = np.roots(coeffs_high_to_low)
    real = [z.real for z in r if abs(z.imag) < 1e-12 and 0.0 < z.real < 1.0]
    assert len(real) == 1, r
    return real[0]


def _sigma_of_x(x):
    return -1.0 / math.log(x)


def _row(orc, g, v, k):
    idx, dist = orc.knn_full(g, k, sources=np.array([v]))
    rho, sigma, a = orc.smooth_knn(dist)
    return idx[0], dist[0].astype(int), float(rho[0]), float(sigma[0]), a[0]


def check_sigma_closed_forms(orc):
    T15 = math.log2(15)
    # star leaf: 1 + 14 x = log2 15
    idx, d, rho, sigma, a = _row(orc, gg.star(40), 5, 15)
    x = (T15 - 1.0) / 14.0
    assert rho == 1.0
    assert abs(sigma - _sigma_of_x(x)) <= 1e-12 * _sigma_of_x(x), (sigma, _sigma_of_x(x))
    assert abs(a[0] - 1.0) == 0.0 and np.allclose(a[1:], x, rtol=1e-12, atol=0)
    # star centre: all 15 at d = rho, no root -> sigma floor 1e-3 * mean(d) = 1e-3, weights 1
    idx, d, rho, sigma, a = _row(orc, gg.star(40), 0, 15)
    assert abs(sigma - 1e-3) <= 1e-15 and np.all(a == 1.0)
    # grid top-edge vertex: 3 + 5x + 7x^2 = log2 15
    idx, d, rho, sigma, a = _row(orc, gg.grid(9, 9), 4, 15)
    x = (-5.0 + math.sqrt(25.0 + 28.0 * (T15 - 3.0))) / 14.0
    assert abs(sigma - _sigma_of_x(x)) <= 1e-12 * _sigma_of_x(x)
    want = np.array([x ** (dd - 1) for dd in d])
    assert np.allclose(a, want, rtol=1e-11, atol=0)
    # grid interior, k = 50: 4 + 8x + 12x^2 + 16x^3 + 10x^4 = log2 50
    idx, d, rho, sigma, a = _row(orc, gg.grid(21, 21), 10 * 21 + 10, 50)
    x = _root_in_unit([10.0, 16.0, 12.0, 8.0, 4.0 - math.log2(50)])
    assert abs(sigma - _sigma_of_x(x)) <= 1e-10 * _sigma_of_x(x)
    assert np.allclose(a, [x ** (dd - 1) for dd in d], rtol=1e-9, atol=0)
    # path interior, k = 15: 2 + 2x + ... + 2x^6 + x^7 = log2 15
    idx, d, rho, sigma, a = _row(orc, gg.path(40), 20, 15)
    x = _root_in_unit([1.0, 2, 2, 2, 2, 2, 2, 2.0 - T15])
    assert abs(sigma - _sigma_of_x(x)) <= 1e-10 * _sigma_of_x(x)
    # grid interior, k = 15: 4 at d = rho > log2 15: no root, sigma = 1e-3 * mean d
    idx, d, rho, sigma, a = _row(orc, gg.grid(9, 9), 40, 15)
    mean = (4 * 1 + 8 * 2 + 3 * 3) / 15.0
    assert abs(sigma - 1e-3 * mean) <= 1e-15
    assert np.all(a[:4] == 1.0) and np.all(a[4:] < 1e-200)
    # complete graph: every weight 1
    idx, d, rho, sigma, a = _row(orc, gg.complete(20), 3, 15)
    assert np.all(a == 1.0)
    # component of 3 vertices with k = 15: 2 valid entries <= log2 15, sigma = inf, weights 1
    idx, d, rho, sigma, a = _row(orc, gg.path(3), 0, 15)
    assert math.isinf(sigma) and a[0] == 1.0 and a[1] == 1.0 and np.all(a[2:] == 0.0)
    # isolated vertex: nothing valid
    idx, d, rho, sigma, a = _row(orc, gg.disjoint_union([gg.path(1), gg.path(4)]), 0, 5)
    assert rho == 0.0 and sigma == 0.0 and np.all(a == 0.0)


def check_sigma_residual(orc):
    """Wherever a root exists, f(sigma) hits log2 k to 1e-12 relative."""
    for g, k in ((gg.barabasi_albert(500, 3, 31), 15), (gg.random_tree(400, 32), 15),
                 (gg.gnp(300, 0.03, 33), 30)):
        idx, dist = orc.knn_full(g, k)
        rho, sigma, a = orc.smooth_knn(dist)
        T = math.log2(k)
        checked = 0
        for i in range(g.n):
            d = dist[i][dist[i] != INF16].astype(np.float64)
            if d.size == 0:
                continue
            c_eq = int(np.sum(d == rho[i]))
            if not (c_eq < T < d.size):
                continue
            f = float(np.sum(np.exp(-np.maximum(0.0, d - rho[i]) / sigma[i])))
            assert abs(f - T) <= 1e-12 * T, (g.name, i, f, T)
            checked += 1
        assert checked > 0


# --------------------------------------------------------------------------
# fuzzy union
# --------------------------------------------------------------------------

def check_union_star(orc):
    """Star with centre 0 and leaves 1..39, k = 15. A leaf j lists the centre
    (a = 1) and the 14 smallest other leaves (a = x, x = (log2 15 - 1)/14);
    the centre lists leaves 1..15 (a = 1). So w(i, j) = 1 when either end is
    the centre, 2x - x^2 between two leaves that list each other and x when
    only one does."""
    n, k = 40, 15
    g = gg.star(n)
    r = orc.knn_pipeline(g, k)
    x = (math.log2(15) - 1.0) / 14.0

    def listed(i, j):  # does i list j?
        if i == 0:
            return 1 <= j <= 15
        if j == 0:
            return True
        others = [v for v in range(1, n) if v != i][:14]
        return j in others

    for i in range(n):
        for t in range(k):
            j = int(r["idx"][i, t])
            if i == 0 or j == 0:
                want = 1.0
            else:
                want = 2 * x - x * x if listed(j, i) else x
            assert abs(r["w"][i, t] - want) <= 1e-13, (i, j, r["w"][i, t], want)
    row, col, w = r["coo"]
    pairs = {(int(a), int(b)): float(c) for a, b, c in zip(row, col, w)}
    expected = set()
    for i in range(n):
        for j in range(n):
            if i != j and (listed(i, j) or listed(j, i)):
                expected.add((i, j))
    assert set(pairs) == expected
    for (i, j), v in pairs.items():
        if i == 0 or j == 0:
            want = 1.0
        else:
            want = 2 * x - x * x if (listed(i, j) and listed(j, i)) else x
        assert abs(v - want) <= 1e-13, (i, j, v, want)


def check_union_properties(orc):
    for g, k in ((gg.barabasi_albert(300, 3, 41), 15), (gg.grid(12, 9), 15),
                 (gg.disjoint_union([gg.random_tree(80, 42), gg.path(2)]), 10)):
        r = orc.knn_pipeline(g, k)
        row, col, w = r["coo"]
        key = row.astype(np.int64) * g.n + col
        assert np.all(np.diff(key) > 0), "COO not strictly sorted"
        assert np.all((w >= 0) & (w <= 1))
        pairs = {(int(a), int(b)): float(c) for a, b, c in zip(row, col, w)}
        for (i, j), v in pairs.items():
            assert pairs.get((j, i)) == v, "COO not symmetric"
        valid = int(np.sum(r["idx"] >= 0))
        assert valid <= row.shape[0] <= 2 * valid
        for i in range(g.n):
            for t in range(k):
                j = int(r["idx"][i, t])
                if j < 0:
                    assert r["w"][i, t] == 0.0
                    continue
                assert abs(pairs[(i, j)] - r["w"][i, t]) <= 1e-15
                if r["dist"][i, t] == r["rho"][i]:
                    assert r["w"][i, t] == 1.0


# --------------------------------------------------------------------------
# quality metrics of a drawing (Section 4.1.3)
# --------------------------------------------------------------------------

def _quality_graph(name, n):
    if name == "path":
        return gg.path(n)
    if name == "star":
        return gg.star(n)
    if name == "complete":
        return gg.complete(n)
    if name == "two_k2":
        return gg.disjoint_union([gg.path(2), gg.path(2)], "two_k2")
    raise ValueError(name)


def _closed_value(expr):
    return {"(sqrt(2) - 1)^2 / 3": (math.sqrt(2.0) - 1.0) ** 2 / 3.0, "2/3": 2.0 / 3.0, "0": 0.0}[expr]


def check_np_golden(orc):
    with open(QUALITY_GOLDEN) as f:
        cases = json.load(f)["np_cases"]
    for case in cases:
        g = _quality_graph(case["graph"], case["n"])
        X = np.asarray(case["X"], dtype=np.float32)
        c, inter, total = orc.np_metric(g, X, case["r"])
        assert c.tolist() == case["c"], (case["why"], c.tolist())
        assert inter.tolist() == case["inter"], (case["why"], inter.tolist())
        assert abs(total - case["sum_num"] / case["sum_den"]) <= 1e-12, (case["why"], total)


def check_np_grid_on_its_coordinates(orc):
    """A grid drawn at its integer coordinates: the hop ball of radius r <= 2
    is exactly the set of lattice points at squared distance <= r^2 (1, 2, 4
    for r = 2; the next squared distance is 5), so N_D = N_G at every vertex."""
    for W, H in ((7, 5), (3, 9), (12, 12), (1, 6)):
        g = gg.grid(W, H)
        X = np.array([[v % W, v // W] for v in range(g.n)], dtype=np.float32)
        for r in (1, 2):
            c, inter, total = orc.np_metric(g, X, r)
            for v in range(g.n):
                i, j = v // W, v % W
                want = sum(1 for a in range(H) for b in range(W) if 0 < abs(a - i) + abs(b - j) <= r)
                assert c[v] == want, (W, H, r, v, c[v], want)
            assert np.array_equal(inter, c)
            assert total == float(g.n)


def _np_brute(g, X, r):
    """Neighbourhood preservation from the Floyd-Warshall matrix and a numpy
    lexicographic sort by (FP32 squared distance, id)."""
    D = floyd_warshall(g)
    X = np.asarray(X, dtype=np.float32)
    n = g.n
    cs, inters, total = [], [], 0.0
    for v in range(n):
        others = np.array([u for u in range(n) if u != v], dtype=np.int64)
        ng = set(int(u) for u in others if D[v, u] <= r)
        d2 = np.zeros(len(others), dtype=np.float32)
        for c in range(X.shape[1]):
            dx = (X[others, c] - X[v, c]).astype(np.float32)
            d2 = (d2 + (dx * dx).astype(np.float32)).astype(np.float32)
        order = others[np.lexsort((others, d2))]
        nd = set(int(u) for u in order[:len(ng)])
        inter = len(ng & nd)
        cs.append(len(ng))
        inters.append(inter)
        total += 1.0 if not ng else inter / len(ng | nd)
    return np.array(cs), np.array(inters), total


def check_np_brute_force(orc):
    rng = np.random.default_rng(77)
    for g in tiny_graphs():
        if g.n < 2:
            continue
        for layout in ("normal", "lattice"):
            if layout == "normal":
                X = rng.standard_normal((g.n, 2)).astype(np.float32)
            else:  # small integer lattice: many equal distances, the tie rule decides
                X = rng.integers(0, 4, size=(g.n, 2)).astype(np.float32)
            for r in (1, 2, 3):
                c, inter, total = orc.np_metric(g, X, r)
                bc, bi, bt = _np_brute(g, X, r)
                assert np.array_equal(c, bc) and np.array_equal(inter, bi), (g.name, layout, r)
                assert abs(total - bt) <= 1e-12 * max(1.0, bt), (g.name, layout, r, total, bt)


def check_stress_golden(orc):
    with open(QUALITY_GOLDEN) as f:
        cases = json.load(f)["stress_cases"]
    for case in cases:
        g = _quality_graph(case["graph"], case["n"])
        total, rows = orc.stress(g, np.asarray(case["X"], dtype=np.float32))
        assert abs(total - _closed_value(case["stress"])) <= 1e-14, (case["why"], total)
        assert abs(rows.sum() / (g.n * g.n - g.n) - total) <= 1e-14


def check_stress_star_circle(orc):
    """Star with L leaves on the unit circle around its centre: centre-leaf
    pairs have d = 1 = |X_i - X_j|; leaves a, b have d = 2 and chord length
    2 sin(pi |a - b| / L), so their term is (1 - sin(pi |a - b| / L))^2."""
    for L in (3, 5, 8):
        g = gg.star(L + 1)
        X = np.zeros((L + 1, 2), dtype=np.float32)
        ang = 2.0 * math.pi * np.arange(L) / L
        X[1:, 0] = np.cos(ang)
        X[1:, 1] = np.sin(ang)
        want = 0.0
        for a in range(L):
            for b in range(L):
                if a != b:
                    want += (1.0 - math.sin(math.pi * abs(a - b) / L)) ** 2
        n = L + 1
        want /= n * n - n
        total, _ = orc.stress(g, X)
        # the drawing is rounded to float32, the closed form is exact: 1e-6 covers the rounding
        assert abs(total - want) <= 1e-6, (L, total, want)


def check_stress_brute_force(orc):
    rng = np.random.default_rng(78)
    for g in tiny_graphs():
        if g.n < 2:
            continue
        X = (3.0 * rng.standard_normal((g.n, 3))).astype(np.float32)
        D = floyd_warshall(g)
        Xd = X.astype(np.float64)
        G = np.sqrt(((Xd[:, None, :] - Xd[None, :, :]) ** 2).sum(axis=2))
        with np.errstate(divide="ignore", invalid="ignore"):
            T = ((D - G) / D) ** 2
        T[np.isinf(D)] = 1.0
        np.fill_diagonal(T, 0.0)
        want_rows = T.sum(axis=1)
        want = want_rows.sum() / (g.n * g.n - g.n)
        total, rows = orc.stress(g, X)
        assert np.allclose(rows, want_rows, rtol=1e-12, atol=1e-12), g.name
        assert abs(total - want) <= 1e-12 * max(1.0, want), (g.name, total, want)


ALL_CHECKS = [check_apsp_floyd_warshall, check_knn_brute_force, check_closed_form_distances,
              check_golden_lists, check_full_equals_partial, check_partial_work,
              check_sigma_closed_forms, check_sigma_residual, check_union_star,
              check_union_properties, check_np_golden, check_np_grid_on_its_coordinates,
              check_np_brute_force, check_stress_golden, check_stress_star_circle, check_stress_brute_force]
