"""Pins for the spectral-layout oracle (oracle/spectral.py), independent of
its own code: closed-form eigenvectors of paths, cycles, tori and complete
graphs, a disconnected graph and an isolated vertex, and the defining
identities (L x = mu D x, D-orthonormality, orthogonality to the trivial
vector, Rayleigh quotients) on weighted graphs.

Each ``check_*`` takes a module exposing ``spectral_layout`` and raises
AssertionError on a mismatch; ``test_oracle_pins.py`` runs them on the real
module, ``test_oracle_mutations.py`` on copies with planted mistakes.

Closed forms used (D^-1 W is the random walk of the graph):
  * path P_n: x_t = cos(pi k t / (n - 1)), mu_k = 1 - cos(pi k / (n - 1));
  * cycle C_n: span{cos(2 pi t / n), sin(2 pi t / n)}, mu = 1 - cos(2 pi / n);
  * torus C_W x C_H (W > H): span{cos(2 pi x / W), sin(2 pi x / W)},
    mu = (1 - cos(2 pi / W)) / 2;
  * complete graph K_n: every nontrivial mu = n / (n - 1).
"""
from __future__ import annotations

import math

import numpy as np

from paper_2509_19703_gb300 import graphgen as gg


def coo_of(g, w=None):
    row = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    return row, np.asarray(g.col), (np.ones(g.nnz) if w is None else w)


def torus_coo(W, H):
    row, col = [], []
    for y in range(H):
        for x in range(W):
            v = y * W + x
            for u in (y * W + (x + 1) % W, y * W + (x - 1) % W, ((y + 1) % H) * W + x, ((y - 1) % H) * W + x):
                row.append(v)
                col.append(u)
    return np.array(row), np.array(col), np.ones(len(row))


def degrees(n, row, w):
    return np.bincount(np.asarray(row), weights=np.asarray(w, dtype=np.float64), minlength=n)


def max_principal_sine(A, B, d):
    """Largest sine of the principal angles between span(A) and span(B) in
    the inner product <x, y> = x^T diag(d) y."""
    s = np.sqrt(d)[:, None]
    qa, _ = np.linalg.qr(A * s)
    qb, _ = np.linalg.qr(B * s)
    if qa.shape[1] != qb.shape[1]:
        return 1.0
    resid = qa - qb @ (qb.T @ qa)  # the part of span(A) outside span(B)
    return float(np.linalg.norm(resid, 2))


def _unit_d(v, d):
    return v / math.sqrt(float(v @ (d * v)))


def check_path_closed_form(sp):
    for n in (9, 30, 101):
        g = gg.path(n)
        row, col, w = coo_of(g)
        d = degrees(n, row, w)
        X, mu = sp.spectral_layout(n, row, col, w, dim=3)
        t = np.arange(n)
        for k in (1, 2, 3):
            assert abs(mu[k - 1] - (1.0 - math.cos(math.pi * k / (n - 1)))) <= 1e-12, (n, k, mu)
            c = _unit_d(np.cos(math.pi * k * t / (n - 1)), d)
            x = X[:, k - 1]
            assert min(np.max(np.abs(x - c)), np.max(np.abs(x + c))) <= 1e-9, (n, k)


def check_cycle_subspace(sp):
    for n in (7, 20, 33):
        g = gg.cycle(n)
        row, col, w = coo_of(g)
        d = degrees(n, row, w)
        X, mu = sp.spectral_layout(n, row, col, w, dim=2)
        t = np.arange(n)
        want = np.stack([np.cos(2 * math.pi * t / n), np.sin(2 * math.pi * t / n)], axis=1)
        assert np.allclose(mu, 1.0 - math.cos(2 * math.pi / n), atol=1e-12), (n, mu)
        assert max_principal_sine(X, want, d) <= 1e-9, n


def check_torus_subspace(sp):
    for W, H in ((8, 5), (12, 7)):
        row, col, w = torus_coo(W, H)
        n = W * H
        d = degrees(n, row, w)
        X, mu = sp.spectral_layout(n, row, col, w, dim=2)
        xs = np.arange(n) % W
        want = np.stack([np.cos(2 * math.pi * xs / W), np.sin(2 * math.pi * xs / W)], axis=1)
        assert np.allclose(mu, 0.5 * (1.0 - math.cos(2 * math.pi / W)), atol=1e-12), (W, H, mu)
        assert max_principal_sine(X, want, d) <= 1e-9, (W, H)


def check_complete_graph(sp):
    for n in (4, 9):
        g = gg.complete(n)
        row, col, w = coo_of(g)
        d = degrees(n, row, w)
        X, mu = sp.spectral_layout(n, row, col, w, dim=2)
        assert np.allclose(mu, n / (n - 1), atol=1e-12), mu
        assert np.allclose(X.sum(axis=0), 0.0, atol=1e-12)
        assert np.allclose(X.T @ (d[:, None] * X), np.eye(2), atol=1e-12)


def _check_identities(sp, n, row, col, w, dim, tag):
    Wm = np.zeros((n, n))
    Wm[row, col] = w
    d = Wm.sum(axis=1)
    X, mu = sp.spectral_layout(n, row, col, w, dim=dim)
    L = np.diag(d) - Wm
    for c in range(dim):
        x = X[:, c]
        r = L @ x - mu[c] * d * x
        assert np.linalg.norm(r) <= 1e-10 * max(1.0, np.linalg.norm(d * x)), (tag, c)
    assert np.allclose(X.T @ (d[:, None] * X), np.eye(dim), atol=1e-10), tag
    assert np.allclose(X.T @ d, 0.0, atol=1e-10), tag
    assert np.all(np.diff(mu) >= -1e-12), (tag, mu)
    # Courant-Fischer: no vector D-orthogonal to the constant has a smaller
    # Rayleigh quotient than the first nontrivial mu
    rng = np.random.default_rng(5)
    for _ in range(50):
        z = rng.standard_normal(n)
        z -= (z @ d) / d.sum()
        q = (z @ L @ z) / (z @ (d * z))
        assert q >= mu[0] - 1e-10, (tag, q, mu[0])


def check_weighted_identities(sp):
    rng = np.random.default_rng(11)
    for g in (gg.barabasi_albert(60, 3, 12), gg.grid(7, 6), gg.gnp(40, 0.2, 13), gg.random_tree(35, 14)):
        row, col, _ = coo_of(g)
        # symmetric positive weights
        wmat = {}
        for a, b in zip(row, col):
            key = (min(a, b), max(a, b))
            if key not in wmat:
                wmat[key] = float(rng.uniform(0.05, 1.0))
        w = np.array([wmat[(min(a, b), max(a, b))] for a, b in zip(row, col)])
        _check_identities(sp, g.n, row, col, w, 3, g.name)


def check_disconnected_and_isolated(sp):
    # P_7 and P_5 side by side, then an isolated vertex: the first column is
    # the eigenvalue-0 direction orthogonal to the trivial one (constant on
    # each path, D-orthogonal to the constant); the second is P_7's own first
    # eigenvector (its mu, 1 - cos(pi/6), is below P_5's 1 - cos(pi/4)),
    # zero on P_5; the isolated vertex stays at 0.
    g = gg.disjoint_union([gg.path(7), gg.path(5), gg.path(1)], "p7p5p1")
    row, col, w = coo_of(g)
    n = g.n
    d = degrees(n, row, w)
    X, mu = sp.spectral_layout(n, row, col, w, dim=2)
    assert abs(mu[0]) <= 1e-12 and abs(mu[1] - (1.0 - math.cos(math.pi / 6))) <= 1e-12, mu
    a = np.zeros(n)
    a[:7] = 1.0 / d[:7].sum()
    a[7:12] = -1.0 / d[7:12].sum()
    assert max_principal_sine(X[:12, :1], a[:12, None], d[:12]) <= 1e-9
    c = np.zeros(n)
    c[:7] = np.cos(math.pi * np.arange(7) / 6)
    c = _unit_d(c, d)
    assert min(np.max(np.abs(X[:, 1] - c)), np.max(np.abs(X[:, 1] + c))) <= 1e-9
    assert np.all(X[12] == 0.0)


ALL_CHECKS = [check_path_closed_form, check_cycle_subspace, check_torus_subspace, check_complete_graph,
              check_weighted_identities, check_disconnected_and_isolated]
