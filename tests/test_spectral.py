"""Spectral layout of the union kNN graph on the GPU (Lanczos in FP64)
against the CPU oracle's dense FP64 eigensolve, through the C ABI.

Two comparisons per graph: with the oracle run on the GPU's own union COO
(float weights widened to FP64), which isolates the eigensolver (eigenvalues
within 1e-9, eigenvectors within 2e-5 after the float32 output rounding);
and with the oracle's whole pipeline (FP64 weights), whose 1e-7-level weight
differences move the eigenvectors by about that over the spectral gap
(within 1e-4). Columns of a repeated eigenvalue are compared as subspaces
(largest principal-angle sine in the D inner product)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import oracle_pins
from oracle import spectral
from paper_2509_19703_gb300 import graphgen as gg
from paper_2509_19703_gb300 import gumap

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gumap.load()


def principal_sine(A, B, d):
    s = np.sqrt(d)[:, None]
    qa, _ = np.linalg.qr(A * s)
    qb, _ = np.linalg.qr(B * s)
    return float(np.linalg.norm(qa - qb @ (qb.T @ qa), 2))


def compare(X, mu, Xr, mur, d, vec_tol, mu_tol, tag):
    """X, mu: the GPU's dim columns; Xr, mur: the oracle's, every nontrivial
    one. Eigenvalues within mu_tol; a column of a simple eigenvalue equal
    up to sign; the columns of a repeated eigenvalue inside the oracle's whole
    eigenspace of it (largest principal-angle sine)."""
    dim = X.shape[1]
    assert np.allclose(mu, mur[:dim], atol=mu_tol, rtol=0), (tag, mu, mur[:dim])
    c = 0
    while c < dim:
        group = np.flatnonzero(np.abs(mur - mur[c]) <= 1e-6)
        e = min(dim, int(group.max()) + 1)
        if group.size == 1:
            x, xr = X[:, c], Xr[:, c]
            err = min(np.max(np.abs(x - xr)), np.max(np.abs(x + xr)))
            assert err <= vec_tol * max(1.0, np.max(np.abs(xr))), (tag, c, err)
        else:
            assert principal_sine(X[:, c:e], Xr[:, group], d) <= vec_tol * 10, (tag, c, e)
        c = e


def cases():
    gs = [(gg.grid(13, 29), 15, "full"), (gg.barabasi_albert(1500, 3, 71), 15, "partial"),
          (gg.path(600), 7, "full"), (gg.cycle(101), 6, "full"), (gg.random_tree(700, 72), 15, "partial"),
          (gg.gnp(900, 0.01, 73), 15, "partial"), (gg.star(150), 10, "full"),
          (gg.disjoint_union([gg.grid(6, 7), gg.path(30), gg.gnp(60, 0.1, 74)], "disj"), 8, "full")]
    gs += [(g, min(5, g.n - 1), "full") for g in oracle_pins.tiny_graphs() if g.n >= 6 and g.nnz > 0]
    return gs


CASES = cases()


@pytest.mark.parametrize("g,k,mode", CASES, ids=[f"{g.name}-k{k}-{m}" for g, k, m in CASES])
@pytest.mark.parametrize("dim", [2, 3])
def test_spectral_layout_matches_oracle(g, k, mode, dim):
    m = gumap.FULL if mode == "full" else gumap.PARTIAL
    with gumap.KnnGraph.from_graph(g, k, mode=m) as kg:
        kg.run()
        row, col, w = kg.coo()
        X, mu, info = kg.spectral_layout(dim)
        kg.check()
        X = X.cpu().numpy().astype(np.float64)
        row, col, w = row.cpu().numpy(), col.cpu().numpy(), w.cpu().numpy().astype(np.float64)
    assert info["converged"] == 1, info
    d = np.bincount(row, weights=w, minlength=g.n)
    live = d > 0
    assert np.all(X[~live] == 0.0)
    extra = int(np.sum(live)) - 1  # every nontrivial eigenvector: whole eigenspaces of repeated eigenvalues
    Xr, mur = spectral.spectral_layout(g.n, row, col, w, extra)
    ok = ~np.isnan(mur[:dim])
    dd = np.where(live, d, 1.0)
    compare(X[:, ok], mu[ok], Xr, mur, dd, 2e-5, 1e-9, f"{g.name} own COO")
    # against the oracle's whole pipeline (FP64 weights)
    ref = oracle.knn_pipeline(g, k, mode)
    rr, rc, rw = ref["coo"]
    Xp, mup = spectral.spectral_layout(g.n, rr, rc, rw, extra)
    compare(X[:, ok], mu[ok], Xp, mup, dd, 1e-4, 1e-6, f"{g.name} pipeline")


def test_spectral_needs_a_union_run():
    with gumap.KnnGraph.from_graph(gg.gnp(20, 0.0, 5), 3) as kg:  # no edge: no union graph to draw
        kg.run()
        with pytest.raises(gumap.GumapError) as e:
            kg.spectral_layout(2)
        assert e.value.status == gumap.ERR_INVALID_ARG
    g = gg.grid(5, 5)
    with gumap.KnnGraph.from_graph(g, 4, flags=gumap.WEIGHTS_DIRECTED) as kg:
        kg.run()
        with pytest.raises(gumap.GumapError) as e:
            kg.spectral_layout(2)
        assert e.value.status == gumap.ERR_INVALID_ARG
    with gumap.KnnGraph.from_graph(g, 4) as kg:
        with pytest.raises(gumap.GumapError) as e:
            kg.spectral_layout(2)  # no run yet
        assert e.value.status == gumap.ERR_INVALID_ARG
        kg.run()
        with pytest.raises(gumap.GumapError) as e:
            kg.spectral_layout(9)
        assert e.value.status == gumap.ERR_INVALID_ARG
