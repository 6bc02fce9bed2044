"""Spectral layout oracle (TEST INFRASTRUCTURE; FP64, dense, tiny graphs only).

Only the tests and the benchmark's CPU-baseline leg use this module. It
shares nothing with the CUDA library.

What it computes: the initial coordinates of the layout stage, "initialize
the coordinates in X using spectral layout" (Algorithm 1; Section 3.2, after
Koren's spectral graph drawing), for the graph the layout stage draws, the
kNN graph G_k with its fuzzy-union weights w (the symmetric COO of the path).
Koren's degree-normalised eigenvectors are the solutions of

    L x = mu D x,   L = D - W,   D = diag(W 1),

ordered by mu; mu_0 = 0 with x constant is trivial, and the layout takes the
next `dim` of them, D-normalised (x^T D x = 1, pairwise x^T D y = 0).

The computation follows that definition with a library eigensolver as its
one step: y = D^(1/2) x turns the pencil into the symmetric matrix
L_sym = I - D^(-1/2) W D^(-1/2) with L_sym y = mu y; numpy.linalg.eigh gives
its eigenpairs in ascending order; x = D^(-1/2) y.

Readings where the paper is silent:
  * graph: the layout stage draws G_k (Algorithm 1, C2 on G_k), so the
    weights are the fuzzy-union weights of the kNN path;
  * the trivial eigenvector is D^(1/2) 1 alone: on a disconnected G_k the
    other eigenvectors of eigenvalue 0 (component indicators orthogonal to
    it) come next, like any eigenvector;
  * a vertex with no edge (weighted degree 0) gets coordinate 0 and is left
    out of the eigenproblem;
  * sign: each column is scaled so that its entry of largest magnitude
    (the first such index) is positive; within a repeated eigenvalue the
    basis is any D-orthonormal one, so comparisons there are of subspaces.
"""
from __future__ import annotations

import numpy as np


def dense_weights(n: int, row, col, w) -> np.ndarray:
    """The symmetric weight matrix of a COO (each (i, j) entry once)."""
    W = np.zeros((n, n), dtype=np.float64)
    W[np.asarray(row, dtype=np.int64), np.asarray(col, dtype=np.int64)] = np.asarray(w, dtype=np.float64)
    return W


def spectral_layout(n: int, row, col, w, dim: int = 2):
    """(X float64 [n, dim], mu float64 [dim]) of the weighted graph given by
    the COO (row, col, w); see the module docstring."""
    W = dense_weights(n, row, col, w)
    deg = W.sum(axis=1)
    live = np.flatnonzero(deg > 0)
    X = np.zeros((n, dim), dtype=np.float64)
    mu = np.full(dim, np.nan)
    m = live.size
    if m < 2:
        return X, mu
    Wl = W[np.ix_(live, live)]
    s = 1.0 / np.sqrt(deg[live])
    L_sym = np.eye(m) - (s[:, None] * Wl) * s[None, :]
    L_sym = 0.5 * (L_sym + L_sym.T)
    evals, evecs = np.linalg.eigh(L_sym)
    # drop the trivial eigenvector D^(1/2) 1 (eigenvalue 0): remove its
    # direction from the eigenvalue-0 eigenspace, keep the rest of the order
    t = np.sqrt(deg[live])
    t /= np.linalg.norm(t)
    zero = np.flatnonzero(np.abs(evals) <= 1e-9)
    if zero.size:
        Z = evecs[:, zero]
        Z = Z - np.outer(t, t @ Z)          # project the trivial direction out
        u, sv, _ = np.linalg.svd(Z, full_matrices=False)
        Z = u[:, sv > 1e-6]                 # the projection removed one dimension
        rest = np.flatnonzero(np.abs(evals) > 1e-9)
        evecs = np.concatenate([Z, evecs[:, rest]], axis=1)
        evals = np.concatenate([np.zeros(Z.shape[1]), evals[rest]])
    take = min(dim, evecs.shape[1])
    Y = evecs[:, :take]
    Xl = Y * s[:, None]
    for c in range(take):
        j = int(np.argmax(np.abs(Xl[:, c])))
        if Xl[j, c] < 0:
            Xl[:, c] = -Xl[:, c]
    X[live, :take] = Xl
    mu[:take] = evals[:take]
    return X, mu
