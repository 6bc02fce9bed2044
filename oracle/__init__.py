"""CPU oracle for the graph-kNN + UMAP-weight path (TEST INFRASTRUCTURE).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package. It shares no code with the CUDA library: the C
source ``gumap_oracle.c`` is compiled on its own with gcc into ``_build/``
and loaded through ctypes. Everything is FP64.

Functions (see the C file for the passage each one follows):
  knn_full(g, k, sources)      BFS to completion per source, (dist, id) sort
  knn_partial(g, k, sources)   level-by-level BFS stopped at the level that
                               reaches k (Algorithm 4 reading), (dist, id) sort
  smooth_knn(dist, k)          rho, sigma, directed weights a_ij (Section 2.1)
  slot_union(idx, a)           per-slot fuzzy union a + b - ab
  coo_union(idx, a)            symmetric COO of the union, sorted (row, col)
  apsp(g)                      n x n hop-distance matrix (uint16, 0xFFFF = inf)
  np_metric(g, X, r)           neighbourhood preservation of a drawing (Section 4.1.3)
  stress(g, X)                 aggregated stress of a drawing (Section 4.1.3)
  spectral_layout(...)         Laplacian eigenvectors for the initial layout (oracle/spectral.py)

Parity pins: the ``-m "not gpu"`` tests check these against Floyd-Warshall,
closed forms on grids/paths/cycles/stars/complete graphs and polynomial
roots of the calibration equation.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gumap_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()

INF16 = 0xFFFF


def compile_source(src: str, out: str) -> str:
    """gcc-compile an oracle source file into a shared library at ``out``."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    # -ffp-contract=off: every float operation rounds on its own (no fused
    # multiply-add), so the FP32 squared distances are the IEEE single steps
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no CUDA involved); returns the .so path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        compile_source(_SRC, _LIB)
    return _LIB


def _bind(lib):
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.oracle_bfs.argtypes = [vp, vp, i32, i32, vp, vp]
    lib.oracle_bfs.restype = ctypes.c_int
    lib.oracle_apsp.argtypes = [vp, vp, i32, vp]
    lib.oracle_apsp.restype = ctypes.c_int
    lib.oracle_knn_full.argtypes = [vp, vp, i32, i32, vp, i32, vp, vp]
    lib.oracle_knn_full.restype = ctypes.c_int
    lib.oracle_knn_partial.argtypes = [vp, vp, i32, i32, vp, i32, vp, vp, vp]
    lib.oracle_knn_partial.restype = ctypes.c_int
    lib.oracle_smooth_knn.argtypes = [vp, i32, i32, vp, vp, vp]
    lib.oracle_smooth_knn.restype = None
    lib.oracle_slot_union.argtypes = [vp, vp, i32, i32, vp]
    lib.oracle_slot_union.restype = None
    lib.oracle_coo_union.argtypes = [vp, vp, i32, i32, vp, vp, vp]
    lib.oracle_coo_union.restype = i64
    lib.oracle_np.argtypes = [vp, vp, i32, vp, i32, i32, vp, i32, vp, vp]
    lib.oracle_np.restype = ctypes.c_double
    lib.oracle_stress.argtypes = [vp, vp, i32, vp, i32, vp, i32, vp]
    lib.oracle_stress.restype = ctypes.c_double
    return lib


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    if col.size == 0:
        col = np.zeros(1, dtype=np.int32)
    return rp, col


def _sources(g, sources):
    if sources is None:
        return None, g.n
    s = np.ascontiguousarray(sources, dtype=np.int32)
    return s, int(s.shape[0])


class Oracle:
    """The oracle bound to one compiled library (the default one, or a copy
    that a test mutated on purpose to show the pins catch the mistake)."""

    def __init__(self, libpath: str):
        self.lib = _bind(ctypes.CDLL(libpath))

    def bfs(self, g, s: int) -> np.ndarray:
        rp, col = _csr(g)
        dist = np.empty(max(g.n, 1), dtype=np.int32)
        q = np.empty(max(g.n, 1), dtype=np.int32)
        if self.lib.oracle_bfs(rp.ctypes.data, col.ctypes.data, g.n, s, dist.ctypes.data, q.ctypes.data):
            raise ValueError("bad source")
        return dist[:g.n]

    def apsp(self, g) -> np.ndarray:
        rp, col = _csr(g)
        D = np.empty((g.n, g.n), dtype=np.uint16)
        if self.lib.oracle_apsp(rp.ctypes.data, col.ctypes.data, g.n, D.ctypes.data):
            raise MemoryError
        return D

    def knn_full(self, g, k: int, sources=None):
        """(idx int32 [n_src, k], dist uint16 [n_src, k]) by full BFS per source."""
        rp, col = _csr(g)
        s, n_src = _sources(g, sources)
        idx = np.empty((n_src, k), dtype=np.int32)
        dist = np.empty((n_src, k), dtype=np.uint16)
        rc = self.lib.oracle_knn_full(rp.ctypes.data, col.ctypes.data, g.n, k,
                                      None if s is None else s.ctypes.data, n_src,
                                      idx.ctypes.data, dist.ctypes.data)
        if rc:
            raise ValueError("oracle_knn_full failed")
        return idx, dist

    def knn_partial(self, g, k: int, sources=None, return_work: bool = False):
        """Partial BFS per source; optionally the scanned adjacency entries."""
        rp, col = _csr(g)
        s, n_src = _sources(g, sources)
        idx = np.empty((n_src, k), dtype=np.int32)
        dist = np.empty((n_src, k), dtype=np.uint16)
        work = np.empty(max(n_src, 1), dtype=np.int64)
        rc = self.lib.oracle_knn_partial(rp.ctypes.data, col.ctypes.data, g.n, k,
                                         None if s is None else s.ctypes.data, n_src,
                                         idx.ctypes.data, dist.ctypes.data, work.ctypes.data)
        if rc:
            raise ValueError("oracle_knn_partial failed")
        return (idx, dist, work[:n_src]) if return_work else (idx, dist)

    def smooth_knn(self, dist: np.ndarray):
        """rho [r], sigma [r], a [r, k] (FP64) from a distance list [r, k]."""
        d = np.ascontiguousarray(dist, dtype=np.uint16)
        r, k = d.shape
        rho = np.empty(r, dtype=np.float64)
        sigma = np.empty(r, dtype=np.float64)
        a = np.empty((r, k), dtype=np.float64)
        self.lib.oracle_smooth_knn(d.ctypes.data, r, k, rho.ctypes.data, sigma.ctypes.data, a.ctypes.data)
        return rho, sigma, a

    def slot_union(self, idx: np.ndarray, a: np.ndarray) -> np.ndarray:
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        a = np.ascontiguousarray(a, dtype=np.float64)
        n, k = idx.shape
        w = np.empty((n, k), dtype=np.float64)
        self.lib.oracle_slot_union(idx.ctypes.data, a.ctypes.data, n, k, w.ctypes.data)
        return w

    def coo_union(self, idx: np.ndarray, a: np.ndarray):
        """(row int32, col int32, w float64) sorted by (row, col)."""
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        a = np.ascontiguousarray(a, dtype=np.float64)
        n, k = idx.shape
        cap = max(2 * n * k, 1)
        row = np.empty(cap, dtype=np.int32)
        col = np.empty(cap, dtype=np.int32)
        w = np.empty(cap, dtype=np.float64)
        nnz = self.lib.oracle_coo_union(idx.ctypes.data, a.ctypes.data, n, k,
                                        row.ctypes.data, col.ctypes.data, w.ctypes.data)
        if nnz < 0:
            raise MemoryError
        return row[:nnz], col[:nnz], w[:nnz]

    def np_metric(self, g, X, r: int = 2, vertices=None):
        """(c int32, inter int32, total float): |N_G(v, r)|, |N_G ∩ N_D| per
        vertex (all, or the given ones) and the sum of |∩| / |∪| over them, for
        the drawing X (float32 [n, dim])."""
        rp, col = _csr(g)
        X = np.ascontiguousarray(X, dtype=np.float32)
        assert X.ndim == 2 and X.shape[0] == g.n
        vs, nv = _sources(g, vertices)
        c = np.empty(max(nv, 1), dtype=np.int32)
        inter = np.empty(max(nv, 1), dtype=np.int32)
        total = self.lib.oracle_np(rp.ctypes.data, col.ctypes.data, g.n, X.ctypes.data, X.shape[1], int(r),
                                   None if vs is None else vs.ctypes.data, nv, c.ctypes.data, inter.ctypes.data)
        if total < 0:
            raise ValueError("oracle_np failed")
        return c[:nv], inter[:nv], float(total)

    def stress(self, g, X, vertices=None):
        """(stress, per-row sums float64) of the drawing X (float32 [n, dim]);
        with `vertices`, only those rows (the first value is then their sum
        over n^2 - n)."""
        rp, col = _csr(g)
        X = np.ascontiguousarray(X, dtype=np.float32)
        assert X.ndim == 2 and X.shape[0] == g.n
        vs, nv = _sources(g, vertices)
        rows = np.empty(max(nv, 1), dtype=np.float64)
        total = self.lib.oracle_stress(rp.ctypes.data, col.ctypes.data, g.n, X.ctypes.data, X.shape[1],
                                       None if vs is None else vs.ctypes.data, nv, rows.ctypes.data)
        if total < 0:
            raise ValueError("oracle_stress failed")
        return float(total), rows[:nv]

    def knn_pipeline(self, g, k: int, mode: str = "full"):
        """The whole path for all vertices: idx, dist, rho, sigma, a, w, coo."""
        idx, dist = self.knn_full(g, k) if mode == "full" else self.knn_partial(g, k)
        rho, sigma, a = self.smooth_knn(dist)
        w = self.slot_union(idx, a)
        coo = self.coo_union(idx, a)
        return dict(idx=idx, dist=dist, rho=rho, sigma=sigma, a=a, w=w, coo=coo)


_default = None


def default() -> Oracle:
    global _default
    with _lock:
        if _default is None:
            _default = Oracle(build())
    return _default


def bfs(g, s):
    return default().bfs(g, s)


def apsp(g):
    return default().apsp(g)


def knn_full(g, k, sources=None):
    return default().knn_full(g, k, sources)


def knn_partial(g, k, sources=None, return_work=False):
    return default().knn_partial(g, k, sources, return_work)


def smooth_knn(dist):
    return default().smooth_knn(dist)


def slot_union(idx, a):
    return default().slot_union(idx, a)


def coo_union(idx, a):
    return default().coo_union(idx, a)


def knn_pipeline(g, k, mode="full"):
    return default().knn_pipeline(g, k, mode)


def np_metric(g, X, r=2, vertices=None):
    return default().np_metric(g, X, r, vertices)


def stress(g, X, vertices=None):
    return default().stress(g, X, vertices)
