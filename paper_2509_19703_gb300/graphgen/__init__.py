"""Seeded synthetic input graphs (CSR, int32), shared by the CUDA path's
tests/bench and by the CPU oracle's tests.

The module holds none of the method's arithmetic: it only draws random graphs
and lays them out as CSR. The generators stand in for the paper's datasets
(Section 4.1.2, Table 2: scale-free, GION and mesh graphs), which are not
available: Barabasi-Albert for scale-free, grids for meshes, G(n, p) and
uniform random trees for the dense and the large-diameter ends.

The C source (``graphgen.c``) is compiled with gcc into ``_build/`` on first
use; ``build()`` compiles it eagerly.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "_build", "libgraphgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator library; returns its path."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.POINTER(ctypes.c_int32)),
                ("col", ctypes.POINTER(ctypes.c_int32))]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(_Csr)
            i32, i64, u64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            for name, args in [("gg_grid", [i32, i32]), ("gg_path", [i32]), ("gg_cycle", [i32]),
                               ("gg_star", [i32]), ("gg_complete", [i32]),
                               ("gg_ba", [i32, i32, u64]), ("gg_gnp", [i32, dbl, u64]),
                               ("gg_tree", [i32, u64]),
                               ("gg_from_edges", [i32, i64, ctypes.c_void_p, ctypes.c_void_p])]:
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = P
            lib.gg_free.argtypes = [P]
            lib.gg_free.restype = None
            lib.gg_uniform.argtypes = [u64, i64, ctypes.c_void_p]
            lib.gg_uniform.restype = None
            _lib = lib
    return _lib


@dataclass
class Graph:
    """Undirected graph as symmetric CSR with sorted rows."""
    n: int
    row_ptr: np.ndarray  # int32 [n+1]
    col: np.ndarray      # int32 [nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    @property
    def m(self) -> int:
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))


def _take(ptr, name: str) -> Graph:
    if not ptr:
        raise ValueError(f"graph generator failed for {name}")
    c = ptr.contents
    n, nnz = int(c.n), int(c.nnz)
    rp = np.ctypeslib.as_array(c.row_ptr, shape=(n + 1,)).copy()
    col = (np.ctypeslib.as_array(c.col, shape=(nnz,)).copy() if nnz > 0
           else np.zeros(0, dtype=np.int32))
    _load().gg_free(ptr)
    return Graph(n=n, row_ptr=rp.astype(np.int32), col=col.astype(np.int32), name=name)


def grid(W: int, H: int | None = None) -> Graph:
    H = W if H is None else H
    return _take(_load().gg_grid(W, H), f"grid{W}x{H}")


def path(n: int) -> Graph:
    return _take(_load().gg_path(n), f"path{n}")


def cycle(n: int) -> Graph:
    return _take(_load().gg_cycle(n), f"cycle{n}")


def star(n: int) -> Graph:
    return _take(_load().gg_star(n), f"star{n}")


def complete(n: int) -> Graph:
    return _take(_load().gg_complete(n), f"K{n}")


def barabasi_albert(n: int, m0: int, seed: int) -> Graph:
    return _take(_load().gg_ba(n, m0, seed), f"ba{n}_m{m0}_s{seed}")


def gnp(n: int, p: float, seed: int) -> Graph:
    return _take(_load().gg_gnp(n, float(p), seed), f"gnp{n}_p{p:g}_s{seed}")


def random_tree(n: int, seed: int) -> Graph:
    return _take(_load().gg_tree(n, seed), f"tree{n}_s{seed}")


def from_edges(n: int, u, v, name: str = "edges") -> Graph:
    """Symmetrised CSR from an edge list; self loops and duplicates dropped."""
    u = np.ascontiguousarray(u, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.int32)
    assert u.shape == v.shape
    return _take(_load().gg_from_edges(n, u.shape[0], u.ctypes.data, v.ctypes.data), name)


def uniform(seed: int, count: int) -> np.ndarray:
    """Seeded uniform doubles in [0, 1) from the same generator family."""
    out = np.empty(count, dtype=np.float64)
    if count:
        _load().gg_uniform(seed, count, out.ctypes.data)
    return out


def disjoint_union(graphs, name: str = "union") -> Graph:
    """Place graphs side by side (ids offset), giving a disconnected graph."""
    rps, cols, off, eoff = [], [], 0, 0
    for g in graphs:
        rps.append(g.row_ptr[:-1].astype(np.int64) + eoff)
        cols.append(g.col.astype(np.int64) + off)
        off += g.n
        eoff += g.nnz
    rp = np.concatenate(rps + [np.array([eoff])]).astype(np.int32)
    col = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    return Graph(n=off, row_ptr=rp, col=col, name=name)


# ---------------------------------------------------------------------------
# Workload recipes (seeded); sizes follow the stated synthetic configurations.
# ---------------------------------------------------------------------------

def config_grid32() -> Graph:
    """32 x 32 grid, n = 1024, m = 1984."""
    return grid(32, 32)


def config_ba20k() -> Graph:
    """Barabasi-Albert, n = 20,000, 5 edges per new vertex (m = 99,985), seed 1."""
    return barabasi_albert(20000, 5, 1)


def config_er5k() -> Graph:
    """G(n = 5,000, p = 0.1), seed 2 (about 1.25 M edges)."""
    return gnp(5000, 0.1, 2)


def config_ba1m() -> Graph:
    """Barabasi-Albert, n = 1,000,000, 4 edges per new vertex, seed 3."""
    return barabasi_albert(1000000, 4, 3)


def config_grid1m() -> Graph:
    """1000 x 1000 grid."""
    return grid(1000, 1000)


@dataclass
class BatchItem:
    graph: Graph
    mode: str   # "full" | "partial"
    k: int
    seed: int
    kind: str


def batch_mix(count: int = 2000, base_seed: int = 4, n_lo: int = 100, n_hi: int = 20000,
              k: int = 15) -> list[BatchItem]:
    """Mixed batch of uneven graphs: n log-uniform in [n_lo, n_hi], the model
    uniform over {grid, BA (2..8 edges per vertex), G(n,p) with mean degree
    U(4, 40), random tree}, mode full/partial 50/50. Graph g gets seed
    base_seed * 10^6 + g."""
    draws = uniform(base_seed, 4 * count).reshape(count, 4)
    out = []
    for g in range(count):
        u_n, u_kind, u_par, u_mode = draws[g]
        n = int(math.floor(math.exp(math.log(n_lo) + u_n * (math.log(n_hi) - math.log(n_lo)))))
        n = max(n, 2)
        seed = base_seed * 10**6 + g
        kind_i = min(int(u_kind * 4), 3)
        if kind_i == 0:
            W = max(1, int(round(math.sqrt(n))))
            H = max(1, int(round(n / W)))
            gr, kind = grid(W, H), "grid"
        elif kind_i == 1:
            m0 = 2 + min(int(u_par * 7), 6)
            gr, kind = barabasi_albert(max(n, m0 + 2), m0, seed), f"ba{m0}"
        elif kind_i == 2:
            mean_deg = 4.0 + 36.0 * u_par
            gr, kind = gnp(n, min(1.0, mean_deg / max(n - 1, 1)), seed), "gnp"
        else:
            gr, kind = random_tree(n, seed), "tree"
        out.append(BatchItem(graph=gr, mode="full" if u_mode < 0.5 else "partial", k=min(k, gr.n - 1),
                             seed=seed, kind=kind))
    return out
