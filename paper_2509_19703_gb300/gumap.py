"""Thin ctypes binding of libgumap (include/gumap.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels. PyTorch supplies device memory (tensors) and streams. There is no
CPU fallback: if ``libgumap.so`` is missing, loading fails with an error.

The functions keep the C names (gumap_knn_create, gumap_knn_run, ...);
``KnnGraph`` is a small convenience wrapper that allocates output tensors.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

from . import _build

# modes, flags, engines, options (mirror include/gumap.h)
FULL, PARTIAL = 0, 1
WEIGHTS_UNION, WEIGHTS_DIRECTED, CSR_ON_DEVICE, EMIT_APSP = 0x0, 0x1, 0x2, 0x4
ENGINE_AUTO, ENGINE_MSBFS, ENGINE_MSBFS_SM, ENGINE_FRONTIER, ENGINE_BATCH = 0, 1, 2, 3, 4
OPT_ENGINE, OPT_BLOCK_BITS, OPT_PROFILE, OPT_STATE_BYTES, OPT_HEAVY_DEGREE = 1, 2, 3, 4, 5
OPT_DIRECTION, OPT_PUSH_DIV, OPT_PULL_WIDTH, OPT_CTAS_PER_SM, OPT_STAGE = 6, 7, 8, 9, 10
OPT_BATCH_WIDTH = 11
OPT_COO_BUILD = 12
OPT_FRONTIER_BUILD = 13
OPT_GRAPH = 14
COO_AUTO, COO_RADIX, COO_ROWS = 0, 1, 2
FRONTIER_AUTO, FRONTIER_THREAD, FRONTIER_WARP, FRONTIER_GROUP = 0, 1, 2, 3
DIRECTION_AUTO, DIRECTION_PULL, DIRECTION_PUSH = 0, 1, 2
MAX_K = 256
DIST_INF = 0xFFFF

OK = 0
ERR_INVALID_ARG, ERR_INVALID_GRAPH, ERR_OOM, ERR_CUDA = 1, 2, 3, 4
ERR_AGAIN, PENDING, ERR_TIMEOUT, ERR_TOO_LARGE, ERR_UNKNOWN_REQUEST = 5, 6, 7, 8, 9

_lock = threading.Lock()
_lib = None


class GumapError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


class _Stats(ctypes.Structure):
    _fields_ = [("engine", ctypes.c_int32), ("block_bits", ctypes.c_int32), ("n_blocks", ctypes.c_int32),
                ("levels_max", ctypes.c_int32), ("bfs_launches", ctypes.c_int64), ("bfs_ms", ctypes.c_double),
                ("bfs_level_sum", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("bfs_init_ms", ctypes.c_double),
                ("bfs_pull_ms", ctypes.c_double), ("bfs_extract_ms", ctypes.c_double),
                ("bfs_push_ms", ctypes.c_double), ("bfs_push_levels", ctypes.c_int64),
                ("bfs_staged_launches", ctypes.c_int64), ("weights_ms", ctypes.c_double),
                ("sort_ms", ctypes.c_double), ("sort_launches", ctypes.c_int64),
                ("batch_model_bytes", ctypes.c_int64), ("graph_replays", ctypes.c_int64)]


class _Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64), ("k", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("max_degree", ctypes.c_int32), ("batch", ctypes.c_int32)]


class _Tune(ctypes.Structure):
    _fields_ = [("from_cache", ctypes.c_int32), ("candidates", ctypes.c_int32), ("best_ms", ctypes.c_double),
                ("default_ms", ctypes.c_double), ("engine", ctypes.c_int32), ("pull_width", ctypes.c_int32),
                ("heavy_mult", ctypes.c_int32), ("direction", ctypes.c_int32), ("state_bytes", ctypes.c_int64),
                ("ctas_per_sm", ctypes.c_int32), ("stage", ctypes.c_int32), ("push_div", ctypes.c_int32),
                ("batch_width", ctypes.c_int32), ("frontier_build", ctypes.c_int32)]


class _SpectralInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("restarts", ctypes.c_int32), ("residual", ctypes.c_double),
                ("converged", ctypes.c_int32)]


class _ServerOpts(ctypes.Structure):
    _fields_ = [("n_streams", ctypes.c_int32), ("max_batch_graphs", ctypes.c_int32),
                ("max_batch_vertices", ctypes.c_int64), ("max_queue", ctypes.c_int32),
                ("staging_bytes", ctypes.c_int64), ("flags", ctypes.c_uint32)]


class _Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("n", ctypes.c_int32), ("k", ctypes.c_int32),
                ("idx", ctypes.c_void_p), ("dist", ctypes.c_void_p), ("w", ctypes.c_void_p),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double), ("t_done", ctypes.c_double),
                ("batch_graphs", ctypes.c_int32), ("engine", ctypes.c_int32)]


class _ServerStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("submitted", "completed", "failed", "released", "launches",
                                              "pending", "running", "arena_bytes", "arena_used_bytes",
                                              "arena_peak_bytes")]


def library_path() -> str:
    return _build.LIB


def _signatures() -> dict:
    """ctypes argument and result types of every entry point of include/gumap.h."""
    vp, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    sig = {
        "gumap_knn_create": [ctypes.POINTER(vp), vp, vp, i32, i64, i32, ctypes.c_int, u32, ctypes.c_int],
        "gumap_knn_run": [vp, vp, i32, vp, vp, vp, vp],
        "gumap_knn_apsp": [vp, vp, i32, vp, vp, vp, vp],
        "gumap_knn_rho_sigma": [vp, vp, vp, vp],
        "gumap_knn_coo": [vp, vp, vp, vp, vp, vp],
        "gumap_knn_check": [vp, vp],
        "gumap_knn_set_option": [vp, ctypes.c_int, i64],
        "gumap_knn_get_stats": [vp, ctypes.POINTER(_Stats)],
        "gumap_knn_reset_stats": [vp],
        "gumap_knn_destroy": [vp],
        "gumap_knn_run_noalloc": [vp, vp, i32, i64, i32, ctypes.c_int, vp, vp, vp, vp],
        "gumap_batch_create": [ctypes.POINTER(vp), i32, vp, vp, vp, i64, i32, vp, u32, ctypes.c_int],
        "gumap_server_create": [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_uint64,
                                ctypes.POINTER(_ServerOpts)],
        "gumap_serve_submit": [vp, vp, vp, i32, i64, i32, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)],
        "gumap_serve_poll": [vp, ctypes.c_uint64, ctypes.POINTER(_Result)],
        "gumap_serve_wait": [vp, ctypes.c_uint64, ctypes.POINTER(_Result), ctypes.c_double],
        "gumap_serve_read": [vp, ctypes.c_uint64, vp, vp, vp, vp],
        "gumap_serve_release": [vp, ctypes.c_uint64],
        "gumap_server_get_stats": [vp, ctypes.POINTER(_ServerStats)],
        "gumap_server_destroy": [vp],
        "gumap_knn_get_info": [vp, ctypes.POINTER(_Info)],
        "gumap_knn_autotune": [vp, ctypes.c_char_p, ctypes.POINTER(_Tune)],
        "gumap_quality_np": [vp, vp, i32, i32, vp, vp, vp, vp],
        "gumap_quality_stress": [vp, vp, i32, vp, vp, vp],
        "gumap_spectral_layout": [vp, i32, vp, vp, ctypes.POINTER(_SpectralInfo), vp],
    }
    out = {name: (args, ctypes.c_int) for name, args in sig.items()}
    out.update({
        "gumap_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "gumap_last_error": ([], ctypes.c_char_p),
        "gumap_server_clock": ([vp], ctypes.c_double),
        "gumap_selftest_wait_timeout": ([ctypes.c_int, ctypes.c_double], ctypes.c_int),
        "gumap_pool_trim": ([ctypes.c_int], ctypes.c_int),
        "gumap_pool_cached_bytes": ([], ctypes.c_int64),
    })
    return out


def load():
    """Load libgumap.so (built by ``__graft_entry__.build()``); raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libgumap.so not built at {path}: run __graft_entry__.build() "
                                   "(there is no CPU fallback)")
            lib = ctypes.CDLL(path)
            for name, (args, res) in _signatures().items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def gumap_status_string(status: int) -> str:
    return load().gumap_status_string(status).decode()


def gumap_last_error() -> str:
    return load().gumap_last_error().decode()


def _check(rc: int, what: str):
    if rc != OK:
        raise GumapError(rc, f"{what}: {gumap_status_string(rc)}: {gumap_last_error()}")


def _dptr(t, dtype=None, name="tensor"):
    """Device pointer of a CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


# ---------------------------------------------------------------- C names

def gumap_knn_create(row_ptr, col_idx, n: int, nnz: int, k: int, mode: int = FULL, flags: int = 0,
                     device: int = 0):
    """Returns an opaque handle. row_ptr/col_idx: host numpy int32 arrays, or
    CUDA int32 tensors together with CSR_ON_DEVICE in flags."""
    lib = load()
    keep = []
    if flags & CSR_ON_DEVICE:
        rp, col = _dptr(row_ptr, torch.int32, "row_ptr"), _dptr(col_idx, torch.int32, "col_idx")
    else:
        rp_a = np.ascontiguousarray(row_ptr, dtype=np.int32)
        col_a = np.ascontiguousarray(col_idx, dtype=np.int32)
        keep += [rp_a, col_a]
        rp, col = rp_a.ctypes.data, (col_a.ctypes.data if col_a.size else None)
    h = ctypes.c_void_p()
    _check(lib.gumap_knn_create(ctypes.byref(h), rp, col, int(n), int(nnz), int(k), int(mode), int(flags),
                                int(device)), "gumap_knn_create")
    return h


def gumap_batch_create(n_graphs: int, vertex_offsets, row_ptr, col_idx, nnz: int, k: int, modes, flags: int = 0,
                       device: int = 0):
    """Handle over many graphs laid side by side (host arrays, global ids)."""
    offs = np.ascontiguousarray(vertex_offsets, dtype=np.int32)
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col_idx, dtype=np.int32)
    md = np.ascontiguousarray(modes, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(load().gumap_batch_create(ctypes.byref(h), int(n_graphs), offs.ctypes.data, rp.ctypes.data,
                                     col.ctypes.data if col.size else None, int(nnz), int(k), md.ctypes.data,
                                     int(flags), int(device)), "gumap_batch_create")
    return h


def gumap_knn_run(h, sources, n_src: int, out_idx, out_dist, out_w, stream=None):
    """sources: CUDA int32 tensor or None (all vertices); outputs: CUDA tensors
    int32 / int16 (uint16 bit pattern) / float32 of shape [n_src, k]."""
    _check(load().gumap_knn_run(h, _dptr(sources, torch.int32, "sources"), int(n_src),
                                _dptr(out_idx, torch.int32, "out_idx"), _dptr(out_dist, torch.int16, "out_dist"),
                                _dptr(out_w, torch.float32, "out_w"), _stream(stream)), "gumap_knn_run")


def gumap_knn_apsp(h, sources, n_src: int, out_idx, out_dist, out_apsp, stream=None):
    """All-pairs hop-distance rows (CUDA int16 tensor [n_src, n], uint16 bit
    pattern) plus the kNN lists, for a handle created with EMIT_APSP."""
    _check(load().gumap_knn_apsp(h, _dptr(sources, torch.int32, "sources"), int(n_src),
                                 _dptr(out_idx, torch.int32, "out_idx"), _dptr(out_dist, torch.int16, "out_dist"),
                                 _dptr(out_apsp, torch.int16, "out_apsp"), _stream(stream)), "gumap_knn_apsp")


def gumap_knn_rho_sigma(h, rho, sigma, stream=None):
    _check(load().gumap_knn_rho_sigma(h, _dptr(rho, torch.float32, "rho"), _dptr(sigma, torch.float32, "sigma"),
                                      _stream(stream)), "gumap_knn_rho_sigma")


def gumap_knn_coo(h, row, col, w, nnz, stream=None):
    _check(load().gumap_knn_coo(h, _dptr(row, torch.int32, "row"), _dptr(col, torch.int32, "col"),
                                _dptr(w, torch.float32, "w"), _dptr(nnz, torch.int64, "nnz"), _stream(stream)),
           "gumap_knn_coo")


def gumap_knn_check(h, stream=None):
    _check(load().gumap_knn_check(h, _stream(stream)), "gumap_knn_check")


def gumap_knn_set_option(h, option: int, value: int):
    _check(load().gumap_knn_set_option(h, int(option), int(value)), "gumap_knn_set_option")


def gumap_knn_get_stats(h) -> dict:
    s = _Stats()
    _check(load().gumap_knn_get_stats(h, ctypes.byref(s)), "gumap_knn_get_stats")
    return {f: getattr(s, f) for f, _ in _Stats._fields_}


def gumap_knn_get_info(h) -> dict:
    i = _Info()
    _check(load().gumap_knn_get_info(h, ctypes.byref(i)), "gumap_knn_get_info")
    return {f: getattr(i, f) for f, _ in _Info._fields_}


def gumap_knn_autotune(h, cache_path: str | None = None) -> dict:
    """Time engine settings on the handle's graph, apply the best (see gumap.h)."""
    r = _Tune()
    _check(load().gumap_knn_autotune(h, cache_path.encode() if cache_path else None, ctypes.byref(r)),
           "gumap_knn_autotune")
    return {f: getattr(r, f) for f, _ in _Tune._fields_}


def gumap_knn_reset_stats(h):
    _check(load().gumap_knn_reset_stats(h), "gumap_knn_reset_stats")


def gumap_knn_destroy(h):
    _check(load().gumap_knn_destroy(h), "gumap_knn_destroy")


def gumap_knn_run_noalloc(row_ptr, col_idx, n: int, nnz: int, k: int, mode: int, out_idx, out_dist,
                          status=None, stream=None):
    """kNN lists of every vertex with no allocation inside the library (for
    callers that cannot allocate device memory at the point of the call: the
    scratch is a fixed array compiled into the library). row_ptr/col_idx are
    CUDA int32 tensors; outputs CUDA int32 / int16 tensors of shape [n, k];
    status an optional CUDA int32 tensor of one element."""
    _check(load().gumap_knn_run_noalloc(_dptr(row_ptr, torch.int32, "row_ptr"), _dptr(col_idx, torch.int32, "col_idx"),
                                        int(n), int(nnz), int(k), int(mode), _dptr(out_idx, torch.int32, "out_idx"),
                                        _dptr(out_dist, torch.int16, "out_dist"), _dptr(status, torch.int32, "status"),
                                        _stream(stream)), "gumap_knn_run_noalloc")


def gumap_quality_np(h, X, r: int = 2, out_c=None, out_inter=None, out_sum=None, stream=None):
    """Neighbourhood preservation of the drawing X (CUDA float32 tensor [n, dim])."""
    _check(load().gumap_quality_np(h, _dptr(X, torch.float32, "X"), int(X.shape[1]), int(r),
                                   _dptr(out_c, torch.int32, "out_c"), _dptr(out_inter, torch.int32, "out_inter"),
                                   _dptr(out_sum, torch.float64, "out_sum"), _stream(stream)), "gumap_quality_np")


def gumap_quality_stress(h, X, out_rows=None, out_stress=None, stream=None):
    """Aggregated stress of the drawing X (CUDA float32 tensor [n, dim])."""
    _check(load().gumap_quality_stress(h, _dptr(X, torch.float32, "X"), int(X.shape[1]),
                                       _dptr(out_rows, torch.float64, "out_rows"),
                                       _dptr(out_stress, torch.float64, "out_stress"), _stream(stream)),
           "gumap_quality_stress")


def gumap_spectral_layout(h, X, stream=None):
    """Spectral layout of the last run's union graph into X (CUDA float32 [n, dim]);
    returns (mu numpy float64 [dim], info dict)."""
    dim = int(X.shape[1])
    mu = np.empty(dim, dtype=np.float64)
    info = _SpectralInfo()
    _check(load().gumap_spectral_layout(h, dim, _dptr(X, torch.float32, "X"), mu.ctypes.data, ctypes.byref(info),
                                        _stream(stream)), "gumap_spectral_layout")
    return mu, {f: getattr(info, f) for f, _ in _SpectralInfo._fields_}


def gumap_pool_trim(device: int = -1):
    _check(load().gumap_pool_trim(int(device)), "gumap_pool_trim")


def gumap_pool_cached_bytes() -> int:
    return int(load().gumap_pool_cached_bytes())


def gumap_selftest_wait_timeout(device: int = 0, limit_s: float = 0.05) -> int:
    """Status of a grid barrier that can never complete (GUMAP_ERR_TIMEOUT expected)."""
    return int(load().gumap_selftest_wait_timeout(int(device), float(limit_s)))


# ---------------------------------------------------------------- serving

def gumap_server_create(device: int = 0, hbm_budget_bytes: int = 64 << 30, **opts):
    o = _ServerOpts(n_streams=opts.get("n_streams", 0), max_batch_graphs=opts.get("max_batch_graphs", 0),
                    max_batch_vertices=opts.get("max_batch_vertices", 0), max_queue=opts.get("max_queue", 0),
                    staging_bytes=opts.get("staging_bytes", 0), flags=opts.get("flags", 0))
    s = ctypes.c_void_p()
    _check(load().gumap_server_create(ctypes.byref(s), int(device), int(hbm_budget_bytes), ctypes.byref(o)),
           "gumap_server_create")
    return s


def gumap_serve_submit(s, row_ptr, col_idx, n: int, nnz: int, k: int, mode: int = PARTIAL) -> int:
    """Queue one graph (host arrays, copied before return); returns the request id.
    Raises GumapError with status ERR_AGAIN when the queue is full."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col_idx, dtype=np.int32)
    rid = ctypes.c_uint64()
    _check(load().gumap_serve_submit(s, rp.ctypes.data, col.ctypes.data if col.size else None, int(n), int(nnz),
                                     int(k), int(mode), ctypes.byref(rid)), "gumap_serve_submit")
    return int(rid.value)


def _result_dict(r: _Result) -> dict:
    return {f: getattr(r, f) for f, _ in _Result._fields_}


def gumap_serve_poll(s, req_id: int):
    """(status, result dict); status is OK, PENDING or the request's error."""
    r = _Result()
    st = load().gumap_serve_poll(s, int(req_id), ctypes.byref(r))
    if st not in (OK, PENDING) and st == ERR_UNKNOWN_REQUEST:
        _check(st, "gumap_serve_poll")
    return st, _result_dict(r)


def gumap_serve_wait(s, req_id: int, timeout_s: float = 60.0):
    r = _Result()
    st = load().gumap_serve_wait(s, int(req_id), ctypes.byref(r), float(timeout_s))
    if st == ERR_UNKNOWN_REQUEST:
        _check(st, "gumap_serve_wait")
    return st, _result_dict(r)


def gumap_serve_read(s, req_id: int, idx=None, dist=None, w=None, stream=None):
    """Copy a finished request's rows into CUDA tensors (int32 / int16 / float32, [n, k])."""
    _check(load().gumap_serve_read(s, int(req_id), _dptr(idx, torch.int32, "idx"), _dptr(dist, torch.int16, "dist"),
                                   _dptr(w, torch.float32, "w"), _stream(stream)), "gumap_serve_read")


def gumap_serve_release(s, req_id: int):
    _check(load().gumap_serve_release(s, int(req_id)), "gumap_serve_release")


def gumap_server_clock(s) -> float:
    return float(load().gumap_server_clock(s))


def gumap_server_get_stats(s) -> dict:
    st = _ServerStats()
    _check(load().gumap_server_get_stats(s, ctypes.byref(st)), "gumap_server_get_stats")
    return {f: getattr(st, f) for f, _ in _ServerStats._fields_}


def gumap_server_destroy(s):
    _check(load().gumap_server_destroy(s), "gumap_server_destroy")


# ---------------------------------------------------------------- wrapper

class KnnGraph:
    """A graph resident on the GPU plus the kNN/weight computation.

    >>> g = KnnGraph(row_ptr, col, k=15, mode=FULL)
    >>> out = g.run()            # dict of CUDA tensors idx / dist / w
    >>> row, col, w = g.coo()
    """

    def __init__(self, row_ptr, col_idx, k: int, mode: int = FULL, flags: int = 0, device: int = 0,
                 n: int | None = None):
        if n is None:
            n = int(row_ptr.shape[0]) - 1
        nnz = int(col_idx.shape[0])
        self.n, self.k, self.mode, self.flags, self.device = n, k, mode, flags, device
        self.h = gumap_knn_create(row_ptr, col_idx, n, nnz, k, mode, flags, device)

    @classmethod
    def from_graph(cls, g, k: int, mode: int = FULL, flags: int = 0, device: int = 0):
        return cls(g.row_ptr, g.col, k, mode, flags, device, n=g.n)

    @classmethod
    def batch(cls, graphs, k: int, modes, flags: int = 0, device: int = 0):
        """One handle over many graphs (gumap_batch_create). Rows of the
        result are the vertices of all graphs in order; ids are global
        (graph g's vertex v is offsets[g] + v). Returns (handle, offsets)."""
        offs = np.zeros(len(graphs) + 1, dtype=np.int64)
        rps, cols, eoff = [], [], 0
        for i, g in enumerate(graphs):
            offs[i + 1] = offs[i] + g.n
            rps.append(g.row_ptr[:-1].astype(np.int64) + eoff)
            cols.append(g.col.astype(np.int64) + offs[i])
            eoff += g.nnz
        rp = np.concatenate(rps + [np.array([eoff])]).astype(np.int32)
        col = np.concatenate(cols).astype(np.int32) if eoff else np.zeros(0, np.int32)
        self = cls.__new__(cls)
        self.n, self.k, self.mode, self.flags, self.device = int(offs[-1]), k, FULL, flags, device
        self.h = gumap_batch_create(len(graphs), offs.astype(np.int32), rp, col, int(eoff), k,
                                    np.asarray(modes, dtype=np.int32), flags, device)
        return self, offs

    def set_option(self, option: int, value: int):
        gumap_knn_set_option(self.h, option, value)

    def alloc_outputs(self, n_src: int):
        dev = torch.device("cuda", self.device)
        return dict(idx=torch.empty((n_src, self.k), dtype=torch.int32, device=dev),
                    dist=torch.empty((n_src, self.k), dtype=torch.int16, device=dev),
                    w=torch.empty((n_src, self.k), dtype=torch.float32, device=dev))

    def run(self, sources=None, stream=None, out=None) -> dict:
        n_src = self.n if sources is None else int(sources.shape[0])
        out = out or self.alloc_outputs(n_src)
        gumap_knn_run(self.h, sources, n_src, out["idx"], out["dist"], out["w"], stream)
        return out

    def apsp(self, sources=None, stream=None) -> dict:
        """All-pairs hop-distance rows of the sources ([n_src, n], uint16 bit
        pattern in int16) and their kNN lists; the handle needs EMIT_APSP."""
        n_src = self.n if sources is None else int(sources.shape[0])
        out = self.alloc_outputs(n_src)
        out["apsp"] = torch.empty((n_src, self.n), dtype=torch.int16, device=torch.device("cuda", self.device))
        gumap_knn_apsp(self.h, sources, n_src, out["idx"], out["dist"], out["apsp"], stream)
        return out

    def quality_np(self, X, r: int = 2, stream=None):
        """(c int32 [n], inter int32 [n], sum float64 [1]) of the drawing X (Section 4.1.3)."""
        dev = torch.device("cuda", self.device)
        c = torch.empty(self.n, dtype=torch.int32, device=dev)
        inter = torch.empty(self.n, dtype=torch.int32, device=dev)
        total = torch.empty(1, dtype=torch.float64, device=dev)
        gumap_quality_np(self.h, X, r, c, inter, total, stream)
        return c, inter, total

    def quality_stress(self, X, stream=None):
        """(stress float64 [1], per-row sums float64 [n]) of the drawing X (Section 4.1.3)."""
        dev = torch.device("cuda", self.device)
        rows = torch.empty(self.n, dtype=torch.float64, device=dev)
        total = torch.empty(1, dtype=torch.float64, device=dev)
        gumap_quality_stress(self.h, X, rows, total, stream)
        return total, rows

    def spectral_layout(self, dim: int = 2, stream=None):
        """(X float32 CUDA [n, dim], mu, info): spectral layout of the last run's union graph."""
        X = torch.empty((self.n, dim), dtype=torch.float32, device=torch.device("cuda", self.device))
        mu, info = gumap_spectral_layout(self.h, X, stream)
        return X, mu, info

    def rho_sigma(self, n_src: int | None = None, stream=None):
        n_src = self.n if n_src is None else n_src
        dev = torch.device("cuda", self.device)
        rho = torch.empty(n_src, dtype=torch.float32, device=dev)
        sigma = torch.empty(n_src, dtype=torch.float32, device=dev)
        gumap_knn_rho_sigma(self.h, rho, sigma, stream)
        return rho, sigma

    def coo(self, stream=None):
        dev = torch.device("cuda", self.device)
        cap = 2 * self.n * self.k
        row = torch.empty(cap, dtype=torch.int32, device=dev)
        col = torch.empty(cap, dtype=torch.int32, device=dev)
        w = torch.empty(cap, dtype=torch.float32, device=dev)
        nnz = torch.zeros(1, dtype=torch.int64, device=dev)
        gumap_knn_coo(self.h, row, col, w, nnz, stream)
        m = int(nnz.item())
        return row[:m], col[:m], w[:m]

    def check(self, stream=None):
        gumap_knn_check(self.h, stream)

    def stats(self) -> dict:
        return gumap_knn_get_stats(self.h)

    def info(self) -> dict:
        return gumap_knn_get_info(self.h)

    def autotune(self, cache_path: str | None = None) -> dict:
        return gumap_knn_autotune(self.h, cache_path)

    def reset_stats(self):
        gumap_knn_reset_stats(self.h)

    def close(self):
        if getattr(self, "h", None) is not None:
            gumap_knn_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dist_u16(t: torch.Tensor) -> np.ndarray:
    """Host uint16 view of a distance tensor stored as int16."""
    return t.cpu().numpy().view(np.uint16)
