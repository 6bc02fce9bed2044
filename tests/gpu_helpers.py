"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and compare with the CPU oracle element by element."""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2509_19703_gb300 import gumap

W_TOL = 1e-5       # absolute tolerance on FP32 weights vs the FP64 oracle
SIGMA_RTOL = 1e-5  # relative tolerance on sigma


def run_gpu(g, k, mode="full", engine=None, block_bits=None, sources=None, directed=False, coo=True,
            direction=None, coo_build=None, frontier_build=None, batch_width=None):
    flags = gumap.WEIGHTS_DIRECTED if directed else gumap.WEIGHTS_UNION
    m = gumap.FULL if mode == "full" else gumap.PARTIAL
    with gumap.KnnGraph.from_graph(g, k, mode=m, flags=flags) as kg:
        if engine is not None:
            kg.set_option(gumap.OPT_ENGINE, engine)
        if block_bits is not None:
            kg.set_option(gumap.OPT_BLOCK_BITS, block_bits)
        if direction is not None:
            kg.set_option(gumap.OPT_DIRECTION, direction)
        if coo_build is not None:
            kg.set_option(gumap.OPT_COO_BUILD, coo_build)
        if frontier_build is not None:
            kg.set_option(gumap.OPT_FRONTIER_BUILD, frontier_build)
        if batch_width is not None:
            kg.set_option(gumap.OPT_BATCH_WIDTH, batch_width)
        src_t = None
        if sources is not None:
            src_t = torch.as_tensor(np.asarray(sources, dtype=np.int32), device="cuda")
        out = kg.run(sources=src_t)
        n_src = g.n if sources is None else len(sources)
        rho, sigma = kg.rho_sigma(n_src)
        res = {}
        if coo and not directed:
            r, c, w = kg.coo()
            res["coo"] = (r.cpu().numpy(), c.cpu().numpy(), w.cpu().numpy().astype(np.float64))
        kg.check()
        torch.cuda.synchronize()
        res.update(idx=out["idx"].cpu().numpy(), dist=gumap.dist_u16(out["dist"]),
                   w=out["w"].cpu().numpy().astype(np.float64), rho=rho.cpu().numpy().astype(np.float64),
                   sigma=sigma.cpu().numpy().astype(np.float64), stats=kg.stats())
    return res


def oracle_ref(g, k, mode="full", sources=None, directed=False, coo=True):
    if mode == "full":
        idx, dist = oracle.knn_full(g, k, sources)
    else:
        idx, dist = oracle.knn_partial(g, k, sources)
    rho, sigma, a = oracle.smooth_knn(dist)
    ref = dict(idx=idx, dist=dist, rho=rho, sigma=sigma, a=a)
    if directed:
        ref["w"] = a
    else:
        ref["w"] = oracle.slot_union(idx, a)
        if coo:
            ref["coo"] = oracle.coo_union(idx, a)
    return ref


def assert_sigma_close(got, want, tag=""):
    both_inf = np.isinf(got) & np.isinf(want)
    assert np.array_equal(np.isinf(got), np.isinf(want)), f"{tag}: sigma inf pattern differs"
    fin = ~both_inf
    g, w = got[fin], want[fin]
    zero = w == 0.0
    assert np.all(g[zero] == 0.0), f"{tag}: sigma zero pattern differs"
    rel = np.abs(g[~zero] - w[~zero]) / w[~zero]
    assert rel.size == 0 or float(rel.max()) <= SIGMA_RTOL, f"{tag}: sigma rel err {rel.max():.3g}"


def assert_parity(res, ref, tag="", rows=None):
    """Bit-exact indices/distances; weights within W_TOL; rho exact; sigma
    within SIGMA_RTOL; COO structure exact and weights within W_TOL. Returns
    the max weight error."""
    sel = slice(None) if rows is None else rows
    gi, gd = res["idx"][sel], res["dist"][sel]
    if not np.array_equal(gi, ref["idx"]):
        bad = np.argwhere(np.any(gi != ref["idx"], axis=1))[:3, 0]
        raise AssertionError(f"{tag}: idx differs at rows {bad.tolist()}: gpu {gi[bad].tolist()} "
                             f"oracle {ref['idx'][bad].tolist()}")
    assert np.array_equal(gd, ref["dist"]), f"{tag}: dist differs"
    werr = float(np.max(np.abs(res["w"][sel] - ref["w"]))) if ref["w"].size else 0.0
    assert werr <= W_TOL, f"{tag}: max |dw| = {werr}"
    assert np.array_equal(res["rho"][sel], ref["rho"]), f"{tag}: rho differs"
    assert_sigma_close(res["sigma"][sel], ref["sigma"], tag)
    if "coo" in ref and "coo" in res:
        gr, gc, gw = res["coo"]
        rr, rc, rw = ref["coo"]
        assert np.array_equal(gr, rr) and np.array_equal(gc, rc), f"{tag}: COO structure differs"
        cerr = float(np.max(np.abs(gw - rw))) if rw.size else 0.0
        assert cerr <= W_TOL, f"{tag}: COO max |dw| = {cerr}"
        werr = max(werr, cerr)
    return werr
