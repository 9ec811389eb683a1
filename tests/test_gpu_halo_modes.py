"""The two halo modes of one NMP layer against the FP64 oracle, row by row
(needs a GB300).

* "None" mode (GNN_HALO_NONE; the paper's standard, inconsistent layer of its
  Sec. III-B comparison): Eq. 5c-5d are skipped, so every copy of a shared node
  keeps its own sub-graph's partial aggregate. The GPU forward and backward
  are compared with the oracle's ``halo=False`` layer.
* Consistent mode: the rows the copy-sum touches (every row of a node held by
  two or more sub-graphs) are checked one by one, so that a single wrong copy
  cannot hide inside a whole-tensor norm.

Tolerances: FP32 1e-5 relative L2 per tensor; BF16 2e-2 on outputs and 5e-2 on
gradients. Per row (copy rows only): FP32 1e-4, BF16 5e-2 on outputs and 1e-1
on gradients."""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import model as om
from paper_2410_01657_gb300 import _build
from paper_2410_01657_gb300 import binding as B
from paper_2410_01657_gb300 import nn as gnn
from paper_2410_01657_gb300.graph import MeshGraph

from gpu_util import max_row_rel, oracle_subgraphs, rel_l2, split_edges, split_rows

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    B.load()


def _bf16(a):
    return torch.as_tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)


def _inputs(part, H, seed):
    rng = np.random.default_rng(seed)
    gid = part.array("row_gid")
    recv, col = part.receivers(), part.array("col")
    uk, inv = np.unique(gid[recv] * part.graph.n_nodes + gid[col], return_inverse=True)
    x = rng.standard_normal((part.graph.n_nodes, H))[gid]
    e = _bf16(rng.standard_normal((uk.size, H))[inv])
    dx1 = rng.standard_normal((part.graph.n_nodes, H))[gid] / part.array("node_deg")[:, None]
    de1 = _bf16(rng.standard_normal((uk.size, H))[inv] * 0.5)
    return x, e, dx1, de1


def _run(G, params, H, x, e, dx1, de1, precision, halo):
    net = gnn.ConsistentGNN(params, precision=precision, device=DEV)
    layer = net.layers[0]
    edt = torch.bfloat16 if precision == "bf16" else torch.float32
    t = lambda a, d=torch.float32: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=DEV).to(d)
    xt, et = t(x), t(e, edt)
    tens = layer.edge.tensors() + layer.node.tensors()
    W = gnn.mp_params(layer.edge.dims, layer.node.dims, tens)
    cfg = gnn.mp_config(H, precision, halo=halo)
    xo, eo, a = torch.empty_like(xt), torch.empty_like(et), torch.empty_like(xt)
    gnn.gnn_mp_forward(G, cfg, W, xt, et, xo, eo, a)
    dparams = [torch.zeros_like(p) for p in tens]
    dxi, dei = torch.empty_like(xt), torch.empty_like(et)
    gnn.gnn_mp_backward(G, cfg, W, xt, et, a, t(dx1), t(de1, edt), dxi, dei,
                        gnn.mp_params(layer.edge.dims, layer.node.dims, dparams))
    B.call("gnn_check", None)
    out = {"x'": xo, "e'": eo, "a*": a, "dL/dx": dxi, "dL/de": dei}
    return {k: v.float().cpu().numpy() for k, v in out.items()}, [d.cpu().numpy() for d in dparams]


def _oracle(params, subs, x, e, dx1, de1, halo):
    lp = params["layers"][0]
    x1, e1, cache = om.layer_forward(lp, subs, split_rows(x, subs), split_edges(e, subs), halo=halo)
    dx0, de0, g = om.layer_backward(lp, subs, cache, split_rows(dx1, subs), split_edges(de1, subs), halo=halo)
    ref = {"x'": np.concatenate(x1), "e'": np.concatenate(e1), "a*": np.concatenate(cache["a_star"]),
           "dL/dx": np.concatenate(dx0), "dL/de": np.concatenate(de0)}
    gref = []
    for m in ("edge", "node"):
        gref += list(g[m]["W"]) + list(g[m]["b"]) + [g[m]["gamma"], g[m]["beta"]]
    return ref, gref


def _tols(precision):
    return (1e-5, 1e-5, 1e-4, 1e-4) if precision == "fp32" else (2e-2, 5e-2, 5e-2, 1e-1)


CASES = [((4, 3, 3), 3, 3, 16), ((4, 4, 4), 3, 8, 64), ((4, 3, 3), 3, 4, 128)]


@pytest.mark.parametrize("nel,p,R,H", CASES)
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_none_mode_matches_oracle_without_halo(nel, p, R, H, precision):
    brick, subs = oracle_subgraphs(nel, p, R)
    part = MeshGraph(nel, p).partition(R, "rcb")
    G = part.to_device(DEV)
    params = syn.gnn_params(61, H, 2, 1, randomize_affine=True)
    x, e, dx1, de1 = _inputs(part, H, 62)
    out, grads = _run(G, params, H, x, e, dx1, de1, precision, halo=False)
    ref, gref = _oracle(params, subs, x, e, dx1, de1, halo=False)
    lo, lg, ro, rg = _tols(precision)
    for k in ("x'", "e'", "a*"):
        assert rel_l2(out[k], ref[k]) < lo, (k, rel_l2(out[k], ref[k]))
    for k in ("dL/dx", "dL/de"):
        assert rel_l2(out[k], ref[k]) < lg, (k, rel_l2(out[k], ref[k]))
    for i, (got, r) in enumerate(zip(grads, gref)):
        assert rel_l2(got, r) < lg, (i, rel_l2(got, r))
    # the rows of shared nodes are where the two modes part: each copy keeps its
    # own partial aggregate, so copies of one node differ, and differ from the
    # consistent layer's
    shared = part.array("node_deg") > 1
    assert shared.sum() > 0
    assert max_row_rel(out["a*"], ref["a*"], shared) < ro
    cons, _ = _oracle(params, subs, x, e, dx1, de1, halo=True)
    assert rel_l2(out["a*"][shared], cons["a*"][shared]) > 0.1


@pytest.mark.parametrize("nel,p,R,H", CASES)
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_consistent_copy_rows_one_by_one(nel, p, R, H, precision):
    brick, subs = oracle_subgraphs(nel, p, R)
    part = MeshGraph(nel, p).partition(R, "rcb")
    G = part.to_device(DEV)
    params = syn.gnn_params(71, H, 2, 1, randomize_affine=True)
    x, e, dx1, de1 = _inputs(part, H, 72)
    out, grads = _run(G, params, H, x, e, dx1, de1, precision, halo=True)
    ref, gref = _oracle(params, subs, x, e, dx1, de1, halo=True)
    lo, lg, ro, rg = _tols(precision)
    shared = part.array("node_deg") > 1
    assert shared.sum() > 0
    for k in ("x'", "a*"):
        assert max_row_rel(out[k], ref[k], shared) < ro, (k, max_row_rel(out[k], ref[k], shared))
    # the input gradient of a node is the sum over its copies (each copy holds its
    # sub-graph's share): compare per global id
    gid = part.array("row_gid")
    N = part.graph.n_nodes
    gsum = np.zeros((N, H))
    rsum = np.zeros((N, H))
    np.add.at(gsum, gid, out["dL/dx"])
    np.add.at(rsum, gid, ref["dL/dx"])
    sg = np.unique(gid[shared])
    assert max_row_rel(gsum, rsum, sg) < rg
    # every edge whose receiver is a shared node (its aggregate reaches the copy-sum)
    recv = part.receivers()
    shared_e = shared[recv]
    assert max_row_rel(out["e'"], ref["e'"], shared_e) < ro
    assert max_row_rel(out["dL/de"], ref["dL/de"], shared_e) < rg
