"""Error of every output and gradient of one consistent NMP layer against the
FP64 oracle (needs a GB300), on p = 3/5/7 bricks split into sub-graphs, for
the FP32 path and the BF16 path at H = 16, 64 and 128.

Each case runs one layer forward (x', e', a*) and backward (dL/dx, dL/de and
the gradient of every weight, bias, gamma and beta of both MLPs) from seeded
inputs, and compares element by element with the oracle's FP64 result
(relative L2 over each tensor). The table is printed (``pytest -s``) and every
entry is held to the tolerances of the path: FP32 1e-5; BF16 2e-2 on outputs,
5e-2 on gradients."""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import model as om
from paper_2410_01657_gb300 import _build
from paper_2410_01657_gb300 import binding as B
from paper_2410_01657_gb300 import nn as gnn
from paper_2410_01657_gb300.graph import MeshGraph

from gpu_util import oracle_subgraphs, rel_l2, split_edges, split_rows

pytestmark = pytest.mark.gpu
DEV = "cuda"

# (name, elements per axis, order, sub-graphs, H, MLP hidden layers)
CASES = [
    ("4^3 p=3, 2 slabs, H=16", (4, 4, 4), 3, 2, 16, 2),
    ("4^3 p=5, 8 RCB parts, H=64", (4, 4, 4), 5, 8, 64, 2),
    ("4x3x3 p=7, 4 RCB parts, H=128", (4, 3, 3), 7, 4, 128, 2),
]


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    B.load()


def _bf16(a):
    return torch.as_tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)


def _case(nel, p, R, H, nh, seed=5):
    brick, subs = oracle_subgraphs(nel, p, R, "slab" if R == 2 else "rcb")
    part = MeshGraph(nel, p).partition(R, "slab" if R == 2 else "rcb")
    G = part.to_device(DEV)
    params = syn.gnn_params(seed, H, nh, 1, randomize_affine=True)
    rng = np.random.default_rng(seed + 1)
    gid = part.array("row_gid")
    recv, col = part.receivers(), part.array("col")
    uk, inv = np.unique(gid[recv] * part.graph.n_nodes + gid[col], return_inverse=True)
    x = rng.standard_normal((part.graph.n_nodes, H))[gid]
    e = _bf16(rng.standard_normal((uk.size, H))[inv])
    dx1 = rng.standard_normal((part.graph.n_nodes, H))[gid] / np.maximum(part.array("node_deg")[:, None], 1)
    de1 = _bf16(rng.standard_normal((uk.size, H))[inv] * 0.5)
    lp = params["layers"][0]
    x1, e1, cache = om.layer_forward(lp, subs, split_rows(x, subs), split_edges(e, subs))
    dx0, de0, g = om.layer_backward(lp, subs, cache, split_rows(dx1, subs), split_edges(de1, subs))
    ref = {"x'": np.concatenate(x1), "e'": np.concatenate(e1), "a*": np.concatenate(cache["a_star"]),
           "dL/dx": np.concatenate(dx0), "dL/de": np.concatenate(de0)}
    gref = []
    for m in ("edge", "node"):
        gref += [(f"{m} W{k}", w) for k, w in enumerate(g[m]["W"])]
        gref += [(f"{m} b{k}", b) for k, b in enumerate(g[m]["b"])]
        gref += [(f"{m} gamma", g[m]["gamma"]), (f"{m} beta", g[m]["beta"])]
    return G, params, x, e, dx1, de1, ref, gref


def _run(G, params, H, x, e, dx1, de1, precision):
    net = gnn.ConsistentGNN(params, precision=precision, device=DEV)
    layer = net.layers[0]
    edt = torch.bfloat16 if precision == "bf16" else torch.float32
    t = lambda a, d=torch.float32: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=DEV).to(d)
    xt, et = t(x), t(e, edt)
    tens = layer.edge.tensors() + layer.node.tensors()
    W = gnn.mp_params(layer.edge.dims, layer.node.dims, tens)
    cfg = gnn.mp_config(H, precision)
    xo, eo, a = torch.empty_like(xt), torch.empty_like(et), torch.empty_like(xt)
    gnn.gnn_mp_forward(G, cfg, W, xt, et, xo, eo, a)
    dparams = [torch.zeros_like(p) for p in tens]
    dxi, dei = torch.empty_like(xt), torch.empty_like(et)
    gnn.gnn_mp_backward(G, cfg, W, xt, et, a, t(dx1), t(de1, edt), dxi, dei,
                        gnn.mp_params(layer.edge.dims, layer.node.dims, dparams))
    B.call("gnn_check", None)
    out = {"x'": xo, "e'": eo, "a*": a, "dL/dx": dxi, "dL/de": dei}
    return {k: v.float().cpu().numpy() for k, v in out.items()}, [d.cpu().numpy() for d in dparams]


@pytest.mark.parametrize("name,nel,p,R,H,nh", CASES)
def test_precision_report(name, nel, p, R, H, nh):
    G, params, x, e, dx1, de1, ref, gref = _case(nel, p, R, H, nh)
    lines = []
    for precision in ("fp32", "bf16"):
        out, grads = _run(G, params, H, x, e, dx1, de1, precision)
        for k, r in ref.items():
            err = rel_l2(out[k], r)
            lim = 1e-5 if precision == "fp32" else (2e-2 if k in ("x'", "e'", "a*") else 5e-2)
            lines.append((precision, k, err))
            assert err < lim, (name, precision, k, err)
        errs = [(gn, rel_l2(gv, gr)) for (gn, gr), gv in zip(gref, grads)]
        for gn, err in errs:
            assert err < (1e-5 if precision == "fp32" else 5e-2), (name, precision, gn, err)
        worst = max(errs, key=lambda t: t[1])
        lines.append((precision, f"parameter gradients ({len(errs)} tensors), max: {worst[0]}", worst[1]))
        lines.append((precision, "parameter gradients, median", float(np.median([e for _, e in errs]))))
    print(f"\n{name}")
    for precision, k, err in lines:
        print(f"  {precision:4s}  {k:52s} {err:.2e}")
