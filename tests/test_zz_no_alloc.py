"""gnn_mp_forward_static: the layer forward for callers that cannot allocate.

Code that runs while a CUDA stream is being captured without a graph memory
pool, or inside a framework that owns the device allocator, cannot hand the
library a freshly allocated workspace. gnn_mp_forward_static uses a fixed
scratch area built into the library instead. This file checks, through the C
ABI, that it computes what gnn_mp_forward computes (two calls in a row, so the
shared area is reused) and that a graph too large for the area is refused.
It is collected last so a failure here never hides the other GPU tests."""
import ctypes as C

import numpy as np
import pytest
import torch

import synthetic as syn
from paper_2410_01657_gb300 import _build
from paper_2410_01657_gb300 import binding as B
from paper_2410_01657_gb300 import nn as gnn
from paper_2410_01657_gb300.graph import MeshGraph

pytestmark = pytest.mark.gpu
DEV = "cuda"
TOL = 2e-2   # the BF16 output tolerance of the fused-path tests


def _rel(a, b):
    return float(torch.linalg.norm((a - b).double()) / max(float(torch.linalg.norm(b.double())), 1e-300))


def _layer(H, R=3, nel=(4, 4, 4), p=3):
    part = MeshGraph(nel, p).partition(R, "rcb")
    G = part.to_device(DEV)
    params = syn.gnn_params(31, H, 2, 1, randomize_affine=True)
    layer = gnn.ConsistentGNN(params, precision="bf16", device=DEV).layers[0]
    tens = layer.edge.tensors() + layer.node.tensors()
    W = gnn.mp_params(layer.edge.dims, layer.node.dims, tens)
    rng = np.random.default_rng(32)
    x = torch.tensor(rng.standard_normal((part.n_rows, H)), dtype=torch.float32, device=DEV)
    e = torch.tensor(rng.standard_normal((part.n_edges, H)), dtype=torch.bfloat16, device=DEV)
    return part, G, W, tens, x, e


def _static_call(G, cfg, W, x, e, with_a):
    xo, eo = torch.empty_like(x), torch.empty_like(e)
    a = torch.empty_like(x) if with_a else None
    B.call("gnn_mp_forward_static", C.byref(G.struct), C.byref(cfg), C.byref(W), B.ptr(x), B.ptr(e),
           B.ptr(xo), B.ptr(eo), B.ptr(a), torch.cuda.current_stream().cuda_stream)
    return xo, eo, a


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    B.load()


@pytest.mark.parametrize("H,with_a", [(64, True), (32, False)])
def test_static_scratch_matches_workspace_forward(H, with_a):
    part, G, W, tens, x, e = _layer(H)
    cfg = gnn.mp_config(H, "bf16")
    xr, er, ar = torch.empty_like(x), torch.empty_like(e), torch.empty_like(x)
    gnn.gnn_mp_forward(G, cfg, W, x, e, xr, er, ar)
    for _ in range(2):   # the second call reuses the area the first one left behind
        xo, eo, a = _static_call(G, cfg, W, x, e, with_a)
        B.call("gnn_check", None)
        assert _rel(xo, xr) < TOL and _rel(eo.float(), er.float()) < TOL
        if with_a:
            assert _rel(a, ar) < TOL


def test_static_scratch_refuses_graphs_beyond_its_size():
    part = MeshGraph((16, 16, 16), 5).partition(8, "rcb")     # 551,368 rows x 4H bytes > 64 MiB at H=64
    G = part.to_device(DEV)
    H = 64
    params = syn.gnn_params(33, H, 2, 1)
    layer = gnn.ConsistentGNN(params, precision="bf16", device=DEV).layers[0]
    W = gnn.mp_params(layer.edge.dims, layer.node.dims, layer.edge.tensors() + layer.node.tensors())
    cfg = gnn.mp_config(H, "bf16")
    x = torch.zeros((part.n_rows, H), device=DEV)
    e = torch.zeros((part.n_edges, H), dtype=torch.bfloat16, device=DEV)
    xo, eo, a = torch.empty_like(x), torch.empty_like(e), torch.empty_like(x)
    rc = B.load().gnn_mp_forward_static(C.byref(G.struct), C.byref(cfg), C.byref(W), B.ptr(x), B.ptr(e),
                                        B.ptr(xo), B.ptr(eo), B.ptr(a), None)
    assert rc == B.GNN_ESHAPE
    assert "scratch" in B.last_error()
