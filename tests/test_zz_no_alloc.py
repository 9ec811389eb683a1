"""gnn_mp_forward_static: the layer forward for callers that cannot allocate.

Code that runs while a CUDA stream is being captured without a graph memory
pool, or inside a framework that owns the device allocator, cannot hand the
library a freshly allocated workspace. gnn_mp_forward_static uses a fixed
scratch area built into the library instead. This file checks, through the C
ABI, that it computes bit for bit what gnn_mp_forward computes (two calls in a
row with a call on another graph between them, so the shared area is reused
and holds other data) and that a graph too large for the area is refused.
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


@pytest.mark.parametrize("H,with_a", [(64, True), (64, False), (32, False), (128, True)])
def test_static_scratch_matches_workspace_forward(H, with_a):
    # The static entry point runs the same deterministic kernels on the same
    # tiles as gnn_mp_forward, so the results must agree bit for bit. Between
    # the two static calls on this graph a call on another graph (another size,
    # other inputs) leaves different data in the shared area; the second call
    # must not see any of it.
    part, G, W, tens, x, e = _layer(H)
    cfg = gnn.mp_config(H, "bf16")
    xr, er, ar = torch.empty_like(x), torch.empty_like(e), torch.empty_like(x)
    gnn.gnn_mp_forward(G, cfg, W, x, e, xr, er, ar if with_a else None)
    _, G2, W2, _, x2, e2 = _layer(H, R=2, nel=(3, 5, 4), p=2)
    for call in range(2):
        if call == 1:
            _static_call(G2, cfg, W2, 3.0 * x2, e2, with_a)
        xo, eo, a = _static_call(G, cfg, W, x, e, with_a)
        B.call("gnn_check", None)
        assert torch.equal(xo, xr), (call, _rel(xo, xr))
        assert torch.equal(eo, er), (call, _rel(eo.float(), er.float()))
        if with_a:
            assert torch.equal(a, ar), (call, _rel(a, ar))
        # and within the fused path's BF16 tolerance of the plain FP32 path
        cfg32 = gnn.mp_config(H, "fp32")
        x32, e32 = torch.empty_like(x), torch.empty(e.shape, device=DEV)
        gnn.gnn_mp_forward(G, cfg32, W, x, e.float(), x32, e32, torch.empty_like(x))
        assert _rel(xo, x32) < TOL and _rel(eo.float(), e32) < TOL


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
