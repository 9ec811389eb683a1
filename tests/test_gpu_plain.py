"""Parity of the plain FP32 GPU path with the FP64 oracle (needs a GB300).

Tolerances (rel-L2 over the whole tensor): FP32 path vs FP64 oracle 1e-5 per
output and per gradient; FP32 partitioned vs unpartitioned 1e-6."""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import graph as og
from oracle import model as om
from paper_2410_01657_gb300 import _build
from paper_2410_01657_gb300 import binding as B
from paper_2410_01657_gb300 import nn as gnn
from paper_2410_01657_gb300.graph import MeshGraph

from gpu_util import flat_grads, node_field, oracle_network, oracle_subgraphs, rel_l2, split_edges, split_rows

pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    B.load()


def _lib_graph(nel, p, R, method="rcb", weights=None, periodic=(False, False, False)):
    part = MeshGraph(nel, p, periodic=periodic).partition(R, method, weights)
    return part, part.to_device(DEV)


def _to(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device=DEV)


@pytest.mark.parametrize("R,method", [(1, "rcb"), (2, "slab")])
def test_config1_encoders_and_one_layer(R, method):
    # 4x4x4 elements at p=3 (2197 nodes), H=16, node/edge encoders + one consistent layer
    nel, p, H = (4, 4, 4), 3, 16
    brick, subs = oracle_subgraphs(nel, p, R, method)
    part, G = _lib_graph(nel, p, R, method)
    params = syn.gnn_params(0, H, 2, 1, randomize_affine=True)
    u = node_field(brick)
    us = [u[sg.gid] for sg in subs]
    attr = [og.edge_attributes(brick.pos, sg) for sg in subs]
    x0 = [om.mlp_forward(params["enc_node"], a)[0] for a in us]
    e0 = [om.mlp_forward(params["enc_edge"], a)[0] for a in attr]
    x1, e1, cache = om.layer_forward(params["layers"][0], subs, x0, e0)

    net = gnn.ConsistentGNN(params, precision="fp32", device=DEV)
    u_t = _to(np.concatenate(us))
    attr_t = G.edge_attr()
    with torch.no_grad():
        x, e = net.encode(G, u_t, attr_t)
        xo, eo = net.process(G, x, e)
    assert rel_l2(x.cpu().numpy(), np.concatenate(x0)) < 1e-5
    assert rel_l2(e.cpu().numpy(), np.concatenate(e0)) < 1e-5
    assert rel_l2(xo.cpu().numpy(), np.concatenate(x1)) < 1e-5
    assert rel_l2(eo.cpu().numpy(), np.concatenate(e1)) < 1e-5


def test_config1_partitioned_equals_unpartitioned_fp32():
    nel, p, H = (4, 4, 4), 3, 16
    params = syn.gnn_params(1, H, 2, 2, randomize_affine=True)
    outs = {}
    for R, method in [(1, "rcb"), (2, "slab"), (8, "rcb")]:
        part, G = _lib_graph(nel, p, R, method)
        pos = part.array("row_pos")
        u = syn.fourier_field(pos, syn.fourier_modes(0, 8))
        net = gnn.ConsistentGNN(params, precision="fp32", device=DEV)
        with torch.no_grad():
            y = net(G, _to(u), G.edge_attr()).cpu().numpy()
        glob = np.zeros((part.graph.n_nodes, 3))
        glob[part.array("row_gid")] = y
        outs[R] = glob
        if R > 1:   # copies of a node agree bitwise
            gid = part.array("row_gid")
            order = np.argsort(gid, kind="stable")
            same = gid[order][1:] == gid[order][:-1]
            assert np.array_equal(y[order][1:][same], y[order][:-1][same])
    for R in (2, 8):
        assert rel_l2(outs[R], outs[1]) < 1e-6


def test_halo_exchange_sums_copies():
    part, G = _lib_graph((3, 3, 3), 2, 5, "rcb", [1, 2, 1, 3, 1])
    rng = np.random.default_rng(0)
    a = rng.standard_normal((part.n_rows, 7)).astype(np.float32)
    t = _to(a)
    gnn.gnn_halo_exchange(G, t)
    out = t.cpu().numpy()
    gid = part.array("row_gid")
    ref = np.zeros((part.graph.n_nodes, 7))
    np.add.at(ref, gid, a.astype(np.float64))
    np.testing.assert_allclose(out, ref[gid], rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("R,method,weights", [(1, "rcb", None), (3, "rcb", [1, 2, 1])])
def test_network_forward_backward_fp32_vs_oracle(R, method, weights):
    nel, p, H, M = (3, 3, 2), 2, 16, 2
    brick, subs = oracle_subgraphs(nel, p, R, method, weights)
    part, G = _lib_graph(nel, p, R, method, weights)
    params = syn.gnn_params(3, H, 2, M, randomize_affine=True)
    u = node_field(brick, 1)
    target = node_field(brick, 2)
    ys, L, g, _ = oracle_network(params, brick, subs, u, target)
    net = gnn.ConsistentGNN(params, precision="fp32", device=DEV)
    u_t = _to(np.concatenate([u[sg.gid] for sg in subs]))
    t_t = _to(np.concatenate([target[sg.gid] for sg in subs]))
    y = net(G, u_t, G.edge_attr())
    loss = gnn.consistent_loss(y, t_t, G)
    loss.backward()
    assert rel_l2(y.detach().cpu().numpy(), np.concatenate(ys)) < 1e-5
    assert abs(loss.item() - L) <= 1e-5 * abs(L)
    gg = dict(flat_grads(net.grads_numpy()))
    for name, ref in flat_grads(g):
        err = rel_l2(gg[name], ref)
        assert err < 1e-4, (name, err)


def test_layer_backward_fp32_vs_oracle_with_edge_grad():
    # single layer with upstream gradients on both x' and e' (de_out != 0)
    nel, p, H, R = (3, 2, 3), 2, 32, 4
    brick, subs = oracle_subgraphs(nel, p, R, "rcb")
    part, G = _lib_graph(nel, p, R, "rcb")
    params = syn.gnn_params(4, H, 2, 1, randomize_affine=True)
    lp = params["layers"][0]
    rng = np.random.default_rng(7)
    x = rng.standard_normal((part.n_rows, H))
    e = rng.standard_normal((part.n_edges, H))
    # coincident copies must carry equal states: take x per global id
    gid = part.array("row_gid")
    xg = rng.standard_normal((part.graph.n_nodes, H))
    x = xg[gid]
    xs, es = split_rows(x, subs), split_edges(e, subs)
    x1, e1, cache = om.layer_forward(lp, subs, xs, es)
    dx1 = [rng.standard_normal(a.shape) for a in x1]
    de1 = [rng.standard_normal(a.shape) for a in e1]
    dx0, de0, g = om.layer_backward(lp, subs, cache, dx1, de1)
    layer = gnn.ConsistentGNN(params, precision="fp32", device=DEV).layers[0]
    tens = layer.edge.tensors() + layer.node.tensors()
    xt, et = _to(x).requires_grad_(True), _to(e).requires_grad_(True)
    xo, eo = gnn.ConsistentMPFunction.apply(xt, et, G, (H, "fp32", True, 1e-5, 0), layer.edge.dims,
                                            layer.node.dims, True, *tens)
    assert rel_l2(xo.detach().cpu().numpy(), np.concatenate(x1)) < 1e-5
    assert rel_l2(eo.detach().cpu().numpy(), np.concatenate(e1)) < 1e-5
    torch.autograd.backward([xo, eo], [_to(np.concatenate(dx1)), _to(np.concatenate(de1))])
    assert rel_l2(xt.grad.cpu().numpy(), np.concatenate(dx0)) < 1e-5
    assert rel_l2(et.grad.cpu().numpy(), np.concatenate(de0)) < 1e-5
    for which, m in (("edge", layer.edge), ("node", layer.node)):
        refs = list(g[which]["W"]) + list(g[which]["b"]) + [g[which]["gamma"], g[which]["beta"]]
        for k, (t, ref) in enumerate(zip(m.tensors(), refs)):
            assert rel_l2(t.grad.cpu().numpy(), ref) < 1e-5, (which, k)


def test_plain_path_is_deterministic():
    part, G = _lib_graph((4, 4, 4), 2, 4, "rcb")
    params = syn.gnn_params(5, 32, 2, 2, randomize_affine=True)
    u = _to(syn.fourier_field(part.array("row_pos"), syn.fourier_modes(0, 8)))
    t = _to(np.cos(u.cpu().numpy()))
    res = []
    for _ in range(2):
        net = gnn.ConsistentGNN(params, precision="fp32", device=DEV)
        loss = gnn.consistent_loss(net(G, u, G.edge_attr()), t, G)
        loss.backward()
        res.append((loss.item(), [p.grad.clone() for p in net.parameters()]))
    assert res[0][0] == res[1][0]
    for a, b in zip(res[0][1], res[1][1]):
        assert torch.equal(a, b)


def test_empty_graph_is_a_noop():
    # zero rows / edges: entry points return without launching anything
    import ctypes as C
    G = B.gnn_graph_dev()
    cfg = gnn.mp_config(16, "fp32")
    params = syn.gnn_params(0, 16, 2, 1)
    layer = gnn.ConsistentGNN(params, precision="fp32", device=DEV).layers[0]
    W = gnn.mp_params(layer.edge.dims, layer.node.dims, layer.edge.tensors() + layer.node.tensors())
    f, b = C.c_size_t(), C.c_size_t()
    B.call("gnn_mp_workspace_size", C.byref(G), C.byref(cfg), C.byref(W), C.byref(f), C.byref(b))
    ws = torch.empty(max(f.value, b.value, 1), dtype=torch.uint8, device=DEV)
    B.call("gnn_mp_forward", C.byref(G), C.byref(cfg), C.byref(W), None, None, None, None, None, B.ptr(ws),
           ws.numel(), None)
    B.call("gnn_check", None)
