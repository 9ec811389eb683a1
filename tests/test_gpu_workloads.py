"""The benchmark workload families at test size, BF16 fused path vs the FP64 oracle.

* batching form: a jittered brick cut into 64 RCB sub-graphs of log-uniform
  element counts (uneven sizes), several consistent layers forward and backward,
  partitioned == unpartitioned;
* inference form: H=32 layers forward only, the last one without writing its
  edge state (GNN_FLAG_NO_EDGE_OUT)."""
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

from gpu_util import rel_l2, split_edges, split_rows

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    B.load()


def _bf16(a):
    return torch.as_tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)


def _uneven_case(p=2, seed=3):
    n, w = syn.uneven_brick(64, 1, 12, seed)
    brick0 = og.build_brick((n, n, n), p)
    jit = syn.jitter_unit(brick0.n_nodes, seed + 1)
    brick = og.build_brick((n, n, n), p, jitter=jit, jitter_frac=0.2)
    part_o = og.partition_rcb(brick, 64, w)
    subs = og.build_subgraphs(brick, part_o, 64)
    lib = MeshGraph((n, n, n), p, jitter=jit, jitter_frac=0.2)
    np.testing.assert_allclose(lib.pos(), brick.pos, atol=1e-14)
    part = lib.partition(64, "rcb", w)
    return brick, subs, part


@pytest.mark.parametrize("save_act", [False, True])
def test_uneven_64_subgraphs_layers_fwd_bwd(save_act):
    H, M = 64, 2
    brick, subs, part = _uneven_case()
    sizes = part.array("part_stats")[:, 0]
    assert sizes.max() > 4 * sizes.min()                      # uneven sub-graphs
    G = part.to_device(DEV)
    params = syn.gnn_params(40, H, 2, M, randomize_affine=True)
    gid = part.array("row_gid")
    rng = np.random.default_rng(41)
    x = rng.standard_normal((brick.n_nodes, H))[gid]
    attr = [og.edge_attributes(brick.pos, sg) for sg in subs]
    e = _bf16(np.concatenate([om.mlp_forward(params["enc_edge"], a)[0] for a in attr]))
    xs, es = split_rows(x, subs), split_edges(e, subs)
    caches = []
    for lp in params["layers"]:
        xs, es, c = om.layer_forward(lp, subs, xs, es)
        caches.append(c)
    net = gnn.ConsistentGNN(params, precision="bf16", device=DEV)
    layers = [(l.edge.tensors(), l.node.tensors(), l.edge.dims, l.node.dims) for l in net.layers]
    stack = gnn.LayerStack(G, layers, H, "bf16", torch.tensor(x, dtype=torch.float32, device=DEV),
                           torch.tensor(e, dtype=torch.float32, device=DEV), save_act=save_act)
    stack.forward()
    B.call("gnn_check", None)
    assert rel_l2(stack.x[M].cpu().numpy(), np.concatenate(xs)) < 2e-2
    assert rel_l2(stack.e[M].float().cpu().numpy(), np.concatenate(es)) < 2e-2
    # coincident copies agree bitwise across the 64 sub-graphs
    xo = stack.x[M].cpu().numpy()
    order = np.argsort(gid, kind="stable")
    same = gid[order][1:] == gid[order][:-1]
    assert np.array_equal(xo[order][1:][same], xo[order][:-1][same])
    # backward: upstream gradient on x only, weight gradients vs the oracle
    dxg = rng.standard_normal((brick.n_nodes, H))
    dx_top = dxg[gid] / part.array("node_deg")[:, None]
    stack.backward(torch.tensor(dx_top, dtype=torch.float32, device=DEV))
    B.call("gnn_check", None)
    dx, de = split_rows(dx_top, subs), [np.zeros_like(a) for a in es]
    grads = [None] * M
    for li in range(M - 1, -1, -1):
        dx, de, grads[li] = om.layer_backward(params["layers"][li], subs, caches[li], dx, de)
    assert rel_l2(stack.dx[0].cpu().numpy(), np.concatenate(dx)) < 5e-2
    for li in range(M):
        g = grads[li]
        refs = list(g["edge"]["W"]) + list(g["edge"]["b"]) + [g["edge"]["gamma"], g["edge"]["beta"]] \
            + list(g["node"]["W"]) + list(g["node"]["b"]) + [g["node"]["gamma"], g["node"]["beta"]]
        for k, (got, ref) in enumerate(zip(stack.dparams[li], refs)):
            assert rel_l2(got.cpu().numpy(), ref) < 5e-2, (li, k)


def test_uneven_partitioned_equals_unpartitioned():
    H = 64
    brick, subs, part = _uneven_case(seed=5)
    params = syn.gnn_params(42, H, 2, 2, randomize_affine=True)
    out = {}
    for R, prt in ((64, part), (1, part.graph.partition(1, "rcb"))):
        G = prt.to_device(DEV)
        net = gnn.ConsistentGNN(params, precision="bf16", device=DEV)
        u = torch.tensor(syn.fourier_field(prt.array("row_pos"), syn.fourier_modes(6, 8)), dtype=torch.float32,
                         device=DEV)
        with torch.no_grad():
            y = net(G, u, G.edge_attr()).cpu().numpy()
        glob = np.zeros((brick.n_nodes, 3))
        glob[prt.array("row_gid")] = y
        out[R] = glob
    assert rel_l2(out[64], out[1]) < 2e-2


def test_inference_h32_last_layer_without_edge_output():
    H, M = 32, 3
    nel, p = (4, 4, 3), 3
    brick = og.build_brick(nel, p)
    subs = og.build_subgraphs(brick, og.partition_rcb(brick, 4), 4)
    part = MeshGraph(nel, p).partition(4, "rcb")
    G = part.to_device(DEV)
    params = syn.gnn_params(43, H, 2, M, randomize_affine=True)
    gid = part.array("row_gid")
    rng = np.random.default_rng(44)
    x = rng.standard_normal((brick.n_nodes, H))[gid]
    key = gid[part.receivers()] * brick.n_nodes + gid[part.array("col")]
    _, inv = np.unique(key, return_inverse=True)
    e = _bf16(rng.standard_normal((inv.max() + 1, H))[inv])
    xs, es = split_rows(x, subs), split_edges(e, subs)
    for lp in params["layers"]:
        xs, es, _ = om.layer_forward(lp, subs, xs, es)
    net = gnn.ConsistentGNN(params, precision="bf16", device=DEV)
    xt = torch.tensor(x, dtype=torch.float32, device=DEV)
    et = torch.tensor(e, dtype=torch.bfloat16, device=DEV)
    for li, layer in enumerate(net.layers):
        last = li == M - 1
        cfg = gnn.mp_config(H, "bf16", flags=B.GNN_FLAG_NO_EDGE_OUT if last else 0)
        W = gnn.mp_params(layer.edge.dims, layer.node.dims, layer.edge.tensors() + layer.node.tensors())
        xo = torch.empty_like(xt)
        eo = None if last else torch.empty_like(et)
        gnn.gnn_mp_forward(G, cfg, W, xt, et, xo, eo)
        xt, et = xo, eo
    B.call("gnn_check", None)
    assert rel_l2(xt.cpu().numpy(), np.concatenate(xs)) < 2e-2


def _stack_case(H=64, M=3, inference=False, seed=50, save_act=False):
    brick, subs, part = _uneven_case(seed=seed)
    G = part.to_device(DEV)
    params = syn.gnn_params(seed, H, 2, M, randomize_affine=True)
    net = gnn.ConsistentGNN(params, precision="bf16", device=DEV)
    layers = [(l.edge.tensors(), l.node.tensors(), l.edge.dims, l.node.dims) for l in net.layers]
    g = torch.Generator(device=DEV).manual_seed(seed)
    x0 = torch.randn(part.n_rows, H, device=DEV, generator=g)
    e0 = torch.randn(part.n_edges, H, device=DEV, generator=g).to(torch.bfloat16)
    dx = 1e-3 * torch.randn(part.n_rows, H, device=DEV, generator=g)
    stack = gnn.LayerStack(G, layers, H, "bf16", x0, e0, inference=inference, save_act=save_act)
    return part, G, layers, x0, e0, dx, stack


def test_inference_stack_equals_training_forward():
    H, M = 32, 4
    part, G, layers, x0, e0, dx, tr = _stack_case(H, M)
    inf = gnn.LayerStack(G, layers, H, "bf16", x0, e0, inference=True)
    tr.forward()
    inf.forward()
    inf.forward()                     # repeated steps read the same inputs
    torch.cuda.synchronize()
    assert torch.equal(inf.x_out, tr.x[M])
    assert len(inf.e) == 3 and len(inf.x) == 3


@pytest.mark.parametrize("H,M,save_act", [(64, 3, False), (64, 3, True), (128, 2, False)])
def test_cuda_graph_replay_matches_eager_step(H, M, save_act):
    # H = 128 captures the layered adjoint (recomputation, per-Linear kernels, reductions)
    part, G, layers, x0, e0, dx, stack = _stack_case(H, M, save_act=save_act)
    stack.zero_grad()
    stack.step(dx)
    torch.cuda.synchronize()
    x_ref = stack.x[-1].clone()
    g_ref = [t.clone() for t in stack.dparams[0]]
    stack.capture(dx)
    stack.zero_grad()
    stack.replay()
    torch.cuda.synchronize()
    assert torch.equal(stack.x[-1], x_ref)
    for t, r in zip(stack.dparams[0], g_ref):
        assert torch.equal(t, r)
    B.call("gnn_check", None)


def test_autotune_keeps_results_and_caches(tmp_path):
    part, G, layers, x0, e0, dx, stack = _stack_case(H=32, M=2, inference=True, seed=60)
    stack.forward()
    torch.cuda.synchronize()
    ref = stack.x_out.clone()
    cache = str(tmp_path / "tune.json")
    rep = stack.autotune(tile_caps=(128, 64, 32), reps=2, cache_file=cache)
    assert not rep["cached"] and rep["tile_edges"] in (128, 64, 32)
    assert len(rep["candidates"]) == 3
    kinds = {c[0] for c in rep["candidates"][0]["fwd_choices"]}
    assert kinds == {B.GNN_EDGE_FWD_RT, B.GNN_EDGE_FWD_WS, B.GNN_EDGE_FWD_ONE}
    assert G.tile_edges == rep["tile_edges"] and part.tile_edges == rep["tile_edges"]
    stack.forward()
    torch.cuda.synchronize()
    # the tuned launch choice may differ from the default one: launch choices agree to FP32
    # rounding except where a last-bit difference flips a BF16 rounding of an activation or of
    # the edge state (about 1e-4 per layer, see test_edge_forward_kernel_choices_agree), and
    # such flips carry into the next layer
    assert rel_l2(stack.x_out.cpu().numpy(), ref.cpu().numpy()) < 1e-3
    gnn._TUNED.clear()
    rep2 = stack.autotune(tile_caps=(128, 64, 32), reps=2, cache_file=cache)
    assert rep2["cached"] and rep2["tile_edges"] == rep["tile_edges"]
