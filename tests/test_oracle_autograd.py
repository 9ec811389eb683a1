"""The oracle's hand-written adjoint of the partitioned consistent layer (Eq. 3)
against torch float64 autograd of the same layer written with library routines
(CPU only).

The torch version is written here from Eq. 5a-5e independently of
``oracle.model``: torch.nn modules for the MLPs, index_select for the edge
gather, index_add for the 1/d-weighted aggregation (Eq. 5b) and for the halo
swap + sync (Eq. 5c-5d, the copies of a global id summed over the ranks that
hold it). Only the reduced sub-graphs (oracle.graph) are shared. Autograd then
gives dL/dx, dL/de and every parameter gradient for a random linear functional
L of the outputs, which the oracle's layer_backward must reproduce."""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import graph, model

from test_oracle_model import _torch_mlp


def _torch_layer(layer, subs, n_global, xs, es):
    """Eq. 5a-5e on every rank with torch ops; returns (x', e') per rank."""
    edge_mlp, node_mlp = _torch_mlp(layer["edge"]), _torch_mlp(layer["node"])
    H = xs[0].shape[1]
    a_loc = []
    e_new = []
    for r, sg in enumerate(subs):
        recv = torch.from_numpy(sg.recv)
        send = torch.from_numpy(sg.send)
        inp = torch.cat([xs[r].index_select(0, recv), xs[r].index_select(0, send), es[r]], dim=1)
        en = es[r] + edge_mlp(inp)                                        # Eq. 5a
        w = torch.from_numpy(1.0 / sg.edge_deg.astype(np.float64)).unsqueeze(1)
        a = torch.zeros(sg.n_local, H, dtype=torch.float64).index_add(0, recv, w * en)   # Eq. 5b
        e_new.append(en)
        a_loc.append(a)
    # Eq. 5c-5d: every copy of a global id gets the sum over the ranks holding it
    tot = torch.zeros(n_global, H, dtype=torch.float64)
    for r, sg in enumerate(subs):
        tot = tot.index_add(0, torch.from_numpy(sg.gid), a_loc[r])
    x_new = []
    for r, sg in enumerate(subs):
        a_star = tot.index_select(0, torch.from_numpy(sg.gid))
        x_new.append(xs[r] + node_mlp(torch.cat([a_star, xs[r]], dim=1)))   # Eq. 5e
    mods = (edge_mlp, node_mlp)
    return x_new, e_new, mods


def _grads_of(mod, P):
    lin = [m for m in mod if isinstance(m, torch.nn.Linear)]
    g = {"W": [m.weight.grad.numpy() for m in lin], "b": [m.bias.grad.numpy() for m in lin]}
    if "gamma" in P:
        ln = [m for m in mod if isinstance(m, torch.nn.LayerNorm)][0]
        g["gamma"], g["beta"] = ln.weight.grad.numpy(), ln.bias.grad.numpy()
    return g


@pytest.mark.parametrize("R,method", [(1, "rcb"), (3, "rcb"), (4, "slab")])
def test_layer_adjoint_matches_torch_autograd(R, method):
    H = 6
    brick = graph.build_brick((3, 2, 4), 2)
    part = graph.partition_slab_z(brick, R) if method == "slab" else graph.partition_rcb(brick, R)
    subs = graph.build_subgraphs(brick, part, R) if R > 1 else graph.unpartitioned(brick)
    params = syn.gnn_params(5, H, 2, 1, randomize_affine=True)
    layer = params["layers"][0]
    rng = np.random.default_rng(6)
    xg = rng.standard_normal((brick.n_nodes, H))
    xs_np = [xg[sg.gid] for sg in subs]
    es_np = [rng.standard_normal((sg.n_edges, H)) for sg in subs]
    # the oracle, forward and hand-written adjoint
    x1, e1, cache = model.layer_forward(layer, subs, xs_np, es_np)
    dx1 = [rng.standard_normal(a.shape) for a in x1]
    de1 = [rng.standard_normal(a.shape) for a in e1]
    dx, de, g = model.layer_backward(layer, subs, cache, dx1, de1)
    # torch autograd of L = sum <dx1, x'> + <de1, e'>
    xs = [torch.tensor(a, requires_grad=True) for a in xs_np]
    es = [torch.tensor(a, requires_grad=True) for a in es_np]
    tx, te, (edge_mod, node_mod) = _torch_layer(layer, subs, brick.n_nodes, xs, es)
    for r in range(len(subs)):
        np.testing.assert_allclose(tx[r].detach().numpy(), x1[r], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(te[r].detach().numpy(), e1[r], rtol=1e-12, atol=1e-12)
    L = sum((tx[r] * torch.from_numpy(dx1[r])).sum() + (te[r] * torch.from_numpy(de1[r])).sum()
            for r in range(len(subs)))
    L.backward()
    for r in range(len(subs)):
        np.testing.assert_allclose(dx[r], xs[r].grad.numpy(), rtol=1e-10, atol=1e-11)
        np.testing.assert_allclose(de[r], es[r].grad.numpy(), rtol=1e-10, atol=1e-11)
    for which, mod in (("edge", edge_mod), ("node", node_mod)):
        tg = _grads_of(mod, layer[which])
        for key in tg:
            for a, b in zip(g[which][key] if isinstance(g[which][key], list) else [g[which][key]],
                            tg[key] if isinstance(tg[key], list) else [tg[key]]):
                np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-11)
