"""Pins of the oracle's MLP, consistent NMP layer, network, loss and adjoint (CPU only).

Pins used: torch.nn reference modules (library routines) for the MLP block and
its gradient; closed-form special cases (zero weights, H=1, constant messages
whose aggregate is the lattice in-degree); a brute-force per-node loop over the
unpartitioned definition on a tiny graph; permutation equivariance; the
consistency property Eq. 2 / Eq. 3 (R-way == R=1); and central finite
differences of the whole network loss; Table 1's parameter counts pin the
MLP layout (tests/golden/table1_param_counts.json)."""
import json
import os

import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import graph, model

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _torch_mlp(P):
    layers = []
    n = len(P["W"])
    for k in range(n):
        lin = torch.nn.Linear(P["W"][k].shape[1], P["W"][k].shape[0]).double()
        with torch.no_grad():
            lin.weight.copy_(torch.from_numpy(P["W"][k]))
            lin.bias.copy_(torch.from_numpy(P["b"][k]))
        layers.append(lin)
        if k < n - 1:
            layers.append(torch.nn.ELU())
    if "gamma" in P:
        ln = torch.nn.LayerNorm(P["W"][-1].shape[0], eps=model.LN_EPS).double()
        with torch.no_grad():
            ln.weight.copy_(torch.from_numpy(P["gamma"]))
            ln.bias.copy_(torch.from_numpy(P["beta"]))
        layers.append(ln)
    return torch.nn.Sequential(*layers)


@pytest.mark.parametrize("dims,ln", [([12, 8, 8, 8, 8], True), ([4, 16, 16], True),
                                     ([8, 8, 8, 8, 3], False), ([6, 5, 5, 5, 5, 5, 5, 5], True)])
def test_mlp_matches_torch_modules(dims, ln):
    rng = np.random.default_rng(0)
    P = syn.xavier_mlp(rng, dims, ln, randomize_affine=True)
    X = rng.standard_normal((37, dims[0])) * 2
    Y, cache = model.mlp_forward(P, X)
    tm = _torch_mlp(P)
    Xt = torch.from_numpy(X).requires_grad_(True)
    Yt = tm(Xt)
    np.testing.assert_allclose(Y, Yt.detach().numpy(), rtol=1e-12, atol=1e-12)
    dY = rng.standard_normal(Y.shape)
    dX, g = model.mlp_backward(P, cache, dY)
    Yt.backward(torch.from_numpy(dY))
    np.testing.assert_allclose(dX, Xt.grad.numpy(), rtol=1e-10, atol=1e-12)
    lins = [m for m in tm if isinstance(m, torch.nn.Linear)]
    for k, lin in enumerate(lins):
        np.testing.assert_allclose(g["W"][k], lin.weight.grad.numpy(), rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(g["b"][k], lin.bias.grad.numpy(), rtol=1e-10, atol=1e-12)
    if ln:
        np.testing.assert_allclose(g["gamma"], tm[-1].weight.grad.numpy(), rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(g["beta"], tm[-1].bias.grad.numpy(), rtol=1e-10, atol=1e-12)


def test_mlp_special_cases():
    rng = np.random.default_rng(1)
    P = syn.xavier_mlp(rng, [6, 4, 4, 4], True, randomize_affine=True)
    X = rng.standard_normal((9, 6))
    # all weights and biases zero: the LayerNorm sees a constant row -> beta
    Z = {"W": [0 * w for w in P["W"]], "b": [0 * b for b in P["b"]],
         "gamma": P["gamma"], "beta": P["beta"]}
    Y, _ = model.mlp_forward(Z, X)
    np.testing.assert_allclose(Y, np.broadcast_to(P["beta"], Y.shape), atol=0)
    # H = 1: LayerNorm of a single feature is beta whatever the input
    P1 = syn.xavier_mlp(rng, [6, 3, 1], True, randomize_affine=True)
    Y1, _ = model.mlp_forward(P1, X)
    np.testing.assert_allclose(Y1, np.broadcast_to(P1["beta"], Y1.shape), atol=0)
    # ELU: identity above 0, e^z - 1 below
    z = np.array([-3.0, -1e-3, 0.0, 2.5])
    np.testing.assert_allclose(model.elu(z), [np.exp(-3) - 1, np.exp(-1e-3) - 1, 0.0, 2.5], rtol=1e-12)


def _array_sizes(tree):
    if isinstance(tree, np.ndarray):
        return tree.size
    if isinstance(tree, dict):
        return sum(_array_sizes(v) for v in tree.values())
    return sum(_array_sizes(v) for v in tree)


def test_table1_parameter_counts():
    # Table 1: 3 node inputs, 3 outputs; (H, layers, MLP hidden layers) -> trainable parameters
    g = json.load(open(os.path.join(GOLD, "table1_param_counts.json")))
    for key in ("small", "large"):
        c = g[key]
        p = syn.gnn_params(0, c["hidden"], c["mlp_hidden_layers"], c["n_layers"])
        assert _array_sizes(p) == c["params"], key
        assert model.network_param_count(p) == c["params"], key
        # the counts single out this layout among the plausible readings
        for kw in ({"f_e": 7}, {"f_e": 3}):   # the text's 7 edge inputs; positions alone
            assert model.network_param_count(
                syn.gnn_params(0, c["hidden"], c["mlp_hidden_layers"], c["n_layers"], **kw)) != c["params"]
        for n_h in (c["mlp_hidden_layers"] - 1, c["mlp_hidden_layers"] + 1):   # Linears counted differently
            assert model.network_param_count(syn.gnn_params(0, c["hidden"], n_h, c["n_layers"])) != c["params"]


def _constant_message_layer(rng, H, c):
    """Edge MLP with zero weights -> message = beta_E = c for every edge."""
    layer = {"edge": syn.xavier_mlp(rng, syn.mlp_dims(3 * H, H, 2, H), True, True),
             "node": syn.xavier_mlp(rng, syn.mlp_dims(2 * H, H, 2, H), True, True)}
    E = layer["edge"]
    E["W"] = [0 * w for w in E["W"]]
    E["b"] = [0 * b for b in E["b"]]
    E["beta"] = c.copy()
    return layer


@pytest.mark.parametrize("R,method,weights", [(1, "slab", None), (2, "slab", None),
                                              (5, "rcb", [1, 3, 2, 7, 1]), (8, "rcb", None)])
def test_aggregate_is_lattice_degree(R, method, weights):
    # With e_in = 0 and constant messages c, Eq. 5b-5d give a*_i = indeg(i) * c
    # on every copy of node i; "None" mode leaves boundary copies short.
    rng = np.random.default_rng(2)
    H = 5
    c = np.array([1.0, -2.0, 0.5, 3.0, 0.25])
    b = graph.build_brick((4, 3, 4), 2)
    part = graph.partition_slab_z(b, R) if method == "slab" else graph.partition_rcb(b, R, weights)
    subs = graph.build_subgraphs(b, part, R) if R > 1 else graph.unpartitioned(b)
    layer = _constant_message_layer(rng, H, c)
    xs = [rng.standard_normal((sg.n_local, H)) for sg in subs]
    es = [np.zeros((sg.n_edges, H)) for sg in subs]
    indeg = np.bincount(b.recv, minlength=b.n_nodes)
    _, e_new, cache = model.layer_forward(layer, subs, xs, es)
    for r, sg in enumerate(subs):
        np.testing.assert_allclose(e_new[r], np.broadcast_to(c, e_new[r].shape), atol=0)
        np.testing.assert_allclose(cache["a_star"][r], indeg[sg.gid][:, None] * c, rtol=1e-14)
    if R > 1:
        _, _, cache_none = model.layer_forward(layer, subs, xs, es, halo=False)
        short = 0
        for r, sg in enumerate(subs):
            got = cache_none["a_star"][r][:, 0]
            full = indeg[sg.gid] * c[0]
            assert np.all(np.abs(got) <= np.abs(full) + 1e-12)
            short += int((np.abs(got - full) > 1e-9).sum())
        assert short > 0


def _brute_force_layer(layer, b, x_glob, e_glob):
    """Unpartitioned Eq. 5a-5e by explicit loops over global ids (torch.nn MLPs)."""
    mE, mN = _torch_mlp(layer["edge"]), _torch_mlp(layer["node"])
    N, H = x_glob.shape
    e_new = {}
    for (i, j), e in e_glob.items():
        inp = torch.from_numpy(np.concatenate([x_glob[i], x_glob[j], e])[None])
        e_new[(i, j)] = e + mE(inp).detach().numpy()[0]
    x_new = np.zeros_like(x_glob)
    for i in range(N):
        a = np.zeros(H)
        for (r, s), e in e_new.items():
            if r == i:
                a += e
        inp = torch.from_numpy(np.concatenate([a, x_glob[i]])[None])
        x_new[i] = x_glob[i] + mN(inp).detach().numpy()[0]
    return x_new, e_new


@pytest.mark.parametrize("R", [1, 2])
def test_layer_matches_brute_force_loops(R):
    rng = np.random.default_rng(3)
    H = 4
    b = graph.build_brick((2, 1, 1), 1, extent=(2.0, 1.0, 1.0))
    layer = {"edge": syn.xavier_mlp(rng, syn.mlp_dims(3 * H, H, 2, H), True, True),
             "node": syn.xavier_mlp(rng, syn.mlp_dims(2 * H, H, 2, H), True, True)}
    x_glob = rng.standard_normal((b.n_nodes, H))
    e_glob = {(int(i), int(j)): rng.standard_normal(H) for i, j in zip(b.recv, b.send)}
    xb, eb = _brute_force_layer(layer, b, x_glob, e_glob)
    subs = graph.unpartitioned(b) if R == 1 else graph.build_subgraphs(b, graph.partition_rcb(b, R), R)
    xs = [x_glob[sg.gid] for sg in subs]
    es = [np.stack([e_glob[(int(sg.gid[i]), int(sg.gid[j]))] for i, j in zip(sg.recv, sg.send)])
          for sg in subs]
    x_new, e_new, _ = model.layer_forward(layer, subs, xs, es)
    for r, sg in enumerate(subs):
        np.testing.assert_allclose(x_new[r], xb[sg.gid], rtol=1e-12, atol=1e-12)
        for k, (i, j) in enumerate(zip(sg.recv, sg.send)):
            np.testing.assert_allclose(e_new[r][k], eb[(int(sg.gid[i]), int(sg.gid[j]))],
                                       rtol=1e-12, atol=1e-12)


def _relabelled(b, perm):
    """Unpartitioned graph with node row perm[g] for global id g, edges shuffled."""
    rng = np.random.default_rng(9)
    order = rng.permutation(b.n_edges)
    return graph.SubGraph(gid=np.argsort(perm), recv=perm[b.recv][order], send=perm[b.send][order],
                          edge_deg=np.ones(b.n_edges, np.int64),
                          node_deg=np.ones(b.n_nodes, np.int64)), order


def test_permutation_equivariance():
    rng = np.random.default_rng(4)
    b = graph.build_brick((2, 2, 2), 2)
    p = syn.gnn_params(5, 6, 2, 2, randomize_affine=True)
    u = rng.standard_normal((b.n_nodes, 3))
    sub = graph.unpartitioned(b)[0]
    y, _ = model.network_forward(p, [sub], [u], [graph.edge_attributes(b.pos, sub)])
    perm = rng.permutation(b.n_nodes)
    sp_, order = _relabelled(b, perm)
    up = np.empty_like(u)
    up[perm] = u
    attr = graph.edge_attributes(b.pos, sub)[order]
    yp, _ = model.network_forward(p, [sp_], [up], [attr])
    np.testing.assert_allclose(yp[0][perm], y[0], rtol=1e-12, atol=1e-12)


def _run_network(b, subs, p, u, halo=True):
    us = [u[sg.gid] for sg in subs]
    attr = [graph.edge_attributes(b.pos, sg) for sg in subs]
    target = [np.cos(us[r]) for r in range(len(subs))]
    ys, cache = model.network_forward(p, subs, us, attr, halo)
    L = model.consistent_loss(subs, ys, target)
    g = model.network_backward(p, subs, cache, model.consistent_loss_grad(subs, ys, target), halo)
    return model.to_global(subs, ys, b.n_nodes), L, g


def _flat(g):
    parts = []
    for key in ("enc_node", "enc_edge", "dec"):
        parts += [*g[key]["W"], *g[key]["b"]] + ([g[key]["gamma"], g[key]["beta"]] if "gamma" in g[key] else [])
    for layer in g["layers"]:
        for key in ("edge", "node"):
            parts += [*layer[key]["W"], *layer[key]["b"], layer[key]["gamma"], layer[key]["beta"]]
    return np.concatenate([x.ravel() for x in parts])


@pytest.mark.parametrize("R", [1, 3, 8])
def test_consistent_loss_is_the_global_mse(R):
    # Eq. 8: with every copy holding its node's value, the 1/d_i weights and
    # N_eff = sum 1/d_i turn the per-rank sums into the plain mean squared
    # error over the unique nodes; the loss gradient summed over a node's
    # copies is 2 (y - t) / (N F)
    b = graph.build_brick((4, 3, 5), 2)
    subs = graph.build_subgraphs(b, graph.partition_rcb(b, R), R) if R > 1 else graph.unpartitioned(b)
    rng = np.random.default_rng(9)
    y, t = rng.standard_normal((b.n_nodes, 3)), rng.standard_normal((b.n_nodes, 3))
    ys, ts = [y[sg.gid] for sg in subs], [t[sg.gid] for sg in subs]
    assert abs(model.consistent_loss(subs, ys, ts) - np.mean((y - t) ** 2)) < 1e-14
    g = np.zeros_like(y)
    for sg, gr in zip(subs, model.consistent_loss_grad(subs, ys, ts)):
        np.add.at(g, sg.gid, gr)
    np.testing.assert_allclose(g, 2 * (y - t) / y.size, rtol=1e-12, atol=1e-15)
    if R > 1:   # the weights matter: without them, shared nodes count several times
        plain = sum(float(((a - c) ** 2).sum()) for a, c in zip(ys, ts)) / (sum(sg.n_local for sg in subs) * 3)
        assert abs(plain - np.mean((y - t) ** 2)) > 1e-6


@pytest.mark.parametrize("R,method,weights", [(2, "slab", None), (8, "rcb", None),
                                              (5, "rcb", [2, 1, 1, 3, 1])])
def test_consistency_eq2_eq3(R, method, weights):
    b = graph.build_brick((4, 4, 4), 2)
    rng = np.random.default_rng(6)
    u = syn.fourier_field(b.pos, syn.fourier_modes(0, 8))
    p = syn.gnn_params(7, 8, 2, 3, randomize_affine=True)
    y1, L1, g1 = _run_network(b, graph.unpartitioned(b), p, u)
    part = graph.partition_slab_z(b, R) if method == "slab" else graph.partition_rcb(b, R, weights)
    subs = graph.build_subgraphs(b, part, R)
    yR, LR, gR = _run_network(b, subs, p, u)
    assert np.abs(yR - y1).max() <= 1e-12 * np.abs(y1).max()
    assert abs(LR - L1) <= 1e-13 * abs(L1)
    f1, fR = _flat(g1), _flat(gR)
    assert np.abs(fR - f1).max() <= 1e-11 * np.abs(f1).max()
    # the paper's "None" mode breaks Eq. 2 on partitioned graphs
    yN, LN, _ = _run_network(b, subs, p, u, halo=False)
    assert np.abs(yN - y1).max() > 1e-4 * np.abs(y1).max()


def test_none_mode_deviation_grows_with_R():
    # Fig. 5 (left): without halo exchange the loss deviates from R=1 more as R grows
    b = graph.build_brick((8, 8, 8), 1)
    u = syn.fourier_field(b.pos, syn.fourier_modes(1, 8))
    p = syn.gnn_params(8, 8, 2, 4)
    _, L1, _ = _run_network(b, graph.unpartitioned(b), p, u)
    dev = []
    for R in (2, 8, 64):
        subs = graph.build_subgraphs(b, graph.partition_rcb(b, R), R)
        _, Lc, _ = _run_network(b, subs, p, u)
        _, Ln, _ = _run_network(b, subs, p, u, halo=False)
        assert abs(Lc - L1) <= 1e-12 * abs(L1)
        dev.append(abs(Ln - L1))
    assert dev[0] < dev[1] < dev[2]


def test_network_adjoint_vs_central_differences():
    b = graph.build_brick((2, 2, 2), 2)
    u = syn.fourier_field(b.pos, syn.fourier_modes(2, 4))
    p = syn.gnn_params(10, 5, 2, 2, randomize_affine=True)
    subs = graph.build_subgraphs(b, graph.partition_rcb(b, 3), 3)
    us = [u[sg.gid] for sg in subs]
    attr = [graph.edge_attributes(b.pos, sg) for sg in subs]
    target = [np.sin(x) for x in us]

    def loss():
        ys, _ = model.network_forward(p, subs, us, attr)
        return model.consistent_loss(subs, ys, target)

    ys, cache = model.network_forward(p, subs, us, attr)
    g = model.network_backward(p, subs, cache, model.consistent_loss_grad(subs, ys, target))
    rng = np.random.default_rng(11)
    arrays = []
    for key in ("enc_node", "enc_edge", "dec"):
        arrays += [(p[key]["W"], g[key]["W"]), (p[key]["b"], g[key]["b"])]
    for li, layer in enumerate(p["layers"]):
        for key in ("edge", "node"):
            arrays += [(layer[key]["W"], g["layers"][li][key]["W"]),
                       (layer[key]["b"], g["layers"][li][key]["b"]),
                       ([layer[key]["gamma"]], [g["layers"][li][key]["gamma"]]),
                       ([layer[key]["beta"]], [g["layers"][li][key]["beta"]])]
    h = 1e-6
    for trial in range(32):
        plist, glist = arrays[rng.integers(len(arrays))]
        k = rng.integers(len(plist))
        flat = plist[k].reshape(-1)
        idx = rng.integers(flat.size)
        old = flat[idx]
        flat[idx] = old + h
        lp = loss()
        flat[idx] = old - h
        lm = loss()
        flat[idx] = old
        fd = (lp - lm) / (2 * h)
        an = glist[k].reshape(-1)[idx]
        assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)) + 1e-9, (trial, fd, an)
