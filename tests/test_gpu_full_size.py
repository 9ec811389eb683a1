"""The benchmarked training step at full size against the FP64 oracle on
sampled nodes (needs a GB300).

The graph, partition, model and launch configuration are the benchmark's: the
16^3-element p=5 GLL brick (531,441 nodes, 3,149,280 directed edges) in 8 RCB
sub-graphs, four consistent layers of width 64 with 2 MLP hidden layers, BF16
fused path recomputing the MLP activations in the backward (and, as the
option, keeping them from the forward). The
inputs are seeded: a state per global node and per directed global edge (so the
copies of a node or edge agree) and an upstream gradient per row. One step runs
on the GPU; the oracle evaluates the same four layers on the ball of 2M + 1 = 9
hops around each sampled node, which gives that node's values exactly (the
sampling is checked on the CPU in test_oracle_ball.py). Compared: x_4 on every
copy of a sampled node, e_4 on every copy of its in-edges, and dL/dx_0, dL/de_0
summed over the copies; relative L2 over the sample, BF16 tolerances (outputs
2e-2, gradients 5e-2). The sample holds nodes with 1, 2, 4 and 8 copies."""
import numpy as np
import pytest
import torch

import bench
import synthetic as syn
from oracle import graph as og
from paper_2410_01657_gb300 import _build
from paper_2410_01657_gb300 import binding as B
from paper_2410_01657_gb300 import nn as gnn

from ball_util import check_sample, neighbour_csr
from gpu_util import rel_l2

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    B.load()


class _Rows:
    """Rows of a host tensor as float64 numpy, indexed on demand."""

    def __init__(self, t):
        self.t = t

    def __getitem__(self, idx):
        return self.t[torch.as_tensor(np.asarray(idx, dtype=np.int64))].double().numpy()


def _sample_ids(L: int, rng) -> list:
    m = L // 2
    lid = lambda i, j, k: i + L * (j + L * k)
    fixed = [lid(m, m, m), lid(m, m, 10), lid(m, 10, 10), lid(0, 0, 0), lid(L - 1, m, 20), lid(3, L - 1, m)]
    return fixed + [int(v) for v in rng.choice(L ** 3, 6, replace=False)]


def _compare(params, b, samples, ed_rows, gid, ekey, node_deg, x0g, e0g, dx_glob, xM, eM, dx0, de0):
    """(got, ref) of x_M, e_M, dL/dx_0, dL/de_0 over the sampled nodes; eM and
    de0 hold the rows of ed_rows (concatenated), xM and dx0 every row."""
    N = b.n_nodes
    ptr, nbr = neighbour_csr(N, b.recv, b.send)
    got = {k: [] for k in ("x", "e", "dx", "de")}
    ref = {k: [] for k in ("x", "e", "dx", "de")}
    o = 0
    for k, rows_e in zip(samples, ed_rows):
        s = check_sample(params["layers"], N, b.recv, b.send, ptr, nbr, k, x0g, e0g, dx_glob)
        rows = np.nonzero(gid == k)[0]
        assert rows.size == node_deg[rows[0]]
        for r in rows:
            got["x"].append(xM[r])
            ref["x"].append(s["x"])
        got["dx"].append(dx0[rows].sum(axis=0))
        ref["dx"].append(s["dx"])
        pos = np.searchsorted(s["eid"], ekey[rows_e])
        assert np.array_equal(s["eid"][pos], ekey[rows_e]) and np.unique(pos).size == s["eid"].size
        n = rows_e.size
        got["e"].append(eM[o:o + n])
        ref["e"].append(s["e"][pos])
        de_sum = np.zeros_like(s["de"])
        np.add.at(de_sum, pos, de0[o:o + n])
        got["de"].append(de_sum)
        ref["de"].append(s["de"])
        o += n
    assert o == eM.shape[0]
    return {k: (np.vstack(got[k]), np.vstack(ref[k])) for k in got}


@pytest.mark.parametrize("save_act", [False, True])
def test_c2_training_step_sampled_vs_oracle(save_act):
    wl = bench.WORKLOADS["c2"]
    H, M, NH = wl["H"], bench.M, bench.NH
    part, nel, N, E = bench.workload_graph(wl, None)
    b = og.build_brick((nel,) * 3, wl["p"])
    assert (b.n_nodes, b.n_edges) == (N, E) == (531_441, 3_149_280)
    gid = part.array("row_gid")
    recv_gid = gid[part.receivers()]
    ekey = np.searchsorted(b.recv * N + b.send, recv_gid * N + gid[part.array("col")])
    node_deg = part.array("node_deg")

    rng = np.random.default_rng(11)
    x0g = rng.standard_normal((N, H)).astype(np.float32)
    e0g = torch.from_numpy(rng.standard_normal((E, H), dtype=np.float32)).to(torch.bfloat16)
    dx_rows = rng.standard_normal((part.n_rows, H), dtype=np.float32)
    dx_glob = torch.zeros(N, H, dtype=torch.float64).index_add_(
        0, torch.from_numpy(gid), torch.from_numpy(dx_rows).double()).numpy()

    # the GPU step, as the benchmark runs it
    G = part.to_device(DEV)
    params = syn.gnn_params(bench.SEED, H, NH, M)
    net = gnn.ConsistentGNN(params, precision="bf16", device=DEV)
    layers = [(l.edge.tensors(), l.node.tensors(), l.edge.dims, l.node.dims) for l in net.layers]
    x0 = torch.from_numpy(x0g[gid]).to(DEV)
    e0 = e0g.to(DEV)[torch.from_numpy(ekey).to(DEV)]
    stack = gnn.LayerStack(G, layers, H, "bf16", x0, e0, save_act=save_act)
    assert all((a is not None) == save_act for a in stack.act)
    stack.step(torch.from_numpy(dx_rows).to(DEV))
    torch.cuda.synchronize()
    B.call("gnn_check", None)

    samples = _sample_ids(nel * wl["p"] + 1, np.random.default_rng(12))
    assert {1, 2, 4, 8} <= {int(node_deg[gid == k][0]) for k in samples}
    ed_rows = [np.nonzero(recv_gid == k)[0] for k in samples]
    idx = torch.from_numpy(np.concatenate(ed_rows)).to(DEV)
    eM = stack.e[M][idx].float().cpu().numpy().astype(np.float64)
    de0 = stack.de[0][idx].float().cpu().numpy().astype(np.float64)
    xM = stack.x[M].cpu().numpy().astype(np.float64)
    dx0 = stack.dx[0].cpu().numpy().astype(np.float64)

    pairs = _compare(params, b, samples, ed_rows, gid, ekey, node_deg, x0g.astype(np.float64), _Rows(e0g),
                     dx_glob, xM, eM, dx0, de0)
    err = {k: rel_l2(g, r) for k, (g, r) in pairs.items()}
    print(f"\nC2 full size (saved activations: {save_act}), sampled rel-L2:",
          {k: f"{v:.2e}" for k, v in err.items()})
    assert err["x"] < 2e-2 and err["e"] < 2e-2, err
    assert err["dx"] < 5e-2 and err["de"] < 5e-2, err


def test_mixed_mesh_training_step_sampled_vs_oracle():
    # the benchmark's mixed-element mesh (64^3 cells, hexahedra and Kuhn
    # tetrahedra, 8 fan cells on one apex of in-degree 4,225 held as co-resident
    # copy rows), 8 RCB parts, the same stack; the apex is checked forward (its
    # M-hop ball), three nodes at least 2M + 2 hops below the fans forward and
    # backward
    wl = bench.WORKLOADS["mixed"]
    H, M, NH = wl["H"], bench.M, bench.NH
    part, n, N, E = bench.workload_graph(wl, None)
    m = syn.mixed_element_mesh(n, bench.SEED, n_fans=8)
    mesh = og.element_mesh(m["pos"], m["elem_ptr"], m["elem_nodes"], m["edge_ptr"], m["edge_pairs"])
    assert (mesh.n_nodes, mesh.n_edges) == (N, E)
    gid = part.array("row_gid")
    recv_gid = gid[part.receivers()]
    ekey = np.searchsorted(mesh.recv * N + mesh.send, recv_gid * N + gid[part.array("col")])
    node_deg = part.array("node_deg")
    hub = N - 1
    assert int((recv_gid == hub).sum()) >= 4225 and int((gid == hub).sum()) > 1

    rng = np.random.default_rng(13)
    x0g = rng.standard_normal((N, H)).astype(np.float32)
    e0g = torch.from_numpy(rng.standard_normal((E, H), dtype=np.float32)).to(torch.bfloat16)
    dx_rows = rng.standard_normal((part.n_rows, H), dtype=np.float32)
    dx_glob = torch.zeros(N, H, dtype=torch.float64).index_add_(
        0, torch.from_numpy(gid), torch.from_numpy(dx_rows).double()).numpy()

    G = part.to_device(DEV)
    params = syn.gnn_params(bench.SEED, H, NH, M)
    net = gnn.ConsistentGNN(params, precision="bf16", device=DEV)
    layers = [(l.edge.tensors(), l.node.tensors(), l.edge.dims, l.node.dims) for l in net.layers]
    stack = gnn.LayerStack(G, layers, H, "bf16", torch.from_numpy(x0g[gid]).to(DEV),
                           e0g.to(DEV)[torch.from_numpy(ekey).to(DEV)])
    stack.step(torch.from_numpy(dx_rows).to(DEV))
    torch.cuda.synchronize()
    B.call("gnn_check", None)

    q = n + 1
    low = np.random.default_rng(14).choice(q * q * (n - 2 * M - 1), 2, replace=False)
    samples = [q // 2 + q * (q // 2 + q * (q // 2))] + [int(v) for v in low]
    ed_rows = [np.nonzero(recv_gid == k)[0] for k in samples]
    idx = torch.from_numpy(np.concatenate(ed_rows)).to(DEV)
    x0d = x0g.astype(np.float64)
    pairs = _compare(params, mesh, samples, ed_rows, gid, ekey, node_deg, x0d, _Rows(e0g), dx_glob,
                     stack.x[M].cpu().numpy().astype(np.float64),
                     stack.e[M][idx].float().cpu().numpy().astype(np.float64),
                     stack.dx[0].cpu().numpy().astype(np.float64),
                     stack.de[0][idx].float().cpu().numpy().astype(np.float64))
    err = {k: rel_l2(g, r) for k, (g, r) in pairs.items()}

    # the apex: every copy row's x_M, every in-edge's e_M
    s = check_sample(params["layers"], N, mesh.recv, mesh.send, *neighbour_csr(N, mesh.recv, mesh.send), hub,
                     x0d, _Rows(e0g), dx_glob, grads=False)
    rows, rows_e = np.nonzero(gid == hub)[0], np.nonzero(recv_gid == hub)[0]
    assert rows.size == node_deg[rows[0]]
    pos = np.searchsorted(s["eid"], ekey[rows_e])
    assert np.array_equal(s["eid"][pos], ekey[rows_e]) and np.unique(pos).size == s["eid"].size == 4225
    eh = stack.e[M][torch.from_numpy(rows_e).to(DEV)].float().cpu().numpy().astype(np.float64)
    err["x_apex"] = rel_l2(stack.x[M][torch.from_numpy(rows).to(DEV)].cpu().numpy(), np.tile(s["x"], (rows.size, 1)))
    err["e_apex"] = rel_l2(eh, s["e"][pos])
    print("\nmixed mesh full size, sampled rel-L2:", {k: f"{v:.2e}" for k, v in err.items()})
    assert max(err["x"], err["e"], err["x_apex"], err["e_apex"]) < 2e-2, err
    assert err["dx"] < 5e-2 and err["de"] < 5e-2, err


# ------------------------------------------------------------------ C3, C4, C5 at full size
#
# These graphs are too large for the host oracle as a whole, so the inputs are
# counter-hashed (regenerated on the device for every row and on the host for
# the rows of a ball) and each sampled node's ball is taken inside a small
# window brick of the same order (tests/fullsize_util.py). The step runs in the
# benchmark's launch form: C3 4 layers at H = 128 fwd+bwd (layered H = 128
# adjoint, recomputing the MLP activations), C4 64 uneven sub-graphs at H = 64
# fwd+bwd replayed as a CUDA graph, C5 the 4-layer H = 32 inference stack whose
# last layer writes no edge state.

def _rows_index(gid):
    order = np.argsort(gid, kind="stable")
    return order, gid[order]


def _fullsize_step(name, grads, use_graph):
    import fullsize_util as fu

    wl = bench.WORKLOADS[name]
    H, M, NH, p = wl["H"], bench.M, wl.get("nh", bench.NH), wl["p"]
    part, nel, N, E = bench.workload_graph(wl, None)
    assert N == (nel * p + 1) ** 3
    G = part.to_device(DEV)
    params = syn.gnn_params(bench.SEED, H, NH, M)
    net = gnn.ConsistentGNN(params, precision="bf16", device=DEV)
    layers = [(l.edge.tensors(), l.node.tensors(), l.edge.dims, l.node.dims) for l in net.layers]
    x0, e0, dx = fu.device_inputs(part, H, N, DEV)
    stack = gnn.LayerStack(G, layers, H, "bf16", x0, e0, inference=not grads, save_act=False)
    del x0, e0
    if use_graph:
        stack.capture(dx if grads else None)
        stack.replay()
    else:
        stack.step(dx if grads else None)
    torch.cuda.synchronize()
    B.call("gnn_check", None)
    return wl, part, nel, N, params, stack


def _fullsize_compare(wl, part, nel, N, params, stack, samples, grads):
    import fullsize_util as fu

    H, M, p = wl["H"], bench.M, wl["p"]
    gid = part.array("row_gid").astype(np.int64)
    node_deg = part.array("node_deg")
    rp = part.array("row_ptr").astype(np.int64)
    col = part.array("col").astype(np.int64)
    order, sgid = _rows_index(gid)

    def dx_glob_of(g):   # the upstream gradient of a node: its rows' hashed rows, summed
        lo, hi = np.searchsorted(sgid, g, "left"), np.searchsorted(sgid, g, "right")
        out = np.zeros((g.size, H))
        for i in range(g.size):
            out[i] = fu.hashed_rows(order[lo[i]:hi[i]], H, fu.SEED_D, 16).sum(axis=0)
        return out

    got = {k: [] for k in ("x", "e", "dx", "de")}
    ref = {k: [] for k in ("x", "e", "dx", "de")}
    xM = stack.x_out
    eM = None if not grads else stack.e[M]
    for k in samples:
        rows = order[np.searchsorted(sgid, k, "left"):np.searchsorted(sgid, k, "right")]
        assert rows.size == node_deg[rows[0]]
        erows = np.concatenate([np.arange(rp[r], rp[r + 1]) for r in rows])
        keys = k * N + gid[col[erows]]
        w = fu.Window((nel,) * 3, p, k, 2 * M + 1 if grads else M)
        s = fu.oracle_at(params["layers"], w, H, dx_glob_of, grads=grads)
        ri = torch.from_numpy(rows).to(DEV)
        for xr in xM[ri].double().cpu().numpy():
            got["x"].append(xr)
            ref["x"].append(s["x"])
        if not grads:
            continue
        ei = torch.from_numpy(erows).to(DEV)
        pos = np.searchsorted(s["keys"], keys)
        assert np.array_equal(s["keys"][pos], keys) and np.unique(pos).size == s["keys"].size
        got["e"].append(eM[ei].double().cpu().numpy())
        ref["e"].append(s["e"][pos])
        got["dx"].append(stack.dx[0][ri].double().cpu().numpy().sum(axis=0, keepdims=True))
        ref["dx"].append(s["dx"][None])
        de_sum = np.zeros_like(s["de"])
        np.add.at(de_sum, pos, stack.de[0][ei].double().cpu().numpy())
        got["de"].append(de_sum)
        ref["de"].append(s["de"])
    return {k: rel_l2(np.vstack(got[k]), np.vstack(ref[k])) for k in got if got[k]}


def _lattice_samples(L, rng, extra=6):
    m = L // 2
    lid = lambda i, j, k: i + L * (j + L * k)
    fixed = [lid(m, m, m), lid(m, m, 10), lid(m, 10, 10), lid(0, 0, 0), lid(L - 1, m, 20), lid(3, L - 1, m)]
    return fixed + [int(v) for v in rng.choice(L ** 3, extra, replace=False)]


def test_c3_training_step_sampled_vs_oracle():
    wl, part, nel, N, params, stack = _fullsize_step("c3", grads=True, use_graph=True)
    node_deg, gid = part.array("node_deg"), part.array("row_gid")
    samples = _lattice_samples(nel * wl["p"] + 1, np.random.default_rng(31))
    assert {1, 2, 4, 8} <= {int(node_deg[gid == k][0]) for k in samples}
    err = _fullsize_compare(wl, part, nel, N, params, stack, samples, grads=True)
    print("\nC3 full size (32^3 p=7, H=128), sampled rel-L2:", {k: f"{v:.2e}" for k, v in err.items()})
    assert err["x"] < 2e-2 and err["e"] < 2e-2, err
    assert err["dx"] < 5e-2 and err["de"] < 5e-2, err


def test_c4_training_step_sampled_vs_oracle():
    wl, part, nel, N, params, stack = _fullsize_step("c4", grads=True, use_graph=True)
    node_deg, gid = part.array("node_deg"), part.array("row_gid")
    rng = np.random.default_rng(41)
    samples = []
    degs = np.unique(node_deg)
    assert degs[0] == 1 and degs.size >= 3
    for d in degs:   # nodes of every copy count the uneven cuts produce, drawn from the rows that have it
        cand = np.unique(gid[node_deg == d])
        samples += [int(v) for v in rng.choice(cand, min(2, cand.size), replace=False)]
    err = _fullsize_compare(wl, part, nel, N, params, stack, samples, grads=True)
    print("\nC4 full size (64 uneven parts), sampled rel-L2:", {k: f"{v:.2e}" for k, v in err.items()})
    assert err["x"] < 2e-2 and err["e"] < 2e-2, err
    assert err["dx"] < 5e-2 and err["de"] < 5e-2, err


def test_c5_inference_sampled_vs_oracle():
    wl, part, nel, N, params, stack = _fullsize_step("c5", grads=False, use_graph=True)
    samples = _lattice_samples(nel * wl["p"] + 1, np.random.default_rng(51))
    err = _fullsize_compare(wl, part, nel, N, params, stack, samples, grads=False)
    print("\nC5 full size (48^3 p=7, H=32, inference), sampled rel-L2:", {k: f"{v:.2e}" for k, v in err.items()})
    assert err["x"] < 2e-2, err
