"""The consistent NMP layer on a general element mesh (needs a GB300).

A mesh of mixed element types (hexahedra, Kuhn tetrahedra, fan cells) whose
apex node has in-degree 289 in the R=1 graph: the partition splits it into
co-resident copies of at most 128 in-edges each, and the Eq. 5c-5d copy-sum
carries their partial aggregates. Every output and gradient of one layer is
compared with the FP64 oracle's (which knows nothing of the split) on the
same inputs: edge rows directly (the library keeps the oracle's edge order),
node rows per (sub-graph, global id), input gradients summed over a node's
copies. Then a whole network step, partitioned against unpartitioned."""
import numpy as np
import pytest
import torch

import synthetic as syn
from paper_2410_01657_gb300 import _build
from paper_2410_01657_gb300 import binding as B
from paper_2410_01657_gb300 import nn as gnn

from elements_util import check_layer, layer_case, mixed_mesh16, partitions
from gpu_util import flat_grads, oracle_network, rel_l2
from test_gpu_precision_report import _run

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    B.load()


@pytest.fixture(scope="module")
def mesh16():
    return mixed_mesh16()


@pytest.mark.parametrize("H,R,how", [(16, 1, None), (32, 3, "fans"), (64, 3, "fans"), (64, 6, "rcb"),
                                     (128, 2, "fans")])
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_layer_on_mixed_elements_vs_oracle(mesh16, H, R, how, precision):
    m, mesh = mesh16
    part, subs = partitions(m, mesh, R, how)
    assert part.info.max_in_degree <= B.GNN_EDGE_TILE
    assert int((part.array("row_gid") == mesh.n_nodes - 1).sum()) >= 3
    case = layer_case(part, mesh, subs, H)
    G = part.to_device(DEV)
    out, grads = _run(G, case["params"], H, case["x"], case["e"], case["dx1"], case["de1"], precision)
    lo, lg = (1e-5, 1e-5) if precision == "fp32" else (2e-2, 5e-2)
    check_layer(part, subs, case, out, grads, lo, lg)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_network_step_on_mixed_elements(mesh16, precision):
    # encoders + 2 consistent layers + decoder + Eq. 8 loss; R = 1, 3 and 6
    m, mesh = mesh16
    H = 32
    params = syn.gnn_params(21, H, 2, 2, randomize_affine=True)
    modes = syn.fourier_modes(1, 8)
    u = syn.fourier_field(mesh.pos, modes)
    target = syn.fourier_field(mesh.pos, modes, phase_advance=0.1)
    tol_o, tol_g = (1e-5, 1e-5) if precision == "fp32" else (2e-2, 5e-2)
    losses = []
    for R, how in ((1, None), (3, "fans"), (6, "rcb")):
        part, subs = partitions(m, mesh, R, how)
        G = part.to_device(DEV)
        gid = part.array("row_gid")
        ys, L, g, _ = oracle_network(params, mesh, subs, u, target)
        net = gnn.ConsistentGNN(params, precision=precision, device=DEV)
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=DEV)
        y = net(G, t(u[gid]), G.edge_attr())
        loss = gnn.consistent_loss(y, t(target[gid]), G)
        loss.backward()
        B.call("gnn_check", None)
        yg = y.detach().cpu().numpy()
        ro = part.array("row_offsets")
        for r, sg in enumerate(subs):
            loc = np.searchsorted(sg.gid, gid[ro[r]:ro[r + 1]])
            assert rel_l2(yg[ro[r]:ro[r + 1]], ys[r][loc]) < tol_o
        assert abs(loss.item() - L) < tol_o * abs(L)
        gg = dict(flat_grads(net.grads_numpy()))
        for name, ref in flat_grads(g):
            assert rel_l2(gg[name], ref) < tol_g, (R, name, rel_l2(gg[name], ref))
        losses.append(loss.item())
    # Eq. 2: the loss does not depend on the partition
    assert max(losses) - min(losses) <= (1e-5 if precision == "fp32" else 5e-3) * abs(losses[0])
