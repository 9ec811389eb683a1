"""The paper's consistency property on the GPU path (Sec. II-B, Eq. 2; the
setting of Fig. 5 in Sec. III-A: a 32^3-element p=1 brick, R = 1 .. 64).

A network of consistent NMP layers gives the same loss for every number of
sub-graphs R; the same network with the halo swap + sync skipped (the paper's
"None" layers) does not, and its error grows as the sub-graphs get smaller.
Training (Adam, target = input, 150 steps) with consistent layers follows the
same loss curve for R = 1 and R = 8; with "None" layers the curves part. Run
with ``-s`` to print the loss table and the curves."""
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
RS = (1, 2, 4, 8, 16, 32, 64)
NEL = (32, 32, 32)


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    B.load()


def _loss(R, precision, halo, H=16):
    graph = MeshGraph(NEL, 1)
    part = graph.partition(R, "rcb")
    G = part.to_device(DEV)
    params = syn.gnn_params(11, H, 2, 4)
    modes = syn.fourier_modes(11, 8)
    pos = part.array("row_pos")
    u = torch.tensor(syn.fourier_field(pos, modes), dtype=torch.float32, device=DEV)
    t = torch.tensor(syn.fourier_field(pos, modes, phase_advance=0.1), dtype=torch.float32, device=DEV)
    net = gnn.ConsistentGNN(params, precision=precision, halo=halo, device=DEV)
    with torch.no_grad():
        y = net(G, u, G.edge_attr())
        loss = gnn.consistent_loss(y, t, G)
    B.call("gnn_check", None)
    return float(loss.item())


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("bf16", 2e-3)])
def test_consistent_loss_is_independent_of_R(precision, tol):
    ref = _loss(1, precision, True)
    rows = [(1, ref, ref)]
    for R in RS[1:]:
        lc, ln = _loss(R, precision, True), _loss(R, precision, False)
        rows.append((R, lc, ln))
        assert abs(lc - ref) <= tol * abs(ref), R
    print(f"\n{precision}: loss vs R on the 32^3 p=1 brick (consistent | None layers)")
    for R, lc, ln in rows:
        print(f"  R={R:3d}  {lc:.8f} ({(lc - ref) / ref:+.1e})  |  {ln:.8f} ({(ln - ref) / ref:+.1e})")


def test_inconsistent_layers_drift_with_R():
    ref = _loss(1, "fp32", False)
    dev = [abs(_loss(R, "fp32", False) - ref) / abs(ref) for R in RS[1:]]
    assert min(dev) > 1e-4                 # every partition changes the result
    assert dev[-1] > 3 * dev[0]             # and more sub-graphs change it more
    assert dev[-1] > dev[2]                 # 64 sub-graphs drift further than 8


def _train(R, precision, halo, steps=150, H=16, lr=2e-3):
    # the paper's training comparison (target = input): Adam on the consistent loss
    graph = MeshGraph(NEL, 1)
    part = graph.partition(R, "rcb")
    G = part.to_device(DEV)
    params = syn.gnn_params(13, H, 2, 2)
    modes = syn.fourier_modes(13, 8)
    u = torch.tensor(syn.fourier_field(part.array("row_pos"), modes), dtype=torch.float32, device=DEV)
    net = gnn.ConsistentGNN(params, precision=precision, halo=halo, device=DEV)
    opt = torch.optim.Adam(net.parameters(), lr=lr)
    attr = G.edge_attr()
    curve = []
    for _ in range(steps):
        opt.zero_grad(set_to_none=True)
        loss = gnn.consistent_loss(net(G, u, attr), u, G)
        loss.backward()
        opt.step()
        curve.append(float(loss.item()))
    B.call("gnn_check", None)
    return np.array(curve)


def _print_curves(title, curves):
    print(f"\n{title}")
    steps = [0, 1, 2, 5, 10, 20, 50, 100, 149]
    print("  step " + " ".join(f"{k:>11s}" for k in curves))
    for i in steps:
        print(f"  {i:4d} " + " ".join(f"{c[i]:11.6f}" for c in curves.values()))


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_training_curve_is_independent_of_R(precision):
    # consistent layers: the R = 8 run follows the R = 1 run step by step (the
    # partitioned loss and its gradient equal the single-graph ones); over 150
    # Adam steps the two runs differ only by the rounding of their sums. In BF16
    # those rounding differences are larger and Adam carries them along, so late
    # in training, where the loss is small and noisy, single steps can part by a
    # few per cent; the whole curve still stays far closer than the "None" run's.
    c1, c8 = _train(1, precision, True), _train(8, precision, True)
    n8 = _train(8, precision, False)
    _print_curves(f"{precision}: training loss, consistent R=1 / R=8 and None R=8",
                  {"R=1": c1, "R=8": c8, "None R=8": n8})
    assert c1[-1] < 0.2 * c1[0]                       # it trains
    dev_c = np.abs(c8 - c1) / np.abs(c1)
    dev_n = np.abs(n8 - c1) / np.abs(c1)
    if precision == "fp32":
        assert np.max(dev_c) < 1e-3
        assert np.max(dev_n) > 10 * np.max(dev_c)
    else:
        assert np.max(dev_c[:100]) < 2e-2 and np.median(dev_c) < 5e-3
        assert np.median(dev_n) > 5 * np.median(dev_c)


def test_inconsistent_training_curve_departs():
    c1, c8 = _train(1, "fp32", False), _train(8, "fp32", False)
    assert np.max(np.abs(c8 - c1) / np.abs(c1)) > 1e-3
