"""The numerators of the bench's roofline figures (CPU only).

FLOPs: counted here Linear by Linear over the MLP shapes of Eq. 5a and 5e
(2 * in * out per row of each Linear), then checked against the closed forms
per layer: edge 2H^2 (n_h + 2) with the first Linear split into per-row x_i / x_j
projections (4H^2 per row), 2H^2 (n_h + 4) unsplit, node 2H^2 (n_h + 3).
Bytes: the method's least traffic per step and the edge forward's designed
traffic, counted field by field."""
import types

import pytest

import bench


def _graph(E, N):
    return types.SimpleNamespace(n_edges=E, n_rows=N)


def _linear_chain(d_in, H, n_lin):
    dims = [d_in] + [H] * n_lin
    return sum(2 * dims[k] * dims[k + 1] for k in range(n_lin))


@pytest.mark.parametrize("H,n_h", [(16, 2), (32, 5), (64, 2), (128, 2), (64, 0)])
@pytest.mark.parametrize("fwd_only", [False, True])
def test_step_flops_by_linear_layers(H, n_h, fwd_only):
    E, N, layers = 3_149_280 + 12_345, 531_441 + 678, 4
    n_lin = n_h + 2
    G = _graph(E, N)
    edge_unsplit = _linear_chain(3 * H, H, n_lin)
    edge_split = edge_unsplit - 2 * (2 * H * H)       # the x_i, x_j blocks of the first Linear ...
    row = _linear_chain(2 * H, H, n_lin) + 2 * (2 * H * H)   # ... move to the rows, once each
    passes = 1 if fwd_only else 3
    assert edge_split == 2 * H * H * (n_h + 2) and edge_unsplit == 2 * H * H * (n_h + 4)
    assert row == 2 * H * H * (n_h + 3) + 4 * H * H
    got = bench.algorithmic_flops_per_step(G, H, n_lin, layers, fwd_only)
    assert got == passes * layers * (E * edge_split + N * row)
    got_model = bench.algorithmic_flops_per_step(G, H, n_lin, layers, fwd_only, split=False)
    assert got_model == passes * layers * (E * edge_unsplit + N * _linear_chain(2 * H, H, n_lin))


def test_c2_edge_forward_sits_below_the_tensor_ridge():
    # per edge at H = 64, n_h = 2, BF16 edge state: 2H^2 * 4 = 32,768 FLOPs over
    # 2 * 2H + 8 = 264 bytes, about 124 FLOP/B, under the ridge of the measured
    # peaks (about 286 FLOP/B): the HBM side of the roofline binds
    G = _graph(3_149_280, 0)
    fl = bench.algorithmic_flops_per_step(G, 64, 4, 4, fwd_only=True)
    by = bench.design_bytes("k_edge_fwd", G, 64, 2, n_lin=4)
    assert fl / by == pytest.approx(32768 / 264, rel=1e-12)
    pk = bench.load_peaks()
    assert fl / by < pk["bf16_tflops"] * 1e12 / (pk["hbm_gbs"] * 1e9)


@pytest.mark.parametrize("se", [2, 4])
def test_method_bytes_field_by_field(se):
    # the method's least traffic per layer, field by field: forward per edge
    # e in + e' out (s_e H each), sender index (4), multiplicity (1); per node
    # x in, x out, a* out, a* in (4H each), CSR pointer (4); the adjoint per
    # edge e_in (s_e H), FP32 de' in and de out (4H each), 5 bytes of indices,
    # per node 28H (x, a* and their FP32 gradients)
    E, N, H, M = 1000, 300, 64, bench.M
    fwd = E * (se * H + se * H + 4 + 1) + N * (4 * H * 4 + 4)
    bwd = E * (se * H + 4 * H + 4 * H + 5) + N * 28 * H
    assert bench.method_bytes_per_step(E, N, H, se) == M * (fwd + bwd)
    assert bench.method_bytes_per_step(E, N, H, se, fwd_only=True) == M * fwd
    # an inference stack's last layer writes no edge state
    assert bench.method_bytes_per_step(E, N, H, se, fwd_only=True, last_layer_no_edge_out=True) == \
        M * fwd - E * se * H


def test_c3_step_roofline_is_hbm_bound():
    # the 32^3 p=7 brick in 8 RCB parts (68,646,144 edges, 11,543,176 rows as
    # partitioned), H = 128, BF16 state, fwd+bwd of 4 layers: about 755 GB and
    # 140 TFLOP per step; at the measured peaks the bytes take longer, so the
    # step's bound is the HBM one (about 112 ms)
    pk = {"hbm_gbs": 6758.2, "bf16_tflops": 1891.8, "bf16_tflops_sustained": 1693.8, "src": "measured"}
    E, N = 68_646_144, 11_543_176
    r = bench.step_roofline(810.8, E, N, 128, 2, 4, False, pk)
    by = 4 * (E * (4 * 128 + 5 + 2 * 128 + 8 * 128 + 5) + N * (16 * 128 + 4 + 28 * 128))
    assert r["bound"] == "hbm" and r["bytes_per_step"] == by
    assert r["hbm_ms"] == pytest.approx(by / 6758.2e9 * 1e3)
    assert r["hbm_ms"] > r["tensor_ms"] and 100 < r["bound_ms"] < 120
    assert r["frac"] == pytest.approx(r["bound_ms"] / 810.8)
    assert r["achieved"] == pytest.approx(by / 0.8108 / 1e9)


@pytest.mark.parametrize("se", [2, 4])
def test_edge_forward_design_bytes_field_by_field(se):
    E, N, H, M = 1000, 300, 64, bench.M
    G = _graph(E, N)
    per_edge = se * H + se * H + 4 + 4            # e in, e' out, sender index, 1/d_ij
    per_row = 2 * H * 2 + 4 * H + 4               # P and Q rows (BF16), a (FP32), CSR pointer
    assert bench.design_bytes("k_edge_fwd", G, H, se) == M * (E * per_edge + N * per_row)
    # an inference stack's last layer writes no edge state
    no_last = bench.design_bytes("k_edge_fwd", G, H, se, last_layer_no_edge_out=True)
    assert no_last == pytest.approx(M * (E * per_edge + N * per_row) - E * se * H)
    # saved activations: the forward also writes h_0 .. h_{L-2} (BF16) of every edge
    n_lin = 4
    saved = bench.design_bytes("k_edge_fwd", G, H, se, n_lin=n_lin, saved_act=True)
    assert saved == M * (E * per_edge + N * per_row) + M * E * (n_lin - 1) * 2 * H


def test_reference_arm_prints_one_contract_line():
    # the reference arm is the oracle on the host cores: it runs here, without a GPU
    import json
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "edges/s" and d["higher_is_better"] is True
    assert d["metric"] == "MP-layer edges/s fwd+bwd" and d["value"] > 0 and d["steps"] == 1
    assert "68,040,000 edges" in d["config"]["workload"] and "H=128" in d["config"]["workload"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_workload_text_names_the_brick_that_ran():
    wl = bench.WORKLOADS["c3"]
    full = bench.workload_config_text(wl, wl["nel"], 1, 2, "fwd+bwd")
    assert f"{wl['nel']}^3 elements: {wl['nel']}^3 elements p=7" in full
    small = bench.workload_config_text(wl, 12, 614_125, 3_641_400, "fwd+bwd")
    assert "12^3 elements: 12^3 elements p=7" in small and f"{wl['nel']}^3" not in small
    assert "(614,125 nodes, 3,641,400 edges)" in small
