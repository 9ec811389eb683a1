#!/usr/bin/env python
"""Throughput of the consistent NMP layer (forward + backward) on one GB300.

One step = M=4 consistent NMP layers forward (Eq. 5a-5e) then their adjoint,
on the 16^3-element p=5 GLL brick (531,441 nodes, 3,149,280 directed edges)
split into 8 RCB sub-graphs resident on the GPU, H=64, MLPs with 2 hidden
layers. Inputs (x0, e0 from the encoders, a seeded upstream gradient) are
resident in HBM; the edge state (>400 MB) is larger than L2, so no flush is
needed between steps. Metric: MP-layer edges/s = 3,149,280 * 4 / step time.

value     -- fused BF16 path (FP32 accumulation and sums), device-timed; the
             training step keeps the MLP activations from the forward to the
             backward (gnn_mp_forward_act / gnn_mp_backward_act).
fp32      -- the plain FP32 SIMT path on the same graph and step.
e2e       -- the full network training step through the public API
             (encoders, 4 layers, decoder, consistent loss, backward) with
             inputs copied from pinned host memory each step and the loss read
             back, in the same metric.
roofline  -- the dominant kernel's algorithmic bytes (or FLOPs) per launch over
             its CUDA-event launch time, against MEASURED_PEAKS.json.
tensor    -- the whole step's algorithmic FLOPs over the step time, against
             the sustained BF16 peak of MEASURED_PEAKS.json.
cpu_baseline -- the FP64 numpy oracle on a bounded sample, host cores.

``--workload`` selects the other graph families (c3: 32^3 p=7 H=128 fwd+bwd,
``--mode fwd`` for its inference form;
c4: 64 uneven sub-graphs of a jittered p=5 brick, H=64 fwd+bwd, autotuned and
replayed as a CUDA graph; c5: 48^3 p=7 H=32 inference); their layer inputs
are seeded random states drawn on the device, and they report no fp32/e2e leg.

``--impl reference`` times the oracle alone (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

P, R, H, NH, M = 5, 8, 64, 2, 4
SEED = 0

# Workload families (sizes of the paper's brick graphs). "c2" is the benchmark
# workload of the JSON line; the others are measured with --workload.
#   inputs "encoders": x0, e0 from the node/edge encoders on the Fourier field
#   inputs "random":   seeded N(0,1) layer states drawn on the device (the
#                      encoders' FP32 workspace would not fit beside them)
WORKLOADS = {
    "c2": dict(nel=16, p=5, parts=8, H=64, mode="fwdbwd", inputs="encoders", graph=False,
               desc="16^3 elements p=5 GLL brick, 8 RCB sub-graphs"),
    "c3": dict(nel=32, p=7, parts=8, H=128, mode="fwdbwd", inputs="random", graph=False,
               desc="32^3 elements p=7 GLL brick, 8 RCB sub-graphs, the precision form (H=128)"),
    "c4": dict(nel=None, p=5, parts=64, H=64, mode="fwdbwd", inputs="random", graph=True, uneven=True,
               desc="jittered p=5 brick in 64 RCB sub-graphs of log-uniform element counts in [50, 5000], "
                    "CUDA graph, autotuned tiles"),
    "c5": dict(nel=48, p=7, parts=16, H=32, mode="fwd", inputs="random", graph=False,
               desc="48^3 elements p=7 GLL brick, 16 RCB sub-graphs, inference: last layer writes no edge state"),
    "mixed": dict(nel=64, p=1, parts=8, H=64, mode="fwdbwd", inputs="encoders", graph=False, mesh="mixed",
                  cells="cells", sample=32, ref_sample=16,
                  desc="mixed element mesh of the unit cube (each cell one hexahedron or its 6 Kuhn tetrahedra, "
                       "drawn 50/50) with 8 fan cells on one apex of in-degree 4,225, held as co-resident copies "
                       "of <= 128 in-edges, 8 RCB sub-graphs"),
    "large": dict(nel=16, p=5, parts=8, H=32, nh=5, mode="fwdbwd", inputs="encoders", graph=False,
                  desc="16^3 elements p=5 GLL brick, 8 RCB sub-graphs, the paper's large model (Table 1: "
                       "H=32, 5 MLP hidden layers)"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp32"])
    ap.add_argument("--mode", default="fwdbwd", choices=["fwdbwd", "fwd"],
                    help="fwd: forward only (inference form of the layer stack)")
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS),
                    help="c2 (default): 16^3 p=5 H=64 fwd+bwd; c3: 32^3 p=7 H=128 fwd+bwd; c4: 64 uneven jittered "
                         "sub-graphs H=64 fwd+bwd; c5: 48^3 p=7 H=32 inference; large: the C2 graph with the "
                         "paper's large model (H=32, 5 MLP hidden layers); mixed: a 64^3-cell mesh of mixed "
                         "element types with a node of in-degree 4,225, H=64 fwd+bwd")
    ap.add_argument("--nel", type=int, default=None,
                    help="elements per axis of the brick (default: the workload's; smaller for profiling)")
    ap.add_argument("--graph", action="store_true", help="time CUDA-graph replays of the step")
    ap.add_argument("--autotune", action="store_true", help="autotune tiles and the edge forward first")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp32", action="store_true")
    return ap.parse_args()


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([v.strip() for v in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            self.proc.wait(timeout=5)

    def summary(self) -> dict:
        sm = [float(s[0]) for s in self.samples if len(s) >= 7 and s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if len(s) >= 7 and s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples if len(s) >= 7
                          for k in range(4) if s[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


# ---------------------------------------------------------------- roofline bookkeeping

def algorithmic_bytes(kernel: str, G, hidden: int, edge_bytes: int, last_layer_no_edge_out: bool = False,
                      n_lin: int = NH + 2, saved_act: bool = False):
    """Least HBM bytes all launches of a kernel move in one step of M layers
    (for the edge forward of an inference stack the last layer writes no edge
    state; with saved activations the edge forward also writes, and the edge
    adjoint reads, h_0 .. h_{L-2} of every edge, and the adjoint gathers no P|Q)."""
    E, N = G.n_edges, G.n_rows
    h2 = 2 * hidden
    if saved_act and kernel == "k_edge_fwd":
        return (algorithmic_bytes(kernel, G, hidden, edge_bytes, last_layer_no_edge_out, n_lin)
                + M * E * (n_lin - 1) * h2)
    if saved_act and kernel == "k_edge_bwd":   # e, de_out in, de_in, dz1 out, col, w, h_0..h_{L-2}; da in, dP out
        return M * (E * (4 * edge_bytes * hidden + 8 + (n_lin - 1) * h2) + N * (2 * 4 * hidden + 4))
    return _algorithmic_bytes(kernel, G, hidden, edge_bytes, last_layer_no_edge_out, n_lin)


def _algorithmic_bytes(kernel: str, G, hidden: int, edge_bytes: int, last_layer_no_edge_out: bool,
                       n_lin: int):
    """Recompute form of ``algorithmic_bytes``.

    Per edge: read e (s_e H), write e' (s_e H), col (4), 1/d (4); per row:
    the row's CSR pointer and node tensors (see the per-kernel notes). The
    layered H = 128 backward counts its scratch rows (BF16 h, dz, [a*, x]) as
    the inputs and outputs of the kernels that read and write them."""
    E, N = G.n_edges, G.n_rows
    se = edge_bytes
    h2 = 2 * hidden                 # one BF16 row
    if kernel == "k_edge_fwd":      # e in/out, col, w, P/Q gathers (bf16 2H per row), a out (fp32 H)
        writes = (M - 1) / M if last_layer_no_edge_out else 1.0
        return M * (E * ((1 + writes) * se * hidden + 8) + N * (2 * 2 * hidden + 4 * hidden + 4))
    if kernel == "k_edge_bwd":      # e in, de_out in, de_in out, dz1 out, col, w; da in, P/Q, dP out per row
        return M * (E * (4 * se * hidden + 8) + N * (4 * hidden + 2 * 2 * hidden + 4 * hidden + 4))
    if kernel == "k_edge_fwd_save":   # e, de_out in, col, w; h_0..h_{L-2}, dz out; da, P/Q per row
        return M * (E * (2 * h2 + 8 + (n_lin - 1) * h2 + h2) + N * (4 * hidden + 2 * h2 + 4))
    if kernel == "k_node_fwd_save":   # a*, x, dx' in (fp32); [a*, x] bf16, h_0..h_{L-2}, dz out
        return M * N * (3 * 4 * hidden + 2 * h2 + (n_lin - 1) * h2 + h2)
    if kernel == "k_bwd_chain":       # per Linear k >= 1: dz_k, h_{k-1} in, dz_{k-1} out
        return M * (n_lin - 1) * (E + N) * 3 * h2
    if kernel == "k_bwd_edge0":       # dz_0, e, de_out in, de_in, dz_0 out; da in, dP out per row
        return M * (E * 5 * h2 + N * 2 * 4 * hidden)
    if kernel == "k_bwd_node0":       # dz_0, [a*, x] bf16, dx' in; da*, dx_in out (fp32)
        return M * N * (h2 + 2 * h2 + 3 * 4 * hidden)
    return None


def measured_traffic(kernel: str, n_edges: int):
    """DRAM bytes per launch of `kernel` from the committed ncu capture, scaled by
    the edge count; None when the kernel sources changed since the capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "edge_kernel_traffic.json")) as fh:
            d = json.load(fh)
        h = hashlib.sha256()
        for f in d["sources_hashed"]:
            with open(os.path.join(ROOT, f), "rb") as fh:
                h.update(fh.read())
        if h.hexdigest() != d["source_hash"] or kernel not in d["bytes_per_edge"]:
            return None
        return d["bytes_per_edge"][kernel] * n_edges
    except (OSError, KeyError, ValueError):
        return None


def sgemm_flops_per_step(G, hidden: int, n_lin: int, layers: int) -> float:
    """FP32 SIMT GEMM FLOPs of one plain-path step (forward, recompute, dgrad, wgrad)."""
    E, N, Hh = G.n_edges, G.n_rows, hidden
    def chain(rows, d0):
        dims = [d0] + [Hh] * n_lin
        return sum(2.0 * rows * dims[k] * dims[k + 1] for k in range(n_lin))
    per_layer_fwd = chain(E, 3 * Hh) + chain(N, 2 * Hh)
    return layers * per_layer_fwd * 4.0     # forward + recompute + dgrad + wgrad


def algorithmic_flops_per_step(G, hidden: int, n_lin: int, layers: int, fwd_only: bool = False,
                               split: bool = True) -> float:
    """Tensor FLOPs one step of the layer stack must compute (Eq. 5a, 5e).

    Forward, per edge: with the first Linear split (its x_i and x_j blocks
    applied once per row) the edge MLP costs 2H^2 * n_lin (the e block and the
    n_lin - 1 hidden Linears); unsplit, 2H^2 * (n_lin + 2). Per row: the node
    MLP 2H^2 * (n_lin + 1) (its 2H-wide first Linear and the rest), plus the
    split's two per-row projections, 4H^2. A training step is 3x the forward
    (forward, input gradients, weight gradients); recomputation is not counted."""
    E, N, Hh = G.n_edges, G.n_rows, hidden
    h2 = 2.0 * Hh * Hh
    edge = h2 * (n_lin if split else n_lin + 2)
    row = h2 * (n_lin + 1) + (2.0 * h2 if split else 0.0)
    return (1.0 if fwd_only else 3.0) * layers * (E * edge + N * row)


def load_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"], "src": "measured",
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained", d["bf16_tflops"]),
                "sm_max_mhz": d.get("sm_max_mhz", 2070.0)}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "src": "fallback",
                "sm_max_mhz": 2070.0}


# ---------------------------------------------------------------- oracle timing (CPU)

def oracle_sample(n_el: int, steps: int = 1, p: int = P, hidden: int = H, parts: int = R, fwd_only: bool = False,
                  nh: int = NH, mesh: str = "brick"):
    """Time the FP64 oracle on an n_el^3 brick of order p (or, mesh="mixed", the
    n_el^3-cell mixed element mesh; RCB parts, 4 layers of width `hidden`,
    forward + backward unless fwd_only): a bounded sample of a workload family.
    Returns (edges/s, seconds per step, description, threads)."""
    import numpy as np

    import synthetic as syn
    from oracle import graph as og
    from oracle import model as om

    if mesh == "mixed":
        m = syn.mixed_element_mesh(n_el, SEED, n_fans=8)
        b = og.element_mesh(m["pos"], m["elem_ptr"], m["elem_nodes"], m["edge_ptr"], m["edge_pairs"])
        subs = og.build_element_subgraphs(b, og.partition_rcb_elements(b, parts), parts)
        what = f"{n_el}^3-cell mixed element mesh"
    else:
        b = og.build_brick((n_el,) * 3, p)
        subs = og.build_subgraphs(b, og.partition_rcb(b, parts), parts)
        what = f"{n_el}^3 elements p={p}"
    params = syn.gnn_params(SEED, hidden, nh, M)
    rng = np.random.default_rng(1)
    xg = rng.standard_normal((b.n_nodes, hidden))
    xs = [xg[sg.gid] for sg in subs]
    es = [rng.standard_normal((sg.n_edges, hidden)) for sg in subs]
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        caches, x, e = [], xs, es
        for lp in params["layers"]:
            x, e, c = om.layer_forward(lp, subs, x, e)
            caches.append(c)
        if not fwd_only:
            dx = [np.ones_like(a) for a in x]
            de = [np.zeros_like(a) for a in e]
            for li in range(M - 1, -1, -1):
                dx, de, _ = om.layer_backward(params["layers"][li], subs, caches[li], dx, de)
        times.append(time.perf_counter() - t0)
    t = statistics.median(times)
    return (b.n_edges * M / t, t,
            f"{what} ({b.n_nodes} nodes, {b.n_edges} edges), {parts} RCB parts, H={hidden}, "
            f"MLP {nh} hidden, 4 layers {'fwd' if fwd_only else 'fwd+bwd'}, FP64 numpy", _blas_threads())


def _blas_threads() -> int:
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 0) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count() or 1


def workload_config_text(wl: dict, n_el, n_unpart, e_unpart, kind: str) -> str:
    """The `config.workload` text of a workload (shared by both arms)."""
    return (f"consistent NMP layers x{M} {kind}, {n_el}^3 {wl.get('cells', 'elements')}: {wl['desc']} "
            f"({n_unpart:,} nodes, {e_unpart:,} edges), H={wl['H']}, MLP {wl.get('nh', NH)} hidden")


def run_reference(args):
    """The reference arm: the FP64 oracle (the method as the paper defines it)
    timed on the host cores, on a bounded sample of the selected workload (same
    order, width, partition count and pass, a smaller brick), reported in the
    GPU arm's metric and config. Rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl = dict(WORKLOADS[args.workload])
    fwd_only = wl["mode"] == "fwd" or args.mode == "fwd"
    kind = "fwd" if fwd_only else "fwd+bwd"
    sample = dict(n_el=wl.get("ref_sample") or {5: 4, 7: 3}[wl["p"]], p=wl["p"], hidden=wl["H"],
                  parts=wl["parts"] if wl["parts"] <= 16 else 8, fwd_only=fwd_only, nh=wl.get("nh", NH),
                  mesh=wl.get("mesh", "brick"))
    for _ in range(args.warmup):
        oracle_sample(**sample)
    vals, secs = [], []
    desc = threads = None
    for _ in range(args.steps):
        v, t, desc, threads = oracle_sample(**sample)
        vals.append(v)
        secs.append(t)
    value = statistics.median(vals)
    if wl.get("uneven") or args.nel:
        workload = f"{wl['desc']}, H={wl['H']}, MLP {wl.get('nh', NH)} hidden, {kind}"
    elif wl.get("mesh") == "mixed":
        n_nodes, n_edges = mixed_mesh_counts(wl["nel"])
        workload = workload_config_text(wl, wl["nel"], n_nodes, n_edges, kind)
    else:
        L = wl["nel"] * wl["p"] + 1
        workload = workload_config_text(wl, wl["nel"], L ** 3, 6 * L * L * (L - 1), kind)
    line = {"impl": "reference", "metric": f"MP-layer edges/s {kind}", "value": value, "unit": "edges/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.median(secs) * 1e3,   # one step = one pass over the sample
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload, "name": args.workload, "inputs": wl["inputs"]},
            "cpu_baseline": {"value": value, "unit": "edges/s", "cores": threads, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- GPU arm

def max_over_ranks(value: float, dist, device) -> float:
    """The slowest rank's time (the whole-job step time of weak-scaled replicas)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def mixed_mesh_counts(n: int):
    """Nodes and directed edges of the n^3-cell mixed mesh (its element lists, counted with numpy)."""
    import numpy as np

    import synthetic as syn

    m = syn.mixed_element_mesh(n, SEED, n_fans=8)
    N = m["pos"].shape[0]
    el = np.repeat(np.arange(m["elem_ptr"].size - 1), np.diff(m["edge_ptr"]))
    base = m["elem_ptr"][el]
    u = m["elem_nodes"][base + m["edge_pairs"][:, 0]]
    v = m["elem_nodes"][base + m["edge_pairs"][:, 1]]
    return N, int(np.unique(np.concatenate([u * N + v, v * N + u])).size)


def workload_graph(wl: dict, nel):
    """(Partition, unpartitioned nodes, unpartitioned directed edges) of a workload."""
    import numpy as np

    import synthetic as syn
    from paper_2410_01657_gb300.graph import MeshGraph

    p = wl["p"]
    if wl.get("mesh") == "mixed":
        n = nel or wl["nel"]
        m = syn.mixed_element_mesh(n, SEED, n_fans=8)
        g = MeshGraph.from_elements(m["pos"], m["elem_ptr"], m["elem_nodes"], m["edge_ptr"], m["edge_pairs"])
        return g.partition(wl["parts"], "rcb"), n, g.n_nodes, g.n_edges
    if wl.get("uneven"):
        n, weights = syn.uneven_brick(wl["parts"], 50, 5000, SEED)
        if nel:
            n, weights = nel, syn.rescale_counts(weights, nel ** 3)
        g0 = MeshGraph((n,) * 3, p)
        jit = syn.jitter_unit(g0.n_nodes, SEED + 1)
        g = MeshGraph((n,) * 3, p, jitter=jit, jitter_frac=0.2)
        part = g.partition(wl["parts"], "rcb", np.asarray(weights, dtype=np.float64))
    else:
        n = nel or wl["nel"]
        g = MeshGraph((n,) * 3, p)
        part = g.partition(wl["parts"], "rcb")
    L = n * p + 1
    return part, n, L ** 3, 6 * L * L * (L - 1)


def build_problem(dev, precision, wl: dict, part):
    import torch

    import synthetic as syn
    from paper_2410_01657_gb300 import nn as gnn

    Hh = wl["H"]
    G = part.to_device(dev)
    params = syn.gnn_params(SEED, Hh, wl.get("nh", NH), M)
    net = gnn.ConsistentGNN(params, precision=precision, device=dev)
    u = t = None
    if wl["inputs"] == "encoders":
        modes = syn.fourier_modes(SEED, 8)
        pos = part.array("row_pos")
        u = torch.tensor(syn.fourier_field(pos, modes), dtype=torch.float32, device=dev)
        t = torch.tensor(syn.fourier_field(pos, modes, phase_advance=0.1), dtype=torch.float32, device=dev)
        with torch.no_grad():
            x0, e0 = net.encode(G, u, G.edge_attr())
    else:
        g = torch.Generator(device=dev).manual_seed(SEED)
        x0 = torch.randn(part.n_rows, Hh, device=dev, generator=g)
        e0 = torch.randn(part.n_edges, Hh, device=dev, generator=g).to(
            torch.bfloat16 if precision == "bf16" else torch.float32)
    layers = [(l.edge.tensors(), l.node.tensors(), l.edge.dims, l.node.dims) for l in net.layers]
    stack = gnn.LayerStack(G, layers, Hh, precision, x0, e0, inference=wl["mode"] == "fwd")
    dx_top = None
    if wl["mode"] == "fwdbwd":
        g = torch.Generator(device=dev).manual_seed(SEED + 7)
        dx_top = 1e-3 * torch.randn(part.n_rows, Hh, device=dev, generator=g)
    return G, net, stack, dx_top, u, t


def _timed(run, steps, profile):
    import torch

    from paper_2410_01657_gb300 import binding as B

    stream = torch.cuda.current_stream()
    if profile:
        B.call("gnn_profile_start", 1 << 16)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        run()
    ev1.record(stream)
    torch.cuda.synchronize()
    if profile:
        B.call("gnn_profile_stop")
    return ev0.elapsed_time(ev1) / steps, (B.profile_report() if profile else {})


def time_stack(stack, dx_top, steps, warmup, profile=True, graph=False):
    """Mean device time of one step (ms) and the per-kernel CUDA-event report.

    Eager: the profiled steps are the timed steps. Graph: the kernel report
    comes from the same number of eager profiled steps, then the step is
    captured once and `steps` replays are timed (the value)."""
    import torch

    run = lambda: stack.step(dx_top)
    for _ in range(warmup):
        run()
    torch.cuda.synchronize()
    ms, report = _timed(run, steps, profile)
    if not graph:
        return ms, report, None
    stack.capture(dx_top)
    for _ in range(warmup):
        stack.replay()
    torch.cuda.synchronize()
    ms_graph, _ = _timed(stack.replay, steps, False)
    return ms_graph, report, ms


def time_e2e(net, G, u, t, steps, warmup, dev):
    """Full training step through the public API with host-resident inputs: the
    step's node field and target are copied from pinned host memory every step;
    the edge attributes are graph geometry and stay on the device with the graph."""
    import torch

    from paper_2410_01657_gb300 import nn as gnn

    u_h = u.cpu().pin_memory()
    t_h = t.cpu().pin_memory()
    attr = G.edge_attr()
    h2d = u_h.numel() * 4 + t_h.numel() * 4

    def one():
        ud = u_h.to(dev, non_blocking=True)
        td = t_h.to(dev, non_blocking=True)
        net.zero_grad(set_to_none=True)
        y = net(G, ud, attr)
        loss = gnn.consistent_loss(y, td, G)
        loss.backward()
        return loss.item()

    for _ in range(warmup):
        one()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(steps):
        one()
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    # the library kernels of one more step, event-timed (torch's own kernels are not listed)
    from paper_2410_01657_gb300 import binding as B
    B.call("gnn_profile_start", 1 << 12)
    one()
    torch.cuda.synchronize()
    B.call("gnn_profile_stop")
    kernels = {k: {"launches": n, "ms": round(v, 4)} for k, (n, v) in B.profile_report().items()}
    return ms, h2d, 4, kernels


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    from paper_2410_01657_gb300 import _build
    from paper_2410_01657_gb300 import binding as B
    _build.build()
    B.load()

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    precision = args.precision
    wl = dict(WORKLOADS[args.workload])
    Hw = wl["H"]
    fwd_only = wl["mode"] == "fwd" or args.mode == "fwd"
    if fwd_only:
        wl["mode"] = "fwd"
    use_graph = args.graph or wl["graph"]
    part, n_el, n_unpart, e_unpart = workload_graph(wl, args.nel)
    G, net, stack, dx_top, u, t = build_problem(dev, precision, wl, part)
    tune = None
    if (args.autotune or wl.get("uneven")) and precision == "bf16":
        tune = stack.autotune(dx_top)
        tune = {k: v for k, v in tune.items() if k != "candidates"} | {
            "candidates": [{k: v for k, v in c.items() if k != "fwd_choices"} for c in tune.get("candidates", [])]}
    peaks = load_peaks()
    barrier()
    with ClockSampler(local) as clk:
        ms, report, ms_eager = time_stack(stack, dx_top, args.steps, args.warmup, graph=use_graph)
    barrier()
    ms = max_over_ranks(ms, dist, dev)
    value = world * e_unpart * M / (ms * 1e-3)
    launches = sum(n for n, _ in report.values())
    total_ms = sum(v for _, v in report.values()) or 1.0
    top = max(report.items(), key=lambda kv: kv[1][1]) if report else ("none", (1, 0.0))
    top_name, (top_n, top_ms) = top
    edge_bytes = 2 if precision == "bf16" else 4
    roof = None
    abytes = algorithmic_bytes(top_name, G, Hw, edge_bytes, last_layer_no_edge_out=fwd_only,
                               n_lin=wl.get("nh", NH) + 2, saved_act=any(a is not None for a in stack.act))
    if abytes is not None:   # bytes of one step over the kernel's device time in one step
        ach = abytes / (top_ms / args.steps * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": top_name, "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"],
                "traffic": measured_traffic(top_name, G.n_edges) if args.workload == "c2" else None,
                "peak_src": peaks["src"], "share": top_ms / total_ms}
    elif top_name == "k_sgemm":
        flops = sgemm_flops_per_step(G, Hw, wl.get("nh", NH) + 2, M) * args.steps
        ach = flops / (top_ms * 1e-3) / 1e12
        peak = 152 * 128 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12
        roof = {"bound": "alu", "kernel": top_name, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": None, "peak_src": "derived: 152 SM x 128 FP32 FMA/clk x 2 x max clock",
                "share": top_ms / total_ms}
    tensor = None
    if precision == "bf16":   # the whole step against the tensor bound (the other side of the roofline max)
        n_lin = wl.get("nh", NH) + 2
        fl = algorithmic_flops_per_step(G, Hw, n_lin, M, fwd_only)
        fl_model = algorithmic_flops_per_step(G, Hw, n_lin, M, fwd_only, split=False)
        ach_t = fl / (ms * 1e-3) / 1e12
        tensor = {"bound": "tensor", "achieved": ach_t, "peak": peaks["bf16_tflops_sustained"], "unit": "TFLOP/s",
                  "frac": ach_t / peaks["bf16_tflops_sustained"], "flops_per_step": fl,
                  "model_flops_per_step": fl_model, "peak_src": peaks["src"] + ", bf16 sustained",
                  "note": "algorithmic FLOPs of the whole step (first Linear split, recompute not counted) "
                          "over the step time"}

    # the cost of consistency: the same stack with Eq. 5c-5d skipped (the paper's "None" layers)
    from paper_2410_01657_gb300 import binding as Bd
    for c in (stack.cfg, stack.cfg_last):
        c.halo_mode = Bd.GNN_HALO_NONE
    stack.graph = None
    ms_none, _, _ = time_stack(stack, dx_top, max(3, args.steps // 2), 2, profile=False)
    for c in (stack.cfg, stack.cfg_last):
        c.halo_mode = Bd.GNN_HALO_SYNC
    inconsistent = {"ms_per_step": ms_none, "cost_of_consistency": (ms_eager or ms) / ms_none,
                    "note": "same stack without the halo swap + sync (inconsistent layers), eager"}

    fp32 = None
    if precision == "bf16" and not args.no_fp32 and wl["inputs"] == "encoders":
        del stack
        torch.cuda.empty_cache()
        _, _, stack32, dx32, _, _ = build_problem(dev, "fp32", wl, part)
        ms32, _, _ = time_stack(stack32, dx32, max(3, args.steps // 2), 2, profile=False)
        fp32 = {"value": e_unpart * M / (ms32 * 1e-3), "unit": "edges/s", "ms_per_step": ms32,
                "speedup_of_bf16": ms32 / ms}
        del stack32
        torch.cuda.empty_cache()

    e2e = None
    if not args.no_e2e and wl["inputs"] == "encoders" and not fwd_only:
        ms_e, h2d, d2h, e2e_k = time_e2e(net, G, u, t, max(3, args.steps // 2), 2, dev)
        e2e = {"value": world * e_unpart * M / (ms_e * 1e-3), "unit": "edges/s", "ms_per_step": ms_e,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "library_kernels_one_step": e2e_k,
               "step": "encoders + 4 layers + decoder + consistent loss, fwd+bwd; node field and target "
                       "copied from pinned host memory each step, loss read back"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        # a bounded sample of the same workload family: a small brick of the same order,
        # width, partition count and pass (about 10-20 s of host time on 16 cores)
        n_s = wl.get("sample") or {5: 8, 7: 5}[wl["p"]]
        v, tsec, desc, threads = oracle_sample(n_s, p=wl["p"], hidden=Hw, parts=wl["parts"] if wl["parts"] <= 16 else 8,
                                               fwd_only=fwd_only, nh=wl.get("nh", NH), mesh=wl.get("mesh", "brick"))
        cpu = {"value": v, "unit": "edges/s", "cores": threads, "kind": "oracle", "sample": desc,
               "seconds": tsec}

    if rank == 0:
        kind = "fwd+bwd" if not fwd_only else "fwd"
        edge_state = e_unpart * Hw * edge_bytes
        line = {"metric": f"MP-layer edges/s {kind}", "value": value, "unit": "edges/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": precision, "data": "synthetic",
                "config": {"workload": workload_config_text(wl, n_el, n_unpart, e_unpart, kind),
                           "name": args.workload, "inputs": wl["inputs"],
                           "rows": part.n_rows, "edges_partitioned": part.n_edges, "tile_edges": G.tile_edges,
                           "l2": f"inputs larger than L2 (edge state {edge_state / 1e6:.0f} MB), no flush",
                           "timing": "CUDA-graph replays; kernel table from as many eager steps" if use_graph
                           else "eager steps",
                           "parallelism": f"replicas x{world}"},
                "nodes_per_s": world * n_unpart * M / (ms * 1e-3),
                "roofline": roof, "tensor": tensor, "fp32": fp32, "e2e": e2e, "cpu_baseline": cpu, "inconsistent": inconsistent,
                "gpu_launches": launches, "kernels": {k: {"launches": n, "ms": v} for k, (n, v) in report.items()},
                "clocks": clk.summary()}
        if ms_eager is not None:
            line["eager_ms_per_step"] = ms_eager
        if tune is not None:
            line["autotune"] = tune
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
