#!/usr/bin/env python
"""Throughput of the consistent NMP layer (forward + backward) on one GB300.

One step = M=4 consistent NMP layers forward (Eq. 5a-5e) then their adjoint
(Eq. 3), recomputing each layer's MLP activations in the backward. The
default workload is the precision form: the 32^3-element p=7 GLL brick
(11,390,625 nodes, 68,040,000 directed edges) split into 8 RCB sub-graphs
resident on the GPU, H=128, MLPs with 2 hidden layers, BF16 GEMM operands with
FP32 accumulation and FP32 sums. The layer inputs x0, e0 come from the node
and edge encoders on a 32-mode Fourier field; they and a seeded upstream
gradient are resident in HBM, and the edge state (17 GB) is far larger than
L2, so no flush is needed between steps. Metric: MP-layer edges/s =
68,040,000 * 4 / step time, the step time being the median of K CUDA-graph
replays, each timed by its own CUDA events with no profiler running.

value     -- fused BF16 path, device-timed (median replay).
roofline  -- the whole step's algorithmic HBM bytes per unit of work (the
             per-edge and per-node figures of the method's forward and
             adjoint, no scratch or saved activations) over the step time,
             against the measured HBM peak, beside the tensor-FLOP side; the
             slower side is the bound. roofline_kernel: the dominant kernel's
             event-timed launches against the bytes it moves as designed.
fp32      -- the plain FP32 SIMT path against the fused BF16 path on the same
             graph (for the H=128 brick, on a 16^3-element p=7 sub-brick:
             the plain path's FP32 per-edge workspace does not fit the
             full graph).
e2e       -- the full network training step through the public API
             (encoders, 4 layers, decoder, consistent loss, backward) with the
             node field and target copied from pinned host memory each step
             and the loss read back, in the same metric.
cpu_baseline -- the FP64 numpy oracle on a bounded sample, host cores.

``--workload`` selects the other graph families (c2: 16^3 p=5 H=64; c4: 64
uneven sub-graphs of a jittered p=5 brick, H=64, autotuned; c5: 48^3 p=7 H=32
inference; large; mixed). ``--save-act`` runs the H <= 64 training step with
the MLP activations kept from the forward (an option; the default
recomputes).

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
    "c2": dict(nel=16, p=5, parts=8, H=64, mode="fwdbwd", inputs="encoders", modes=8, graph=True,
               desc="16^3 elements p=5 GLL brick, 8 RCB sub-graphs"),
    "c3": dict(nel=32, p=7, parts=8, H=128, mode="fwdbwd", inputs="encoders", modes=32, graph=True, fp32_nel=16,
               desc="32^3 elements p=7 GLL brick, 8 RCB sub-graphs, the precision form (H=128)"),
    "c4": dict(nel=None, p=5, parts=64, H=64, mode="fwdbwd", inputs="random", graph=True, uneven=True,
               desc="jittered p=5 brick in 64 RCB sub-graphs of log-uniform element counts in [50, 5000], "
                    "CUDA graph, autotuned tiles"),
    "c5": dict(nel=48, p=7, parts=16, H=32, mode="fwd", inputs="random", graph=True,
               desc="48^3 elements p=7 GLL brick, 16 RCB sub-graphs, inference: last layer writes no edge state"),
    "mixed": dict(nel=64, p=1, parts=8, H=64, mode="fwdbwd", inputs="encoders", modes=8, graph=True, mesh="mixed",
                  cells="cells", sample=32, ref_sample=16,
                  desc="mixed element mesh of the unit cube (each cell one hexahedron or its 6 Kuhn tetrahedra, "
                       "drawn 50/50) with 8 fan cells on one apex of in-degree 4,225, held as co-resident copies "
                       "of <= 128 in-edges, 8 RCB sub-graphs"),
    "large": dict(nel=16, p=5, parts=8, H=32, nh=5, mode="fwdbwd", inputs="encoders", modes=8, graph=True,
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
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS),
                    help="c3 (default): 32^3 p=7 H=128 fwd+bwd; c2: 16^3 p=5 H=64 fwd+bwd; c4: 64 uneven jittered "
                         "sub-graphs H=64 fwd+bwd; c5: 48^3 p=7 H=32 inference; large: the C2 graph with the "
                         "paper's large model (H=32, 5 MLP hidden layers); mixed: a 64^3-cell mesh of mixed "
                         "element types with a node of in-degree 4,225, H=64 fwd+bwd")
    ap.add_argument("--nel", type=int, default=None,
                    help="elements per axis of the brick (default: the workload's; smaller for profiling)")
    ap.add_argument("--eager", action="store_true", help="time eager steps instead of CUDA-graph replays")
    ap.add_argument("--save-act", action="store_true",
                    help="H <= 64 training: keep the MLP activations from the forward (default: recompute)")
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

def method_bytes_per_step(n_edges: int, n_rows: int, hidden: int, edge_bytes: int, layers: int = M,
                          fwd_only: bool = False, last_layer_no_edge_out: bool = False) -> float:
    """Least HBM bytes one step of the layer stack must move: the method's
    per-unit figures, not this implementation's traffic.

    Forward, per layer: per edge read e and write e' (2 s_e H), its sender
    index (4) and multiplicity (1); per node read and write x (FP32), write and
    read a* (FP32) and the CSR pointer (16H + 4). The adjoint adds per edge read
    e_in and read/write FP32 edge gradients (s_e H + 8H + 5) and per node about
    28H (x, a* and their gradients in and out). No scratch, saved activation or
    recomputed row is counted. Units are the partitioned rows and edges the
    sub-graphs hold (halo copies are rows the method processes)."""
    E, N, Hh, se = n_edges, n_rows, hidden, edge_bytes
    fwd = E * (2 * se * Hh + 5) + N * (16 * Hh + 4)
    if fwd_only:
        return layers * fwd - (E * se * Hh if last_layer_no_edge_out else 0)
    bwd = E * (se * Hh + 8 * Hh + 5) + N * 28 * Hh
    return layers * (fwd + bwd)


def step_roofline(step_ms: float, n_edges: int, n_rows: int, hidden: int, edge_bytes: int, n_lin: int,
                  fwd_only: bool, peaks: dict, last_layer_no_edge_out: bool = False) -> dict:
    """The whole step against both sides of the roofline: HBM (method bytes over
    the measured copy bandwidth) and tensor (algorithmic FLOPs over the measured
    sustained BF16 GEMM rate); the slower side is the bound."""
    by = method_bytes_per_step(n_edges, n_rows, hidden, edge_bytes, M, fwd_only, last_layer_no_edge_out)
    G = _Units(n_edges, n_rows)
    fl = algorithmic_flops_per_step(G, hidden, n_lin, M, fwd_only)
    t_hbm = by / (peaks["hbm_gbs"] * 1e9)
    t_ten = fl / (peaks["bf16_tflops_sustained"] * 1e12)
    t = step_ms * 1e-3
    if t_hbm >= t_ten:
        out = {"bound": "hbm", "achieved": by / t / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s"}
    else:
        out = {"bound": "tensor", "achieved": fl / t / 1e12, "peak": peaks["bf16_tflops_sustained"],
               "unit": "TFLOP/s"}
    out["frac"] = out["achieved"] / out["peak"]
    out.update({"scope": "whole step (all launches of the 4-layer fwd+bwd step)" if not fwd_only
                else "whole step (all launches of the 4-layer forward)",
                "bytes_per_step": by, "flops_per_step": fl, "bound_ms": max(t_hbm, t_ten) * 1e3,
                "hbm_ms": t_hbm * 1e3, "tensor_ms": t_ten * 1e3,
                "tensor_frac": fl / t / 1e12 / peaks["bf16_tflops_sustained"],
                "hbm_frac": by / t / 1e9 / peaks["hbm_gbs"],
                "peak_src": peaks["src"] + " (HBM copy; BF16 GEMM sustained)"})
    return out


class _Units:
    def __init__(self, n_edges, n_rows):
        self.n_edges, self.n_rows = n_edges, n_rows


def design_bytes(kernel: str, G, hidden: int, edge_bytes: int, last_layer_no_edge_out: bool = False,
                 n_lin: int = NH + 2, saved_act: bool = False):
    """HBM bytes all launches of a kernel move in one step of M layers as this
    implementation is designed (its inputs, outputs and scratch each once): the
    yardstick of how close a kernel runs to its own streaming time. Unlike
    ``method_bytes_per_step`` this counts the P|Q rows of the split first
    Linear, the H = 128 adjoint's scratch rows and, with saved activations, the
    stored h_0 .. h_{L-2}."""
    E, N = G.n_edges, G.n_rows
    h2 = 2 * hidden
    if saved_act and kernel == "k_edge_fwd":
        return (design_bytes(kernel, G, hidden, edge_bytes, last_layer_no_edge_out, n_lin)
                + M * E * (n_lin - 1) * h2)
    if saved_act and kernel == "k_edge_bwd":   # e, de_out in, de_in, dz1 out, col, w, h_0..h_{L-2}; da in, dP out
        return M * (E * (4 * edge_bytes * hidden + 8 + (n_lin - 1) * h2) + N * (2 * 4 * hidden + 4))
    return _design_bytes(kernel, G, hidden, edge_bytes, last_layer_no_edge_out, n_lin)


def _design_bytes(kernel: str, G, hidden: int, edge_bytes: int, last_layer_no_edge_out: bool, n_lin: int):
    """Recompute form of ``design_bytes``.

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


def measured_traffic(workload: str, kernels: list, n_edges: int):
    """DRAM bytes of one step of the listed kernels (sum over their launches)
    from the committed ncu capture of the workload's family, scaled by the
    partitioned edge count; None when the kernel sources changed since the
    capture or a kernel is missing from it."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", f"step_traffic_{workload}.json")) as fh:
            d = json.load(fh)
        h = hashlib.sha256()
        for f in d["sources_hashed"]:
            with open(os.path.join(ROOT, f), "rb") as fh:
                h.update(fh.read())
        if h.hexdigest() != d["source_hash"]:
            return None
        per = d["bytes_per_edge_per_step"]
        if any(k not in per for k in kernels):
            return None
        return {k: per[k] * n_edges for k in kernels}
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
    """The `config.workload` text of a workload (shared by both arms); a brick size
    given on the command line replaces the default one in the description."""
    desc, pre = wl["desc"], f"{wl.get('nel')}^3 "
    if n_el != wl.get("nel") and desc.startswith(pre):
        desc = f"{n_el}^3 " + desc[len(pre):]
    return (f"consistent NMP layers x{M} {kind}, {n_el}^3 {wl.get('cells', 'elements')}: {desc} "
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


def build_problem(dev, precision, wl: dict, part, save_act: bool = False):
    import torch

    import synthetic as syn
    from paper_2410_01657_gb300 import nn as gnn

    Hh = wl["H"]
    G = part.to_device(dev)
    params = syn.gnn_params(SEED, Hh, wl.get("nh", NH), M)
    net = gnn.ConsistentGNN(params, precision=precision, device=dev)
    u = t = None
    if wl["inputs"] == "encoders":
        modes = syn.fourier_modes(SEED, wl.get("modes", 8))
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
    stack = gnn.LayerStack(G, layers, Hh, precision, x0, e0, inference=wl["mode"] == "fwd", save_act=save_act)
    dx_top = None
    if wl["mode"] == "fwdbwd":
        g = torch.Generator(device=dev).manual_seed(SEED + 7)
        dx_top = 1e-3 * torch.randn(part.n_rows, Hh, device=dev, generator=g)
    return G, net, stack, dx_top, u, t


def _profiled(run, steps):
    """Per-kernel CUDA-event report (launches, ms) of `steps` eager calls of `run`."""
    import torch

    from paper_2410_01657_gb300 import binding as B

    torch.cuda.synchronize()
    B.call("gnn_profile_start", 1 << 16)
    for _ in range(steps):
        run()
    torch.cuda.synchronize()
    B.call("gnn_profile_stop")
    return B.profile_report()


def time_steps(run, steps: int, stream) -> list:
    """Device time (ms) of each of `steps` calls of `run`, each bracketed by its
    own CUDA events on the launching stream; synchronized on both sides."""
    import torch

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    torch.cuda.synchronize()
    for i in range(steps):
        ev[i].record(stream)
        run()
    ev[steps].record(stream)
    torch.cuda.synchronize()
    return [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]


def prepare_timing(stack, dx_top, warmup: int, graph: bool):
    """Warm the step up (eager), capture it as a CUDA graph when asked, and return
    the callable one timed step runs (a graph replay, or an eager step)."""
    import torch

    run = lambda: stack.step(dx_top)
    for _ in range(warmup):
        run()
    torch.cuda.synchronize()
    if not graph:
        return run
    stack.capture(dx_top)
    for _ in range(2):
        stack.replay()
    torch.cuda.synchronize()
    return stack.replay


def time_e2e(net, G, u, t, steps, warmup, dev):
    """Full training step through the public API with host-resident inputs: the
    step's node field and target are copied from pinned host memory every step;
    the edge attributes are graph geometry and stay on the device with the graph.
    Returns (median ms, mean ms, H2D bytes, D2H bytes, library kernels of one step)."""
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
    stream = torch.cuda.current_stream()
    times = time_steps(one, steps, stream)
    report = _profiled(one, 1)
    kernels = {k: {"launches": n, "ms": round(v, 4)} for k, (n, v) in report.items()}
    return statistics.median(times), statistics.mean(times), h2d, 4, kernels


def measure_fp32_peak():
    """FP32 SIMT FMA throughput of this GPU, measured by the library's FMA kernel
    (TFLOP/s, 2 FLOPs per FMA) and its SM count."""
    import ctypes as C

    from paper_2410_01657_gb300 import binding as B
    tf, sms = C.c_double(), C.c_int32()
    B.call("gnn_measure_fp32_fma", C.byref(tf), C.byref(sms), None)
    return float(tf.value), int(sms.value)


def fp32_comparison(dev, wl: dict, part_full, steps: int, warmup: int, ms_bf16_full: float):
    """The plain FP32 SIMT path against the fused BF16 path, same graph and step
    (eager steps, median). For the H=128 brick the comparison graph is the
    16^3-element sub-brick of the same order and partition count."""
    import torch

    sub_nel = wl.get("fp32_nel")
    part = part_full if sub_nel is None else workload_graph(dict(wl, nel=sub_nel), sub_nel)[0]
    res = {}
    sgemm = None
    for prec in ("bf16", "fp32"):
        G, _, stack, dx, _, _ = build_problem(dev, prec, wl, part)
        run = prepare_timing(stack, dx, 2, graph=False)
        res[prec] = statistics.median(time_steps(run, steps, torch.cuda.current_stream()))
        if prec == "fp32":   # the plain path's SIMT GEMMs against the measured FP32 FMA peak
            rep = _profiled(run, 1)
            n_lin = wl.get("nh", NH) + 2
            if "k_sgemm" in rep:
                sgemm = (sgemm_flops_per_step(G, wl["H"], n_lin, M), rep["k_sgemm"][1])
        del stack, G
        torch.cuda.empty_cache()
    L = (sub_nel or wl["nel"]) * wl["p"] + 1 if wl.get("mesh") != "mixed" else None
    e_unpart = 6 * L * L * (L - 1) if L else part.graph.n_edges
    out = {"value": e_unpart * M / (res["fp32"] * 1e-3), "unit": "edges/s", "ms_per_step": res["fp32"],
           "bf16_ms_per_step_same_graph": res["bf16"], "speedup_of_bf16": res["fp32"] / res["bf16"],
           "graph": "the benchmark graph" if sub_nel is None else
           f"{sub_nel}^3 elements p={wl['p']}, {wl['parts']} RCB sub-graphs ({L ** 3:,} nodes, {e_unpart:,} edges): "
           "the plain path keeps FP32 per-edge activations ([E x 3H] input alone 105 GB at 32^3), which do not "
           "fit the full graph", "timing": "eager steps, median"}
    tf, sms = measure_fp32_peak()
    out["simt_peak"] = {"tflops": tf, "sm_count": sms,
                        "src": "measured: the library's FP32 FMA kernel (gnn_measure_fp32_fma)"}
    if sgemm is not None:
        fl, ms_k = sgemm
        out["sgemm"] = {"tflops": fl / (ms_k * 1e-3) / 1e12, "frac": fl / (ms_k * 1e-3) / 1e12 / tf,
                        "ms_per_step": ms_k, "note": "the plain path's k_sgemm launches of one step (forward, "
                                                     "recompute, input and weight gradients) over the SIMT peak"}
    return out


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
    n_lin = wl.get("nh", NH) + 2
    fwd_only = wl["mode"] == "fwd" or args.mode == "fwd"
    if fwd_only:
        wl["mode"] = "fwd"
    use_graph = wl["graph"] and not args.eager
    part, n_el, n_unpart, e_unpart = workload_graph(wl, args.nel)
    G, net, stack, dx_top, u, t = build_problem(dev, precision, wl, part, save_act=args.save_act)
    saved_act = any(a is not None for a in stack.act)
    tune = None
    if (args.autotune or wl.get("uneven")) and precision == "bf16":
        tune = stack.autotune(dx_top)
        tune = {k: v for k, v in tune.items() if k != "candidates"} | {
            "candidates": [{k: v for k, v in c.items() if k != "fwd_choices"} for c in tune.get("candidates", [])]}
    peaks = load_peaks()
    stream = torch.cuda.current_stream()
    run = prepare_timing(stack, dx_top, args.warmup, use_graph)
    barrier()
    with ClockSampler(local) as clk:
        times = time_steps(run, args.steps, stream)
    barrier()
    ms = max_over_ranks(statistics.median(times), dist, dev)
    ms_mean = max_over_ranks(statistics.mean(times), dist, dev)
    value = world * e_unpart * M / (ms * 1e-3)

    # the per-kernel table: separate eager steps with the event profiler on (not timed above)
    n_prof = 2
    report = _profiled(lambda: stack.step(dx_top), n_prof)
    launches_per_step = sum(n for n, _ in report.values()) / n_prof
    total_ms = sum(v for _, v in report.values()) or 1.0
    edge_bytes = 2 if precision == "bf16" else 4
    roof = step_roofline(ms, G.n_edges, G.n_rows, Hw, edge_bytes, n_lin, fwd_only, peaks,
                         last_layer_no_edge_out=fwd_only)
    traffic = measured_traffic(args.workload, list(report), G.n_edges) if not args.nel and not args.save_act else None
    roof["traffic"] = sum(traffic.values()) if traffic else None
    roof_kernel = None
    if report:
        top_name, (top_n, top_ms) = max(report.items(), key=lambda kv: kv[1][1])
        db = design_bytes(top_name, G, Hw, edge_bytes, last_layer_no_edge_out=fwd_only, n_lin=n_lin,
                          saved_act=saved_act)
        roof_kernel = {"kernel": top_name, "share": top_ms / total_ms, "launches_per_step": top_n / n_prof,
                       "ms_per_step": top_ms / n_prof}
        if db is not None:
            ach = db / (top_ms / n_prof * 1e-3) / 1e9
            roof_kernel.update({"bound": "hbm", "design_bytes_per_step": db, "achieved": ach,
                                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": ach / peaks["hbm_gbs"],
                                "traffic": traffic.get(top_name) if traffic else None,
                                "note": "bytes the kernel moves as designed (scratch and stored activations "
                                        "included), over its event-timed launches in profiled eager steps"})
        elif top_name == "k_sgemm":   # the FP32 bench: the SIMT GEMMs against the measured FP32 FMA peak
            tf, sms = measure_fp32_peak()
            flops = sgemm_flops_per_step(G, Hw, n_lin, M)
            ach = flops / (top_ms / n_prof * 1e-3) / 1e12
            roof_kernel.update({"bound": "alu", "achieved": ach, "peak": tf, "unit": "TFLOP/s", "frac": ach / tf,
                                "peak_src": f"measured: FP32 FMA kernel on {sms} SMs"})

    # the cost of consistency: the same stack with Eq. 5c-5d skipped (the paper's "None" layers)
    for c in (stack.cfg, stack.cfg_last):
        c.halo_mode = B.GNN_HALO_NONE
    stack.graph = None
    run_eager = prepare_timing(stack, dx_top, 1, graph=False)
    ms_none = statistics.median(time_steps(run_eager, max(3, args.steps // 4), stream))
    for c in (stack.cfg, stack.cfg_last):
        c.halo_mode = B.GNN_HALO_SYNC
    ms_sync = statistics.median(time_steps(run_eager, max(3, args.steps // 4), stream))
    inconsistent = {"ms_per_step": ms_none, "consistent_ms_per_step": ms_sync, "cost_of_consistency": ms_sync / ms_none,
                    "note": "same stack without the halo swap + sync (inconsistent layers) against the consistent "
                            "stack, eager steps, median"}

    saved = None
    if not saved_act and not fwd_only and precision == "bf16" and Hw <= 64 and args.workload in ("c2", "mixed", "large"):
        # the option: H <= 64 training with the MLP activations kept from the forward
        stack.save_act = True
        stack._alloc_act()
        if any(a is not None for a in stack.act):
            run_s = prepare_timing(stack, dx_top, 2, graph=False)
            ms_s = statistics.median(time_steps(run_s, max(3, args.steps // 4), stream))
            saved = {"value": e_unpart * M / (ms_s * 1e-3), "unit": "edges/s", "ms_per_step": ms_s,
                     "act_bytes_per_step": sum(a.numel() * 2 for a in stack.act),
                     "note": "option: MLP activations stored by the forward, only the last Linear recomputed "
                             "(eager steps, median)"}
        stack.save_act = False
        stack._alloc_act()

    del stack, run, run_eager
    torch.cuda.empty_cache()

    e2e = None
    if not args.no_e2e and wl["inputs"] == "encoders" and not fwd_only:
        torch.cuda.synchronize()
        ms_e, ms_e_mean, h2d, d2h, e2e_k = time_e2e(net, G, u, t, max(3, args.steps // 4), 2, dev)
        enc_path = "fused BF16 row MLPs"
        e2e = {"value": world * e_unpart * M / (ms_e * 1e-3), "unit": "edges/s", "ms_per_step": ms_e,
               "mean_ms_per_step": ms_e_mean, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "library_kernels_one_step": e2e_k,
               "step": f"encoders and decoder ({enc_path}) + 4 layers + consistent loss, fwd+bwd; node field and "
                       "target copied from pinned host memory each step, loss read back; eager steps, median"}
        net.zero_grad(set_to_none=True)
        torch.cuda.empty_cache()

    fp32 = None
    if precision == "bf16" and not args.no_fp32 and wl["inputs"] == "encoders" and not fwd_only:
        del G
        torch.cuda.empty_cache()
        fp32 = fp32_comparison(dev, wl, part, max(3, args.steps // 4), 2, ms)

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
        edge_state = part.n_edges * Hw * edge_bytes
        line = {"metric": f"MP-layer edges/s {kind}", "value": value, "unit": "edges/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "mean_ms_per_step": ms_mean,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": precision,
                "data": "synthetic",
                "config": {"workload": workload_config_text(wl, n_el, n_unpart, e_unpart, kind),
                           "name": args.workload, "inputs": wl["inputs"],
                           "rows": part.n_rows, "edges_partitioned": part.n_edges, "tile_edges": part.tile_edges,
                           "training_form": ("saved activations (option)" if saved_act else
                                             "per-layer recomputation of the MLP activations") if not fwd_only
                           else "inference",
                           "l2": f"inputs larger than L2 (edge state {edge_state / 1e6:.0f} MB), no flush",
                           "timing": ("median of K CUDA-graph replays" if use_graph else "median of K eager steps")
                           + ", each timed by CUDA events on the launching stream, profiler off",
                           "parallelism": f"replicas x{world}"},
                "nodes_per_s": world * n_unpart * M / (ms * 1e-3),
                "roofline": roof, "roofline_kernel": roof_kernel, "fp32": fp32, "e2e": e2e, "cpu_baseline": cpu,
                "inconsistent": inconsistent, "saved_activations": saved,
                "gpu_launches": int(round(launches_per_step * args.steps)),
                "kernels": {k: {"launches_per_step": n / n_prof, "ms_per_step": v / n_prof, "share": v / total_ms}
                            for k, (n, v) in report.items()},
                "clocks": clk.summary()}
        if tune is not None:
            line["autotune"] = tune
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
