"""PyTorch front end of libgnnmp: autograd Functions and the encode-process-decode network.

torch provides device memory, streams and autograd bookkeeping only; every
step of the network runs in libgnnmp's kernels through ``binding``:

* ``ConsistentMPFunction`` -- one consistent NMP layer (Eq. 5a-5e) with its
  hand-written adjoint (``gnn_mp_forward`` / ``gnn_mp_backward``), recomputing
  the layer's MLP activations in the backward pass instead of storing them
  (or, as an option, keeping them: ``gnn_mp_forward_act`` / ``_backward_act``);
* ``RowMLPFunction`` -- node/edge encoders and the node decoder (Sec. III);
* ``ConsistentLossFunction`` -- the consistent MSE loss, Eq. 8a-8c;
* ``ConsistentGNN`` -- encoders, M consistent layers, decoder (Sec. III).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import binding as B
from .graph import DeviceGraph

PRECISIONS = {"fp32": B.GNN_PREC_FP32, "bf16": B.GNN_PREC_BF16}


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def mlp_struct(dims, tensors, has_ln: bool) -> B.gnn_mlp:
    """gnn_mlp view of tensors ordered [W_0..W_{n-1}, b_0..b_{n-1}, (gamma, beta)]."""
    n = len(dims) - 1
    s = B.gnn_mlp()
    s.n_lin = n
    for k, d in enumerate(dims):
        s.dims[k] = int(d)
    for k in range(n):
        s.W[k] = B.ptr(tensors[k])
        s.b[k] = B.ptr(tensors[n + k])
    if has_ln:
        s.gamma = B.ptr(tensors[2 * n])
        s.beta = B.ptr(tensors[2 * n + 1])
    return s


def n_mlp_tensors(dims, has_ln: bool) -> int:
    return 2 * (len(dims) - 1) + (2 if has_ln else 0)


def mp_config(hidden: int, precision: str, halo: bool = True, ln_eps: float = 1e-5, flags: int = 0):
    c = B.gnn_mp_config()
    c.hidden = int(hidden)
    c.precision = PRECISIONS[precision]
    c.halo_mode = B.GNN_HALO_SYNC if halo else B.GNN_HALO_NONE
    c.flags = int(flags)
    c.ln_eps = float(ln_eps)
    return c


def mp_params(edge_dims, node_dims, tensors) -> B.gnn_mp_params:
    ne = n_mlp_tensors(edge_dims, True)
    p = B.gnn_mp_params()
    p.edge = mlp_struct(edge_dims, tensors[:ne], True)
    p.node = mlp_struct(node_dims, tensors[ne:], True)
    return p


def workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def mp_workspace_sizes(G: DeviceGraph, cfg, W) -> tuple:
    f, b = C.c_size_t(), C.c_size_t()
    B.call("gnn_mp_workspace_size", C.byref(G.struct), C.byref(cfg), C.byref(W), C.byref(f), C.byref(b))
    return int(f.value), int(b.value)


def mp_act_bytes(G: DeviceGraph, cfg, W) -> int:
    """Bytes of the saved MLP activations of gnn_mp_forward_act (0: the backward recomputes)."""
    n = C.c_size_t()
    B.call("gnn_mp_act_size", C.byref(G.struct), C.byref(cfg), C.byref(W), C.byref(n))
    return int(n.value)


def act_buffer(G: DeviceGraph, cfg, W, device):
    """A buffer for the saved MLP activations of one layer, or None where none are kept."""
    n = mp_act_bytes(G, cfg, W)
    return torch.empty(n // 2, dtype=torch.bfloat16, device=device) if n else None


def gnn_mp_forward(G: DeviceGraph, cfg, W, x, e, x_out, e_out, a_star=None, ws=None, act=None):
    """Direct call of gnn_mp_forward (gnn_mp_forward_act when ``act`` is given,
    which also stores the MLP activations) on preallocated tensors (no autograd)."""
    if ws is None:
        ws = workspace(mp_workspace_sizes(G, cfg, W)[0], x.device)
    if act is not None:
        B.call("gnn_mp_forward_act", C.byref(G.struct), C.byref(cfg), C.byref(W), B.ptr(x), B.ptr(e), B.ptr(x_out),
               B.ptr(e_out), B.ptr(a_star), B.ptr(act), B.ptr(ws), ws.numel(), _stream())
        return
    B.call("gnn_mp_forward", C.byref(G.struct), C.byref(cfg), C.byref(W), B.ptr(x), B.ptr(e), B.ptr(x_out),
           B.ptr(e_out), B.ptr(a_star), B.ptr(ws), ws.numel(), _stream())


def gnn_mp_backward(G: DeviceGraph, cfg, W, x, e, a_star, dx_out, de_out, dx_in, de_in, dW, ws=None, act=None):
    """Direct call of gnn_mp_backward (gnn_mp_backward_act with the forward's
    saved ``act``) on preallocated tensors; dW accumulates."""
    if ws is None:
        ws = workspace(mp_workspace_sizes(G, cfg, W)[1], x.device)
    if act is not None:
        B.call("gnn_mp_backward_act", C.byref(G.struct), C.byref(cfg), C.byref(W), B.ptr(x), B.ptr(e),
               B.ptr(a_star), B.ptr(act), B.ptr(dx_out), B.ptr(de_out), B.ptr(dx_in), B.ptr(de_in), C.byref(dW),
               B.ptr(ws), ws.numel(), _stream())
        return
    B.call("gnn_mp_backward", C.byref(G.struct), C.byref(cfg), C.byref(W), B.ptr(x), B.ptr(e), B.ptr(a_star),
           B.ptr(dx_out), B.ptr(de_out), B.ptr(dx_in), B.ptr(de_in), C.byref(dW), B.ptr(ws), ws.numel(),
           _stream())


def gnn_halo_exchange(G: DeviceGraph, rows: torch.Tensor) -> None:
    B.call("gnn_halo_exchange", C.byref(G.struct), B.ptr(rows), int(rows.shape[1]), _stream())


class ConsistentMPFunction(torch.autograd.Function):
    """One consistent NMP layer, Eq. 5a-5e, with the hand-written adjoint (Eq. 3).
    The backward recomputes the MLP activations; with ``save`` they are kept
    from the forward instead where the library supports it
    (gnn_mp_forward_act / gnn_mp_backward_act, H <= 64)."""

    @staticmethod
    def forward(ctx, x, e, G, cfg_args, edge_dims, node_dims, save, *params):
        cfg = mp_config(*cfg_args)
        W = mp_params(edge_dims, node_dims, params)
        fwd, _ = mp_workspace_sizes(G, cfg, W)
        x = x.contiguous()
        e = e.contiguous()
        x_out = torch.empty_like(x)
        e_out = torch.empty_like(e)
        a_star = torch.empty_like(x)
        act = act_buffer(G, cfg, W, x.device) if save else None
        gnn_mp_forward(G, cfg, W, x, e, x_out, e_out, a_star, workspace(fwd, x.device), act)
        ctx.act = act
        ctx.G, ctx.cfg_args, ctx.dims = G, cfg_args, (edge_dims, node_dims)
        ctx.save_for_backward(x, e, a_star, *params)
        return x_out, e_out

    @staticmethod
    def backward(ctx, dx_out, de_out):
        x, e, a_star, *params = ctx.saved_tensors
        G = ctx.G
        cfg = mp_config(*ctx.cfg_args)
        W = mp_params(*ctx.dims, params)
        dparams = [torch.zeros_like(p) for p in params]
        dW = mp_params(*ctx.dims, dparams)
        _, bwd = mp_workspace_sizes(G, cfg, W)
        dx = torch.empty_like(x)
        de = torch.empty_like(e)
        dx_out = torch.zeros_like(x) if dx_out is None else dx_out.contiguous()
        de_out = None if de_out is None else de_out.to(e.dtype).contiguous()
        gnn_mp_backward(G, cfg, W, x, e, a_star, dx_out, de_out, dx, de, dW, workspace(bwd, x.device), ctx.act)
        ctx.act = None
        return (dx, de, None, None, None, None, None, *dparams)


def rowmlp_fused_shape(dims, has_ln: bool) -> bool:
    """True when the fused BF16 row MLP covers this block (gnn_mlp_forward_bf16):
    hidden widths H in {16, 32, 64}, an encoder (in <= 16, out H, LayerNorm) or a
    decoder (in H, out <= 16, no LayerNorm); at H = 128 either with 2 to 4
    Linear layers."""
    H = dims[1]
    if len(dims) < 3 or H not in (16, 32, 64, 128) or any(d != H for d in dims[1:-1]):
        return False
    if H == 128 and len(dims) > 5:
        return False
    if has_ln:
        return dims[0] <= 16 and dims[-1] == H
    return dims[0] == H and dims[-1] <= 16


class RowMLPFunction(torch.autograd.Function):
    """Row-wise MLP block (encoders, decoder): the fused BF16 kernels when
    ``fused`` and the shape is covered, else the plain FP32 kernels."""

    @staticmethod
    def forward(ctx, X, dims, has_ln, out_bf16, ln_eps, need_dx, fused, save, *params):
        P = mlp_struct(dims, params, has_ln)
        f, b = C.c_size_t(), C.c_size_t()
        rows = X.shape[0]
        fused = bool(fused) and rowmlp_fused_shape(dims, has_ln)
        sfx = "_bf16" if fused else ""
        B.call("gnn_mlp_workspace_size" + sfx, C.byref(P), rows, C.byref(f), C.byref(b))
        X = X.contiguous()
        Y = torch.empty((rows, dims[-1]), dtype=torch.bfloat16 if out_bf16 else torch.float32, device=X.device)
        act = None
        if fused and save:   # keep the activations for the backward (training)
            n = C.c_size_t()
            B.call("gnn_mlp_act_size_bf16", C.byref(P), rows, C.byref(n))
            act = torch.empty(int(n.value) // 2, dtype=torch.bfloat16, device=X.device) if n.value else None
        if act is not None:
            B.call("gnn_mlp_forward_bf16_act", C.byref(P), rows, B.ptr(X), B.ptr(Y), int(out_bf16), float(ln_eps),
                   B.ptr(act), _stream())
        else:
            ws = workspace(f.value, X.device)
            B.call("gnn_mlp_forward" + sfx, C.byref(P), rows, B.ptr(X), B.ptr(Y), int(out_bf16), float(ln_eps),
                   B.ptr(ws), ws.numel(), _stream())
        ctx.act = act
        ctx.meta = (dims, has_ln, out_bf16, ln_eps, need_dx, int(b.value), sfx)
        ctx.save_for_backward(X, *params)
        return Y

    @staticmethod
    def backward(ctx, dY):
        X, *params = ctx.saved_tensors
        dims, has_ln, out_bf16, ln_eps, need_dx, bwd, sfx = ctx.meta
        P = mlp_struct(dims, params, has_ln)
        dparams = [torch.zeros_like(p) for p in params]
        dP = mlp_struct(dims, dparams, has_ln)
        dY = dY.to(torch.bfloat16 if out_bf16 else torch.float32).contiguous()
        dX = torch.empty_like(X) if need_dx else None
        ws = workspace(bwd, X.device)
        if ctx.act is not None:
            B.call("gnn_mlp_backward_bf16_act", C.byref(P), X.shape[0], B.ptr(X), B.ptr(dY), int(out_bf16),
                   B.ptr(dX), C.byref(dP), float(ln_eps), B.ptr(ctx.act), B.ptr(ws), ws.numel(), _stream())
            ctx.act = None
        else:
            B.call("gnn_mlp_backward" + sfx, C.byref(P), X.shape[0], B.ptr(X), B.ptr(dY), int(out_bf16), B.ptr(dX),
                   C.byref(dP), float(ln_eps), B.ptr(ws), ws.numel(), _stream())
        return (dX, None, None, None, None, None, None, None, *dparams)


class ConsistentLossFunction(torch.autograd.Function):
    """Consistent MSE loss, Eq. 8a-8c (1/d_i-weighted, N_eff-normalised)."""

    @staticmethod
    def forward(ctx, y, t, G):
        y = y.contiguous()
        t = t.contiguous()
        loss = torch.empty((), dtype=torch.float32, device=y.device)
        dy = torch.empty_like(y)
        ws = workspace(1 << 16, y.device)
        B.call("gnn_consistent_loss", C.byref(G.struct), B.ptr(y), B.ptr(t), int(y.shape[1]), B.ptr(loss),
               B.ptr(dy), B.ptr(ws), ws.numel(), _stream())
        ctx.save_for_backward(dy)
        return loss

    @staticmethod
    def backward(ctx, g):
        (dy,) = ctx.saved_tensors
        return dy * g, None, None


def consistent_loss(y, t, G: DeviceGraph):
    return ConsistentLossFunction.apply(y, t, G)


class _MLP(torch.nn.Module):
    def __init__(self, P: dict, device):
        super().__init__()
        self.dims = [P["W"][0].shape[1]] + [w.shape[0] for w in P["W"]]
        self.has_ln = "gamma" in P
        ts = [*P["W"], *P["b"]] + ([P["gamma"], P["beta"]] if self.has_ln else [])
        self.params = torch.nn.ParameterList(
            [torch.nn.Parameter(torch.as_tensor(np.asarray(t), dtype=torch.float32, device=device).contiguous())
             for t in ts])

    def tensors(self):
        return list(self.params)


def gnn_mp_autotune(G: DeviceGraph, cfg, W, x, e, x_out, e_out, a_star=None, ws=None, reps: int = 5):
    """Native autotuner of the edge forward's launch choice on this graph (see
    gnn_mp_autotune in gnnmp.h). Updates ``cfg`` in place; returns the timings
    as [(edge_fwd_kernel, ctas_per_sm, ms)]."""
    if ws is None:
        ws = workspace(mp_workspace_sizes(G, cfg, W)[0], x.device)
    out = (B.gnn_tune_entry * 8)()
    n = C.c_int32()
    B.call("gnn_mp_autotune", C.byref(G.struct), C.byref(cfg), C.byref(W), B.ptr(x), B.ptr(e), B.ptr(x_out),
           B.ptr(e_out), B.ptr(a_star), B.ptr(ws), ws.numel(), int(reps), out, 8, C.byref(n), _stream())
    return [(int(out[i].edge_fwd_kernel), int(out[i].ctas_per_sm), float(out[i].ms)) for i in range(n.value)]


_TUNED: dict = {}


class LayerStack:
    """M consistent NMP layers on preallocated buffers: a training step
    (forward then backward) or, with ``inference=True``, the forward alone.

    Every buffer (node/edge states, saved a*, gradients, workspace) is
    allocated once, so ``step`` / ``forward`` issue library calls only and can
    be captured in a CUDA graph (``capture``). ``layers`` is a list of
    (edge tensors, node tensors, edge dims, node dims) per layer; gradients
    accumulate into ``dparams`` (zeroed by ``zero_grad``).

    Inference keeps the inputs and two edge-state and two node-state buffers
    (ping-pong) and skips the last layer's edge-state write (GNN_FLAG_NO_EDGE_OUT): only the
    aggregates reach the node update, so no per-edge output of the last layer
    touches HBM. Training keeps every layer's input states and a* and two
    node- and two edge-gradient buffers (ping-pong: layer l writes dx[l % 2],
    de[l % 2]; dx[0] ends as dL/dx0); the backward recomputes each layer's MLP
    activations from them. ``save_act=True`` (an option at H <= 64) keeps the
    MLPs' activations from the forward instead, so the backward recomputes only
    the last Linear of each MLP, at the price of 2H(L-1) bytes per edge and
    per row for every layer; the forward then always uses the record-tiled
    edge kernel (the autotuner's choice of forward kernel then only affects
    ``forward`` of an inference stack)."""

    def __init__(self, G: DeviceGraph, layers, hidden: int, precision: str, x0, e0, halo: bool = True,
                 ln_eps: float = 1e-5, inference: bool = False, save_act: bool = False):
        self.G = G
        self.M = len(layers)
        self.hidden = hidden
        self.precision = precision
        self.inference = inference
        self.cfg = mp_config(hidden, precision, halo, ln_eps)
        self.cfg_last = mp_config(hidden, precision, halo, ln_eps, B.GNN_FLAG_NO_EDGE_OUT if inference else 0)
        dev = x0.device
        edt = torch.bfloat16 if precision == "bf16" else torch.float32
        self.W, self.dW, self.dparams = [], [], []
        for (te, tn, de, dn) in layers:
            tens = list(te) + list(tn)
            self.W.append(mp_params(de, dn, tens))
            if not inference:
                dp = [torch.zeros_like(t) for t in tens]
                self.dparams.append(dp)
                self.dW.append(mp_params(de, dn, dp))
        self._keep = [layers]
        NR, E = G.n_rows, G.n_edges
        if inference:
            self.x = [x0.contiguous(), torch.empty(NR, hidden, device=dev), torch.empty(NR, hidden, device=dev)]
            self.e = [e0.to(edt).contiguous()] + [torch.empty(E, hidden, device=dev, dtype=edt)
                                                  for _ in range(min(2, self.M - 1))]
            self.a = []
        else:
            self.x = [x0.contiguous()] + [torch.empty(NR, hidden, device=dev) for _ in range(self.M)]
            self.e = [e0.to(edt).contiguous()] + [torch.empty(E, hidden, device=dev, dtype=edt)
                                                  for _ in range(self.M)]
            self.a = [torch.empty(NR, hidden, device=dev) for _ in range(self.M)]
            self.dx = [torch.empty(NR, hidden, device=dev) for _ in range(2)]
            self.de = [torch.empty(E, hidden, device=dev, dtype=edt) for _ in range(min(2, self.M))]
        self.save_act = not inference and save_act
        self._alloc_act()
        f, b = mp_workspace_sizes(G, self.cfg, self.W[0])
        self.ws = workspace(f if inference else max(f, b), dev)
        self.graph = None

    def _alloc_act(self):
        # the saved activations come in whole edge tiles: their size follows the tiling
        self.act = [None] * self.M   # (frees the old buffers first)
        if self.save_act:
            self.act = [act_buffer(self.G, self.cfg, self.W[l], self.x[0].device) for l in range(self.M)]
        self._act_tiles = int(self.G.struct.n_edge_tiles)

    # buffers of layer l: inputs, outputs, saved a* (ping-pong in inference)
    def _io(self, l: int):
        if not self.inference:
            return self.x[l], self.e[l], self.x[l + 1], self.e[l + 1], self.a[l]
        xi = self.x[0] if l == 0 else self.x[1 + (l - 1) % 2]
        xo = self.x[1 + l % 2]
        ei = self.e[0] if l == 0 else self.e[1 + (l - 1) % 2]
        eo = None if l == self.M - 1 else self.e[1 + l % 2]
        return xi, ei, xo, eo, None

    @property
    def x_out(self):
        return self._io(self.M - 1)[2]

    def zero_grad(self):
        for dp in self.dparams:
            for t in dp:
                t.zero_()

    def forward(self):
        if self._act_tiles != int(self.G.struct.n_edge_tiles):
            self._alloc_act()
        for l in range(self.M):
            xi, ei, xo, eo, a = self._io(l)
            cfg = self.cfg_last if l == self.M - 1 else self.cfg
            gnn_mp_forward(self.G, cfg, self.W[l], xi, ei, xo, eo, a, self.ws, self.act[l])

    def backward(self, dx_top):
        """dx_top: dL/dx of the last layer's output; dL/de of it is zero."""
        assert not self.inference, "an inference stack has no backward"
        dx_out, de_out = dx_top, None
        for l in range(self.M - 1, -1, -1):
            dx_in, de_in = self.dx[l % 2], self.de[l % 2]
            gnn_mp_backward(self.G, self.cfg, self.W[l], self.x[l], self.e[l], self.a[l], dx_out, de_out,
                            dx_in, de_in, self.dW[l], self.ws, self.act[l])
            dx_out, de_out = dx_in, de_in

    def step(self, dx_top=None):
        if self.inference:
            self.forward()
        else:
            self.forward()
            self.backward(dx_top)

    # ------------------------------------------------------------------ CUDA graph
    def capture(self, dx_top=None, warmup: int = 2) -> torch.cuda.CUDAGraph:
        """Capture one ``step`` into a CUDA graph (replay with ``replay``). The
        launch choices and tiles in force now are frozen into the graph."""
        s = torch.cuda.Stream(device=self.ws.device)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(warmup):   # first calls look up device attributes outside the capture
                self.step(dx_top)
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, capture_error_mode="thread_local"):
            self.step(dx_top)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    # ------------------------------------------------------------------ autotuning
    def autotune(self, dx_top=None, tile_caps=(128, 96, 64, 32), reps: int = 3, cache_file: str | None = None):
        """Choose the edge-tile cap (gnn_partition_set_tile_edges) and the edge
        forward's launch choice (gnn_mp_autotune) for this graph by timing:
        for every cap, the native tuner picks the launch choice, then a whole
        ``step`` is timed; the fastest (cap, choice) is kept. Results are
        cached per (device, H, layer shapes, precision, graph size, mode), in
        memory and in ``cache_file`` (JSON) when given. Returns the report."""
        import json
        import os

        if self.precision != "bf16":
            return {"tuned": False, "reason": "the FP32 path has no launch choices"}
        dev = self.ws.device
        key = "|".join(str(v) for v in (torch.cuda.get_device_name(dev), self.hidden, self.W[0].edge.n_lin,
                                          self.W[0].node.n_lin, self.precision, self.G.n_rows, self.G.n_edges,
                                          "inf" if self.inference else "train"))
        cache = dict(_TUNED)
        if cache_file and os.path.exists(cache_file):
            with open(cache_file) as fh:
                cache.update(json.load(fh))
        if key in cache:
            r = cache[key]
            self._apply(r["tile_edges"], r["edge_fwd_kernel"], r["ctas_per_sm"])
            return dict(r, cached=True)
        xi, ei, xo, eo, a = self._io(0)
        scratch_e = eo if eo is not None else torch.empty_like(ei)
        rows = []
        caps = [c for c in tile_caps if self.G.part.info.max_in_degree <= c <= B.GNN_EDGE_TILE]
        for cap in caps:
            self.G.retile(cap)
            cfg = mp_config(self.hidden, self.precision, self.cfg.halo_mode == B.GNN_HALO_SYNC, self.cfg.ln_eps)
            timings = gnn_mp_autotune(self.G, cfg, self.W[0], xi, ei, xo, scratch_e, a, self.ws, reps)
            self._apply(cap, cfg.edge_fwd_kernel, cfg.ctas_per_sm)
            self.step(dx_top)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                self.step(dx_top)
            e1.record()
            torch.cuda.synchronize()
            rows.append({"tile_edges": cap, "edge_fwd_kernel": cfg.edge_fwd_kernel, "ctas_per_sm": cfg.ctas_per_sm,
                         "step_ms": e0.elapsed_time(e1) / reps, "fwd_choices": timings})
        best = min(rows, key=lambda r: r["step_ms"])
        self._apply(best["tile_edges"], best["edge_fwd_kernel"], best["ctas_per_sm"])
        self.zero_grad()
        res = {"tile_edges": best["tile_edges"], "edge_fwd_kernel": best["edge_fwd_kernel"],
               "ctas_per_sm": best["ctas_per_sm"], "step_ms": best["step_ms"], "candidates": rows}
        _TUNED[key] = res
        if cache_file:
            cache[key] = res
            with open(cache_file, "w") as fh:
                json.dump(cache, fh, indent=1)
        return dict(res, cached=False)

    def _apply(self, tile_edges: int, kernel: int, ctas_per_sm: int):
        if self.G.tile_edges != tile_edges:
            self.G.retile(tile_edges)
        for c in (self.cfg, self.cfg_last):
            c.edge_fwd_kernel = int(kernel)
            c.ctas_per_sm = int(ctas_per_sm)
        self.graph = None


class ConsistentGNN(torch.nn.Module):
    """Encode-process-decode GNN with consistent NMP layers (Sec. III).

    ``params`` is the nested dict of arrays made by ``synthetic.gnn_params``
    (float64 arrays are cast to FP32 master weights). Training recomputes each
    layer's MLP activations in the backward; ``save_act=True`` keeps them from
    the forward where the library supports it (H <= 64)."""

    def __init__(self, params: dict, precision: str = "bf16", halo: bool = True, ln_eps: float = 1e-5,
                 device="cuda", save_act: bool = False):
        super().__init__()
        self.precision = precision
        self.save_act = save_act
        self.halo = halo
        self.ln_eps = ln_eps
        self.enc_node = _MLP(params["enc_node"], device)
        self.enc_edge = _MLP(params["enc_edge"], device)
        self.layers = torch.nn.ModuleList()
        for lp in params["layers"]:
            m = torch.nn.Module()
            m.edge = _MLP(lp["edge"], device)
            m.node = _MLP(lp["node"], device)
            self.layers.append(m)
        self.dec = _MLP(params["dec"], device)
        self.hidden = self.enc_node.dims[-1]

    def _row_mlp(self, m: _MLP, X, out_bf16: bool, need_dx: bool):
        return RowMLPFunction.apply(X, m.dims, m.has_ln, out_bf16, self.ln_eps, need_dx, self.precision == "bf16",
                                    torch.is_grad_enabled() and self.save_act, *m.tensors())

    def encode(self, G: DeviceGraph, u, attr):
        x = self._row_mlp(self.enc_node, u, False, False)
        e = self._row_mlp(self.enc_edge, attr, self.precision == "bf16", False)
        return x, e

    def process(self, G: DeviceGraph, x, e):
        cfg_args = (self.hidden, self.precision, self.halo, self.ln_eps, 0)
        for layer in self.layers:
            x, e = ConsistentMPFunction.apply(x, e, G, cfg_args, layer.edge.dims, layer.node.dims,
                                              torch.is_grad_enabled() and self.save_act,
                                              *layer.edge.tensors(), *layer.node.tensors())
        return x, e

    def forward(self, G: DeviceGraph, u, attr):
        x, e = self.encode(G, u, attr)
        x, e = self.process(G, x, e)
        return self._row_mlp(self.dec, x, False, True)

    def grads_numpy(self) -> dict:
        """Parameter gradients in the nested-dict layout of ``synthetic.gnn_params``."""
        def mlp(m: _MLP):
            n = len(m.dims) - 1
            g = [p.grad.double().cpu().numpy() if p.grad is not None else np.zeros(p.shape) for p in m.params]
            out = {"W": g[:n], "b": g[n:2 * n]}
            if m.has_ln:
                out["gamma"], out["beta"] = g[2 * n], g[2 * n + 1]
            return out
        return {"enc_node": mlp(self.enc_node), "enc_edge": mlp(self.enc_edge),
                "layers": [{"edge": mlp(l.edge), "node": mlp(l.node)} for l in self.layers],
                "dec": mlp(self.dec)}
