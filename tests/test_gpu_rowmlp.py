"""The fused BF16 row MLP (encoders and decoder of the network, Sec. III)
against the FP64 oracle's MLP and the plain FP32 path (needs a GB300).

Tolerances as for the layer: 2e-2 relative L2 on outputs, 5e-2 on gradients.
Row counts are ragged (not multiples of the 128-row tile) and span many CTAs."""
import ctypes

import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import model as om
from paper_2410_01657_gb300 import _build
from paper_2410_01657_gb300 import binding as B
from paper_2410_01657_gb300 import nn as gnn

from gpu_util import rel_l2

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    B.load()


def _mlp_params(dims, has_ln, seed):
    rng = np.random.default_rng(seed)
    W = [rng.uniform(-1, 1, (dims[k + 1], dims[k])) * np.sqrt(6.0 / (dims[k] + dims[k + 1]))
         for k in range(len(dims) - 1)]
    b = [0.1 * rng.standard_normal(dims[k + 1]) for k in range(len(dims) - 1)]
    P = {"W": W, "b": b}
    if has_ln:
        P["gamma"] = 1.0 + 0.1 * rng.standard_normal(dims[-1])
        P["beta"] = 0.1 * rng.standard_normal(dims[-1])
    return P


def _run(P, dims, has_ln, X, dY, fused, out_bf16=False, need_dx=False, save=False):
    ts = [torch.nn.Parameter(torch.as_tensor(t, dtype=torch.float32, device=DEV))
          for t in [*P["W"], *P["b"]] + ([P["gamma"], P["beta"]] if has_ln else [])]
    Xt = torch.as_tensor(X, dtype=torch.float32, device=DEV).requires_grad_(need_dx)
    Y = gnn.RowMLPFunction.apply(Xt, dims, has_ln, out_bf16, 1e-5, need_dx, fused, save, *ts)
    Y.backward(torch.as_tensor(dY, dtype=torch.float32, device=DEV).to(Y.dtype))
    B.call("gnn_check", None)
    n = len(dims) - 1
    g = {"W": [t.grad.double().cpu().numpy() for t in ts[:n]], "b": [t.grad.double().cpu().numpy() for t in ts[n:2 * n]]}
    if has_ln:
        g["gamma"], g["beta"] = ts[2 * n].grad.double().cpu().numpy(), ts[2 * n + 1].grad.double().cpu().numpy()
    dx = Xt.grad.double().cpu().numpy() if need_dx else None
    return Y.detach().float().cpu().numpy(), g, dx


def _check(P, dims, has_ln, rows, seed, out_bf16=False, need_dx=False):
    assert gnn.rowmlp_fused_shape(dims, has_ln)
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((rows, dims[0]))
    dY = rng.standard_normal((rows, dims[-1]))
    Yo, cache = om.mlp_forward(P, X)
    dXo, go = om.mlp_backward(P, cache, dY)
    Yf, gf, dxf = _run(P, dims, has_ln, X, dY, True, out_bf16, need_dx)
    Yp, gp, dxp = _run(P, dims, has_ln, X, dY, False, False, need_dx)
    assert rel_l2(Yp, Yo) < 1e-5                      # the plain FP32 reference itself
    assert rel_l2(Yf, Yo) < 2e-2 and rel_l2(Yf, Yp) < 2e-2
    # with saved activations (gnn_mlp_*_bf16_act): the same forward, and the adjoint of the
    # recomputing kernels to FP32 rounding
    Ys, gs, dxs = _run(P, dims, has_ln, X, dY, True, out_bf16, need_dx, save=True)
    assert np.array_equal(Ys, Yf)
    for key in gf:
        for a, ref in zip(gs[key] if isinstance(gs[key], list) else [gs[key]],
                          gf[key] if isinstance(gf[key], list) else [gf[key]]):
            assert rel_l2(a, ref) < 1e-6, (key, rel_l2(a, ref))
    if need_dx:
        assert rel_l2(dxs, dxf) < 1e-6
    for key in gf:
        for a, ref in zip(gf[key] if isinstance(gf[key], list) else [gf[key]],
                          go[key] if isinstance(go[key], list) else [go[key]]):
            assert rel_l2(a, ref) < 5e-2, (key, rel_l2(a, ref))
    if need_dx:
        assert rel_l2(dxf, dXo) < 5e-2


@pytest.mark.parametrize("H", [16, 32, 64])
@pytest.mark.parametrize("n_in,n_hidden", [(3, 2), (4, 2), (4, 0)])
def test_encoder(H, n_in, n_hidden):
    dims = [n_in] + [H] * (n_hidden + 2)
    _check(_mlp_params(dims, True, H + n_in + n_hidden), dims, True, 5003, 7, out_bf16=(n_in == 4))


@pytest.mark.parametrize("H", [16, 32, 64])
@pytest.mark.parametrize("n_hidden", [0, 2])
def test_decoder(H, n_hidden):
    dims = [H] * (n_hidden + 2) + [3]
    _check(_mlp_params(dims, False, H + n_hidden), dims, False, 5003, 8, need_dx=True)


def test_encoder_many_tiles_and_deterministic():
    dims = [4, 64, 64, 64, 64]
    P = _mlp_params(dims, True, 3)
    _check(P, dims, True, 200001, 9)
    rng = np.random.default_rng(10)
    X = rng.standard_normal((70001, 4))
    dY = rng.standard_normal((70001, 64))
    a = _run(P, dims, True, X, dY, True)
    b = _run(P, dims, True, X, dY, True)
    assert np.array_equal(a[0], b[0])
    for k in a[1]:
        for u, v in zip(a[1][k] if isinstance(a[1][k], list) else [a[1][k]],
                        b[1][k] if isinstance(b[1][k], list) else [b[1][k]]):
            assert np.array_equal(u, v)


@pytest.mark.parametrize("n_in,n_hidden,rows,out_bf16,need_dx", [
    (3, 2, 5003, False, False), (4, 2, 70001, True, True), (16, 0, 1000, False, True),
    (1, 1, 127, True, False), (5, 2, 1, False, True)])
def test_encoder_h128(n_in, n_hidden, rows, out_bf16, need_dx):
    # the H = 128 encoder (tensor-memory forward; layered adjoint with the
    # recomputed activations in the workspace): ragged row counts, one row, one tile
    dims = [n_in] + [128] * (n_hidden + 2)
    _check(_mlp_params(dims, True, 128 + n_in + n_hidden), dims, True, rows, 11, out_bf16=out_bf16,
           need_dx=need_dx)


@pytest.mark.parametrize("n_hidden,n_out,rows,need_dx", [
    (2, 3, 5003, True), (1, 16, 70001, True), (0, 1, 1000, False), (2, 5, 1, True)])
def test_decoder_h128(n_hidden, n_out, rows, need_dx):
    # the H = 128 decoder: N = 16 last Linear, its adjoint inside the recomputation,
    # the chain kernel's input pass for dX and dW_0
    dims = [128] * (n_hidden + 2) + [n_out]
    _check(_mlp_params(dims, False, 300 + n_hidden + n_out), dims, False, rows, 12, need_dx=need_dx)


@pytest.mark.parametrize("dims,has_ln", [([4, 128, 128, 128, 128], True), ([128, 128, 128, 128, 3], False)])
def test_row_mlp_h128_chunks_and_determinism(dims, has_ln):
    # A workspace smaller than the one reported runs the adjoint in several chunks
    # of tiles: the same gradients up to the order of the per-chunk sums; two runs
    # with the same workspace agree bit for bit; a workspace below one tile's scratch
    # is refused with GNN_ENOMEM; zero rows is a no-op.
    import ctypes as C

    rows = 200001
    n_in, n_out = dims[0], dims[-1]
    P = _mlp_params(dims, has_ln, 21)
    ts = [torch.as_tensor(t, dtype=torch.float32, device=DEV)
          for t in [*P["W"], *P["b"]] + ([P["gamma"], P["beta"]] if has_ln else [])]
    S = gnn.mlp_struct(dims, ts, has_ln)
    g = torch.Generator(device=DEV).manual_seed(3)
    X = torch.randn(rows, n_in, device=DEV, generator=g)
    dY = torch.randn(rows, n_out, device=DEV, generator=g).to(torch.bfloat16)
    stream = torch.cuda.current_stream().cuda_stream
    f, b = C.c_size_t(), C.c_size_t()
    B.call("gnn_mlp_workspace_size_bf16", C.byref(S), rows, C.byref(f), C.byref(b))

    def bwd(ws_bytes, n=rows):
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device=DEV)
        dts = [torch.zeros_like(t) for t in ts]
        dS = gnn.mlp_struct(dims, dts, has_ln)
        dX = torch.empty(n, n_in, device=DEV)
        B.call("gnn_mlp_backward_bf16", C.byref(S), n, B.ptr(X), B.ptr(dY), 1, B.ptr(dX), C.byref(dS), 1e-5,
               B.ptr(ws), ws_bytes, stream)
        B.call("gnn_check", None)
        return dX, dts

    dX, d1 = bwd(b.value)
    dXa, da = bwd(int(b.value * 0.3))
    dXb, db = bwd(int(b.value * 0.3))
    assert torch.equal(dXa, dX)                 # dX is per row: independent of the chunking
    for u, v, w in zip(d1, da, db):
        assert torch.equal(v, w)
        assert (v - u).norm() <= 1e-5 * u.norm()
    with pytest.raises(B.GnnError) as ei:
        bwd(1 << 20)
    assert ei.value.code == B.GNN_ENOMEM
    _, dz = bwd(b.value, 0)
    assert all(int(torch.count_nonzero(t)) == 0 for t in dz)


@pytest.mark.parametrize("dims,has_ln,rows", [
    ([4, 128, 128, 128, 128], True, 68_646_144),     # the C3 edge encoder's rows (partitioned edges)
    ([128, 128, 128, 128, 3], False, 11_543_176)])   # the C3 decoder's rows (partitioned node rows)
def test_row_mlp_h128_full_size_sampled(dims, has_ln, rows):
    # The fused H = 128 row MLP over the rows of the full C3 graph (the adjoint in
    # many chunks of the default workspace), checked on sampled rows: the outputs row
    # by row against the FP64 oracle, and the gradients by linearity in dY: with dY
    # zero except on the sampled rows, dW, db (and dgamma, dbeta) over all rows are
    # the oracle's gradients over the sampled rows alone, and dX is zero elsewhere.
    import ctypes as C

    n_in, n_out = dims[0], dims[-1]
    P = _mlp_params(dims, has_ln, 31)
    ts = [torch.as_tensor(t, dtype=torch.float32, device=DEV)
          for t in [*P["W"], *P["b"]] + ([P["gamma"], P["beta"]] if has_ln else [])]
    S = gnn.mlp_struct(dims, ts, has_ln)
    g = torch.Generator(device=DEV).manual_seed(7)
    X = torch.randn(rows, n_in, device=DEV, generator=g)
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(8)
    sample = np.unique(np.concatenate([rng.integers(0, rows, 1500), [0, rows - 1, 4_194_303, 4_194_304]]))
    sample = sample[sample < rows]
    bf = int(has_ln)   # the edge encoder's rows in BF16, as the network keeps them
    dt = torch.bfloat16 if bf else torch.float32
    Y = torch.empty(rows, n_out, device=DEV, dtype=dt)
    B.call("gnn_mlp_forward_bf16", C.byref(S), rows, B.ptr(X), B.ptr(Y), bf, 1e-5, None, 0, stream)
    Xs = X[torch.as_tensor(sample, device=DEV)].double().cpu().numpy()
    Yo, cache = om.mlp_forward(P, Xs)
    Ys = Y[torch.as_tensor(sample, device=DEV)].double().cpu().numpy()
    del Y
    # each row's error against the rows' RMS norm (a 3-wide decoder row can be near zero)
    err = np.linalg.norm(Ys - Yo, axis=1) / np.sqrt(np.mean(np.sum(Yo ** 2, axis=1)))
    assert err.max() < 3e-2 and np.sqrt(np.mean(err ** 2)) < 1e-2, (err.max(), np.sqrt(np.mean(err ** 2)))
    # gradients by linearity in dY
    dYs = rng.standard_normal((len(sample), n_out))
    dYs = torch.as_tensor(dYs, dtype=torch.float32).to(dt).double().numpy()   # as the kernel reads them
    dY = torch.zeros(rows, n_out, device=DEV, dtype=dt)
    dY[torch.as_tensor(sample, device=DEV)] = torch.as_tensor(dYs, device=DEV).to(dt)
    f, b = C.c_size_t(), C.c_size_t()
    B.call("gnn_mlp_workspace_size_bf16", C.byref(S), rows, C.byref(f), C.byref(b))
    ws = torch.empty(b.value, dtype=torch.uint8, device=DEV)
    dts = [torch.zeros_like(t) for t in ts]
    dS = gnn.mlp_struct(dims, dts, has_ln)
    dX = torch.empty(rows, n_in, device=DEV)
    B.call("gnn_mlp_backward_bf16", C.byref(S), rows, B.ptr(X), B.ptr(dY), bf, B.ptr(dX), C.byref(dS), 1e-5,
           B.ptr(ws), ws.numel(), stream)
    B.call("gnn_check", None)
    dXo, go = om.mlp_backward(P, cache, dYs)
    n = len(dims) - 1
    got = {"W": [t.double().cpu().numpy() for t in dts[:n]], "b": [t.double().cpu().numpy() for t in dts[n:2 * n]]}
    if has_ln:
        got["gamma"], got["beta"] = dts[2 * n].double().cpu().numpy(), dts[2 * n + 1].double().cpu().numpy()
    for key in got:
        for a, ref in zip(got[key] if isinstance(got[key], list) else [got[key]],
                          go[key] if isinstance(go[key], list) else [go[key]]):
            assert rel_l2(a, ref) < 5e-2, (key, rel_l2(a, ref))
    mask = torch.ones(rows, dtype=torch.bool, device=DEV)
    mask[torch.as_tensor(sample, device=DEV)] = False
    assert int(torch.count_nonzero(dX[mask])) == 0
    assert rel_l2(dX[torch.as_tensor(sample, device=DEV)].double().cpu().numpy(), dXo) < 5e-2


def test_uncovered_shape_is_rejected():
    dims = [8, 24, 24, 5]
    assert not gnn.rowmlp_fused_shape(dims, False)
    s = gnn.mlp_struct(dims, [torch.zeros(1, device=DEV)] * 6, False)
    f, b = ctypes.c_size_t(), ctypes.c_size_t()
    with pytest.raises(B.GnnError) as ei:
        B.call("gnn_mlp_workspace_size_bf16", ctypes.byref(s), 10, ctypes.byref(f), ctypes.byref(b))
    assert ei.value.code == B.GNN_EUNSUPPORTED


@pytest.mark.parametrize("dims,has_ln", [([4, 128, 128, 128, 128], True), ([128, 128, 128, 128, 3], False)])
def test_plain_row_mlp_runs_in_row_blocks(dims, has_ln):
    # The plain FP32 row MLP (the H = 128 encoders and decoder) runs over blocks of 2^22
    # rows with a workspace sized for one block. On 2^22 + 1,000,003 rows its outputs
    # must equal, bit for bit, two calls on the two row ranges, and its weight and input
    # gradients the sum of the two calls' (the blocks accumulate in row order).
    import ctypes as C

    n0, n1 = 1 << 22, 1_000_003
    rows = n0 + n1
    P = _mlp_params(dims, has_ln, 17)
    ts = [torch.as_tensor(t, dtype=torch.float32, device=DEV)
          for t in [*P["W"], *P["b"]] + ([P["gamma"], P["beta"]] if has_ln else [])]
    S = gnn.mlp_struct(dims, ts, has_ln)
    g = torch.Generator(device=DEV).manual_seed(5)
    X = torch.randn(rows, dims[0], device=DEV, generator=g)
    dY = torch.randn(rows, dims[-1], device=DEV, generator=g)
    stream = torch.cuda.current_stream().cuda_stream

    def fwd_bwd(lo, hi):
        n = hi - lo
        f, b = C.c_size_t(), C.c_size_t()
        B.call("gnn_mlp_workspace_size", C.byref(S), n, C.byref(f), C.byref(b))
        ws = gnn.workspace(max(f.value, b.value), DEV)
        Y = torch.empty(n, dims[-1], device=DEV)
        B.call("gnn_mlp_forward", C.byref(S), n, B.ptr(X[lo:hi]), B.ptr(Y), 0, 1e-5, B.ptr(ws), ws.numel(), stream)
        dts = [torch.zeros_like(t) for t in ts]
        dS = gnn.mlp_struct(dims, dts, has_ln)
        dX = torch.empty(n, dims[0], device=DEV)
        B.call("gnn_mlp_backward", C.byref(S), n, B.ptr(X[lo:hi]), B.ptr(dY[lo:hi]), 0, B.ptr(dX), C.byref(dS), 1e-5,
               B.ptr(ws), ws.numel(), stream)
        B.call("gnn_check", None)
        return Y, dX, dts, f.value

    Y, dX, dts, ws_all = fwd_bwd(0, rows)
    Ya, dXa, da, ws_a = fwd_bwd(0, n0)
    Yb, dXb, db, _ = fwd_bwd(n0, rows)
    assert ws_all == ws_a                      # the workspace covers one block
    assert torch.equal(Y[:n0], Ya) and torch.equal(Y[n0:], Yb)
    assert torch.equal(dX[:n0], dXa) and torch.equal(dX[n0:], dXb)
    for t, a, b in zip(dts, da, db):
        assert torch.equal(t, a + b)
