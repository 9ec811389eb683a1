"""Sizes of the saved activations of the training calls (CPU only: the size
queries read shapes, never device memory, so placeholder addresses serve).

gnn_mp_act_size: (L_e - 1) blocks of the edge tiles' rows (tiles * 128) plus
(L_n - 1) node blocks and the node MLP's [a*, x] rows (2H wide), rows rounded up
to whole 128-row tiles, BF16; 0 on the FP32 path, at H = 128 and for tilings
whose tiles would hold mostly padding (edge caps below 128).
gnn_mlp_act_size_bf16: (L - 1) blocks of whole 128-row tiles of H."""
import ctypes as C

import pytest

from paper_2410_01657_gb300 import _build
from paper_2410_01657_gb300 import binding as B
from paper_2410_01657_gb300.graph import MeshGraph

FAKE = 0x1000   # a 16-byte aligned placeholder address (never dereferenced)


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return B.load()


def _mlp(dims, ln):
    m = B.gnn_mlp()
    m.n_lin = len(dims) - 1
    for k, d in enumerate(dims):
        m.dims[k] = d
    for k in range(m.n_lin):
        m.W[k] = FAKE
        m.b[k] = FAKE
    if ln:
        m.gamma = FAKE
        m.beta = FAKE
    return m


def _graph_dev(part):
    g = B.gnn_graph_dev()
    g.n_rows, g.n_edges = part.n_rows, part.n_edges
    for f in ("row_ptr", "col", "edge_w", "t_ptr", "t_eid", "node_w", "halo_ptr", "halo_rows", "edge_tiles",
              "tile_meta"):
        setattr(g, f, FAKE)
    g.n_shared = int(part.info.n_shared)
    g.n_edge_tiles = int(part.info.n_edge_tiles)
    g.max_in_degree = int(part.info.max_in_degree)
    return g


def _act_size(lib, part, H, n_hidden, precision=B.GNN_PREC_BF16):
    cfg = B.gnn_mp_config()
    cfg.hidden, cfg.precision, cfg.ln_eps = H, precision, 1e-5
    W = B.gnn_mp_params()
    W.edge = _mlp([3 * H] + [H] * (n_hidden + 2), True)
    W.node = _mlp([2 * H] + [H] * (n_hidden + 2), True)
    n = C.c_size_t()
    assert lib.gnn_mp_act_size(C.byref(_graph_dev(part)), C.byref(cfg), C.byref(W), C.byref(n)) == B.GNN_OK
    return int(n.value)


@pytest.mark.parametrize("H,n_hidden", [(16, 2), (32, 5), (64, 2), (64, 0)])
def test_layer_activation_layout_size(lib, H, n_hidden):
    part = MeshGraph((5, 4, 3), 3).partition(4, "rcb")
    L = n_hidden + 2
    T = part.info.n_edge_tiles * 128
    R = (part.n_rows + 127) // 128 * 128
    assert _act_size(lib, part, H, n_hidden) == 2 * H * ((L - 1) * T + (L - 1) * R + 2 * R)


def test_no_saved_activations_where_the_backward_recomputes(lib):
    part = MeshGraph((5, 4, 3), 3).partition(4, "rcb")
    assert _act_size(lib, part, 64, 2, B.GNN_PREC_FP32) == 0
    assert _act_size(lib, part, 128, 2) == 0
    assert _act_size(lib, part, 64, 2) > 0
    part.set_tile_edges(64)   # tiles half full: the whole-tile layout would be mostly padding
    assert _act_size(lib, part, 64, 2) == 0
    part.set_tile_edges(B.GNN_EDGE_TILE)
    assert _act_size(lib, part, 64, 2) > 0


@pytest.mark.parametrize("dims,ln,H", [([4, 64, 64, 64, 64], True, 64), ([3, 32, 32, 32], True, 32),
                                       ([64, 64, 64, 64, 3], False, 64), ([16, 16, 16], False, 16)])
def test_row_mlp_activation_size(lib, dims, ln, H):
    m = _mlp(dims, ln)
    n = C.c_size_t()
    for rows in (1, 127, 128, 5003):
        assert lib.gnn_mlp_act_size_bf16(C.byref(m), rows, C.byref(n)) == B.GNN_OK
        assert n.value == (len(dims) - 2) * ((rows + 127) // 128 * 128) * H * 2
    assert lib.gnn_mlp_act_size_bf16(C.byref(m), 0, C.byref(n)) == B.GNN_OK and n.value == 0
    # a shape outside the fused row MLP keeps no activations
    wide = _mlp([4, 48, 48, 48], True)
    assert lib.gnn_mlp_act_size_bf16(C.byref(wide), 1000, C.byref(n)) == B.GNN_OK and n.value == 0


def test_act_calls_reject_missing_or_misaligned_buffers(lib):
    # checked before any device work: a NULL or misaligned act where one is needed is GNN_EINVAL
    part = MeshGraph((5, 4, 3), 3).partition(4, "rcb")
    H = 64
    cfg = B.gnn_mp_config()
    cfg.hidden, cfg.precision, cfg.ln_eps = H, B.GNN_PREC_BF16, 1e-5
    W = B.gnn_mp_params()
    W.edge = _mlp([3 * H] + [H] * 4, True)
    W.node = _mlp([2 * H] + [H] * 4, True)
    G = _graph_dev(part)
    for act in (None, FAKE + 8):
        rc = lib.gnn_mp_forward_act(C.byref(G), C.byref(cfg), C.byref(W), FAKE, FAKE, FAKE + 64, FAKE, FAKE, act,
                                    FAKE, 1 << 30, None)
        assert rc == B.GNN_EINVAL
        rc = lib.gnn_mp_backward_act(C.byref(G), C.byref(cfg), C.byref(W), FAKE, FAKE, FAKE, act, FAKE, None, FAKE,
                                     FAKE, C.byref(W), FAKE, 1 << 30, None)
        assert rc == B.GNN_EINVAL
        m = _mlp([4, H, H, H, H], True)
        assert lib.gnn_mlp_forward_bf16_act(C.byref(m), 1000, FAKE, FAKE, 1, 1e-5, act, None) == B.GNN_EINVAL
        assert lib.gnn_mlp_backward_bf16_act(C.byref(m), 1000, FAKE, FAKE, 1, None, C.byref(m), 1e-5, act, FAKE,
                                             1 << 20, None) == B.GNN_EINVAL
