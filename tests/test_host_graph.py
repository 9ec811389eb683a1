"""libgnnmp's host graph generation and partitioning against the oracle (CPU only).

The library builds the R=1 CSR directly from lattice coordinates and each
sub-graph from lattice/element arithmetic; the oracle deduplicates per-element
stencils with set operations. Bit-exact agreement of every integer array pins
the library's bookkeeping; positions agree to rounding."""
import json
import os

import numpy as np
import pytest

from oracle import graph as og
from paper_2410_01657_gb300 import _build
from paper_2410_01657_gb300 import binding as B
from paper_2410_01657_gb300.graph import MeshGraph

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()


CASES = [((4, 4, 4), 3, (False, False, False)), ((3, 2, 5), 2, (False, False, False)),
         ((2, 1, 1), 1, (False, False, False)), ((3, 4, 3), 2, (True, False, True)),
         ((5, 3, 4), 1, (True, True, True))]


@pytest.mark.parametrize("nel,p,periodic", CASES)
def test_graph_matches_oracle(nel, p, periodic):
    lib = MeshGraph(nel, p, periodic=periodic)
    ora = og.build_brick(nel, p, periodic=periodic)
    assert lib.n_nodes == ora.n_nodes and lib.n_edges == ora.n_edges
    np.testing.assert_allclose(lib.pos(), ora.pos, rtol=0, atol=1e-14)
    rp, col = lib.csr()
    recv = np.repeat(np.arange(lib.n_nodes), np.diff(rp))
    assert np.array_equal(recv, ora.recv) and np.array_equal(col, ora.send)
    assert np.array_equal(lib.elements(), ora.elem_nodes)


def test_jitter_matches_oracle():
    nel, p = (3, 2, 4), 5
    ora0 = og.build_brick(nel, p)
    jit = np.random.default_rng(5).uniform(-1, 1, size=(ora0.n_nodes, 3))
    lib = MeshGraph(nel, p, jitter=jit, jitter_frac=0.2)
    ora = og.build_brick(nel, p, jitter=jit, jitter_frac=0.2)
    np.testing.assert_allclose(lib.pos(), ora.pos, rtol=0, atol=1e-14)


PARTS = [((4, 4, 4), 3, (False,) * 3, 2, "slab", None), ((4, 4, 4), 3, (False,) * 3, 8, "rcb", None),
         ((4, 3, 5), 2, (False,) * 3, 5, "rcb", [1, 3, 2, 7, 1]), ((4, 4, 6), 2, (False,) * 3, 3, "slab", None),
         ((3, 4, 3), 2, (True, False, True), 4, "rcb", None), ((6, 6, 6), 1, (False,) * 3, 27, "rcb", None)]


@pytest.mark.parametrize("nel,p,periodic,R,method,weights", PARTS)
def test_partition_matches_oracle(nel, p, periodic, R, method, weights):
    lib = MeshGraph(nel, p, periodic=periodic).partition(R, method, weights)
    ora = og.build_brick(nel, p, periodic=periodic)
    part = og.partition_slab_z(ora, R) if method == "slab" else og.partition_rcb(ora, R, weights)
    subs = og.build_subgraphs(ora, part, R)
    ro = lib.array("row_offsets")
    eo = lib.array("edge_offsets")
    gid = lib.array("row_gid")
    rp = lib.array("row_ptr").astype(np.int64)
    col = lib.array("col").astype(np.int64)
    ed = lib.array("edge_deg")
    nd = lib.array("node_deg")
    stats = lib.array("part_stats")
    for r, sg in enumerate(subs):
        rows = slice(ro[r], ro[r + 1])
        assert np.array_equal(gid[rows], sg.gid)
        assert np.array_equal(nd[rows], sg.node_deg)
        lrp = rp[ro[r]:ro[r + 1] + 1] - eo[r]
        recv = np.repeat(np.arange(sg.n_local), np.diff(lrp))
        assert np.array_equal(recv, sg.recv)
        assert np.array_equal(col[eo[r]:eo[r + 1]] - ro[r], sg.send)
        assert np.array_equal(ed[eo[r]:eo[r + 1]], sg.edge_deg)
        assert stats[r, 0] == sg.n_local
        assert stats[r, 1] == sg.n_halo
        assert stats[r, 2] == len(sg.neighbours)
    # halo copy list: every shared gid, its copies in increasing part order
    hp = lib.array("halo_ptr")
    hr = lib.array("halo_rows")
    row_part = np.searchsorted(ro, np.arange(lib.n_rows), side="right") - 1
    for s in range(len(hp) - 1):
        rows = hr[hp[s]:hp[s + 1]]
        assert len(rows) >= 2 and len(set(gid[rows])) == 1
        assert np.all(np.diff(row_part[rows]) > 0)
        assert len(rows) == nd[rows[0]]
    assert sum(hp[1:] - hp[:-1]) == int((nd > 1).sum())
    # edge weights, transposed CSR, edge tiles, attributes
    np.testing.assert_array_equal(lib.array("edge_w"), (1.0 / ed).astype(np.float32))
    tp = lib.array("t_ptr").astype(np.int64)
    te = lib.array("t_eid")
    assert np.array_equal(np.repeat(np.arange(lib.n_rows), np.diff(tp)), col[te])
    for s in range(lib.n_rows):
        assert np.all(np.diff(te[tp[s]:tp[s + 1]]) > 0)
    tiles = lib.array("edge_tiles").astype(np.int64)
    assert tiles[0] == 0 and tiles[-1] == lib.n_rows and np.all(np.diff(tiles) > 0)
    assert np.all(rp[tiles[1:]] - rp[tiles[:-1]] <= B.GNN_EDGE_TILE)
    attr = lib.array("edge_attr")
    for r, sg in enumerate(subs):
        np.testing.assert_allclose(attr[eo[r]:eo[r + 1]], og.edge_attributes(ora.pos, sg), rtol=1e-6, atol=1e-7)


def test_table2_r8_row_library():
    g = json.load(open(os.path.join(GOLD, "table2_r8.json")))
    part = MeshGraph((16, 16, 128), 5, periodic=(True, True, True)).partition(g["ranks"], "slab")
    stats = part.array("part_stats")
    for r in range(g["ranks"]):
        assert round(stats[r, 0] / 1000) == g["graph_nodes_thousands"]
        assert stats[r, 1] / 1000 == g["halo_nodes_thousands"]
        assert stats[r, 2] == g["neighbours"]


def test_fig4_library():
    g = json.load(open(os.path.join(GOLD, "fig4_two_elements.json")))
    part = MeshGraph((2, 1, 1), 1, extent=(2.0, 1.0, 1.0)).partition(2, "rcb")
    stats = part.array("part_stats")
    ed = part.array("edge_deg")
    eo = part.array("edge_offsets")
    for r in range(2):
        assert stats[r].tolist() == [g["per_rank_nodes"], g["per_rank_halo_rows"], g["per_rank_neighbours"]]
        assert eo[r + 1] - eo[r] == g["per_rank_directed_edges"]
        assert int((ed[eo[r]:eo[r + 1]] == 2).sum()) == g["shared_face_directed_edges_degree_2"]
    assert part.info.n_shared == 4 and part.info.n_copies == 8


def test_partition_errors():
    g = MeshGraph((2, 2, 2), 1)
    with pytest.raises(B.GnnError) as ei:
        g.partition(9, "rcb")
    assert ei.value.code == B.GNN_EINVAL
    with pytest.raises(B.GnnError):
        g.partition(3, "slab")
    with pytest.raises(B.GnnError):
        g.partition(2, "rcb", [1.0, -1.0])


def test_tile_records_match_partition_arrays():
    part = MeshGraph((4, 3, 5), 2).partition(5, "rcb", [1, 3, 2, 7, 1])
    rec = part.array("tile_meta").reshape(-1, B.GNN_TILE_META_BYTES)
    tiles = part.array("edge_tiles")
    rp = part.array("row_ptr")
    col = part.array("col")
    w = part.array("edge_w")
    assert rec.shape[0] == len(tiles) - 1
    for t in range(rec.shape[0]):
        hdr = rec[t, :16].view(np.int32)
        r0, r1 = tiles[t], tiles[t + 1]
        e0, ne = rp[r0], rp[r1] - rp[r0]
        assert hdr.tolist() == [r0, r1, e0, ne]
        assert np.array_equal(rec[t, 16:16 + 4 * (r1 - r0 + 1)].view(np.int32), rp[r0:r1 + 1] - e0)
        seg = rec[t, 544:544 + 2 * ne].view(np.int16)
        assert np.array_equal(seg, np.repeat(np.arange(r1 - r0), np.diff(rp[r0:r1 + 1])))
        assert np.array_equal(rec[t, 800:800 + 4 * ne].view(np.int32), col[e0:e0 + ne])
        assert np.array_equal(rec[t, 1312:1312 + 4 * ne].view(np.float32), w[e0:e0 + ne])


@pytest.mark.parametrize("cap", [7, 40, 128])
def test_retile_caps_edges_and_keeps_records(cap):
    part = MeshGraph((4, 3, 5), 2).partition(5, "rcb", [1, 3, 2, 7, 1])
    assert part.tile_edges == B.GNN_EDGE_TILE
    n0 = part.info.n_edge_tiles
    part.set_tile_edges(cap)
    assert part.tile_edges == cap
    tiles = part.array("edge_tiles").astype(np.int64)
    rp = part.array("row_ptr").astype(np.int64)
    assert tiles[0] == 0 and tiles[-1] == part.n_rows and np.all(np.diff(tiles) > 0)
    assert np.all(rp[tiles[1:]] - rp[tiles[:-1]] <= cap)
    # greedy: adding the next row to any tile would exceed the cap
    nxt = tiles[1:-1]
    assert np.all(rp[nxt + 1] - rp[tiles[:-2]] > cap)
    if cap < B.GNN_EDGE_TILE:
        assert part.info.n_edge_tiles > n0
    rec = part.array("tile_meta").reshape(-1, B.GNN_TILE_META_BYTES)
    assert rec.shape[0] == len(tiles) - 1
    for t in range(rec.shape[0]):
        hdr = rec[t, :16].view(np.int32)
        assert hdr.tolist() == [tiles[t], tiles[t + 1], rp[tiles[t]], rp[tiles[t + 1]] - rp[tiles[t]]]


def test_retile_rejects_caps_below_degree():
    part = MeshGraph((3, 3, 3), 2).partition(2, "slab")
    with pytest.raises(B.GnnError) as ei:
        part.set_tile_edges(part.info.max_in_degree - 1)
    assert ei.value.code == B.GNN_EINVAL
    with pytest.raises(B.GnnError):
        part.set_tile_edges(B.GNN_EDGE_TILE + 1)
