"""libgnnmp's general element-mesh graphs and their partitions (CPU only).

gnn_graph_build_elements / gnn_partition_elements against the oracle's
element-mesh graph, the library's own lattice builder on the same elements, and
the invariants of the split of high in-degree nodes into co-resident copies:
every row's in-degree fits one edge tile, the copies of a node together hold
exactly the oracle's in-edges of that node with the same d_ij, d_i counts all
copies, and the constant-message aggregate summed over the copy list is the
R=1 in-degree on every row (Eq. 5b-5d)."""
import numpy as np
import pytest

import synthetic as syn
from oracle import graph as og
from paper_2410_01657_gb300 import _build
from paper_2410_01657_gb300 import binding as B
from paper_2410_01657_gb300.graph import MeshGraph

from test_oracle_elements import _fan_split


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()


def _lib_graph(m):
    return MeshGraph.from_elements(m["pos"], m["elem_ptr"], m["elem_nodes"], m["edge_ptr"], m["edge_pairs"])


def _ora_mesh(m):
    return og.element_mesh(m["pos"], m["elem_ptr"], m["elem_nodes"], m["edge_ptr"], m["edge_pairs"])


def _brick_elements(nel, p):
    b = og.build_brick(nel, p)
    pairs = og.local_stencil_pairs(p)
    ne = b.n_elem
    q3 = (p + 1) ** 3
    return b, {"pos": MeshGraph(nel, p).pos(), "elem_ptr": np.arange(ne + 1) * q3,
               "elem_nodes": b.elem_nodes.ravel(), "edge_ptr": np.arange(ne + 1) * len(pairs),
               "edge_pairs": np.tile(pairs, (ne, 1))}


@pytest.mark.parametrize("nel,p", [((3, 2, 4), 1), ((2, 3, 2), 3)])
def test_brick_as_elements_matches_lattice_builder(nel, p):
    b, m = _brick_elements(nel, p)
    lib_e, lib_b = _lib_graph(m), MeshGraph(nel, p)
    assert lib_e.info.kind == B.GNN_GRAPH_ELEMENTS and lib_b.info.kind == B.GNN_GRAPH_BRICK
    rp_e, col_e = lib_e.csr()
    rp_b, col_b = lib_b.csr()
    assert np.array_equal(rp_e, rp_b) and np.array_equal(col_e, col_b)
    assert lib_e.info.max_degree == lib_b.info.max_degree == 6
    assert np.array_equal(lib_e.elements(), lib_b.elements().ravel())
    assert np.array_equal(lib_e.element_ptr(), lib_b.element_ptr())
    # the same element assignment gives identical partitions on both graphs
    part = og.partition_rcb(b, 5, [1, 3, 2, 7, 1])
    pe, pb = lib_e.partition(5, elem_part=part), lib_b.partition(5, elem_part=part)
    for name in ("row_offsets", "edge_offsets", "row_gid", "row_ptr", "col", "edge_deg", "node_deg", "t_ptr",
                 "t_eid", "halo_ptr", "halo_rows", "edge_tiles", "tile_meta", "part_stats"):
        assert np.array_equal(pe.array(name), pb.array(name)), name
    # and the library's own RCB of the brick is that assignment
    pr = lib_b.partition(5, "rcb", [1, 3, 2, 7, 1])
    assert np.array_equal(pr.array("row_gid"), pb.array("row_gid"))
    assert np.array_equal(pr.array("col"), pb.array("col"))


def _exact_check(lib, subs):
    ro, eo = lib.array("row_offsets"), lib.array("edge_offsets")
    gid, nd, ed = lib.array("row_gid"), lib.array("node_deg"), lib.array("edge_deg")
    rp, col = lib.array("row_ptr").astype(np.int64), lib.array("col").astype(np.int64)
    for r, sg in enumerate(subs):
        assert np.array_equal(gid[ro[r]:ro[r + 1]], sg.gid)
        assert np.array_equal(nd[ro[r]:ro[r + 1]], sg.node_deg)
        recv = np.repeat(np.arange(sg.n_local), np.diff(rp[ro[r]:ro[r + 1] + 1]))
        assert np.array_equal(recv, sg.recv)
        assert np.array_equal(col[eo[r]:eo[r + 1]] - ro[r], sg.send)
        assert np.array_equal(ed[eo[r]:eo[r + 1]], sg.edge_deg)


@pytest.mark.parametrize("R,how", [(1, None), (3, "slab"), (5, "rcb"), (4, "fans")])
def test_element_partition_matches_oracle(R, how):
    m = syn.mixed_element_mesh(5, 1, n_fans=3)
    mesh, lib = _ora_mesh(m), _lib_graph(m)
    assert lib.n_nodes == mesh.n_nodes and lib.n_edges == mesh.n_edges
    rp, col = lib.csr()
    assert np.array_equal(np.repeat(np.arange(lib.n_nodes), np.diff(rp)), mesh.recv)
    assert np.array_equal(col, mesh.send)
    if R == 1:
        part = lib.partition(1, "rcb")
        subs = og.element_mesh_unpartitioned(mesh)
    elif how == "fans":
        ep = _fan_split(m, R)
        part, subs = lib.partition(R, elem_part=ep), og.build_element_subgraphs(mesh, ep, R)
    elif how == "slab":
        part = lib.partition(R, "slab")
        subs = og.build_element_subgraphs(mesh, og.partition_slab_elements(mesh, R), R)
    else:
        w = [1, 3, 2, 7, 1]
        part = lib.partition(R, "rcb", w)
        subs = og.build_element_subgraphs(mesh, og.partition_rcb_elements(mesh, R, w), R)
    assert part.info.max_in_degree <= B.GNN_EDGE_TILE
    _exact_check(part, subs)


def _check_split(lib, subs, mesh):
    """Invariants of a partition whose high in-degree nodes are split into copies."""
    ro, eo = lib.array("row_offsets"), lib.array("edge_offsets")
    gid, nd, ed = lib.array("row_gid"), lib.array("node_deg"), lib.array("edge_deg")
    rp, col = lib.array("row_ptr").astype(np.int64), lib.array("col").astype(np.int64)
    deg = np.diff(rp)
    assert deg.max() <= B.GNN_EDGE_TILE and lib.info.max_in_degree == deg.max()
    rows_of_gid = np.bincount(gid, minlength=mesh.n_nodes)
    assert np.array_equal(nd, rows_of_gid[gid])                    # d_i counts every row
    recv = np.repeat(np.arange(lib.n_rows), deg)
    for r, sg in enumerate(subs):
        g = gid[ro[r]:ro[r + 1]]
        assert np.all(np.diff(g) >= 0) and np.array_equal(np.unique(g), sg.gid)
        e = slice(eo[r], eo[r + 1])
        # the edges of the copies, in row order, are the oracle's edges in order
        assert np.array_equal(gid[recv[e]], sg.gid[sg.recv])
        assert np.array_equal(gid[col[e]], sg.gid[sg.send])
        assert np.array_equal(ed[e], sg.edge_deg)
        # the copies' in-degrees differ by at most one (near-equal runs)
        for u in np.unique(g[np.diff(np.r_[g, -1]) == 0]):
            d = deg[ro[r] + np.nonzero(g == u)[0]]
            assert d.max() - d.min() <= 1 and d.sum() == int((sg.gid[sg.recv] == u).sum())
        # a copy sends to the nodes it receives from
        for t in range(eo[r], eo[r + 1]):
            s = col[t]
            if rows_of_gid[gid[s]] > 1 and np.sum(g == gid[s]) > 1:
                assert gid[recv[t]] in gid[col[rp[s]:rp[s + 1]]]
    # Eq. 5b-5d with unit messages: the copy-summed aggregate is the R=1 in-degree
    a = np.bincount(recv, weights=1.0 / ed.astype(np.float64), minlength=lib.n_rows)
    hp, hr = lib.array("halo_ptr"), lib.array("halo_rows")
    for s in range(len(hp) - 1):
        rows = hr[hp[s]:hp[s + 1]]
        assert len(set(gid[rows])) == 1 and len(rows) == nd[rows[0]] and np.all(np.diff(rows) > 0)
        a[rows] = a[rows].sum()
    np.testing.assert_allclose(a, np.bincount(mesh.recv, minlength=mesh.n_nodes)[gid], rtol=1e-14)


@pytest.mark.parametrize("R,how", [(1, None), (2, "fans"), (3, "fans"), (6, "rcb")])
def test_high_in_degree_split(R, how):
    # n = 16, two fans of 9 x 17 top-face nodes: the apex has in-degree 289
    # (3 copies) in the R=1 graph and 153 (2 copies) in a sub-graph of one fan
    m = syn.mixed_element_mesh(16, 3, n_fans=2)
    mesh, lib = _ora_mesh(m), _lib_graph(m)
    assert lib.info.max_degree == 289
    apex = mesh.n_nodes - 1
    if R == 1:
        part, subs = lib.partition(1, "rcb"), og.element_mesh_unpartitioned(mesh)
        expect_rows = 3
    elif how == "fans":
        ep = _fan_split(m, R)
        part, subs = lib.partition(R, elem_part=ep), og.build_element_subgraphs(mesh, ep, R)
        expect_rows = 4
    else:
        part = lib.partition(R, "rcb")
        subs = og.build_element_subgraphs(mesh, og.partition_rcb_elements(mesh, R), R)
        expect_rows = None
    _check_split(part, subs, mesh)
    n_apex = int((part.array("row_gid") == apex).sum())
    if expect_rows is not None:
        assert n_apex == expect_rows
    assert n_apex >= 3


def test_tile_records_of_split_partition():
    m = syn.mixed_element_mesh(16, 3, n_fans=2)
    part = _lib_graph(m).partition(2, elem_part=_fan_split(m, 2))
    rec = part.array("tile_meta").reshape(-1, B.GNN_TILE_META_BYTES)
    tiles, rp = part.array("edge_tiles"), part.array("row_ptr")
    for t in range(rec.shape[0]):
        r0, r1 = tiles[t], tiles[t + 1]
        assert rec[t, :16].view(np.int32).tolist() == [r0, r1, rp[r0], rp[r1] - rp[r0]]
        assert rp[r1] - rp[r0] <= B.GNN_EDGE_TILE


def test_element_mesh_errors():
    pos = np.zeros((5, 3))
    ok = dict(pos=pos, elem_ptr=[0, 4, 8], elem_nodes=[0, 1, 2, 3, 1, 2, 3, 4], edge_ptr=[0, 6, 12],
              edge_pairs=np.concatenate([syn.TET_EDGES, syn.TET_EDGES]))
    g = MeshGraph.from_elements(**ok)
    assert g.n_edges == 18 and g.info.n_elem == 2 and g.info.n_elem_nodes == 8
    bad = [dict(ok, elem_nodes=[0, 1, 2, 3, 1, 2, 3, 5]),              # id out of range
           dict(ok, pos=np.zeros((6, 3))),                                # node 5 in no element
           dict(ok, elem_nodes=[0, 1, 2, 3, 1, 2, 3, 3]),              # pair joins a node to itself
           dict(ok, edge_pairs=np.concatenate([syn.TET_EDGES, [[0, 1]] * 5 + [[0, 4]]])),  # local index 4
           dict(ok, elem_ptr=[0, 4, 4]),                                  # element without nodes
           dict(ok, pos=np.zeros((6, 3)), elem_ptr=[0, 4, 9], elem_nodes=[0, 1, 2, 3, 1, 2, 3, 4, 5])]  # no edge
    for kw in bad:
        with pytest.raises(B.GnnError) as ei:
            MeshGraph.from_elements(**kw)
        assert ei.value.code == B.GNN_EINVAL
    for R, ep in ((2, [0, 2]), (2, [0, 0]), (3, [0, 1])):
        with pytest.raises(B.GnnError) as ei:
            g.partition(R, elem_part=ep)
        assert ei.value.code == B.GNN_EINVAL
    # a node that would need more than 255 rows is refused
    n = 4100
    star = dict(pos=np.zeros((n, 3)), elem_ptr=[0, n], elem_nodes=np.arange(n), edge_ptr=[0, n - 1],
                edge_pairs=np.stack([np.zeros(n - 1), np.arange(1, n)], axis=1))
    p = MeshGraph.from_elements(**star).partition(1, "rcb")
    assert int((p.array("row_gid") == 0).sum()) == (n - 1 + 127) // 128
    n = 128 * 256 + 2
    star = dict(pos=np.zeros((n, 3)), elem_ptr=[0, n], elem_nodes=np.arange(n), edge_ptr=[0, n - 1],
                edge_pairs=np.stack([np.zeros(n - 1), np.arange(1, n)], axis=1))
    with pytest.raises(B.GnnError) as ei:
        MeshGraph.from_elements(**star).partition(1, "rcb")
    assert ei.value.code == B.GNN_EUNSUPPORTED


@pytest.mark.parametrize("R,how", [(1, None), (3, "fans"), (6, "rcb")])
def test_split_partition_evaluates_to_the_oracle_layer(R, how):
    # the library's rows (split copies, copy list, d_i, d_ij) run through the
    # oracle's own layer give the oracle's results on its unsplit sub-graphs
    from oracle import model as om
    from elements_util import check_layer, layer_case, library_view, mixed_mesh16, partitions
    from gpu_util import split_edges, split_rows

    m, mesh = mixed_mesh16()
    part, subs = partitions(m, mesh, R, how)
    case = layer_case(part, mesh, subs, 8, round_edges=False)
    view = library_view(part)
    lp = case["params"]["layers"][0]
    x1, e1, cache = om.layer_forward(lp, view, split_rows(case["x"], view), split_edges(case["e"], view))
    dx0, de0, g = om.layer_backward(lp, view, cache, split_rows(case["dx1"], view), split_edges(case["de1"], view))
    out = {"x'": np.concatenate(x1), "e'": np.concatenate(e1), "a*": np.concatenate(cache["a_star"]),
           "dL/dx": np.concatenate(dx0), "dL/de": np.concatenate(de0)}
    grads = []
    for mm in ("edge", "node"):
        grads += list(g[mm]["W"]) + list(g[mm]["b"]) + [g[mm]["gamma"], g[mm]["beta"]]
    check_layer(part, subs, case, out, grads, 1e-12, 1e-11)
