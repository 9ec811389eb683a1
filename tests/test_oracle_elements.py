"""Pins of the oracle's general element-mesh graph and of the layer on it (CPU only).

Sec. II-A notes that the graph construction and its distribution apply to any
mesh made of finite elements. Pins used: closed forms of the Kuhn (Freudenthal)
triangulation of a cube lattice (3n(n+1)^2 + 3n^2(n+1) + n^3 undirected edges,
interior degree 14, the 6 tetrahedra of a cell fill it); hexahedral cells
listed as elements give the lattice builder's p=1 brick; a hand-counted
two-tetrahedron mesh (d_i, d_ij of Eq. 5b / 8b); constant messages whose
aggregate is the in-degree on every copy; a brute-force loop over the
unpartitioned definition; and Eq. 2 / Eq. 3 consistency (R-way == R=1) on a
mesh of mixed element types with a node of in-degree above 128."""
import numpy as np
import pytest

import synthetic as syn
from oracle import graph as og
from oracle import model as om

from test_oracle_model import _brute_force_layer, _constant_message_layer, _flat


def _mesh(n, seed=0, **kw):
    m = syn.mixed_element_mesh(n, seed, **kw)
    return og.element_mesh(m["pos"], m["elem_ptr"], m["elem_nodes"], m["edge_ptr"], m["edge_pairs"]), m


@pytest.mark.parametrize("n", [1, 2, 3])
def test_kuhn_triangulation_closed_forms(n):
    mesh, m = _mesh(n, tet_fraction=1.0, n_fans=0, jitter=0.0)
    assert mesh.n_nodes == (n + 1) ** 3
    assert mesh.n_edges == 2 * (3 * n * (n + 1) ** 2 + 3 * n * n * (n + 1) + n ** 3)
    deg = np.bincount(mesh.recv, minlength=mesh.n_nodes)
    assert deg[0] == 7                       # 3 axis + 3 face diagonals + 1 body diagonal
    if n >= 2:
        c = 1 + (n + 1) * (1 + (n + 1))       # lattice point (1, 1, 1)
        assert deg[c] == 14
    # the 6 tetrahedra of every cell fill it: volumes sum to the unit cube
    vol = 0.0
    for e in range(mesh.n_elem):
        v = mesh.pos[mesh.element(e)[0]]
        vol += abs(np.linalg.det(v[1:] - v[0])) / 6.0
    assert abs(vol - 1.0) < 1e-12
    assert mesh.n_elem == 6 * n ** 3


def test_hex_cells_give_the_p1_brick():
    n = 3
    mesh, _ = _mesh(n, tet_fraction=0.0, n_fans=0, jitter=0.0)
    b = og.build_brick((n, n, n), 1)
    np.testing.assert_array_equal(mesh.recv, b.recv)
    np.testing.assert_array_equal(mesh.send, b.send)
    np.testing.assert_allclose(mesh.pos, b.pos, rtol=0, atol=1e-15)


def test_two_tetrahedra_hand_counts():
    # tetrahedra (0,1,2,3) and (1,2,3,4) share the face (1,2,3)
    pos = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]], dtype=np.float64)
    pairs = np.concatenate([syn.TET_EDGES, syn.TET_EDGES])
    mesh = og.element_mesh(pos, [0, 4, 8], [0, 1, 2, 3, 1, 2, 3, 4], [0, 6, 12], pairs)
    assert mesh.n_edges == 18
    np.testing.assert_array_equal(np.bincount(mesh.recv), [3, 4, 4, 4, 3])
    subs = og.build_element_subgraphs(mesh, np.array([0, 1]), 2)
    np.testing.assert_array_equal(subs[0].gid, [0, 1, 2, 3])
    np.testing.assert_array_equal(subs[1].gid, [1, 2, 3, 4])
    np.testing.assert_array_equal(subs[0].node_deg, [1, 2, 2, 2])
    np.testing.assert_array_equal(subs[1].node_deg, [2, 2, 2, 1])
    for sg, apex in zip(subs, (0, 4)):
        assert sg.n_edges == 12
        on_face = (sg.gid[sg.recv] != apex) & (sg.gid[sg.send] != apex)
        np.testing.assert_array_equal(sg.edge_deg, np.where(on_face, 2, 1))
        assert int(on_face.sum()) == 6
    assert subs[0].n_halo == 3 and subs[1].n_halo == 3


def _fan_split(m, R):
    """Element -> part: cells by x-slab over R-1 parts, the fans alternating
    over all R parts (so the apex is held by several sub-graphs)."""
    kind = m["kind"]
    cells = np.nonzero(kind != 2)[0]
    part = np.zeros(kind.shape[0], dtype=np.int64)
    part[cells] = (np.arange(cells.shape[0]) * max(R - 1, 1)) // cells.shape[0]
    fans = np.nonzero(kind == 2)[0]
    part[fans] = (np.arange(fans.shape[0]) + 1) % R
    return part


@pytest.mark.parametrize("R,how", [(1, None), (3, "slab"), (5, "rcb"), (4, "fans")])
def test_aggregate_is_in_degree(R, how):
    rng = np.random.default_rng(2)
    H = 5
    c = np.array([1.0, -2.0, 0.5, 3.0, 0.25])
    mesh, m = _mesh(5, seed=1, n_fans=3)
    if R == 1:
        subs = og.element_mesh_unpartitioned(mesh)
    else:
        part = {"slab": lambda: og.partition_slab_elements(mesh, R),
                "rcb": lambda: og.partition_rcb_elements(mesh, R, [1, 3, 2, 7, 1]),
                "fans": lambda: _fan_split(m, R)}[how]()
        subs = og.build_element_subgraphs(mesh, part, R)
    layer = _constant_message_layer(rng, H, c)
    xs = [rng.standard_normal((sg.n_local, H)) for sg in subs]
    es = [np.zeros((sg.n_edges, H)) for sg in subs]
    indeg = np.bincount(mesh.recv, minlength=mesh.n_nodes)
    _, _, cache = om.layer_forward(layer, subs, xs, es)
    for r, sg in enumerate(subs):
        np.testing.assert_allclose(cache["a_star"][r], indeg[sg.gid][:, None] * c, rtol=1e-14)


@pytest.mark.parametrize("R", [1, 2])
def test_layer_matches_brute_force_loops_on_elements(R):
    rng = np.random.default_rng(3)
    H = 4
    mesh, m = _mesh(1, seed=4, tet_fraction=1.0, n_fans=1)
    layer = {"edge": syn.xavier_mlp(rng, syn.mlp_dims(3 * H, H, 2, H), True, True),
             "node": syn.xavier_mlp(rng, syn.mlp_dims(2 * H, H, 2, H), True, True)}
    x_glob = rng.standard_normal((mesh.n_nodes, H))
    e_glob = {(int(i), int(j)): rng.standard_normal(H) for i, j in zip(mesh.recv, mesh.send)}
    xb, eb = _brute_force_layer(layer, mesh, x_glob, e_glob)
    subs = (og.element_mesh_unpartitioned(mesh) if R == 1
            else og.build_element_subgraphs(mesh, _fan_split(m, R), R))
    xs = [x_glob[sg.gid] for sg in subs]
    es = [np.stack([e_glob[(int(sg.gid[i]), int(sg.gid[j]))] for i, j in zip(sg.recv, sg.send)])
          for sg in subs]
    x_new, e_new, _ = om.layer_forward(layer, subs, xs, es)
    for r, sg in enumerate(subs):
        np.testing.assert_allclose(x_new[r], xb[sg.gid], rtol=1e-12, atol=1e-12)
        for k, (i, j) in enumerate(zip(sg.recv, sg.send)):
            np.testing.assert_allclose(e_new[r][k], eb[(int(sg.gid[i]), int(sg.gid[j]))], rtol=1e-12, atol=1e-12)


def _run_network(mesh, subs, p, u):
    us = [u[sg.gid] for sg in subs]
    attr = [og.edge_attributes(mesh.pos, sg) for sg in subs]
    target = [np.cos(us[r]) for r in range(len(subs))]
    ys, cache = om.network_forward(p, subs, us, attr)
    L = om.consistent_loss(subs, ys, target)
    g = om.network_backward(p, subs, cache, om.consistent_loss_grad(subs, ys, target))
    return om.to_global(subs, ys, mesh.n_nodes), L, g


@pytest.mark.parametrize("R,how", [(4, "rcb"), (3, "fans")])
def test_consistency_eq2_eq3_mixed_elements(R, how):
    # n = 12 with two fans: the apex has in-degree 13^2 = 169 in the R=1 graph
    mesh, m = _mesh(12, seed=5, n_fans=2)
    assert np.bincount(mesh.recv).max() == 169
    u = syn.fourier_field(mesh.pos, syn.fourier_modes(0, 8))
    p = syn.gnn_params(7, 8, 2, 2, randomize_affine=True)
    y1, L1, g1 = _run_network(mesh, og.element_mesh_unpartitioned(mesh), p, u)
    part = og.partition_rcb_elements(mesh, R) if how == "rcb" else _fan_split(m, R)
    yR, LR, gR = _run_network(mesh, og.build_element_subgraphs(mesh, part, R), p, u)
    assert np.abs(yR - y1).max() <= 1e-12 * np.abs(y1).max()
    assert abs(LR - L1) <= 1e-13 * abs(L1)
    f1, fR = _flat(g1), _flat(gR)
    assert np.abs(fR - f1).max() <= 1e-11 * np.abs(f1).max()


def test_mixed_mesh_recipe_by_loops():
    # the generator's element lists, rebuilt cell by cell from its documented recipe
    n, seed, tf, nf = 3, 11, 0.4, 2
    m = syn.mixed_element_mesh(n, seed, tet_fraction=tf, n_fans=nf)
    rng = np.random.default_rng(seed)
    q = n + 1
    rng.uniform(-0.5, 0.5, size=(q ** 3, 3))          # the jitter draw comes first
    draw = rng.uniform(size=n ** 3)
    nodes, pairs, kind = [], [], []
    for c in range(n ** 3):
        ci, cj, ck = c % n, (c // n) % n, c // (n * n)
        hexn = [(ci + (v & 1)) + q * ((cj + ((v >> 1) & 1)) + q * (ck + ((v >> 2) & 1))) for v in range(8)]
        if draw[c] < tf:
            for t in syn.kuhn_tets():
                nodes.append([hexn[v] for v in t]); pairs.append(syn.TET_EDGES); kind.append(1)
        else:
            nodes.append(hexn); pairs.append(syn.HEX_EDGES); kind.append(0)
    for f in range(nf):
        lo, hi = (f * n) // nf, ((f + 1) * n) // nf
        top = [i + q * (j + q * n) for i in range(lo, hi + 1) for j in range(q)]
        nodes.append([q ** 3] + top)
        pairs.append(np.array([(0, k + 1) for k in range(len(top))], dtype=np.int32)); kind.append(2)
    assert np.array_equal(m["elem_ptr"], np.concatenate([[0], np.cumsum([len(x) for x in nodes])]))
    assert np.array_equal(m["elem_nodes"], np.concatenate([np.asarray(x) for x in nodes]))
    assert np.array_equal(m["edge_ptr"], np.concatenate([[0], np.cumsum([len(x) for x in pairs])]))
    assert np.array_equal(m["edge_pairs"], np.concatenate(pairs))
    assert np.array_equal(m["kind"], kind)
    assert m["pos"].shape == (q ** 3 + 1, 3) and np.allclose(m["pos"][-1], (0.5, 0.5, 1 + 1 / n))
