"""Pins of the oracle's graph generation and partitioning (CPU only).

Each test checks oracle.graph against something other than itself: closed
forms, the paper's printed Table 2 / Fig. 3 / Fig. 4 numbers, or invariants
(Eq. 8c) that a dropped term or wrong index would break."""
import json
import os

import numpy as np
import pytest

from oracle import graph

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _lattice_in_degree(L, periodic=(False, False, False)):
    """Closed form: number of lattice neighbours of each node (6-stencil)."""
    iz, iy, ix = np.meshgrid(np.arange(L[2]), np.arange(L[1]), np.arange(L[0]), indexing="ij")
    deg = np.zeros(ix.size, dtype=np.int64)
    for a, idx in enumerate((ix.ravel(), iy.ravel(), iz.ravel())):
        if periodic[a]:
            deg += 2
        else:
            deg += (idx > 0).astype(np.int64) + (idx < L[a] - 1).astype(np.int64)
    return deg


def test_gll_closed_forms():
    # p=1: endpoints; p=2: {-1,0,1}; p=3: +-1/sqrt(5); p=4: 0, +-sqrt(3/7);
    # p=5: +-sqrt(1/3 -+ 2 sqrt(7)/21) (roots of P_p').
    np.testing.assert_allclose(graph.gll_points(1), [-1, 1], atol=0)
    np.testing.assert_allclose(graph.gll_points(2), [-1, 0, 1], atol=1e-15)
    s5 = 1 / np.sqrt(5)
    np.testing.assert_allclose(graph.gll_points(3), [-1, -s5, s5, 1], atol=1e-15)
    s37 = np.sqrt(3 / 7)
    np.testing.assert_allclose(graph.gll_points(4), [-1, -s37, 0, s37, 1], atol=1e-15)
    a = np.sqrt(1 / 3 - 2 * np.sqrt(7) / 21)
    b = np.sqrt(1 / 3 + 2 * np.sqrt(7) / 21)
    np.testing.assert_allclose(graph.gll_points(5), [-1, -b, -a, a, b, 1], atol=1e-14)


@pytest.mark.parametrize("p", [1, 2, 3, 5, 7])
def test_gll_quadrature_exactness(p):
    # GLL weights w_k = 2 / (p (p+1) P_p(x_k)^2) integrate degree <= 2p-1 exactly.
    x = graph.gll_points(p)
    Pp = np.polynomial.legendre.Legendre.basis(p)(x)
    w = 2.0 / (p * (p + 1) * Pp ** 2)
    for deg in range(2 * p):
        exact = 0.0 if deg % 2 else 2.0 / (deg + 1)
        assert abs(np.sum(w * x ** deg) - exact) < 1e-12


@pytest.mark.parametrize("nel,p", [((4, 4, 4), 3), ((3, 2, 5), 2), ((2, 2, 2), 1), ((16, 16, 16), 5)])
def test_graph_closed_form_counts(nel, p):
    b = graph.build_brick(nel, p)
    L = [n * p + 1 for n in nel]
    assert b.n_nodes == L[0] * L[1] * L[2]
    n_und = (L[0] - 1) * L[1] * L[2] + L[0] * (L[1] - 1) * L[2] + L[0] * L[1] * (L[2] - 1)
    assert b.n_edges == 2 * n_und
    # receiver-sorted, senders ascending, no self loops, symmetric
    key = b.recv * b.n_nodes + b.send
    assert np.all(np.diff(key) > 0)
    assert np.all(b.recv != b.send)
    rev = np.sort(b.send * b.n_nodes + b.recv)
    assert np.array_equal(rev, key)
    np.testing.assert_array_equal(np.bincount(b.recv, minlength=b.n_nodes), _lattice_in_degree(L))


def test_config_sizes_closed_form():
    # N = L^3, E = 6 L^2 (L - 1) with L = n p + 1 for the benchmark bricks
    for n, p, N, E in [(4, 3, 2197, 12168), (16, 5, 531441, 3149280),
                       (32, 7, 11390625, 68040000), (48, 7, 38272753, 228955104)]:
        L = n * p + 1
        assert L ** 3 == N and 6 * L * L * (L - 1) == E


def test_positions_are_gll_lattice():
    b = graph.build_brick((2, 1, 1), 3, extent=(2.0, 1.0, 1.0))
    xi = graph.gll_points(3)
    xs = np.unique(b.pos[:, 0])
    expect = np.unique(np.concatenate([(xi + 1) / 2, 1 + (xi + 1) / 2]))
    np.testing.assert_allclose(xs, expect, atol=1e-15)


def test_edge_attribute_sign_and_norm():
    # single p=1 unit element: node 0 at the origin receives from nodes 1, 2, 4
    b = graph.build_brick((1, 1, 1), 1)
    sub = graph.unpartitioned(b)[0]
    attr = graph.edge_attributes(b.pos, sub)
    m = sub.recv == 0
    assert sorted(sub.send[m].tolist()) == [1, 2, 4]
    np.testing.assert_allclose(np.sort(attr[m][:, :3], axis=0)[::-1].sum(axis=0), [1, 1, 1])
    assert np.all(attr[m][:, :3] >= 0)            # d = pos(sender) - pos(receiver)
    np.testing.assert_allclose(attr[:, 3], 1.0)
    np.testing.assert_allclose(np.linalg.norm(attr[:, :3], axis=1), attr[:, 3])


def test_fig3_local_coincident_collapse():
    # Fig. 3: 2x2x2 elements at p=5 on one rank; coincident face nodes collapse
    b = graph.build_brick((2, 2, 2), 5, with_edges=False)
    assert b.elem_nodes.size == 8 * 6 ** 3
    assert np.unique(b.elem_nodes).size == 11 ** 3 == b.n_nodes


def test_fig4_two_element_halo():
    g = json.load(open(os.path.join(GOLD, "fig4_two_elements.json")))
    b = graph.build_brick((2, 1, 1), 1, extent=(2.0, 1.0, 1.0))
    part = graph.partition_rcb(b, 2)
    assert part.tolist() == [0, 1]
    subs = graph.build_subgraphs(b, part, 2)
    for r, sg in enumerate(subs):
        assert sg.n_local == g["per_rank_nodes"]
        assert sg.n_halo == g["per_rank_halo_rows"]
        assert len(sg.neighbours) == g["per_rank_neighbours"]
        assert sg.n_edges == g["per_rank_directed_edges"]
        assert int((sg.edge_deg == 2).sum()) == g["shared_face_directed_edges_degree_2"]
        shared = sg.gid[sg.node_deg == 2]
        np.testing.assert_allclose(b.pos[shared, 0], 1.0)     # the shared face x = 1
        # halo rows point at the same global ids on the other rank
        other = subs[1 - r]
        assert np.array_equal(other.gid[sg.halo_src_row], sg.gid[sg.halo_local_row])


def test_table2_r8_row():
    g = json.load(open(os.path.join(GOLD, "table2_r8.json")))
    b = graph.build_brick((16, 16, 128), 5, periodic=(True, True, True), with_edges=False)
    part = graph.partition_slab_z(b, g["ranks"])
    nodes = graph.partition_nodes(b, part, g["ranks"])
    for r in range(g["ranks"]):
        assert round(nodes[r].size / 1000) == g["graph_nodes_thousands"]
        halo = 0
        neigh = 0
        for s in range(g["ranks"]):
            if s != r:
                k = np.intersect1d(nodes[r], nodes[s], assume_unique=True).size
                halo += k
                neigh += k > 0
        assert halo / 1000 == g["halo_nodes_thousands"]
        assert neigh == g["neighbours"]
        assert nodes[r].size == 80 * 80 * 81


@pytest.mark.parametrize("R,method,weights", [(2, "slab", None), (8, "rcb", None),
                                              (5, "rcb", [1, 3, 2, 7, 1]), (3, "slab", None)])
def test_eq8c_effective_counts(R, method, weights):
    # Eq. 8c: sum over ranks of sum 1/d_i equals N; the edge analogue equals E
    b = graph.build_brick((4, 4, 4), 3)
    part = graph.partition_slab_z(b, R) if method == "slab" else graph.partition_rcb(b, R, weights)
    subs = graph.build_subgraphs(b, part, R)
    n_eff = sum((1.0 / sg.node_deg).sum() for sg in subs)
    e_eff = sum((1.0 / sg.edge_deg).sum() for sg in subs)
    assert abs(n_eff - b.n_nodes) < 1e-9
    assert abs(e_eff - b.n_edges) < 1e-9
    # an edge lies on at most 4 elements (an element edge line); irregular cuts can give d = 3
    assert set(np.unique(np.concatenate([sg.edge_deg for sg in subs])).tolist()) <= {1, 2, 3, 4}
    # every unpartitioned edge appears on at least one rank
    keys = np.unique(np.concatenate([sg.gid[sg.recv] * b.n_nodes + sg.gid[sg.send] for sg in subs]))
    assert np.array_equal(keys, b.recv * b.n_nodes + b.send)


def test_rcb_uniform_octants_and_weights():
    b = graph.build_brick((4, 4, 4), 1, with_edges=False)
    part = graph.partition_rcb(b, 8)
    for r in range(8):
        ijk = b.elem_ijk[part == r]
        assert ijk.shape[0] == 8
        assert np.all(ijk.max(axis=0) - ijk.min(axis=0) == 1)   # each part a 2x2x2 octant
    w = np.array([1.0, 3.0])
    part = graph.partition_rcb(b, 2, w)
    assert (part == 0).sum() == 16 and (part == 1).sum() == 48


def test_jitter_bounds_and_boundary():
    nel, p, frac = (3, 3, 3), 5, 0.2
    b0 = graph.build_brick(nel, p)
    jit = np.random.default_rng(3).uniform(-1, 1, size=(b0.n_nodes, 3))
    b1 = graph.build_brick(nel, p, jitter=jit, jitter_frac=frac)
    L = b0.L[0]
    c = np.unique(b0.pos[:, 0])
    sp = np.minimum(np.r_[np.inf, np.diff(c)], np.r_[np.diff(c), np.inf])
    iz, iy, ix = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    idx = [ix.ravel(), iy.ravel(), iz.ravel()]
    for a in range(3):
        off = b1.pos[:, a] - b0.pos[:, a]
        assert np.all(np.abs(off) <= frac * sp[idx[a]] + 1e-15)
        on_face = (idx[a] == 0) | (idx[a] == L - 1)
        assert np.all(off[on_face] == 0.0)
        assert np.abs(off[~on_face]).max() > 0.5 * frac * sp.min()


def test_uneven_partition_recipe():
    import synthetic as syn
    n, w = syn.uneven_brick(64, 50, 5000, 0)
    assert n == 41 and w.sum() == 41 ** 3 and w.min() >= 1
    c = syn.log_uniform_counts(64, 50, 5000, 0)
    assert np.all((c >= 50) & (c <= 5000))
    r = syn.rescale_counts([1, 2, 3], 12)
    assert r.sum() == 12 and list(r) == [2, 4, 6]
