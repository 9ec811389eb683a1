"""The sampling the full-size GPU checks rely on (CPU only): the oracle's
M-layer stack evaluated on a ball of 2M + 1 hops around a node gives, at that
node, the values of the stack on the whole graph (outputs and input gradients,
to rounding), and a ball of M hops does not give the gradients."""
import numpy as np
import pytest

import synthetic as syn
from oracle import graph as og

from ball_util import ball, check_sample, neighbour_csr, stack_on_nodes


@pytest.fixture(scope="module")
def case():
    b = og.build_brick((6, 6, 6), 2)
    H, M = 6, 3
    params = syn.gnn_params(3, H, 1, M, randomize_affine=True)
    rng = np.random.default_rng(4)
    x0 = rng.standard_normal((b.n_nodes, H))
    e0 = rng.standard_normal((b.n_edges, H))
    dx_top = rng.standard_normal((b.n_nodes, H))
    full = stack_on_nodes(params["layers"], b.n_nodes, b.recv, b.send, np.arange(b.n_nodes), x0, e0, dx_top)
    return b, params["layers"], x0, e0, dx_top, full


def test_edges_sorted_and_symmetric(case):
    b = case[0]
    N = b.n_nodes
    k = b.recv * N + b.send
    assert np.all(np.diff(k) > 0)
    assert np.array_equal(np.sort(b.send * N + b.recv), k)


def test_ball_is_the_lattice_l1_ball(case):
    b = case[0]
    ptr, nbr = neighbour_csr(b.n_nodes, b.recv, b.send)
    L = np.array([13, 13, 13])
    ijk = np.stack(np.unravel_index(np.arange(b.n_nodes), L[::-1]), axis=1)[:, ::-1]
    c = int(np.ravel_multi_index((4, 3, 5)[::-1], L[::-1]))
    for r in (0, 1, 3, 6):
        want = np.nonzero(np.abs(ijk - ijk[c]).sum(axis=1) <= r)[0]
        assert np.array_equal(ball(ptr, nbr, c, r), want)


@pytest.mark.parametrize("centre", [0, 57, 1098, 1500])
def test_ball_of_2m_plus_1_hops_is_exact(case, centre):
    b, layers, x0, e0, dx_top, (eid_f, xM, eM, dx0, de0) = case
    ptr, nbr = neighbour_csr(b.n_nodes, b.recv, b.send)
    s = check_sample(layers, b.n_nodes, b.recv, b.send, ptr, nbr, centre, x0, e0, dx_top)
    assert ball(ptr, nbr, centre, 2 * len(layers) + 1).size < b.n_nodes // 3   # a real truncation
    assert s["eid"].size == int((b.recv == centre).sum()) > 0
    np.testing.assert_allclose(s["x"], xM[centre], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(s["dx"], dx0[centre], rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(s["e"], eM[s["eid"]], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(s["de"], de0[s["eid"]], rtol=1e-11, atol=1e-12)


def test_smaller_ball_misses_gradient_terms(case):
    b, layers, x0, e0, dx_top, (eid_f, xM, eM, dx0, de0) = case
    ptr, nbr = neighbour_csr(b.n_nodes, b.recv, b.send)
    c = 1098   # the lattice centre (6, 6, 6)
    M = len(layers)
    nodes = ball(ptr, nbr, c, M)
    _, xs, _, dxs, _ = stack_on_nodes(layers, b.n_nodes, b.recv, b.send, nodes, x0, e0, dx_top)
    k = int(np.searchsorted(nodes, c))
    np.testing.assert_allclose(xs[k], xM[c], rtol=1e-12, atol=1e-12)   # M hops: the forward is exact
    assert np.abs(dxs[k] - dx0[c]).max() > 1e-6 * np.abs(dx0[c]).max()
    s = check_sample(layers, b.n_nodes, b.recv, b.send, ptr, nbr, c, x0, e0, dx_top, grads=False)
    np.testing.assert_allclose(s["x"], xM[c], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(s["e"], eM[s["eid"]], rtol=1e-12, atol=1e-12)
