"""The window sampling of the full-size GPU checks (CPU only).

* The counter-hashed input generator gives the same values on numpy arrays and
  torch tensors, on grids that BF16 (8 bits) and FP32 (16 bits) hold exactly.
* On a brick small enough for the whole-graph oracle, the oracle evaluated on
  the ball of a node inside a window brick (``fullsize_util.oracle_at``) equals
  the whole-graph stack at that node: outputs, input gradients and the
  in-edges' values, for centres in the interior, on faces and at corners."""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import graph as og

import fullsize_util as fu
from ball_util import stack_on_nodes


def test_hashed_values_agree_between_numpy_and_torch():
    c = np.arange(0, 200_000, dtype=np.int64) * 7919 + (1 << 44) + 3
    for bits in (8, 16):
        a = syn.hashed_values(c, 9, bits)
        t = syn.hashed_values(torch.from_numpy(c), 9, bits)
        assert t.dtype == torch.float32
        assert np.array_equal(a, t.double().numpy())
        step = 4.0 / (1 << bits)
        assert a.min() >= -2.0 and a.max() < 2.0
        assert np.array_equal(np.round(a / step) * step, a)           # on the grid
        n, k = c.size, 1 << bits      # grid points hit: as many as uniform draws hit on average
        assert abs(np.unique(a).size - k * (1 - np.exp(-n / k))) < 0.01 * k
        assert abs(a.mean()) < 0.02 and abs(a.std() - 4 / np.sqrt(12)) < 0.02
    a8 = syn.hashed_values(c, 9, 8)
    assert np.array_equal(torch.from_numpy(a8).float().to(torch.bfloat16).double().numpy(), a8)
    # different seeds and neighbouring counters give unrelated values
    assert np.corrcoef(syn.hashed_values(c, 9, 16), syn.hashed_values(c, 10, 16))[0, 1] < 0.02
    assert np.corrcoef(syn.hashed_values(c, 9, 16), syn.hashed_values(c + 1, 9, 16))[0, 1] < 0.02


@pytest.fixture(scope="module")
def case():
    nel, p, H, M = (5, 4, 6), 2, 5, 2
    b = og.build_brick(nel, p)
    N = b.n_nodes
    params = syn.gnn_params(7, H, 1, M, randomize_affine=True)
    x0 = fu.hashed_rows(np.arange(N), H, fu.SEED_X, 16)
    e0 = fu.hashed_rows(b.recv * N + b.send, H, fu.SEED_E, 8)
    dx_top = fu.hashed_rows(np.arange(N), H, fu.SEED_D, 16)
    full = stack_on_nodes(params["layers"], N, b.recv, b.send, np.arange(N), x0, e0, dx_top)
    return nel, p, H, b, params["layers"], dx_top, full


@pytest.mark.parametrize("ijk", [(5, 4, 6), (0, 0, 0), (10, 8, 12), (3, 0, 7), (7, 8, 1)])
@pytest.mark.parametrize("grads", [True, False])
def test_window_ball_equals_whole_graph(case, ijk, grads):
    nel, p, H, b, layers, dx_top, (eid_f, xM, eM, dx0, de0) = case
    L = b.L
    centre = ijk[0] + L[0] * (ijk[1] + L[1] * ijk[2])
    w = fu.Window(nel, p, centre, 2 * len(layers) + 1 if grads else len(layers))
    assert w.Nw < b.n_nodes or ijk == (5, 4, 6)
    assert np.array_equal(w.glob(w.local(np.arange(w.Nw) * 0 + centre)), [centre] * w.Nw)
    s = fu.oracle_at(layers, w, H, lambda g: dx_top[g], grads=grads)
    N = b.n_nodes
    keys_full = b.recv * N + b.send
    mine = b.recv == centre
    assert np.array_equal(s["keys"], keys_full[mine])
    assert np.allclose(s["x"], xM[centre], rtol=0, atol=1e-12)
    assert np.allclose(s["e"], eM[mine], rtol=0, atol=1e-12)
    if grads:
        assert np.allclose(s["dx"], dx0[centre], rtol=0, atol=1e-12)
        assert np.allclose(s["de"], de0[mine], rtol=0, atol=1e-12)
