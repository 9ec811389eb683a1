"""Full-size sampled parity on GLL bricks too large for the host oracle as a
whole: the oracle runs on the ball of a sampled node inside a small window
brick, and the inputs are counter-hashed so that any row can be regenerated on
either side.

* Window: the elements covering the lattice box centre +- radius. On a
  conforming brick the graph between the window's nodes is the window brick's
  own graph (an edge joins lattice neighbours of one element, and an element
  holding two window nodes' edge is a window element), and every path of at
  most `radius` hops from the centre stays in the box, so the ball found in the
  window is the ball of the full graph.
* Inputs (``synthetic.hashed_values``): x0 of global node g from counter
  g * H + c (16-bit grid, exact in FP32), e0 of the directed edge (receiver r,
  sender s) from counter (r * N + s) * H + c (8-bit grid, exact in BF16), the
  upstream gradient of partition row i from counter i * H + c."""
from __future__ import annotations

import numpy as np
import torch

import synthetic as syn
from oracle import graph as og

from ball_util import ball, neighbour_csr, stack_on_nodes

SEED_X, SEED_E, SEED_D = 101, 202, 303


def hashed_rows(keys, H: int, seed: int, bits: int):
    """[len(keys), H] hashed values of the given int64 row keys (numpy float64 or
    torch float32 on the keys' device)."""
    if isinstance(keys, np.ndarray):
        return syn.hashed_values(keys.astype(np.int64)[:, None] * H + np.arange(H, dtype=np.int64), seed, bits)
    cols = torch.arange(H, dtype=torch.int64, device=keys.device)
    return syn.hashed_values(keys[:, None] * H + cols, seed, bits)


class Window:
    """The window brick around a lattice point of the nel^3-element brick of order p."""

    def __init__(self, nel, p: int, centre: int, radius: int):
        self.L = tuple(n * p + 1 for n in nel)
        self.N = self.L[0] * self.L[1] * self.L[2]
        c = (centre % self.L[0], (centre // self.L[0]) % self.L[1], centre // (self.L[0] * self.L[1]))
        first = [max(0, (c[a] - radius) // p) for a in range(3)]
        last = [min(nel[a] - 1, -(-(c[a] + radius) // p) - 1) for a in range(3)]
        self.off = np.array([f * p for f in first], dtype=np.int64)
        self.brick = og.build_brick(tuple(last[a] - first[a] + 1 for a in range(3)), p)
        self.Lw = self.brick.L
        self.Nw = self.brick.n_nodes
        self.centre = int(self.local(np.array([centre]))[0])

    def glob(self, local):
        """Global lattice ids of window node ids."""
        local = np.asarray(local, dtype=np.int64)
        i = local % self.Lw[0] + self.off[0]
        j = (local // self.Lw[0]) % self.Lw[1] + self.off[1]
        k = local // (self.Lw[0] * self.Lw[1]) + self.off[2]
        return i + self.L[0] * (j + self.L[1] * k)

    def local(self, g):
        """Window node ids of global lattice ids (which must lie in the window)."""
        g = np.asarray(g, dtype=np.int64)
        i = g % self.L[0] - self.off[0]
        j = (g // self.L[0]) % self.L[1] - self.off[1]
        k = g // (self.L[0] * self.L[1]) - self.off[2]
        assert (i >= 0).all() and (j >= 0).all() and (k >= 0).all()
        assert (i < self.Lw[0]).all() and (j < self.Lw[1]).all() and (k < self.Lw[2]).all()
        return i + self.Lw[0] * (j + self.Lw[1] * k)


class _Lazy:
    def __init__(self, fn):
        self.fn = fn

    def __getitem__(self, idx):
        return self.fn(np.asarray(idx, dtype=np.int64))


def oracle_at(layers, w: Window, H: int, dx_glob_of, grads: bool = True) -> dict:
    """The oracle's exact values at the window's centre node: x_M (and dL/dx_0),
    and, keyed by global (receiver, sender) pair keys, e_M (and dL/de_0) of its
    in-edges. dx_glob_of(global ids) -> [n, H] upstream gradient summed over
    each node's rows."""
    M = len(layers)
    b = w.brick
    ptr, nbr = neighbour_csr(w.Nw, b.recv, b.send)
    nodes = ball(ptr, nbr, w.centre, 2 * M + 1 if grads else M)
    x0 = _Lazy(lambda idx: hashed_rows(w.glob(idx), H, SEED_X, 16))
    e0 = _Lazy(lambda idx: hashed_rows(w.glob(b.recv[idx]) * w.N + w.glob(b.send[idx]), H, SEED_E, 8))
    dx = _Lazy(lambda idx: dx_glob_of(w.glob(idx)))
    eid, xM, eM, dx0, de0 = stack_on_nodes(layers, w.Nw, b.recv, b.send, nodes, x0, e0, dx, backward=grads)
    k = int(np.searchsorted(nodes, w.centre))
    mine = b.recv[eid] == w.centre
    keys = w.glob(b.recv[eid[mine]]) * w.N + w.glob(b.send[eid[mine]])
    out = {"x": xM[k], "keys": keys, "e": eM[mine]}
    if grads:
        out["dx"], out["de"] = dx0[k], de0[mine]
    return out


def device_inputs(part, H: int, N: int, dev, edge_dtype=torch.bfloat16, chunk: int = 1 << 21):
    """x0 [n_rows, H] FP32, e0 [n_edges, H] and the upstream gradient [n_rows, H]
    of the partition's rows and edges, generated on the device."""
    gid = torch.from_numpy(part.array("row_gid").astype(np.int64)).to(dev)
    x0 = hashed_rows(gid, H, SEED_X, 16)
    dx = hashed_rows(torch.arange(part.n_rows, dtype=torch.int64, device=dev), H, SEED_D, 16)
    rp = torch.from_numpy(part.array("row_ptr").astype(np.int64)).to(dev)
    recv = torch.repeat_interleave(torch.arange(part.n_rows, dtype=torch.int64, device=dev), rp[1:] - rp[:-1])
    col = torch.from_numpy(part.array("col").astype(np.int64)).to(dev)
    e0 = torch.empty(part.n_edges, H, dtype=edge_dtype, device=dev)
    for a in range(0, part.n_edges, chunk):
        b = min(part.n_edges, a + chunk)
        key = gid[recv[a:b]] * N + gid[col[a:b]]
        e0[a:b] = hashed_rows(key, H, SEED_E, 8).to(edge_dtype)
    del recv, col, rp
    return x0, e0, dx
