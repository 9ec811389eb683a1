"""The oracle's layer stack on a graph ball, for checking sampled outputs of a
graph too large for the oracle as a whole.

M layers of Eq. 5a-5e read one hop per layer: a node's output after layer l
depends only on the inputs within l hops of it. So on the sub-graph induced by
the nodes within r hops of a centre node c (every edge between two of them,
weights of the unpartitioned graph, d = 1), the forward values of a node at
distance s are exact through layer r - s. The adjoint (Eq. 3) of the input at c
collects the outputs within M hops of c, each of which reads the inputs within M
hops of it: r = 2M + 1 makes dL/dx_0 at c and dL/de_0 on c's in-edges exact as
well (the extra hop covers the sender of an in-edge)."""
from __future__ import annotations

import numpy as np

from oracle import graph as og
from oracle import model as om


def neighbour_csr(N: int, recv: np.ndarray, send: np.ndarray):
    """(ptr, nbr): the in-neighbours of node v are nbr[ptr[v]:ptr[v + 1]] (the
    mesh graph holds both directions of every edge, so these are all its
    neighbours)."""
    order = np.argsort(recv, kind="stable")
    ptr = np.zeros(N + 1, dtype=np.int64)
    ptr[1:] = np.cumsum(np.bincount(recv, minlength=N))
    return ptr, send[order]


def ball(ptr: np.ndarray, nbr: np.ndarray, centre: int, radius: int) -> np.ndarray:
    """Global ids within `radius` hops of `centre`, ascending (breadth-first)."""
    seen = {int(centre)}
    frontier = [int(centre)]
    for _ in range(radius):
        nxt = []
        for v in frontier:
            for u in nbr[ptr[v]:ptr[v + 1]]:
                u = int(u)
                if u not in seen:
                    seen.add(u)
                    nxt.append(u)
        frontier = nxt
    return np.array(sorted(seen), dtype=np.int64)


def stack_on_nodes(layers: list, N: int, recv: np.ndarray, send: np.ndarray, nodes: np.ndarray,
                   x0: np.ndarray, e0: np.ndarray, dx_top: np.ndarray, backward: bool = True):
    """Forward and adjoint of the layers on the sub-graph induced by `nodes`.

    recv/send: the global directed edges, sorted by recv * N + send (the edge
    id indexes e0); x0 [N, H], e0 [E, H]: layer inputs; dx_top [N, H]: dL/dx of
    the last layer's output (dL/de of it is zero). Returns (edge ids of the
    sub-graph, x_M and dL/dx_0 per node of `nodes`, e_M and dL/de_0 per edge id)."""
    inside = np.zeros(N, dtype=bool)
    inside[nodes] = True
    eid = np.nonzero(inside[recv] & inside[send])[0]
    sub = og.subgraphs_of_sets(N, [nodes], [recv[eid] * N + send[eid]], with_halo=False)[0]
    xs, es = [x0[nodes]], [e0[eid]]
    caches = []
    for lp in layers:
        xs, es, c = om.layer_forward(lp, [sub], xs, es)
        caches.append(c)
    if not backward:
        return eid, xs[0], es[0], None, None
    dx, de = [dx_top[nodes]], [np.zeros_like(es[0])]
    for lp, c in zip(reversed(layers), reversed(caches)):
        dx, de, _ = om.layer_backward(lp, [sub], c, dx, de)
    return eid, xs[0], es[0], dx[0], de[0]


def check_sample(layers, N, recv, send, ptr, nbr, centre, x0, e0, dx_top, grads: bool = True):
    """Exact (up to rounding) oracle values at one centre node: x_M and dL/dx_0
    of the node, and e_M and dL/de_0 of its in-edges (global edge ids). With
    grads=False the ball has M hops, enough for x_M and e_M only."""
    M = len(layers)
    nodes = ball(ptr, nbr, centre, 2 * M + 1 if grads else M)
    eid, xM, eM, dx0, de0 = stack_on_nodes(layers, N, recv, send, nodes, x0, e0, dx_top, backward=grads)
    k = int(np.searchsorted(nodes, centre))
    mine = recv[eid] == centre
    if not grads:
        return {"x": xM[k], "eid": eid[mine], "e": eM[mine]}
    return {"x": xM[k], "dx": dx0[k], "eid": eid[mine], "e": eM[mine], "de": de0[mine]}
