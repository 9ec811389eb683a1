"""Mesh-based graph generation and partitioning, plain numpy (oracle side).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Follows Sec. II-A of the paper:
* nodes sit at the Gauss-Legendre-Lobatto (GLL) quadrature points of each
  hexahedral element, (p+1)^3 per element, non-uniformly spaced;
* undirected edges connect neighbouring quadrature nodes inside an element
  (here: the 6-neighbour lattice stencil, so p=1 gives the element edges);
* local coincident nodes (same global id, same rank) are collapsed, giving
  the "reduced" distributed graph of Fig. 3(c);
* non-local coincident nodes (same global id on different ranks) get halo
  rows appended on each rank (Fig. 4); edges held by several ranks carry the
  edge degree d_ij of Eq. 5b, nodes the node degree d_i of Eq. 8b.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def gll_points(p: int) -> np.ndarray:
    """GLL points on [-1, 1] for polynomial order p (Sec. II-A): the two
    endpoints plus the p-1 roots of the derivative of the Legendre polynomial P_p."""
    if p < 1:
        raise ValueError("polynomial order must be >= 1")
    inner = np.polynomial.legendre.Legendre.basis(p).deriv().roots()
    inner = np.sort(np.real(inner))
    return np.concatenate([[-1.0], inner, [1.0]])


@dataclass
class Brick:
    """A brick of nel[0] x nel[1] x nel[2] hex elements of order p."""
    nel: tuple
    p: int
    extent: tuple
    periodic: tuple
    L: tuple                 # lattice points per axis
    pos: np.ndarray          # [N, 3] node positions, row = global id
    elem_nodes: np.ndarray   # [n_elem, (p+1)^3] global ids of each element's GLL nodes
    elem_ijk: np.ndarray     # [n_elem, 3] integer element coordinates
    recv: np.ndarray         # [E] receiver global id of each directed edge (sorted)
    send: np.ndarray         # [E] sender global id

    @property
    def n_nodes(self) -> int:
        return self.pos.shape[0]

    @property
    def n_edges(self) -> int:
        return self.recv.shape[0]

    @property
    def n_elem(self) -> int:
        return self.elem_nodes.shape[0]


def _axis_coords(n_el: int, p: int, length: float, periodic: bool) -> np.ndarray:
    """1-D lattice coordinates: element e, local GLL index k -> lattice index e*p+k."""
    xi = gll_points(p)
    n_pts = n_el * p + (0 if periodic else 1)
    h = length / n_el
    c = np.empty(n_pts)
    for e in range(n_el):
        for k in range(p + 1):
            g = e * p + k
            if g < n_pts:
                c[g] = (e + 0.5 * (xi[k] + 1.0)) * h
    return c


def _axis_min_spacing(c: np.ndarray, length: float, periodic: bool) -> np.ndarray:
    """Smallest distance from each lattice point to its neighbours along the axis."""
    n = c.shape[0]
    left = np.full(n, np.inf)
    right = np.full(n, np.inf)
    left[1:] = c[1:] - c[:-1]
    right[:-1] = c[1:] - c[:-1]
    if periodic:
        wrap = c[0] + length - c[-1]
        left[0] = wrap
        right[-1] = wrap
    return np.minimum(left, right)


def local_stencil_pairs(p: int) -> np.ndarray:
    """Undirected (u, v) pairs of element-local node indices joined by the
    6-neighbour stencil; local index = i + (p+1)*(j + (p+1)*k)."""
    q = p + 1
    pairs = []
    for k in range(q):
        for j in range(q):
            for i in range(q):
                u = i + q * (j + q * k)
                if i < p:
                    pairs.append((u, u + 1))
                if j < p:
                    pairs.append((u, u + q))
                if k < p:
                    pairs.append((u, u + q * q))
    return np.array(pairs, dtype=np.int64)


def build_brick(nel, p, extent=(1.0, 1.0, 1.0), periodic=(False, False, False),
                jitter=None, jitter_frac: float = 0.0, with_edges: bool = True) -> Brick:
    """Build the R=1 graph of a GLL brick.

    Global node id of lattice point (ix, iy, iz) is ix + L0*(iy + L1*iz).
    ``jitter`` ([N,3] in [-1,1]) displaces each global node by
    jitter*jitter_frac*(smallest adjacent GLL spacing on that axis), except the
    normal coordinate of nodes on a non-periodic domain face.
    Directed edges (receiver, sender) are unique and sorted by receiver, then sender.
    """
    nel = tuple(int(v) for v in nel)
    periodic = tuple(bool(v) for v in periodic)
    extent = tuple(float(v) for v in extent)
    for a in range(3):
        if periodic[a] and nel[a] * p < 3:
            raise ValueError("periodic axis needs at least 3 lattice points")
    coords = [_axis_coords(nel[a], p, extent[a], periodic[a]) for a in range(3)]
    L = tuple(c.shape[0] for c in coords)
    N = L[0] * L[1] * L[2]
    iz, iy, ix = np.meshgrid(np.arange(L[2]), np.arange(L[1]), np.arange(L[0]), indexing="ij")
    ix, iy, iz = ix.ravel(), iy.ravel(), iz.ravel()          # row = global id
    idx = (ix, iy, iz)
    pos = np.stack([coords[a][idx[a]] for a in range(3)], axis=1)
    if jitter is not None and jitter_frac != 0.0:
        jitter = np.asarray(jitter, dtype=np.float64)
        for a in range(3):
            sp = _axis_min_spacing(coords[a], extent[a], periodic[a])[idx[a]]
            off = jitter[:, a] * jitter_frac * sp
            if not periodic[a]:
                off = np.where((idx[a] == 0) | (idx[a] == L[a] - 1), 0.0, off)
            pos[:, a] = pos[:, a] + off

    q = p + 1
    ez, ey, ex = np.meshgrid(np.arange(nel[2]), np.arange(nel[1]), np.arange(nel[0]), indexing="ij")
    elem_ijk = np.stack([ex.ravel(), ey.ravel(), ez.ravel()], axis=1)      # element id = ex + nx*(ey + ny*ez)
    lk, lj, li = np.meshgrid(np.arange(q), np.arange(q), np.arange(q), indexing="ij")
    li, lj, lk = li.ravel(), lj.ravel(), lk.ravel()                         # local index = i + q*(j + q*k)
    gx = (elem_ijk[:, 0:1] * p + li[None, :]) % L[0]
    gy = (elem_ijk[:, 1:2] * p + lj[None, :]) % L[1]
    gz = (elem_ijk[:, 2:3] * p + lk[None, :]) % L[2]
    elem_nodes = gx + L[0] * (gy + L[1] * gz)

    if with_edges:
        pairs = local_stencil_pairs(p)
        u = elem_nodes[:, pairs[:, 0]].ravel()
        v = elem_nodes[:, pairs[:, 1]].ravel()
        key = np.unique(np.concatenate([u * N + v, v * N + u]))
        recv, send = key // N, key % N
    else:
        recv = np.zeros(0, dtype=np.int64)
        send = np.zeros(0, dtype=np.int64)
    return Brick(nel=nel, p=p, extent=extent, periodic=periodic, L=L, pos=pos,
                 elem_nodes=elem_nodes, elem_ijk=elem_ijk, recv=recv, send=send)


# --------------------------------------------------------------------------- partitioning

def partition_slab_z(brick: Brick, R: int) -> np.ndarray:
    """Element -> part: R contiguous z-layers, part r holding layers
    [floor(r*nz/R), floor((r+1)*nz/R))."""
    nz = brick.nel[2]
    if not (1 <= R <= nz):
        raise ValueError("slab partition needs 1 <= R <= nz")
    ez = brick.elem_ijk[:, 2]
    bounds = [(r * nz) // R for r in range(R + 1)]
    part = np.empty(brick.n_elem, dtype=np.int64)
    for r in range(R):
        part[(ez >= bounds[r]) & (ez < bounds[r + 1])] = r
    return part


def partition_rcb(brick: Brick, R: int, target_weights=None) -> np.ndarray:
    """Element -> part by recursive coordinate bisection of element centres.

    Element centres are the undeformed lattice centres ((e_a + 0.5) * h_a).
    A set holding parts [r0, r0+R) splits into the first floor(R/2) parts and
    the rest, along the axis of largest centre extent (lowest axis on ties),
    after a stable sort by (coordinate, element id); the left share is
    floor(n * W_left / W + 0.5) elements, clamped so every part keeps at
    least one element. W sums the target weights of the parts on each side."""
    h = [brick.extent[a] / brick.nel[a] for a in range(3)]
    centre = np.stack([(brick.elem_ijk[:, a] + 0.5) * h[a] for a in range(3)], axis=1)
    return rcb_of_centres(centre, R, target_weights)


def rcb_of_centres(centre: np.ndarray, R: int, target_weights=None) -> np.ndarray:
    """Element -> part by recursive coordinate bisection of the given element
    centres ([n_elem, 3]), by the rule of ``partition_rcb``."""
    n_elem = centre.shape[0]
    if not (1 <= R <= n_elem):
        raise ValueError("RCB needs 1 <= R <= number of elements")
    w = np.ones(R) if target_weights is None else np.asarray(target_weights, dtype=np.float64)
    if w.shape != (R,) or np.any(w <= 0):
        raise ValueError("target weights must be R positive numbers")
    part = np.empty(n_elem, dtype=np.int64)

    def split(elems: np.ndarray, r0: int, nr: int):
        if nr == 1:
            part[elems] = r0
            return
        ext = [centre[elems, a].max() - centre[elems, a].min() for a in range(3)]
        axis = 0
        for a in (1, 2):
            if ext[a] > ext[axis]:
                axis = a
        order = np.lexsort((elems, centre[elems, axis]))
        elems = elems[order]
        nl = nr // 2
        wl = 0.0
        for k in range(r0, r0 + nl):
            wl += w[k]
        wr = 0.0
        for k in range(r0 + nl, r0 + nr):
            wr += w[k]
        n = elems.shape[0]
        cut = int(np.floor(float(n) * wl / (wl + wr) + 0.5))
        cut = min(max(cut, nl), n - (nr - nl))
        split(elems[:cut], r0, nl)
        split(elems[cut:], r0 + nl, nr - nl)

    split(np.arange(n_elem, dtype=np.int64), 0, R)
    return part


# --------------------------------------------------------------------------- reduced sub-graphs

@dataclass
class SubGraph:
    """Rank-r reduced sub-graph: local rows are the rank's unique global ids,
    ascending; edges are receiver-sorted local (recv, send) row pairs."""
    gid: np.ndarray          # [n_local] global id of each local row
    recv: np.ndarray         # [E_r] local receiver row
    send: np.ndarray         # [E_r] local sender row
    edge_deg: np.ndarray     # [E_r] d_ij: ranks holding this directed edge (Eq. 5b)
    node_deg: np.ndarray     # [n_local] d_i: ranks holding this node (Eq. 8b)
    # halo rows appended after the local rows (Fig. 4): one per (neighbour rank s, shared gid)
    halo_rank: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))   # s
    halo_src_row: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))  # local row k on rank s
    halo_local_row: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))  # row on this rank with the same gid

    @property
    def n_local(self) -> int:
        return self.gid.shape[0]

    @property
    def n_edges(self) -> int:
        return self.recv.shape[0]

    @property
    def n_halo(self) -> int:
        return self.halo_rank.shape[0]

    @property
    def neighbours(self) -> np.ndarray:
        return np.unique(self.halo_rank)


def partition_nodes(brick: Brick, part: np.ndarray, R: int) -> list:
    """Global ids held by each rank (union of its elements' nodes), ascending."""
    return [np.unique(brick.elem_nodes[part == r]) for r in range(R)]


def build_subgraphs(brick: Brick, part: np.ndarray, R: int, with_halo: bool = True) -> list:
    """Reduced distributed graph (Fig. 3(c)) with halo rows (Fig. 4).

    Each rank keeps the nodes and the stencil edges of its own elements; local
    coincident nodes are one row. d_ij counts the ranks whose element set
    produces the directed edge (i, j); d_i counts the ranks holding node i."""
    N = brick.n_nodes
    pairs = local_stencil_pairs(brick.p)
    node_sets = partition_nodes(brick, part, R)
    edge_sets = []
    for r in range(R):
        en = brick.elem_nodes[part == r]
        u = en[:, pairs[:, 0]].ravel()
        v = en[:, pairs[:, 1]].ravel()
        edge_sets.append(np.unique(np.concatenate([u * N + v, v * N + u])))
    return subgraphs_of_sets(N, node_sets, edge_sets, with_halo)


def subgraphs_of_sets(N: int, node_sets: list, edge_sets: list, with_halo: bool = True) -> list:
    """Reduced sub-graphs from each rank's global node ids (ascending) and
    directed edge keys recv*N + send (ascending): d_ij and d_i count the ranks
    holding each edge and node; halo rows as in ``build_subgraphs``."""
    R = len(node_sets)
    node_count = np.zeros(N, dtype=np.int64)
    for s in node_sets:
        node_count[s] += 1
    all_keys, key_count = np.unique(np.concatenate(edge_sets), return_counts=True)

    subs = []
    for r in range(R):
        gid = node_sets[r]
        row_of = {int(g): i for i, g in enumerate(gid)} if gid.shape[0] < 4096 else None
        keys = edge_sets[r]
        rg, sg = keys // N, keys % N
        if row_of is not None:
            recv = np.array([row_of[int(g)] for g in rg], dtype=np.int64)
            send = np.array([row_of[int(g)] for g in sg], dtype=np.int64)
        else:
            recv = np.searchsorted(gid, rg)
            send = np.searchsorted(gid, sg)
        edeg = key_count[np.searchsorted(all_keys, keys)]
        subs.append(SubGraph(gid=gid, recv=recv, send=send, edge_deg=edeg,
                             node_deg=node_count[gid]))
    if with_halo and R > 1:
        for r in range(R):
            hr, hsrc, hloc = [], [], []
            for s in range(R):
                if s == r:
                    continue
                shared = np.intersect1d(node_sets[r], node_sets[s], assume_unique=True)
                if shared.shape[0] == 0:
                    continue
                hr.append(np.full(shared.shape[0], s, dtype=np.int64))
                hsrc.append(np.searchsorted(node_sets[s], shared))
                hloc.append(np.searchsorted(node_sets[r], shared))
            if hr:
                subs[r].halo_rank = np.concatenate(hr)
                subs[r].halo_src_row = np.concatenate(hsrc)
                subs[r].halo_local_row = np.concatenate(hloc)
    return subs


def edge_attributes(pos: np.ndarray, sub: SubGraph) -> np.ndarray:
    """Edge input features [dx, dy, dz, |d|] with d = pos(sender) - pos(receiver)."""
    d = pos[sub.gid[sub.send]] - pos[sub.gid[sub.recv]]
    return np.concatenate([d, np.linalg.norm(d, axis=1, keepdims=True)], axis=1)


def unpartitioned(brick: Brick) -> list:
    """The R=1 graph as a one-rank sub-graph list (rows = global ids)."""
    N = brick.n_nodes
    return [SubGraph(gid=np.arange(N, dtype=np.int64), recv=brick.recv.copy(),
                     send=brick.send.copy(), edge_deg=np.ones(brick.n_edges, dtype=np.int64),
                     node_deg=np.ones(N, dtype=np.int64))]


# --------------------------------------------------------------------------- general element meshes

@dataclass
class ElementMesh:
    """A mesh of elements of any types (Sec. II-A: the graph construction and
    its distribution apply to any mesh made of finite elements). Element e
    holds the global nodes elem_nodes[elem_ptr[e]:elem_ptr[e+1]] and the
    undirected edges between its local nodes edge_pairs[k] = (u, v),
    k in [edge_ptr[e], edge_ptr[e+1])."""
    pos: np.ndarray
    elem_ptr: np.ndarray
    elem_nodes: np.ndarray
    edge_ptr: np.ndarray
    edge_pairs: np.ndarray
    recv: np.ndarray         # [E] receiver global id of each directed edge (sorted)
    send: np.ndarray         # [E] sender global id

    @property
    def n_nodes(self) -> int:
        return self.pos.shape[0]

    @property
    def n_edges(self) -> int:
        return self.recv.shape[0]

    @property
    def n_elem(self) -> int:
        return self.elem_ptr.shape[0] - 1

    def element(self, e: int):
        """Global node ids and global (u, v) edge pairs of element e."""
        nodes = self.elem_nodes[self.elem_ptr[e]:self.elem_ptr[e + 1]]
        pr = self.edge_pairs[self.edge_ptr[e]:self.edge_ptr[e + 1]]
        return nodes, nodes[pr[:, 0]], nodes[pr[:, 1]]


def element_mesh(pos, elem_ptr, elem_nodes, edge_ptr, edge_pairs) -> ElementMesh:
    """The R=1 graph of an element mesh: every element edge in both directions,
    unique, sorted by receiver and then sender."""
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    mesh = ElementMesh(pos=pos, elem_ptr=np.asarray(elem_ptr, dtype=np.int64),
                       elem_nodes=np.asarray(elem_nodes, dtype=np.int64),
                       edge_ptr=np.asarray(edge_ptr, dtype=np.int64),
                       edge_pairs=np.asarray(edge_pairs, dtype=np.int64).reshape(-1, 2),
                       recv=np.zeros(0, np.int64), send=np.zeros(0, np.int64))
    N = mesh.n_nodes
    keys = _element_edge_keys(mesh, range(mesh.n_elem))
    mesh.recv, mesh.send = keys // N, keys % N
    return mesh


def _element_edge_keys(mesh: ElementMesh, elems) -> np.ndarray:
    N = mesh.n_nodes
    ks = [np.zeros(0, np.int64)]
    for e in elems:
        _, u, v = mesh.element(e)
        ks.append(u * N + v)
        ks.append(v * N + u)
    return np.unique(np.concatenate(ks))


def element_centres(mesh: ElementMesh) -> np.ndarray:
    """Mean position of each element's nodes."""
    return np.stack([mesh.pos[mesh.element(e)[0]].mean(axis=0) for e in range(mesh.n_elem)])


def partition_rcb_elements(mesh: ElementMesh, R: int, target_weights=None) -> np.ndarray:
    return rcb_of_centres(element_centres(mesh), R, target_weights)


def partition_slab_elements(mesh: ElementMesh, R: int) -> np.ndarray:
    """R runs of the elements sorted by (centre z, element id); run r holds
    sorted positions [floor(r*n/R), floor((r+1)*n/R))."""
    n = mesh.n_elem
    if not (1 <= R <= n):
        raise ValueError("slab partition needs 1 <= R <= number of elements")
    order = np.lexsort((np.arange(n), element_centres(mesh)[:, 2]))
    part = np.empty(n, dtype=np.int64)
    for r in range(R):
        part[order[(r * n) // R:((r + 1) * n) // R]] = r
    return part


def build_element_subgraphs(mesh: ElementMesh, part: np.ndarray, R: int, with_halo: bool = True) -> list:
    """Reduced distributed graph of an element mesh: rank r keeps the nodes and
    edges of its elements (Fig. 3(c)), with halo rows (Fig. 4)."""
    node_sets, edge_sets = [], []
    for r in range(R):
        elems = np.nonzero(np.asarray(part) == r)[0]
        node_sets.append(np.unique(np.concatenate([mesh.element(e)[0] for e in elems])))
        edge_sets.append(_element_edge_keys(mesh, elems))
    return subgraphs_of_sets(mesh.n_nodes, node_sets, edge_sets, with_halo)


def element_mesh_unpartitioned(mesh: ElementMesh) -> list:
    """The R=1 graph of an element mesh as a one-rank sub-graph list."""
    N = mesh.n_nodes
    return [SubGraph(gid=np.arange(N, dtype=np.int64), recv=mesh.recv.copy(), send=mesh.send.copy(),
                     edge_deg=np.ones(mesh.n_edges, dtype=np.int64), node_deg=np.ones(N, dtype=np.int64))]
