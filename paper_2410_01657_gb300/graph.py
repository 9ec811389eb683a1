"""Mesh graphs and partitions of libgnnmp as Python objects.

``MeshGraph`` wraps ``gnn_graph_build`` (the R=1 GLL-brick graph, Sec. II-A)
and ``gnn_graph_build_elements`` (a mesh of elements of any types),
``Partition`` wraps ``gnn_partition_halo`` / ``gnn_partition_elements``
(reduced sub-graphs, multiplicities and the halo copy list, Figs. 3-4), and
``DeviceGraph`` holds the partition's
arrays in device memory (allocated by torch) together with the
``gnn_graph_dev`` struct that the compute entry points take.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import binding as B


class MeshGraph:
    """R=1 graph of a brick of nel[0] x nel[1] x nel[2] hex elements of order p
    (or, built by ``from_elements``, of a general element mesh)."""

    def __init__(self, nel, p, extent=(1.0, 1.0, 1.0), periodic=(False, False, False),
                 jitter=None, jitter_frac=0.0):
        B.load()
        d = B.gnn_mesh_desc()
        for a in range(3):
            d.nel[a] = int(nel[a])
            d.extent[a] = float(extent[a])
            d.periodic[a] = 1 if periodic[a] else 0
        d.p = int(p)
        d.jitter_frac = float(jitter_frac)
        self._jitter = None
        if jitter is not None:
            self._jitter = np.ascontiguousarray(jitter, dtype=np.float64)
            d.jitter = self._jitter.ctypes.data_as(C.POINTER(C.c_double))
        h = C.c_void_p()
        B.call("gnn_graph_build", C.byref(d), C.byref(h))
        self._h = h
        self.info = B.gnn_graph_info()
        B.call("gnn_graph_get_info", self._h, C.byref(self.info))
        self.nel, self.p = tuple(int(v) for v in nel), int(p)

    @classmethod
    def from_elements(cls, pos, elem_ptr, elem_nodes, edge_ptr, edge_pairs) -> "MeshGraph":
        """Graph of a general element mesh: element e holds the global nodes
        elem_nodes[elem_ptr[e]:elem_ptr[e+1]] and the undirected edges between
        its local nodes edge_pairs[k] = (u, v), k in [edge_ptr[e], edge_ptr[e+1])."""
        B.load()
        arrs = [np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3),
                np.ascontiguousarray(elem_ptr, dtype=np.int64),
                np.ascontiguousarray(elem_nodes, dtype=np.int64),
                np.ascontiguousarray(edge_ptr, dtype=np.int64),
                np.ascontiguousarray(edge_pairs, dtype=np.int32).reshape(-1, 2)]
        d = B.gnn_elem_mesh_desc()
        d.n_nodes = arrs[0].shape[0]
        d.n_elem = arrs[1].shape[0] - 1
        d.pos, d.elem_ptr, d.elem_nodes, d.edge_ptr, d.edge_pairs = (B.ptr(a) for a in arrs)
        self = cls.__new__(cls)
        h = C.c_void_p()
        B.call("gnn_graph_build_elements", C.byref(d), C.byref(h))
        self._h = h
        self._jitter = None
        self.info = B.gnn_graph_info()
        B.call("gnn_graph_get_info", self._h, C.byref(self.info))
        self.nel, self.p = None, 0
        return self

    @property
    def is_brick(self) -> bool:
        return int(self.info.kind) == B.GNN_GRAPH_BRICK

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            B.load().gnn_graph_destroy(h)
            self._h = None

    @property
    def n_nodes(self) -> int:
        return int(self.info.n_nodes)

    @property
    def n_edges(self) -> int:
        return int(self.info.n_edges)

    @property
    def L(self) -> tuple:
        return tuple(int(v) for v in self.info.L)

    def pos(self) -> np.ndarray:
        out = np.empty((self.n_nodes, 3), dtype=np.float64)
        B.call("gnn_graph_copy_pos", self._h, B.ptr(out))
        return out

    def csr(self):
        rp = np.empty(self.n_nodes + 1, dtype=np.int64)
        col = np.empty(self.n_edges, dtype=np.int64)
        B.call("gnn_graph_copy_csr", self._h, B.ptr(rp), B.ptr(col))
        return rp, col

    def elements(self) -> np.ndarray:
        """Brick: [n_elem, (p+1)^3] node ids; element mesh: the flat node lists
        (offsets from ``element_ptr``)."""
        out = np.empty(int(self.info.n_elem_nodes), dtype=np.int64)
        B.call("gnn_graph_copy_elements", self._h, B.ptr(out))
        return out.reshape(int(self.info.n_elem), -1) if self.is_brick else out

    def element_ptr(self) -> np.ndarray:
        out = np.empty(int(self.info.n_elem) + 1, dtype=np.int64)
        B.call("gnn_graph_copy_element_ptr", self._h, B.ptr(out))
        return out

    def partition(self, R: int, method: str = "rcb", target_weights=None, elem_part=None) -> "Partition":
        """R sub-graphs by ``method`` ("rcb" or "slab"), or by the given
        element -> sub-graph map ``elem_part``."""
        return Partition(self, R, method, target_weights, elem_part)


_ARRAYS = {
    "row_offsets": (B.GNN_P_ROW_OFFSETS, np.int64, lambda i: (i.n_parts + 1,)),
    "edge_offsets": (B.GNN_P_EDGE_OFFSETS, np.int64, lambda i: (i.n_parts + 1,)),
    "row_gid": (B.GNN_P_ROW_GID, np.int64, lambda i: (i.n_rows,)),
    "row_ptr": (B.GNN_P_ROW_PTR, np.int32, lambda i: (i.n_rows + 1,)),
    "col": (B.GNN_P_COL, np.int32, lambda i: (i.n_edges,)),
    "edge_deg": (B.GNN_P_EDGE_DEG, np.uint8, lambda i: (i.n_edges,)),
    "edge_w": (B.GNN_P_EDGE_W, np.float32, lambda i: (i.n_edges,)),
    "node_deg": (B.GNN_P_NODE_DEG, np.uint8, lambda i: (i.n_rows,)),
    "node_w": (B.GNN_P_NODE_W, np.float32, lambda i: (i.n_rows,)),
    "t_ptr": (B.GNN_P_T_PTR, np.int32, lambda i: (i.n_rows + 1,)),
    "t_eid": (B.GNN_P_T_EID, np.int32, lambda i: (i.n_edges,)),
    "halo_ptr": (B.GNN_P_HALO_PTR, np.int32, lambda i: (i.n_shared + 1,)),
    "halo_rows": (B.GNN_P_HALO_ROWS, np.int32, lambda i: (i.n_copies,)),
    "edge_tiles": (B.GNN_P_EDGE_TILES, np.int32, lambda i: (i.n_edge_tiles + 1,)),
    "edge_attr": (B.GNN_P_EDGE_ATTR, np.float32, lambda i: (i.n_edges, 4)),
    "row_pos": (B.GNN_P_ROW_POS, np.float64, lambda i: (i.n_rows, 3)),
    "part_stats": (B.GNN_P_PART_STATS, np.int64, lambda i: (i.n_parts, 3)),
    "tile_meta": (B.GNN_P_TILE_META, np.uint8, lambda i: (i.n_edge_tiles * B.GNN_TILE_META_BYTES,)),
}


class Partition:
    """R reduced sub-graphs of a MeshGraph, concatenated (host arrays)."""

    def __init__(self, graph: MeshGraph, R: int, method: str = "rcb", target_weights=None, elem_part=None):
        h = C.c_void_p()
        if elem_part is not None:
            ep = np.ascontiguousarray(elem_part, dtype=np.int32)
            if ep.shape != (int(graph.info.n_elem),):
                raise ValueError("elem_part must hold one sub-graph index per element")
            B.call("gnn_partition_elements", graph._h, int(R), B.ptr(ep), C.byref(h))
        else:
            m = {"slab": B.GNN_PART_SLAB_Z, "slab_z": B.GNN_PART_SLAB_Z, "rcb": B.GNN_PART_RCB}[method]
            w = None
            if target_weights is not None:
                w = np.ascontiguousarray(target_weights, dtype=np.float64)
            B.call("gnn_partition_halo", graph._h, int(R), m, B.ptr(w), C.byref(h))
        self._h = h
        self.graph = graph
        self.info = B.gnn_partition_info()
        B.call("gnn_partition_get_info", self._h, C.byref(self.info))
        self._cache = {}

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            B.load().gnn_partition_destroy(h)
            self._h = None

    @property
    def n_parts(self) -> int:
        return int(self.info.n_parts)

    @property
    def n_rows(self) -> int:
        return int(self.info.n_rows)

    @property
    def n_edges(self) -> int:
        return int(self.info.n_edges)

    def array(self, name: str) -> np.ndarray:
        if name not in self._cache:
            what, dt, shape = _ARRAYS[name]
            out = np.empty(shape(self.info), dtype=dt)
            B.call("gnn_partition_copy", self._h, what, B.ptr(out), out.nbytes)
            self._cache[name] = out
        return self._cache[name]

    @property
    def tile_edges(self) -> int:
        return int(self.info.tile_edges)

    def set_tile_edges(self, tile_edges: int) -> "Partition":
        """Rebuild the edge tiles with at most `tile_edges` edges each (device
        copies made before keep the old tiles)."""
        B.call("gnn_partition_set_tile_edges", self._h, int(tile_edges))
        B.call("gnn_partition_get_info", self._h, C.byref(self.info))
        self._cache.pop("edge_tiles", None)
        self._cache.pop("tile_meta", None)
        return self

    def receivers(self) -> np.ndarray:
        rp = self.array("row_ptr").astype(np.int64)
        return np.repeat(np.arange(self.n_rows, dtype=np.int64), np.diff(rp))

    def to_device(self, device="cuda") -> "DeviceGraph":
        return DeviceGraph(self, device)


class DeviceGraph:
    """A partition's arrays in device memory plus the ``gnn_graph_dev`` view of them."""

    def __init__(self, part: Partition, device="cuda"):
        import torch

        self.part = part
        self.device = torch.device(device)
        t = {}
        for name in ("row_ptr", "col", "edge_w", "t_ptr", "t_eid", "node_w", "halo_ptr", "halo_rows",
                     "edge_tiles", "tile_meta"):
            t[name] = torch.from_numpy(part.array(name)).to(self.device)
        self.t = t
        g = B.gnn_graph_dev()
        g.n_rows = part.n_rows
        g.n_edges = part.n_edges
        g.row_ptr = B.ptr(t["row_ptr"])
        g.col = B.ptr(t["col"])
        g.edge_w = B.ptr(t["edge_w"])
        g.t_ptr = B.ptr(t["t_ptr"])
        g.t_eid = B.ptr(t["t_eid"])
        g.node_w = B.ptr(t["node_w"])
        g.n_shared = int(part.info.n_shared)
        g.halo_ptr = B.ptr(t["halo_ptr"])
        g.halo_rows = B.ptr(t["halo_rows"])
        g.n_edge_tiles = int(part.info.n_edge_tiles)
        g.edge_tiles = B.ptr(t["edge_tiles"])
        g.max_in_degree = int(part.info.max_in_degree)
        g.tile_meta = B.ptr(t["tile_meta"])
        self.struct = g
        self._tile_edges = part.tile_edges

    @property
    def n_rows(self) -> int:
        return self.part.n_rows

    @property
    def n_edges(self) -> int:
        return self.part.n_edges

    @property
    def tile_edges(self) -> int:
        """Edge cap of the tiles held on the device."""
        return self._tile_edges

    def retile(self, tile_edges: int) -> "DeviceGraph":
        """Re-tile the partition (at most `tile_edges` edges per edge tile) and
        upload only the tile arrays; every other device array is kept."""
        import torch

        part = self.part
        if part.tile_edges != tile_edges:
            part.set_tile_edges(tile_edges)
        for name in ("edge_tiles", "tile_meta"):
            self.t[name] = torch.from_numpy(part.array(name)).to(self.device)
        self.struct.n_edge_tiles = int(part.info.n_edge_tiles)
        self.struct.edge_tiles = B.ptr(self.t["edge_tiles"])
        self.struct.tile_meta = B.ptr(self.t["tile_meta"])
        self._tile_edges = int(tile_edges)
        return self

    def edge_attr(self):
        """Edge attributes [dx, dy, dz, |d|] (graph geometry, FP32 [n_edges x 4]),
        uploaded on first use and kept on the device with the graph."""
        import torch
        if "edge_attr" not in self.t:
            self.t["edge_attr"] = torch.from_numpy(self.part.array("edge_attr")).to(self.device)
        return self.t["edge_attr"]
