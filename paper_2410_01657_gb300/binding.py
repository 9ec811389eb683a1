"""ctypes binding of libgnnmp (include/gnnmp.h): argument marshalling only.

Every step of the consistent message-passing path runs inside libgnnmp's CUDA
kernels; this module only converts Python/torch arguments into the C structs
and pointers the library expects. There is no fallback: if the shared library
is missing or fails to load, importing the symbols raises.
"""
from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libgnnmp.so")

GNN_OK = 0
GNN_EINVAL, GNN_ESHAPE, GNN_EDTYPE, GNN_ECUDA = -1, -2, -3, -4
GNN_EHALO, GNN_ETIMEOUT, GNN_ENOMEM, GNN_EUNSUPPORTED = -5, -6, -7, -8

GNN_PART_SLAB_Z, GNN_PART_RCB = 0, 1
GNN_GRAPH_BRICK, GNN_GRAPH_ELEMENTS = 0, 1
GNN_PREC_FP32, GNN_PREC_BF16 = 0, 1
GNN_HALO_SYNC, GNN_HALO_NONE = 0, 1
GNN_FLAG_NO_EDGE_OUT = 1
GNN_FLAG_ADJ_ONE_LINEAR = 2
GNN_EDGE_FWD_AUTO, GNN_EDGE_FWD_RT, GNN_EDGE_FWD_WS, GNN_EDGE_FWD_ONE, GNN_EDGE_FWD_TM = 0, 1, 2, 3, 4
GNN_MAX_LIN = 8
GNN_EDGE_TILE = 128
GNN_NODE_TILE = 128

(GNN_P_ROW_OFFSETS, GNN_P_EDGE_OFFSETS, GNN_P_ROW_GID, GNN_P_ROW_PTR, GNN_P_COL, GNN_P_EDGE_DEG,
 GNN_P_EDGE_W, GNN_P_NODE_DEG, GNN_P_NODE_W, GNN_P_T_PTR, GNN_P_T_EID, GNN_P_HALO_PTR,
 GNN_P_HALO_ROWS, GNN_P_EDGE_TILES, GNN_P_EDGE_ATTR, GNN_P_ROW_POS, GNN_P_PART_STATS,
 GNN_P_TILE_META) = range(18)
GNN_TILE_META_BYTES = 2048


class GnnError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libgnnmp error {code}: {msg}")
        self.code = code


class gnn_mesh_desc(C.Structure):
    _fields_ = [("nel", C.c_int32 * 3), ("p", C.c_int32), ("extent", C.c_double * 3),
                ("periodic", C.c_int32 * 3), ("jitter_frac", C.c_double),
                ("jitter", C.POINTER(C.c_double))]


class gnn_elem_mesh_desc(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("pos", C.c_void_p), ("n_elem", C.c_int64),
                ("elem_ptr", C.c_void_p), ("elem_nodes", C.c_void_p), ("edge_ptr", C.c_void_p),
                ("edge_pairs", C.c_void_p)]


class gnn_graph_info(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_edges", C.c_int64), ("n_elem", C.c_int64),
                ("L", C.c_int32 * 3), ("p", C.c_int32), ("n_elem_nodes", C.c_int64),
                ("kind", C.c_int32), ("max_degree", C.c_int32)]


class gnn_partition_info(C.Structure):
    _fields_ = [("n_parts", C.c_int32), ("max_in_degree", C.c_int32), ("n_rows", C.c_int64),
                ("n_edges", C.c_int64), ("n_shared", C.c_int64), ("n_copies", C.c_int64),
                ("n_edge_tiles", C.c_int64), ("n_node_tiles", C.c_int64), ("tile_edges", C.c_int32),
                ("reserved", C.c_int32)]


class gnn_tune_entry(C.Structure):
    _fields_ = [("edge_fwd_kernel", C.c_int32), ("ctas_per_sm", C.c_int32), ("ms", C.c_float)]


class gnn_graph_dev(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("n_edges", C.c_int64),
                ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("edge_w", C.c_void_p),
                ("t_ptr", C.c_void_p), ("t_eid", C.c_void_p), ("node_w", C.c_void_p),
                ("n_shared", C.c_int64), ("halo_ptr", C.c_void_p), ("halo_rows", C.c_void_p),
                ("n_edge_tiles", C.c_int64), ("edge_tiles", C.c_void_p),
                ("max_in_degree", C.c_int32), ("tile_meta", C.c_void_p)]


class gnn_mlp(C.Structure):
    _fields_ = [("n_lin", C.c_int32), ("dims", C.c_int32 * (GNN_MAX_LIN + 1)),
                ("W", C.c_void_p * GNN_MAX_LIN), ("b", C.c_void_p * GNN_MAX_LIN),
                ("gamma", C.c_void_p), ("beta", C.c_void_p)]


class gnn_mp_params(C.Structure):
    _fields_ = [("edge", gnn_mlp), ("node", gnn_mlp)]


class gnn_mp_config(C.Structure):
    _fields_ = [("hidden", C.c_int32), ("precision", C.c_int32), ("halo_mode", C.c_int32),
                ("flags", C.c_int32), ("ln_eps", C.c_float), ("edge_fwd_kernel", C.c_int32),
                ("ctas_per_sm", C.c_int32)]


_P = C.c_void_p
_SIGS = {
    "gnn_last_error": (C.c_char_p, []),
    "gnn_version": (C.c_int, []),
    "gnn_check": (C.c_int, [_P]),
    "gnn_graph_build": (C.c_int, [C.POINTER(gnn_mesh_desc), C.POINTER(_P)]),
    "gnn_graph_destroy": (None, [_P]),
    "gnn_graph_get_info": (C.c_int, [_P, C.POINTER(gnn_graph_info)]),
    "gnn_graph_copy_pos": (C.c_int, [_P, _P]),
    "gnn_graph_copy_csr": (C.c_int, [_P, _P, _P]),
    "gnn_graph_copy_elements": (C.c_int, [_P, _P]),
    "gnn_graph_build_elements": (C.c_int, [C.POINTER(gnn_elem_mesh_desc), C.POINTER(_P)]),
    "gnn_graph_copy_element_ptr": (C.c_int, [_P, _P]),
    "gnn_partition_halo": (C.c_int, [_P, C.c_int32, C.c_int32, _P, C.POINTER(_P)]),
    "gnn_partition_elements": (C.c_int, [_P, C.c_int32, _P, C.POINTER(_P)]),
    "gnn_partition_destroy": (None, [_P]),
    "gnn_partition_get_info": (C.c_int, [_P, C.POINTER(gnn_partition_info)]),
    "gnn_partition_copy": (C.c_int, [_P, C.c_int32, _P, C.c_size_t]),
    "gnn_partition_set_tile_edges": (C.c_int, [_P, C.c_int32]),
    "gnn_mp_workspace_size": (C.c_int, [C.POINTER(gnn_graph_dev), C.POINTER(gnn_mp_config),
                                        C.POINTER(gnn_mp_params), C.POINTER(C.c_size_t),
                                        C.POINTER(C.c_size_t)]),
    "gnn_mp_autotune": (C.c_int, [C.POINTER(gnn_graph_dev), C.POINTER(gnn_mp_config), C.POINTER(gnn_mp_params),
                                  _P, _P, _P, _P, _P, _P, C.c_size_t, C.c_int32, C.POINTER(gnn_tune_entry),
                                  C.c_int32, C.POINTER(C.c_int32), _P]),
    "gnn_mp_forward": (C.c_int, [C.POINTER(gnn_graph_dev), C.POINTER(gnn_mp_config),
                                 C.POINTER(gnn_mp_params), _P, _P, _P, _P, _P, _P, C.c_size_t, _P]),
    "gnn_mp_backward": (C.c_int, [C.POINTER(gnn_graph_dev), C.POINTER(gnn_mp_config),
                                  C.POINTER(gnn_mp_params), _P, _P, _P, _P, _P, _P, _P,
                                  C.POINTER(gnn_mp_params), _P, C.c_size_t, _P]),
    "gnn_mp_act_size": (C.c_int, [C.POINTER(gnn_graph_dev), C.POINTER(gnn_mp_config), C.POINTER(gnn_mp_params),
                                  C.POINTER(C.c_size_t)]),
    "gnn_mp_forward_act": (C.c_int, [C.POINTER(gnn_graph_dev), C.POINTER(gnn_mp_config),
                                     C.POINTER(gnn_mp_params), _P, _P, _P, _P, _P, _P, _P, C.c_size_t, _P]),
    "gnn_mp_backward_act": (C.c_int, [C.POINTER(gnn_graph_dev), C.POINTER(gnn_mp_config),
                                      C.POINTER(gnn_mp_params), _P, _P, _P, _P, _P, _P, _P, _P,
                                      C.POINTER(gnn_mp_params), _P, C.c_size_t, _P]),
    "gnn_mp_forward_static": (C.c_int, [C.POINTER(gnn_graph_dev), C.POINTER(gnn_mp_config),
                                        C.POINTER(gnn_mp_params), _P, _P, _P, _P, _P, _P]),
    "gnn_halo_exchange": (C.c_int, [C.POINTER(gnn_graph_dev), _P, C.c_int32, _P]),
    "gnn_mlp_workspace_size": (C.c_int, [C.POINTER(gnn_mlp), C.c_int64, C.POINTER(C.c_size_t),
                                         C.POINTER(C.c_size_t)]),
    "gnn_mlp_forward": (C.c_int, [C.POINTER(gnn_mlp), C.c_int64, _P, _P, C.c_int32, C.c_float, _P,
                                  C.c_size_t, _P]),
    "gnn_mlp_backward": (C.c_int, [C.POINTER(gnn_mlp), C.c_int64, _P, _P, C.c_int32, _P,
                                   C.POINTER(gnn_mlp), C.c_float, _P, C.c_size_t, _P]),
    "gnn_mlp_workspace_size_bf16": (C.c_int, [C.POINTER(gnn_mlp), C.c_int64, C.POINTER(C.c_size_t),
                                              C.POINTER(C.c_size_t)]),
    "gnn_mlp_forward_bf16": (C.c_int, [C.POINTER(gnn_mlp), C.c_int64, _P, _P, C.c_int32, C.c_float, _P,
                                       C.c_size_t, _P]),
    "gnn_mlp_backward_bf16": (C.c_int, [C.POINTER(gnn_mlp), C.c_int64, _P, _P, C.c_int32, _P,
                                        C.POINTER(gnn_mlp), C.c_float, _P, C.c_size_t, _P]),
    "gnn_mlp_act_size_bf16": (C.c_int, [C.POINTER(gnn_mlp), C.c_int64, C.POINTER(C.c_size_t)]),
    "gnn_mlp_forward_bf16_act": (C.c_int, [C.POINTER(gnn_mlp), C.c_int64, _P, _P, C.c_int32, C.c_float, _P, _P]),
    "gnn_mlp_backward_bf16_act": (C.c_int, [C.POINTER(gnn_mlp), C.c_int64, _P, _P, C.c_int32, _P,
                                            C.POINTER(gnn_mlp), C.c_float, _P, _P, C.c_size_t, _P]),
    "gnn_consistent_loss": (C.c_int, [C.POINTER(gnn_graph_dev), _P, _P, C.c_int32, _P, _P, _P,
                                      C.c_size_t, _P]),
    "gnn_profile_start": (C.c_int, [C.c_int32]),
    "gnn_profile_stop": (C.c_int, []),
    "gnn_profile_report": (C.c_int, [C.c_char_p, C.c_size_t]),
    "gnn_measure_fp32_fma": (C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_int32), _P]),
    "gnn_selftest_bounded_wait": (C.c_int, [C.c_uint64, _P, _P]),
}


def profile_report() -> dict:
    """{kernel name: (launches, total_ms)} of the last gnn_profile_start/stop window."""
    buf = C.create_string_buffer(1 << 16)
    call("gnn_profile_report", buf, len(buf))
    out = {}
    for line in buf.value.decode().splitlines():
        if line and not line.startswith("#"):
            name, n, ms = line.split()
            out[name] = (int(n), float(ms))
    return out

_lib = None


def load(path: str | None = None) -> C.CDLL:
    """Load libgnnmp.so (built in-tree by ``_build.build``) and declare its symbols."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libgnnmp.so not found at {path}; run paper_2410_01657_gb300._build.build() first")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


def last_error() -> str:
    return load().gnn_last_error().decode()


def check(code: int) -> None:
    if code != GNN_OK:
        raise GnnError(code, last_error())


def call(name: str, *args) -> None:
    """Call a libgnnmp entry point that returns a status code; raise on failure."""
    check(getattr(load(), name)(*args))


def ptr(t) -> int | None:
    """Device/host address of a torch tensor or numpy array (None for None)."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr() if t.numel() else None
    return t.ctypes.data if t.size else None
