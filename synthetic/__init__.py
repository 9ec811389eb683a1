"""Seeded synthetic inputs shared by the oracle and the GPU path.

This module only draws random numbers and evaluates the input fields; it holds
none of the arithmetic of the consistent message-passing method. Both sides of
every parity test receive the arrays made here, so neither side has to
reproduce the other's random stream.

Recipes (all numpy PCG64 via ``numpy.random.default_rng(seed)``):

* MLP parameters: Xavier-uniform weights with gain 1 (bound sqrt(6/(fan_in+fan_out))),
  biases 0, LayerNorm gamma 1 and beta 0; ``randomize_affine=True`` draws biases
  U[-0.5,0.5], gamma U[0.5,1.5] and beta U[-0.5,0.5] instead, so that tests do
  not hide mistakes behind zeros and ones.
* Node field: a sum of K Fourier modes per velocity component,
  u_c(p) = sum_m A_mc sin(2 pi k_m . p + phi_mc), A ~ N(0,1),
  k_m uniform on {-4..4}^3 without 0, phi ~ U[0, 2 pi). It stands in for the
  smooth low-wavenumber Taylor-Green velocity the paper trains on (Sec. III-B).
* Mesh jitter: U[-1,1] per global node and axis; the graph builder scales it.
* Partition sizes: element counts drawn log-uniform on [lo, hi].
* Mixed element mesh (``mixed_element_mesh``): a unit cube of n^3 lattice
  cells, each drawn (U[0,1) < tet_fraction) as one 8-node hexahedron or as
  its 6 Kuhn tetrahedra, plus fan cells joining one apex above the top face to
  bands of top-face nodes; interior nodes jittered U[-1/2,1/2]*jitter/n.
* Counter-hashed states (``hashed_values``): for inputs of graphs too large to
  draw on the host, each value is a fixed function of an integer counter (a
  global node id or a directed edge key times the width, plus the column), so
  any subset of rows can be regenerated on either side without the rest. The
  counter's two 32-bit halves pass through the "lowbias32" integer hash
  (x ^= x >> 16; x *= 0x7feb352d; x ^= x >> 15; x *= 0x846ca68b; x ^= x >> 16,
  mod 2^32), seeded by xor; the top bits give uniform values on a grid that
  BF16 (8 bits) or FP32 (16 bits) holds exactly. The same integer steps run on
  numpy arrays and on torch tensors (any device), so the values agree bit for bit.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "mlp_dims",
    "xavier_mlp",
    "fourier_modes",
    "fourier_field",
    "jitter_unit",
    "log_uniform_counts",
    "normal",
    "hashed_values",
]


def mlp_dims(n_in: int, hidden: int, n_hidden: int, n_out: int) -> list[int]:
    """Widths of the n_hidden+2 Linear layers: in -> H, n_hidden x (H -> H), H -> out."""
    return [n_in] + [hidden] * (n_hidden + 1) + [n_out]


def xavier_mlp(rng: np.random.Generator, dims: list[int], layernorm: bool,
               randomize_affine: bool = False, dtype=np.float64) -> dict:
    """Parameters of one MLP as a dict of arrays.

    ``W[k]`` has shape [dims[k+1], dims[k]] (out x in, row-major), ``b[k]`` [dims[k+1]],
    and ``gamma``/``beta`` [dims[-1]] when ``layernorm`` is set.
    """
    W, b = [], []
    for k in range(len(dims) - 1):
        fan_in, fan_out = dims[k], dims[k + 1]
        bound = np.sqrt(6.0 / (fan_in + fan_out))
        W.append(rng.uniform(-bound, bound, size=(fan_out, fan_in)).astype(dtype))
        if randomize_affine:
            b.append(rng.uniform(-0.5, 0.5, size=fan_out).astype(dtype))
        else:
            b.append(np.zeros(fan_out, dtype=dtype))
    out = {"W": W, "b": b}
    if layernorm:
        if randomize_affine:
            out["gamma"] = rng.uniform(0.5, 1.5, size=dims[-1]).astype(dtype)
            out["beta"] = rng.uniform(-0.5, 0.5, size=dims[-1]).astype(dtype)
        else:
            out["gamma"] = np.ones(dims[-1], dtype=dtype)
            out["beta"] = np.zeros(dims[-1], dtype=dtype)
    return out


def fourier_modes(seed: int, n_modes: int, n_comp: int = 3) -> dict:
    """Draw the wave vectors, amplitudes and phases of the synthetic velocity field."""
    rng = np.random.default_rng(seed)
    k = np.zeros((n_modes, 3), dtype=np.int64)
    for m in range(n_modes):
        while True:
            cand = rng.integers(-4, 5, size=3)
            if np.any(cand != 0):
                k[m] = cand
                break
    amp = rng.standard_normal((n_modes, n_comp))
    phase = rng.uniform(0.0, 2.0 * np.pi, size=(n_modes, n_comp))
    return {"k": k, "amp": amp, "phase": phase}


def fourier_field(pos: np.ndarray, modes: dict, phase_advance: float = 0.0) -> np.ndarray:
    """Evaluate the field at positions ``pos`` [N,3]; returns [N, n_comp] float64.

    ``phase_advance`` shifts every phase by ``phase_advance * |k_m|`` (the seeded
    "next step" target field)."""
    pos = np.asarray(pos, dtype=np.float64)
    k = modes["k"].astype(np.float64)
    amp, phase = modes["amp"], modes["phase"]
    shift = phase_advance * np.linalg.norm(k, axis=1)
    out = np.zeros((pos.shape[0], amp.shape[1]), dtype=np.float64)
    for m in range(k.shape[0]):
        arg = 2.0 * np.pi * (pos @ k[m])
        for c in range(amp.shape[1]):
            out[:, c] += amp[m, c] * np.sin(arg + phase[m, c] + shift[m])
    return out


def jitter_unit(n_nodes: int, seed: int) -> np.ndarray:
    """U[-1,1] offsets per global node and axis, [n_nodes, 3] float64."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(n_nodes, 3))


def log_uniform_counts(n: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """``n`` integer counts drawn log-uniform on [lo, hi], rounded, at least 1."""
    rng = np.random.default_rng(seed)
    v = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n))
    return np.maximum(1, np.rint(v)).astype(np.int64)


def normal(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """Standard-normal array (float64) scaled by ``scale``."""
    return scale * np.random.default_rng(seed).standard_normal(shape)


def gnn_params(seed: int, hidden: int, n_hidden: int, n_layers: int, f_x: int = 3,
               f_e: int = 4, f_y: int = 3, randomize_affine: bool = False) -> dict:
    """Parameters of the encode-process-decode network (float64).

    Shapes: node encoder f_x -> H, edge encoder f_e -> H, per layer an edge MLP
    3H -> H and a node MLP 2H -> H (all with LayerNorm), decoder H -> f_y
    (no LayerNorm). Drawn in that order from one generator."""
    rng = np.random.default_rng(seed)
    H = hidden
    p = {
        "enc_node": xavier_mlp(rng, mlp_dims(f_x, H, n_hidden, H), True, randomize_affine),
        "enc_edge": xavier_mlp(rng, mlp_dims(f_e, H, n_hidden, H), True, randomize_affine),
        "layers": [],
    }
    for _ in range(n_layers):
        p["layers"].append({
            "edge": xavier_mlp(rng, mlp_dims(3 * H, H, n_hidden, H), True, randomize_affine),
            "node": xavier_mlp(rng, mlp_dims(2 * H, H, n_hidden, H), True, randomize_affine),
        })
    p["dec"] = xavier_mlp(rng, mlp_dims(H, H, n_hidden, f_y), False, randomize_affine)
    return p


def rescale_counts(counts, total: int) -> np.ndarray:
    """Scale integer counts to sum to ``total`` by largest-remainder rounding
    (ties to the lower index), keeping every count >= 1."""
    c = np.asarray(counts, dtype=np.float64)
    raw = c * (total / c.sum())
    out = np.maximum(1, np.floor(raw)).astype(np.int64)
    rem = raw - np.floor(raw)
    order = sorted(range(len(c)), key=lambda i: (-rem[i], i))
    k = 0
    while out.sum() < total:
        out[order[k % len(c)]] += 1
        k += 1
    k = 0
    while out.sum() > total:
        i = order[::-1][k % len(c)]
        if out[i] > 1:
            out[i] -= 1
        k += 1
    return out


def uneven_brick(n_parts: int, lo: float, hi: float, seed: int):
    """Element counts of ``n_parts`` sub-graphs drawn log-uniform on [lo, hi],
    the smallest cube n^3 holding them, and the counts rescaled to n^3
    (the RCB target weights of the batching workload)."""
    counts = log_uniform_counts(n_parts, lo, hi, seed)
    n = int(np.ceil(round(counts.sum() ** (1.0 / 3.0), 9)))
    while n ** 3 < counts.sum():
        n += 1
    return n, rescale_counts(counts, n ** 3)


# local node index of a p=1 hexahedron: i + 2*(j + 2*k)
HEX_EDGES = np.array([(0, 1), (2, 3), (4, 5), (6, 7),        # along x
                      (0, 2), (1, 3), (4, 6), (5, 7),        # along y
                      (0, 4), (1, 5), (2, 6), (3, 7)],       # along z
                     dtype=np.int32)
TET_EDGES = np.array([(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)], dtype=np.int32)


def kuhn_tets() -> list:
    """The 6 Kuhn tetrahedra of the unit cube as hex-local vertex indices: for
    each order (a, b, c) of the axes, the path 0 -> +e_a -> +e_b -> +e_c = 7."""
    out = []
    for a, b, c in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
        v1 = 1 << a
        v2 = v1 | (1 << b)
        out.append((0, v1, v2, 7))
    return out


def mixed_element_mesh(n: int, seed: int, tet_fraction: float = 0.5, n_fans: int = 2,
                       jitter: float = 0.2) -> dict:
    """Element lists of a mixed mesh on the unit cube (input structure only).

    Lattice node (i, j, k), 0 <= i, j, k <= n, has id i + (n+1)*(j + (n+1)*k)
    and sits at (i, j, k)/n, interior nodes moved by jitter*U[-1/2,1/2]/n per
    axis; the apex (id (n+1)^3, present when n_fans > 0) sits at
    (1/2, 1/2, 1 + 1/n). Cells in order
    i + n*(j + n*k) become one hexahedron (8 nodes, ``HEX_EDGES``) or, when
    U[0,1) < tet_fraction, 6 tetrahedra (``kuhn_tets``, ``TET_EDGES``). Then
    fan f < n_fans holds the apex (local 0) and the top-face nodes of the
    columns floor(f*n/n_fans) .. floor((f+1)*n/n_fans) (neighbouring fans share
    a column) with a spoke from the apex to each. Returns pos, elem_ptr,
    elem_nodes, edge_ptr, edge_pairs and the element kind (0 hex, 1 tet, 2 fan)."""
    rng = np.random.default_rng(seed)
    m = n + 1
    N = m ** 3 + (1 if n_fans > 0 else 0)
    k, j, i = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    ijk = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
    pos = np.zeros((N, 3))
    interior = np.all((ijk > 0) & (ijk < n), axis=1)
    off = rng.uniform(-0.5, 0.5, size=(m ** 3, 3)) * jitter / n
    pos[:m ** 3] = ijk / n + np.where(interior[:, None], off, 0.0)
    if n_fans > 0:
        pos[m ** 3] = (0.5, 0.5, 1.0 + 1.0 / n)
    draw = rng.uniform(size=n ** 3)
    c = np.arange(n ** 3)
    ci, cj, ck = c % n, (c // n) % n, c // (n * n)
    v = np.arange(8)
    hexn = ((ci[:, None] + (v & 1)) + m * ((cj[:, None] + ((v >> 1) & 1)) + m * (ck[:, None] + ((v >> 2) & 1))))
    tet = draw < tet_fraction
    kuhn = np.array(kuhn_tets())
    # elements in cell order: a hexahedron, or the cell's 6 tetrahedra
    n_el = np.where(tet, 6, 1)
    first = np.concatenate([[0], np.cumsum(n_el)])
    kind = np.zeros(first[-1], dtype=np.int8)
    size = np.full(first[-1], 8, dtype=np.int64)
    npair = np.full(first[-1], len(HEX_EDGES), dtype=np.int64)
    tet_el = (first[:-1][tet][:, None] + np.arange(6)).ravel()
    kind[tet_el], size[tet_el], npair[tet_el] = 1, 4, len(TET_EDGES)
    cell_ptr = np.concatenate([[0], np.cumsum(np.where(tet, 24, 8))])
    cell_nodes = np.empty(cell_ptr[-1], dtype=np.int64)
    hex_cells = np.nonzero(~tet)[0]
    cell_nodes[(cell_ptr[hex_cells][:, None] + v).ravel()] = hexn[hex_cells].ravel()
    tet_cells = np.nonzero(tet)[0]
    cell_nodes[(cell_ptr[tet_cells][:, None] + np.arange(24)).ravel()] = hexn[tet_cells][:, kuhn].ravel()
    pair_ptr = np.concatenate([[0], np.cumsum(npair)])
    k = np.arange(pair_ptr[-1]) - np.repeat(pair_ptr[:-1], npair)
    kk = np.repeat(kind, npair)
    edge_pairs = np.where((kk == 0)[:, None], HEX_EDGES[np.minimum(k, len(HEX_EDGES) - 1)],
                          TET_EDGES[np.minimum(k, len(TET_EDGES) - 1)])
    fan_nodes, fan_pairs = [], []
    for f in range(n_fans):
        lo, hi = (f * n) // n_fans, ((f + 1) * n) // n_fans
        ii, jj = np.meshgrid(np.arange(lo, hi + 1), np.arange(m), indexing="ij")
        top = (ii + m * (jj + m * n)).ravel()
        fan_nodes.append(np.concatenate([[m ** 3], top]))
        fan_pairs.append(np.stack([np.zeros(top.size), np.arange(1, top.size + 1)], axis=1).astype(np.int32))
    sizes = np.concatenate([size, [x.size for x in fan_nodes]]).astype(np.int64)
    npairs = np.concatenate([npair, [x.shape[0] for x in fan_pairs]]).astype(np.int64)
    return {"pos": pos, "elem_ptr": np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64),
            "elem_nodes": np.concatenate([cell_nodes] + fan_nodes).astype(np.int64),
            "edge_ptr": np.concatenate([[0], np.cumsum(npairs)]).astype(np.int64),
            "edge_pairs": np.concatenate([edge_pairs] + fan_pairs).astype(np.int32),
            "kind": np.concatenate([kind, np.full(n_fans, 2, dtype=np.int8)])}


_M32 = 0xFFFFFFFF


def _lowbias32(x):
    """The lowbias32 integer hash on values in [0, 2^32) held in int64 (numpy or
    torch): only the low 32 bits of each product are kept."""
    x = x ^ (x >> 16)
    x = (x * 0x7FEB352D) & _M32
    x = x ^ (x >> 15)
    x = (x * 0x846CA68B) & _M32
    return x ^ (x >> 16)


def hashed_values(counter, seed: int, bits: int):
    """Uniform values on [-2, 2) on a grid of 2^bits points, one per non-negative
    int64 counter (numpy array or torch tensor; the result has its type and
    device, float64 for numpy, float32 for torch). bits = 8 gives values BF16
    holds exactly, bits = 16 values FP32 holds exactly."""
    assert 1 <= bits <= 16
    lo = counter & _M32
    hi = (counter >> 32) & _M32
    h = _lowbias32(lo ^ _lowbias32(hi ^ (seed & _M32)))
    q = (h >> (32 - bits)) - (1 << (bits - 1))      # integer in [-2^(bits-1), 2^(bits-1))
    scale = 2.0 / (1 << (bits - 1))
    if isinstance(q, np.ndarray):
        return q.astype(np.float64) * scale
    return q.float() * scale
