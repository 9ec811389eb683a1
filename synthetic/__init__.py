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
