"""Shared helpers of the GPU parity tests: oracle runs on the same seeded
inputs as the library, concatenated in the library's row/edge order."""
from __future__ import annotations

import numpy as np

import synthetic as syn
from oracle import graph as og
from oracle import model as om


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def oracle_subgraphs(nel, p, R, method="rcb", weights=None, periodic=(False, False, False)):
    brick = og.build_brick(nel, p, periodic=periodic)
    if R == 1:
        return brick, og.unpartitioned(brick)
    part = og.partition_slab_z(brick, R) if method == "slab" else og.partition_rcb(brick, R, weights)
    return brick, og.build_subgraphs(brick, part, R)


def node_field(brick, seed=0, n_modes=8):
    return syn.fourier_field(brick.pos, syn.fourier_modes(seed, n_modes))


def split_rows(arr, subs):
    out, o = [], 0
    for sg in subs:
        out.append(arr[o:o + sg.n_local])
        o += sg.n_local
    return out


def split_edges(arr, subs):
    out, o = [], 0
    for sg in subs:
        out.append(arr[o:o + sg.n_edges])
        o += sg.n_edges
    return out


def flat_grads(g: dict) -> list:
    """(name, array) pairs of a nested gradient dict in a fixed order."""
    out = []

    def mlp(prefix, m):
        for k, w in enumerate(m["W"]):
            out.append((f"{prefix}.W{k}", w))
        for k, b in enumerate(m["b"]):
            out.append((f"{prefix}.b{k}", b))
        if "gamma" in m:
            out.append((f"{prefix}.gamma", m["gamma"]))
            out.append((f"{prefix}.beta", m["beta"]))

    mlp("enc_node", g["enc_node"])
    mlp("enc_edge", g["enc_edge"])
    for i, layer in enumerate(g["layers"]):
        mlp(f"L{i}.edge", layer["edge"])
        mlp(f"L{i}.node", layer["node"])
    mlp("dec", g["dec"])
    return out


def oracle_network(params, brick, subs, u, target, attr=None, halo=True):
    us = [u[sg.gid] for sg in subs]
    ts = [target[sg.gid] for sg in subs]
    at = attr if attr is not None else [og.edge_attributes(brick.pos, sg) for sg in subs]
    ys, cache = om.network_forward(params, subs, us, at, halo)
    L = om.consistent_loss(subs, ys, ts)
    g = om.network_backward(params, subs, cache, om.consistent_loss_grad(subs, ys, ts), halo)
    return ys, L, g, cache


def max_row_rel(got, ref, rows=None) -> float:
    """Largest per-row relative L2 error over ``rows`` (all rows when None); a
    row's norm is floored at 1e-3 of the mean row norm of ``ref``."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if rows is not None:
        got, ref = got[rows], ref[rows]
    if ref.shape[0] == 0:
        return 0.0
    rn = np.linalg.norm(ref, axis=1)
    floor = 1e-3 * max(float(rn.mean()), 1e-300)
    return float((np.linalg.norm(got - ref, axis=1) / np.maximum(rn, floor)).max())
