"""Consistent NMP network in FP64 with its hand-written adjoint (oracle side).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Every rank r holds a reduced sub-graph (``oracle.graph.SubGraph``) with its
node rows x_r and edge rows e_r. One consistent NMP layer is Eq. 5a-5e of the
paper, evaluated rank by rank exactly as written:

  Eq. 5a  e_ij  <- e_ij + MLP_E([x_i, x_j, e_ij])          (i receiver, j sender)
  Eq. 5b  a_i    = sum_{j in N(i)} e_ij / d_ij
  Eq. 5c  halo rows of rank r receive a_s(k) where G_r(i) = G_s(k)
  Eq. 5d  a*_i   = sum of a over the rows of rank r with the same global id
  Eq. 5e  x_i   <- x_i + MLP_N([a*_i, x_i])

MLP blocks (Sec. III; layout pinned by Table 1's parameter counts): Linear
layers in -> H, n_hidden x (H -> H), H -> out, ELU (alpha 1) after every Linear
but the last, then an affine LayerNorm (eps 1e-5, biased variance) in the
encoders and the processor; the decoder has no LayerNorm. The processor MLPs
add their input state as a residual after the LayerNorm.

The encode-process-decode network follows Sec. III (node/edge encoders, M
consistent layers, node decoder) and the consistent loss follows Eq. 8a-8c.
The adjoint of Eq. 5c+5d is the same symmetric copy-sum (the gradient of the
differentiable halo exchange), and the weight gradient is the sum of the
per-rank gradients of the one global loss (Eq. 3).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

LN_EPS = 1e-5


# --------------------------------------------------------------------------- MLP block

def elu(z: np.ndarray) -> np.ndarray:
    """ELU with alpha = 1."""
    return np.where(z > 0.0, z, np.expm1(np.minimum(z, 0.0)))


def elu_deriv(z: np.ndarray) -> np.ndarray:
    return np.where(z > 0.0, 1.0, np.exp(np.minimum(z, 0.0)))


def mlp_forward(P: dict, X: np.ndarray, eps: float = LN_EPS):
    """Linear -> ELU -> ... -> Linear [-> LayerNorm]; returns (Y, cache)."""
    n = len(P["W"])
    inputs, pre = [], []
    h = X
    z = None
    for k in range(n):
        inputs.append(h)
        z = h @ P["W"][k].T + P["b"][k]
        pre.append(z)
        h = elu(z) if k < n - 1 else z
    cache = {"inputs": inputs, "pre": pre}
    if "gamma" in P:
        mu = z.mean(axis=1, keepdims=True)
        var = ((z - mu) ** 2).mean(axis=1, keepdims=True)
        rstd = 1.0 / np.sqrt(var + eps)
        xhat = (z - mu) * rstd
        cache["xhat"] = xhat
        cache["rstd"] = rstd
        h = xhat * P["gamma"] + P["beta"]
    return h, cache


def mlp_backward(P: dict, cache: dict, dY: np.ndarray):
    """Adjoint of ``mlp_forward``: returns (dX, grads) with grads shaped like P."""
    n = len(P["W"])
    grads = {"W": [None] * n, "b": [None] * n}
    g = dY
    if "gamma" in P:
        xhat, rstd = cache["xhat"], cache["rstd"]
        grads["gamma"] = (g * xhat).sum(axis=0)
        grads["beta"] = g.sum(axis=0)
        dxh = g * P["gamma"]
        g = rstd * (dxh - dxh.mean(axis=1, keepdims=True)
                    - xhat * (dxh * xhat).mean(axis=1, keepdims=True))
    for k in range(n - 1, -1, -1):
        if k < n - 1:
            g = g * elu_deriv(cache["pre"][k])
        grads["W"][k] = g.T @ cache["inputs"][k]
        grads["b"][k] = g.sum(axis=0)
        g = g @ P["W"][k]
    return g, grads


def mlp_param_count(P: dict) -> int:
    n = sum(w.size for w in P["W"]) + sum(b.size for b in P["b"])
    if "gamma" in P:
        n += P["gamma"].size + P["beta"].size
    return int(n)


def network_param_count(params: dict) -> int:
    n = mlp_param_count(params["enc_node"]) + mlp_param_count(params["enc_edge"])
    n += mlp_param_count(params["dec"])
    for layer in params["layers"]:
        n += mlp_param_count(layer["edge"]) + mlp_param_count(layer["node"])
    return n


# --------------------------------------------------------------------------- graph operators

def aggregation_matrix(sub) -> sp.csr_matrix:
    """[n_local x E_r] matrix with 1/d_ij at (receiver(e), e): Eq. 5b as A @ e."""
    E = sub.n_edges
    return sp.csr_matrix((1.0 / sub.edge_deg.astype(np.float64), (sub.recv, np.arange(E))),
                         shape=(sub.n_local, E))


def gather_matrix(rows: np.ndarray, n_rows: int) -> sp.csr_matrix:
    """[E x n] one-hot selection matrix: (G @ x)[e] = x[rows[e]]."""
    E = rows.shape[0]
    return sp.csr_matrix((np.ones(E), (np.arange(E), rows)), shape=(E, n_rows))


def halo_swap(subs: list, a: list) -> list:
    """Eq. 5c: the halo rows of rank r take a_s(k) for the matching global id."""
    return [a[0][:0].reshape(0, a[0].shape[1]) if sg.n_halo == 0 else
            np.stack([a[s][k] for s, k in zip(sg.halo_rank, sg.halo_src_row)])
            for sg in subs]


def synchronize(subs: list, a: list, a_halo: list) -> list:
    """Eq. 5d: a*_i = own row + halo rows with the same global id (in halo order)."""
    out = []
    for r, sg in enumerate(subs):
        s = a[r].copy()
        np.add.at(s, sg.halo_local_row, a_halo[r])
        out.append(s)
    return out


def synchronize_adjoint(subs: list, da_star: list) -> list:
    """Adjoint of Eq. 5c+5d: every halo row sends its gradient back to its
    source row on the neighbour rank (the reverse exchange)."""
    da = [d.copy() for d in da_star]
    for r, sg in enumerate(subs):
        da_halo = da_star[r][sg.halo_local_row]
        for h in range(sg.n_halo):
            da[sg.halo_rank[h]][sg.halo_src_row[h]] += da_halo[h]
    return da


# --------------------------------------------------------------------------- consistent NMP layer

def layer_forward(layer: dict, subs: list, xs: list, es: list, halo: bool = True,
                  eps: float = LN_EPS):
    """One consistent NMP layer (Eq. 5a-5e) on every rank; ``halo=False`` is the
    paper's "None" mode (Eq. 5c-5d skipped, an inconsistent standard layer)."""
    e_new, a, c_edge = [], [], []
    for r, sg in enumerate(subs):
        inp = np.concatenate([xs[r][sg.recv], xs[r][sg.send], es[r]], axis=1)
        m, c = mlp_forward(layer["edge"], inp, eps)
        en = es[r] + m                                   # Eq. 5a (residual MLP)
        e_new.append(en)
        a.append(aggregation_matrix(sg) @ en)            # Eq. 5b
        c_edge.append(c)
    a_star = synchronize(subs, a, halo_swap(subs, a)) if halo else a   # Eq. 5c, 5d
    x_new, c_node = [], []
    for r in range(len(subs)):
        m, c = mlp_forward(layer["node"], np.concatenate([a_star[r], xs[r]], axis=1), eps)
        x_new.append(xs[r] + m)                          # Eq. 5e (residual MLP)
        c_node.append(c)
    cache = {"c_edge": c_edge, "c_node": c_node, "a": a, "a_star": a_star}
    return x_new, e_new, cache


def layer_backward(layer: dict, subs: list, cache: dict, dx_new: list, de_new: list,
                   halo: bool = True):
    """Adjoint of ``layer_forward``: returns (dx, de, grads summed over ranks)."""
    R = len(subs)
    H = dx_new[0].shape[1]
    g_node = None
    da_star, dx = [], []
    for r in range(R):
        d_inp, g = mlp_backward(layer["node"], cache["c_node"][r], dx_new[r])
        da_star.append(d_inp[:, :H])
        dx.append(dx_new[r] + d_inp[:, H:])
        g_node = g if g_node is None else add_grads(g_node, g)
    da = synchronize_adjoint(subs, da_star) if halo else da_star
    g_edge = None
    de = []
    for r, sg in enumerate(subs):
        de_tot = de_new[r] + aggregation_matrix(sg).T @ da[r]
        d_inp, g = mlp_backward(layer["edge"], cache["c_edge"][r], de_tot)
        de.append(de_tot + d_inp[:, 2 * H:])
        dx[r] = (dx[r] + gather_matrix(sg.recv, sg.n_local).T @ d_inp[:, :H]
                 + gather_matrix(sg.send, sg.n_local).T @ d_inp[:, H:2 * H])
        g_edge = g if g_edge is None else add_grads(g_edge, g)
    return dx, de, {"edge": g_edge, "node": g_node}


# --------------------------------------------------------------------------- network and loss

def network_forward(params: dict, subs: list, u: list, attr: list, halo: bool = True,
                    eps: float = LN_EPS):
    """Encode-process-decode (Sec. III): returns (y per rank, cache)."""
    xs, es, c_enc_n, c_enc_e = [], [], [], []
    for r in range(len(subs)):
        x, c = mlp_forward(params["enc_node"], u[r], eps)
        xs.append(x)
        c_enc_n.append(c)
        e, c = mlp_forward(params["enc_edge"], attr[r], eps)
        es.append(e)
        c_enc_e.append(c)
    c_layers = []
    for layer in params["layers"]:
        xs, es, c = layer_forward(layer, subs, xs, es, halo, eps)
        c_layers.append(c)
    ys, c_dec = [], []
    for r in range(len(subs)):
        y, c = mlp_forward(params["dec"], xs[r], eps)
        ys.append(y)
        c_dec.append(c)
    return ys, {"enc_n": c_enc_n, "enc_e": c_enc_e, "layers": c_layers, "dec": c_dec,
                "x_final": xs, "e_final": es}


def consistent_loss(subs: list, ys: list, targets: list) -> float:
    """Eq. 8a-8c: sum of 1/d_i-weighted squared errors over local rows of all
    ranks, divided by N_eff * F_y with N_eff = sum of 1/d_i."""
    S = 0.0
    n_eff = 0.0
    for r, sg in enumerate(subs):
        w = 1.0 / sg.node_deg.astype(np.float64)
        S += float((w[:, None] * (ys[r] - targets[r]) ** 2).sum())
        n_eff += float(w.sum())
    return S / (n_eff * ys[0].shape[1])


def consistent_loss_grad(subs: list, ys: list, targets: list) -> list:
    n_eff = sum(float((1.0 / sg.node_deg).sum()) for sg in subs)
    F = ys[0].shape[1]
    return [2.0 * (ys[r] - targets[r]) / (sg.node_deg[:, None] * n_eff * F)
            for r, sg in enumerate(subs)]


def network_backward(params: dict, subs: list, cache: dict, dys: list, halo: bool = True):
    """Adjoint of ``network_forward`` given dL/dy per rank; returns grads shaped like params."""
    R = len(subs)
    g_dec = None
    dx = []
    for r in range(R):
        d, g = mlp_backward(params["dec"], cache["dec"][r], dys[r])
        dx.append(d)
        g_dec = g if g_dec is None else add_grads(g_dec, g)
    de = [np.zeros_like(e) for e in cache["e_final"]]
    g_layers = [None] * len(params["layers"])
    for li in range(len(params["layers"]) - 1, -1, -1):
        dx, de, g_layers[li] = layer_backward(params["layers"][li], subs,
                                              cache["layers"][li], dx, de, halo)
    g_enc_n = g_enc_e = None
    for r in range(R):
        _, g = mlp_backward(params["enc_node"], cache["enc_n"][r], dx[r])
        g_enc_n = g if g_enc_n is None else add_grads(g_enc_n, g)
        _, g = mlp_backward(params["enc_edge"], cache["enc_e"][r], de[r])
        g_enc_e = g if g_enc_e is None else add_grads(g_enc_e, g)
    return {"enc_node": g_enc_n, "enc_edge": g_enc_e, "layers": g_layers, "dec": g_dec}


def add_grads(a: dict, b: dict) -> dict:
    out = {"W": [x + y for x, y in zip(a["W"], b["W"])],
           "b": [x + y for x, y in zip(a["b"], b["b"])]}
    if "gamma" in a:
        out["gamma"] = a["gamma"] + b["gamma"]
        out["beta"] = a["beta"] + b["beta"]
    return out


def to_global(subs: list, rows: list, n_global: int) -> np.ndarray:
    """Scatter per-rank local rows into global-id order (copies must agree;
    the last rank's copy is the one kept)."""
    out = np.zeros((n_global,) + rows[0].shape[1:])
    for r, sg in enumerate(subs):
        out[sg.gid] = rows[r]
    return out
