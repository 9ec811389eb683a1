"""Shared helpers of the element-mesh layer tests: one consistent layer's
inputs in the library's row space (split copies included), the oracle's
results on its own sub-graphs, and the comparison of the two."""
from __future__ import annotations

import numpy as np
import torch

import synthetic as syn
from oracle import graph as og
from oracle import model as om

from gpu_util import max_row_rel, rel_l2


def _bf16(a):
    return torch.as_tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)


def library_view(part) -> list:
    """The library partition's own rows as oracle sub-graphs: the copies of a
    split node are extra rows, and every copy of a global id (in the same or
    another sub-graph) is a halo row of each of the others (Eq. 5c-5d)."""
    ro, eo = part.array("row_offsets"), part.array("edge_offsets")
    gid, nd, ed = part.array("row_gid"), part.array("node_deg"), part.array("edge_deg")
    recv, col = part.receivers(), part.array("col").astype(np.int64)
    row_part = np.searchsorted(ro, np.arange(part.n_rows), side="right") - 1
    R = len(ro) - 1
    halo = [([], [], []) for _ in range(R)]
    hp, hr = part.array("halo_ptr"), part.array("halo_rows")
    for s in range(len(hp) - 1):
        rows = hr[hp[s]:hp[s + 1]]
        for k in rows:
            for m in rows:
                if m != k:
                    pk, pm = row_part[k], row_part[m]
                    halo[pk][0].append(pm)
                    halo[pk][1].append(m - ro[pm])
                    halo[pk][2].append(k - ro[pk])
    subs = []
    for r in range(R):
        e = slice(eo[r], eo[r + 1])
        sg = og.SubGraph(gid=gid[ro[r]:ro[r + 1]].astype(np.int64), recv=recv[e] - ro[r], send=col[e] - ro[r],
                         edge_deg=ed[e].astype(np.int64), node_deg=nd[ro[r]:ro[r + 1]].astype(np.int64))
        sg.halo_rank, sg.halo_src_row, sg.halo_local_row = (np.asarray(v, dtype=np.int64) for v in halo[r])
        subs.append(sg)
    return subs


def layer_case(part, mesh, subs, H, seed=11, round_edges=True):
    """Seeded inputs of one layer (one value per global node / directed global
    edge, replicated to every copy; the upstream node gradient split evenly
    over a node's rows) and the oracle's forward and adjoint on ``subs``."""
    params = syn.gnn_params(seed, H, 2, 1, randomize_affine=True)
    rng = np.random.default_rng(seed + 1)
    N = mesh.n_nodes
    rnd = _bf16 if round_edges else (lambda a: a)
    xg = rng.standard_normal((N, H))
    keys = mesh.recv * N + mesh.send
    eg, deg1 = rnd(rng.standard_normal((keys.size, H))), rnd(rng.standard_normal((keys.size, H)) * 0.5)
    dxg = rng.standard_normal((N, H))
    gid = part.array("row_gid")
    ekey = np.searchsorted(keys, gid[part.receivers()] * N + gid[part.array("col")])
    nd = part.array("node_deg").astype(np.float64)
    lp = params["layers"][0]
    okey = [np.searchsorted(keys, sg.gid[sg.recv] * N + sg.gid[sg.send]) for sg in subs]
    x1, e1, cache = om.layer_forward(lp, subs, [xg[sg.gid] for sg in subs], [eg[k] for k in okey])
    dx0, de0, g = om.layer_backward(lp, subs, cache, [dxg[sg.gid] / sg.node_deg[:, None] for sg in subs],
                                    [deg1[k] for k in okey])
    gref = []
    for m in ("edge", "node"):
        gref += list(g[m]["W"]) + list(g[m]["b"]) + [g[m]["gamma"], g[m]["beta"]]
    return {"params": params, "x": xg[gid], "e": eg[ekey], "dx1": dxg[gid] / nd[:, None], "de1": deg1[ekey],
            "x'": x1, "e'": e1, "a*": cache["a_star"], "dL/dx": dx0, "dL/de": de0, "grads": gref}


def check_layer(part, subs, case, out, grads, lo, lg):
    """Edge rows compare directly (the library keeps the oracle's edge order);
    node rows per (sub-graph, global id); input gradients summed over copies."""
    errs = {"e'": rel_l2(out["e'"], np.concatenate(case["e'"])),
            "dL/de": rel_l2(out["dL/de"], np.concatenate(case["dL/de"]))}
    assert errs["e'"] < lo and errs["dL/de"] < lg, errs
    ro, gid = part.array("row_offsets"), part.array("row_gid")
    nd = part.array("node_deg")
    # per row, on the rows the copy-sum touches (nodes shared between sub-graphs
    # and the copies of split high-degree nodes), so one wrong copy row shows
    row_o, row_g = (1e-4, 1e-4) if lo <= 1e-5 else (5e-2, 1e-1)
    for r, sg in enumerate(subs):
        rows = slice(ro[r], ro[r + 1])
        loc = np.searchsorted(sg.gid, gid[rows])
        assert rel_l2(out["x'"][rows], case["x'"][r][loc]) < lo
        assert rel_l2(out["a*"][rows], case["a*"][r][loc]) < lo
        copies = nd[rows] > 1
        assert max_row_rel(out["x'"][rows], case["x'"][r][loc], copies) < row_o
        assert max_row_rel(out["a*"][rows], case["a*"][r][loc], copies) < row_o
        dsum = np.zeros((sg.n_local, out["dL/dx"].shape[1]))
        np.add.at(dsum, loc, out["dL/dx"][rows])
        assert rel_l2(dsum, case["dL/dx"][r]) < lg
        assert max_row_rel(dsum, case["dL/dx"][r], np.unique(loc[copies])) < row_g
    for k, (got, ref) in enumerate(zip(grads, case["grads"])):
        assert rel_l2(got, ref) < lg, (k, rel_l2(got, ref))


def mixed_mesh16():
    """n = 16 mixed mesh with two fans: the apex has in-degree 289 at R=1."""
    m = syn.mixed_element_mesh(16, 3, n_fans=2)
    return m, og.element_mesh(m["pos"], m["elem_ptr"], m["elem_nodes"], m["edge_ptr"], m["edge_pairs"])


def partitions(m, mesh, R, how):
    """The library partition and the oracle's sub-graphs for R = 1, the fan
    split (``how`` = "fans") or RCB of the element centres."""
    from paper_2410_01657_gb300.graph import MeshGraph
    from test_oracle_elements import _fan_split

    lib = MeshGraph.from_elements(m["pos"], m["elem_ptr"], m["elem_nodes"], m["edge_ptr"], m["edge_pairs"])
    if R == 1:
        return lib.partition(1, "rcb"), og.element_mesh_unpartitioned(mesh)
    if how == "fans":
        ep = _fan_split(m, R)
        return lib.partition(R, elem_part=ep), og.build_element_subgraphs(mesh, ep, R)
    return lib.partition(R, "rcb"), og.build_element_subgraphs(mesh, og.partition_rcb_elements(mesh, R), R)
