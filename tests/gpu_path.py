"""Helpers that run the CUDA path through the C ABI for the tests."""
import numpy as np


def as_u64(t) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint64)


def run_gpu(g, vertices=False, edges=False, options=None, export=False, device="cuda:0"):
    """Prepare + count one graph on the GPU through the C ABI; returns numpy results."""
    import torch
    from paper_1812_00283_gb300 import ButterflyGraph, bfc
    off = torch.from_numpy(np.ascontiguousarray(g.off_u)).to(device)
    adj = torch.from_numpy(np.ascontiguousarray(g.adj_u if g.num_edges else np.zeros(1, np.int32))).to(device)
    if not g.num_edges:
        adj = adj[:0]
    G = ButterflyGraph(off, adj, g.num_u, g.num_l, options)
    try:
        out = dict(total=G.count(), info=G.info())
        out["retries"] = int(G.export(bfc.BFC_RETRIES)[0])
        if vertices:
            pu, pl, t = G.count_vertices()
            out.update(pv_u=as_u64(pu), pv_l=as_u64(pl), total_v=t)
        if edges:
            pe, t = G.count_edges()
            out.update(pe=as_u64(pe), total_e=t)
        if vertices and edges:
            # the combined pass must give exactly the separate passes' outputs
            pu, pl, pe, t = G.count_all()
            out.update(all_pv_u=as_u64(pu), all_pv_l=as_u64(pl), all_pe=as_u64(pe), total_all=t)
        if export:
            out["rank_u"] = G.export(bfc.BFC_RANK_U).cpu().numpy()
            out["rank_l"] = G.export(bfc.BFC_RANK_L).cpu().numpy()
            out["off"] = G.export(bfc.BFC_PROJ_OFF).cpu().numpy()
            out["adj"] = G.export(bfc.BFC_PROJ_ADJ).cpu().numpy()
            out["eid"] = G.export(bfc.BFC_PROJ_EID).cpu().numpy()
            out["cut"] = G.export(bfc.BFC_CUT).cpu().numpy()
            out["work"] = as_u64(G.export(bfc.BFC_WORK))
        G.sync()
        return out
    finally:
        G.release()
