"""Exact butterfly counting on one GB300 GPU (vertex-priority method of
Wang et al., "Efficient Butterfly Counting for Large Bipartite Networks").

The work happens in libbfc (hand-written CUDA for sm_103a behind a C ABI,
include/bfc.h).  This package binds it (``bfc``) and adds a small PyTorch
convenience layer: tensors in, tensors out, on the current CUDA stream.
"""
from __future__ import annotations

import importlib

__all__ = ["bfc", "BfcError", "ButterflyGraph", "count_butterflies", "estimate_butterflies"]


def __getattr__(name):
    # libbfc is loaded on first use, so that the build step can import this
    # package before the library exists; a missing library raises ImportError.
    if name == "bfc":
        return importlib.import_module(".bfc", __name__)
    if name == "BfcError":
        return importlib.import_module(".bfc", __name__).BfcError
    raise AttributeError(name)


def _lib():
    return importlib.import_module(".bfc", __name__)


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream), s


class ButterflyGraph:
    """A prepared graph (steps a1-a5) on the current device.

    ``off_u`` (int32[num_u + 1]) and ``adj_u`` (int32[num_edges]) are the U-side
    CSR as CUDA tensors; they may be freed once the constructor returns.
    """

    def __init__(self, off_u, adj_u, num_u: int, num_l: int, options=None, stream=None):
        import torch
        if off_u.dtype != torch.int32 or adj_u.dtype != torch.int32:
            raise TypeError("off_u and adj_u must be int32")
        if not (off_u.is_cuda and adj_u.is_cuda):
            raise TypeError("off_u and adj_u must be CUDA tensors")
        off_u = off_u.contiguous()
        adj_u = adj_u.contiguous()
        self.num_u, self.num_l, self.num_edges = int(num_u), int(num_l), int(adj_u.numel())
        self.device = off_u.device
        sp, _ = _stream(stream)
        bfc = _lib()
        self._h = bfc.bfc_prepare(self.num_u, self.num_l, self.num_edges, off_u.data_ptr(),
                                  adj_u.data_ptr() if self.num_edges else 0, options, sp)
        self._total = torch.zeros(1, dtype=torch.int64, device=self.device)

    # -- a6-a7 --------------------------------------------------------------
    def count_async(self, out=None, stream=None):
        """Launches the count; returns a 1-element int64 tensor holding ⋈_G
        (bit pattern of the uint64)."""
        import torch
        out = self._total if out is None else out
        sp, _ = _stream(stream)
        _lib().bfc_count(self._h, sp, out.data_ptr())
        return out

    def count(self, stream=None) -> int:
        out = self.count_async(stream=stream)
        sp, _ = _stream(stream)
        _lib().bfc_sync(self._h, sp)
        return int(out.item()) & ((1 << 64) - 1)

    # -- a8 -----------------------------------------------------------------
    def count_vertices(self, stream=None):
        """Returns (per_u, per_l, total) with per-vertex counts in original ids."""
        import torch
        pu = torch.empty(max(self.num_u, 1), dtype=torch.int64, device=self.device)
        pl = torch.empty(max(self.num_l, 1), dtype=torch.int64, device=self.device)
        sp, _ = _stream(stream)
        bfc = _lib()
        bfc.bfc_count_vertices(self._h, sp, pu.data_ptr(), pl.data_ptr(), self._total.data_ptr())
        bfc.bfc_sync(self._h, sp)
        return pu[:self.num_u], pl[:self.num_l], int(self._total.item()) & ((1 << 64) - 1)

    # -- a9 -----------------------------------------------------------------
    def count_edges(self, stream=None):
        """Returns (per_edge, total); per_edge is indexed by U-side slot."""
        import torch
        pe = torch.empty(max(self.num_edges, 1), dtype=torch.int64, device=self.device)
        sp, _ = _stream(stream)
        bfc = _lib()
        bfc.bfc_count_edges(self._h, sp, pe.data_ptr(), self._total.data_ptr())
        bfc.bfc_sync(self._h, sp)
        return pe[:self.num_edges], int(self._total.item()) & ((1 << 64) - 1)

    def count_all(self, stream=None):
        """Returns (per_u, per_l, per_edge, total) from one combined pass."""
        import torch
        pu = torch.empty(max(self.num_u, 1), dtype=torch.int64, device=self.device)
        pl = torch.empty(max(self.num_l, 1), dtype=torch.int64, device=self.device)
        pe = torch.empty(max(self.num_edges, 1), dtype=torch.int64, device=self.device)
        sp, _ = _stream(stream)
        bfc = _lib()
        bfc.bfc_count_all(self._h, sp, pu.data_ptr(), pl.data_ptr(), pe.data_ptr(), self._total.data_ptr())
        bfc.bfc_sync(self._h, sp)
        return (pu[:self.num_u], pl[:self.num_l], pe[:self.num_edges],
                int(self._total.item()) & ((1 << 64) - 1))

    def count_pairs(self, stream=None) -> int:
        """⋈_G by Section 6.3's pair formulation (sort of the wedge pairs)."""
        import torch
        out = torch.zeros(1, dtype=torch.int64, device=self.device)
        sp, _ = _stream(stream)
        bfc = _lib()
        bfc.bfc_count_pairs(self._h, sp, out.data_ptr())
        bfc.bfc_sync(self._h, sp)
        return int(out.item()) & ((1 << 64) - 1)

    # -- derived statistics (Section 1) ----------------------------------------
    def caterpillars(self, stream=None) -> int:
        """Three-paths: Σ over edges (deg u − 1)(deg v − 1)."""
        import torch
        out = torch.zeros(1, dtype=torch.int64, device=self.device)
        sp, _ = _stream(stream)
        bfc = _lib()
        bfc.bfc_caterpillars(self._h, sp, out.data_ptr())
        bfc.bfc_sync(self._h, sp)
        return int(out.item()) & ((1 << 64) - 1)

    def clustering_coefficient(self, stream=None) -> float:
        """Bipartite clustering coefficient 4·⋈_G / caterpillars (0 without
        three-paths), computed by the library from a fresh count."""
        import torch
        tot = self.count_async(stream=stream)
        cat = torch.zeros(1, dtype=torch.int64, device=self.device)
        coef = torch.zeros(1, dtype=torch.float64, device=self.device)
        sp, _ = _stream(stream)
        bfc = _lib()
        bfc.bfc_clustering_coefficient(self._h, sp, tot.data_ptr(), cat.data_ptr(), coef.data_ptr())
        bfc.bfc_sync(self._h, sp)
        return float(coef.item())

    def info(self) -> dict:
        return _lib().bfc_graph_info(self._h)

    def export(self, which: int, stream=None):
        """Copies an internal array (bfc.BFC_*) into a new tensor."""
        import torch
        bfc = _lib()
        n = self.num_u + self.num_l
        m = self.num_edges
        spec = {bfc.BFC_RANK_U: (self.num_u, torch.int32), bfc.BFC_RANK_L: (self.num_l, torch.int32),
                bfc.BFC_PROJ_OFF: (n + 1, torch.int64), bfc.BFC_PROJ_ADJ: (2 * m, torch.int32),
                bfc.BFC_PROJ_EID: (2 * m, torch.int32), bfc.BFC_CUT: (n, torch.int32),
                bfc.BFC_WORK: (n, torch.int64), bfc.BFC_RETRIES: (1, torch.int32)}
        info = self.info()
        spec[bfc.BFC_CORE_PRODUCT_U] = (info["core_u"] ** 2, torch.int16)
        spec[bfc.BFC_CORE_PRODUCT_L] = (info["core_l"] ** 2, torch.int16)
        spec = spec[which]
        t = torch.empty(max(spec[0], 1), dtype=spec[1], device=self.device)
        sp, _ = _stream(stream)
        bfc.bfc_export(self._h, which, t.data_ptr(), sp)
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        return t[:spec[0]]

    def sync(self, stream=None):
        sp, _ = _stream(stream)
        _lib().bfc_sync(self._h, sp)

    def release(self):
        if getattr(self, "_h", None):
            _lib().bfc_release(self._h)
            self._h = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


def count_butterflies(off_u, adj_u, num_u: int, num_l: int, options=None) -> int:
    """⋈_G of a U-side CSR given as CUDA tensors."""
    g = ButterflyGraph(off_u, adj_u, num_u, num_l, options)
    try:
        return g.count()
    finally:
        g.release()


def estimate_butterflies(off_u, adj_u, num_u: int, num_l: int, p: float, num_samples: int,
                         seed: int = 0, options=None, stream=None) -> dict:
    """Approximate ⋈_G from num_samples edge-sparsified copies (each edge kept
    with probability p), each counted exactly (Section 7's estimator with this
    counter as its inner block).  Returns the samples' exact counts (uint64
    as an int64 CUDA tensor), the estimate and its standard error."""
    import torch
    if off_u.dtype != torch.int32 or adj_u.dtype != torch.int32:
        raise TypeError("off_u and adj_u must be int32")
    if not (off_u.is_cuda and adj_u.is_cuda):
        raise TypeError("off_u and adj_u must be CUDA tensors")
    off_u, adj_u = off_u.contiguous(), adj_u.contiguous()
    sp, s = _stream(stream)
    counts = torch.zeros(int(num_samples), dtype=torch.int64, device=off_u.device)
    est = torch.zeros(2, dtype=torch.float64, device=off_u.device)
    _lib().bfc_estimate_sparsified(int(num_u), int(num_l), int(adj_u.numel()), off_u.data_ptr(),
                                   adj_u.data_ptr() if adj_u.numel() else 0, p, int(seed),
                                   int(num_samples), options, sp, counts.data_ptr(), est.data_ptr())
    e = est.cpu().tolist()
    return dict(counts=counts, estimate=e[0], std_error=e[1])
