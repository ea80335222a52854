"""Thin ctypes binding of libbfc (include/bfc.h): argument marshalling only.

Every function keeps the C name.  Device pointers are plain integers (for
example ``tensor.data_ptr()``); ``stream`` is a cudaStream_t as an integer
(``torch.cuda.current_stream().cuda_stream``), 0 for the legacy default
stream.  A non-OK status raises :class:`BfcError`.  There is no fallback:
if libbfc.so is missing the import fails.
"""
from __future__ import annotations

import ctypes
import os
import re

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbfc.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "bfc.h")

c_int32, c_int64, c_uint64, c_void_p, c_int = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                               ctypes.c_void_p, ctypes.c_int)

BFC_OK = 0
STATUS = {0: "BFC_OK", 1: "BFC_ERR_INVALID_ARGUMENT", 2: "BFC_ERR_INVALID_GRAPH",
          3: "BFC_ERR_OUT_OF_MEMORY", 4: "BFC_ERR_CUDA", 5: "BFC_ERR_TIMEOUT",
          6: "BFC_ERR_INTERNAL"}
(BFC_RANK_U, BFC_RANK_L, BFC_PROJ_OFF, BFC_PROJ_ADJ, BFC_PROJ_EID, BFC_CUT, BFC_WORK, BFC_RETRIES,
 BFC_CORE_PRODUCT_U, BFC_CORE_PRODUCT_L) = range(10)


class bfc_csr(ctypes.Structure):
    _fields_ = [("num_u", c_int32), ("num_l", c_int32), ("num_edges", c_int64),
                ("off_u", c_void_p), ("adj_u", c_void_p)]


class bfc_options(ctypes.Structure):
    _fields_ = [("validate", c_int32), ("warp_max_work", c_int32), ("hash_max_work", c_int32),
                ("num_ctas", c_int32), ("wide_positions", c_int32), ("orientation", c_int32),
                ("team_max_work", c_int32), ("core_vertices", c_int32), ("use_tuned", c_int32),
                ("reserved", c_int32 * 7)]


class bfc_info(ctypes.Structure):
    _fields_ = [("num_u", c_int32), ("num_l", c_int32), ("num_edges", c_int64),
                ("wedges", c_uint64), ("max_start_work", c_uint64),
                ("starts_with_work", c_int64), ("warp_starts", c_int64), ("hash_starts", c_int64),
                ("dense_starts", c_int64), ("dense_items", c_int64), ("device_bytes", c_int64),
                ("max_deg_u", c_int32), ("max_deg_l", c_int32), ("team_starts", c_int64),
                ("core_u", c_int32), ("core_l", c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class bfc_batch(ctypes.Structure):
    _fields_ = [("num_graphs", c_int32), ("graph_u_start", c_void_p), ("graph_l_start", c_void_p)]


class bfc_batch_shape(ctypes.Structure):
    _fields_ = [("num_u", c_int32), ("num_l", c_int32), ("num_edges", c_int64), ("num_graphs", c_int32),
                ("max_layer", c_int32), ("reserved", c_int32 * 6)]


class bfc_server_config(ctypes.Structure):
    _fields_ = [("memory_budget_bytes", c_int64), ("workers", c_int32), ("max_batch_graphs", c_int32),
                ("max_batch_edges", c_int64), ("warp_max_work", c_int32), ("hash_max_work", c_int32),
                ("team_max_work", c_int32), ("reserved", c_int32 * 7)]


class bfc_server_stats(ctypes.Structure):
    _fields_ = [(k, c_int64) for k in ("submitted", "completed", "failed", "batches",
                                       "max_batch_graphs", "peak_bytes_in_use", "bytes_in_use",
                                       "waiting", "pool_bytes_at_create", "pool_bytes_high")]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class BfcError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


if not os.path.exists(LIB_PATH):
    raise ImportError(f"libbfc.so not built ({LIB_PATH}); run `python -m paper_1812_00283_gb300.build`")

_lib = ctypes.CDLL(LIB_PATH)

_SIGS = {
    "bfc_options_init": (None, [ctypes.POINTER(bfc_options)]),
    "bfc_prepare": (c_int, [ctypes.POINTER(bfc_csr), ctypes.POINTER(bfc_options), c_void_p,
                            ctypes.POINTER(c_void_p)]),
    "bfc_count": (c_int, [c_void_p, c_void_p, c_void_p]),
    "bfc_count_vertices": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "bfc_count_edges": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "bfc_count_all": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "bfc_count_pairs": (c_int, [c_void_p, c_void_p, c_void_p]),
    "bfc_sync": (c_int, [c_void_p, c_void_p]),
    "bfc_graph_info": (c_int, [c_void_p, ctypes.POINTER(bfc_info)]),
    "bfc_export": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "bfc_count_host": (c_int, [c_int32, c_int32, c_int64, c_void_p, c_void_p,
                               ctypes.POINTER(bfc_options), c_void_p, ctypes.POINTER(c_uint64),
                               ctypes.POINTER(c_uint64)]),
    "bfc_count_all_host": (c_int, [c_int32, c_int32, c_int64, c_void_p, c_void_p,
                                   ctypes.POINTER(bfc_options), c_void_p, c_void_p, c_void_p, c_void_p,
                                   ctypes.POINTER(c_uint64), ctypes.POINTER(c_uint64)]),
    "bfc_release": (None, [c_void_p]),
    "bfc_status_string": (ctypes.c_char_p, [c_int]),
    "bfc_last_error": (ctypes.c_char_p, []),
    "bfc_version": (c_int, []),
    "bfc_kernel_launches": (ctypes.c_longlong, []),
    "bfc_caterpillars": (c_int, [c_void_p, c_void_p, c_void_p]),
    "bfc_clustering_coefficient": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "bfc_bench_smem_atomics": (c_int, [c_void_p, c_int32, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]),
    "bfc_prepare_batch": (c_int, [ctypes.POINTER(bfc_csr), ctypes.POINTER(bfc_batch),
                                  ctypes.POINTER(bfc_options), c_void_p, ctypes.POINTER(c_void_p)]),
    "bfc_count_batch": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "bfc_batch_wedges": (c_int, [c_void_p, c_void_p, c_void_p]),
    "bfc_autotune": (c_int, [c_void_p, c_void_p, c_int, ctypes.POINTER(bfc_options)]),
    "bfc_batch_plan_create": (c_int, [ctypes.POINTER(bfc_batch_shape), ctypes.POINTER(bfc_options), c_void_p,
                                      ctypes.POINTER(c_void_p)]),
    "bfc_batch_plan_run": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                   c_void_p]),
    "bfc_batch_plan_destroy": (None, [c_void_p]),
    "bfc_server_config_init": (None, [ctypes.POINTER(bfc_server_config)]),
    "bfc_server_create": (c_int, [ctypes.POINTER(bfc_server_config), ctypes.POINTER(c_void_p)]),
    "bfc_server_submit": (c_int, [c_void_p, c_int32, c_int32, c_int64, c_void_p, c_void_p,
                                  ctypes.POINTER(c_uint64)]),
    "bfc_server_poll": (c_int, [c_void_p, c_uint64, c_int, ctypes.POINTER(c_uint64),
                                ctypes.POINTER(c_int), ctypes.POINTER(ctypes.c_double)]),
    "bfc_server_get_stats": (c_int, [c_void_p, ctypes.POINTER(bfc_server_stats)]),
    "bfc_server_destroy": (None, [c_void_p]),
    "bfc_count_small_noalloc": (c_int, [c_int32, c_int32, c_int64, c_void_p, c_void_p, c_void_p,
                                        c_void_p, c_void_p]),
    "bfc_prepare_sparsified": (c_int, [c_int32, c_int32, c_int64, c_void_p, c_void_p, ctypes.c_double,
                                       c_uint64, c_int32, ctypes.POINTER(bfc_options), c_void_p, c_void_p,
                                       ctypes.POINTER(c_void_p)]),
    "bfc_sparsified_estimate": (c_int, [c_void_p, c_int32, ctypes.c_double, c_void_p, c_void_p]),
    "bfc_estimate_sparsified": (c_int, [c_int32, c_int32, c_int64, c_void_p, c_void_p, ctypes.c_double,
                                        c_uint64, c_int32, ctypes.POINTER(bfc_options), c_void_p, c_void_p,
                                        c_void_p]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def header_functions() -> list[str]:
    """Names of the functions include/bfc.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bfc_\w+)\s*\(", text)))


def _check(rc: int, where: str):
    if rc != BFC_OK:
        raise BfcError(rc, where, (_lib.bfc_last_error() or b"").decode())


def bfc_options_init(**overrides) -> bfc_options:
    o = bfc_options()
    _lib.bfc_options_init(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def bfc_prepare(num_u: int, num_l: int, num_edges: int, off_u: int, adj_u: int,
                options: bfc_options | None = None, stream: int = 0) -> int:
    """Steps a1-a5; returns an opaque graph handle (int)."""
    csr = bfc_csr(num_u, num_l, num_edges, off_u, adj_u)
    h = c_void_p()
    _check(_lib.bfc_prepare(ctypes.byref(csr), ctypes.byref(options) if options else None,
                            stream, ctypes.byref(h)), "bfc_prepare")
    return h.value


def bfc_count(g: int, stream: int, total_dev: int):
    _check(_lib.bfc_count(g, stream, total_dev), "bfc_count")


def bfc_count_vertices(g: int, stream: int, per_u_dev: int | None, per_l_dev: int | None,
                       total_dev: int | None):
    _check(_lib.bfc_count_vertices(g, stream, per_u_dev, per_l_dev, total_dev),
           "bfc_count_vertices")


def bfc_count_edges(g: int, stream: int, per_edge_dev: int, total_dev: int | None):
    _check(_lib.bfc_count_edges(g, stream, per_edge_dev, total_dev), "bfc_count_edges")


def bfc_count_all(g: int, stream: int, per_u_dev: int | None, per_l_dev: int | None,
                  per_edge_dev: int, total_dev: int | None):
    _check(_lib.bfc_count_all(g, stream, per_u_dev, per_l_dev, per_edge_dev, total_dev), "bfc_count_all")


def bfc_count_pairs(g: int, stream: int, total_dev: int):
    _check(_lib.bfc_count_pairs(g, stream, total_dev), "bfc_count_pairs")


def bfc_sync(g: int, stream: int = 0):
    _check(_lib.bfc_sync(g, stream), "bfc_sync")


def bfc_graph_info(g: int) -> dict:
    info = bfc_info()
    _check(_lib.bfc_graph_info(g, ctypes.byref(info)), "bfc_graph_info")
    return info.as_dict()


def bfc_export(g: int, which: int, dst_dev: int, stream: int = 0):
    _check(_lib.bfc_export(g, which, dst_dev, stream), "bfc_export")


def bfc_count_host(num_u: int, num_l: int, num_edges: int, off_u_host: int, adj_u_host: int,
                   options: bfc_options | None = None, stream: int = 0) -> tuple[int, int]:
    """End to end from host memory: returns (total, processed wedges)."""
    t = c_uint64(0)
    w = c_uint64(0)
    _check(_lib.bfc_count_host(num_u, num_l, num_edges, off_u_host, adj_u_host,
                               ctypes.byref(options) if options else None, stream,
                               ctypes.byref(t), ctypes.byref(w)), "bfc_count_host")
    return int(t.value), int(w.value)


def bfc_count_all_host(num_u: int, num_l: int, num_edges: int, off_u_host: int, adj_u_host: int,
                       options: bfc_options | None, stream: int, per_u_host: int | None,
                       per_l_host: int | None, per_edge_host: int | None) -> tuple[int, int]:
    """Steps a1-a9 from host buffers into host buffers; returns (total, W)."""
    tot, wed = c_uint64(0), c_uint64(0)
    _check(_lib.bfc_count_all_host(num_u, num_l, num_edges, off_u_host, adj_u_host,
                                   ctypes.byref(options) if options else None, stream, per_u_host,
                                   per_l_host, per_edge_host, ctypes.byref(tot), ctypes.byref(wed)),
           "bfc_count_all_host")
    return int(tot.value), int(wed.value)


def bfc_prepare_batch(num_u: int, num_l: int, num_edges: int, off_u: int, adj_u: int,
                      num_graphs: int, graph_u_start: int, graph_l_start: int,
                      options: bfc_options | None = None, stream: int = 0) -> int:
    """Steps a1-a5 for a batch given as a disjoint union; returns a graph handle."""
    csr = bfc_csr(num_u, num_l, num_edges, off_u, adj_u)
    b = bfc_batch(num_graphs, graph_u_start, graph_l_start)
    h = c_void_p()
    _check(_lib.bfc_prepare_batch(ctypes.byref(csr), ctypes.byref(b),
                                  ctypes.byref(options) if options else None, stream,
                                  ctypes.byref(h)), "bfc_prepare_batch")
    return h.value


def bfc_batch_plan_create(num_u: int, num_l: int, num_edges: int, num_graphs: int, max_layer: int,
                          options: bfc_options | None = None, stream: int = 0) -> int:
    """A plan for batches of this union shape; returns its handle."""
    shape = bfc_batch_shape(num_u, num_l, num_edges, num_graphs, max_layer)
    h = c_void_p()
    _check(_lib.bfc_batch_plan_create(ctypes.byref(shape), ctypes.byref(options) if options else None,
                                      stream, ctypes.byref(h)), "bfc_batch_plan_create")
    return h.value


def bfc_batch_plan_run(plan: int, off_u: int, adj_u: int, graph_u_start: int, graph_l_start: int,
                       stream: int, totals_dev: int, status_dev: int | None = None):
    _check(_lib.bfc_batch_plan_run(plan, off_u, adj_u, graph_u_start, graph_l_start, stream, totals_dev,
                                   status_dev), "bfc_batch_plan_run")


def bfc_batch_plan_destroy(plan: int):
    _lib.bfc_batch_plan_destroy(plan)


def bfc_count_batch(g: int, stream: int, totals_dev: int, total_dev: int | None = None):
    _check(_lib.bfc_count_batch(g, stream, totals_dev, total_dev), "bfc_count_batch")


def bfc_batch_wedges(g: int, stream: int, wedges_dev: int):
    _check(_lib.bfc_batch_wedges(g, stream, wedges_dev), "bfc_batch_wedges")


def bfc_prepare_sparsified(num_u: int, num_l: int, num_edges: int, off_u: int, adj_u: int, p: float,
                           seed: int, num_samples: int, options: bfc_options | None = None,
                           stream: int = 0, sample_edges_dev: int | None = None) -> int:
    """num_samples edge-sparsified copies of a graph (keep probability p),
    prepared as one batch; returns a graph handle for bfc_count_batch."""
    h = c_void_p()
    _check(_lib.bfc_prepare_sparsified(num_u, num_l, num_edges, off_u, adj_u, float(p),
                                       seed & 0xFFFFFFFFFFFFFFFF, num_samples,
                                       ctypes.byref(options) if options else None, stream,
                                       sample_edges_dev, ctypes.byref(h)), "bfc_prepare_sparsified")
    return h.value


def bfc_sparsified_estimate(sample_counts_dev: int, num_samples: int, p: float, stream: int,
                            estimate_dev: int):
    _check(_lib.bfc_sparsified_estimate(sample_counts_dev, num_samples, float(p), stream, estimate_dev),
           "bfc_sparsified_estimate")


def bfc_estimate_sparsified(num_u: int, num_l: int, num_edges: int, off_u: int, adj_u: int, p: float,
                            seed: int, num_samples: int, options: bfc_options | None, stream: int,
                            sample_counts_dev: int, estimate_dev: int | None = None):
    _check(_lib.bfc_estimate_sparsified(num_u, num_l, num_edges, off_u, adj_u, float(p),
                                        seed & 0xFFFFFFFFFFFFFFFF, num_samples,
                                        ctypes.byref(options) if options else None, stream,
                                        sample_counts_dev, estimate_dev), "bfc_estimate_sparsified")


def bfc_autotune(g: int, stream: int = 0, iters: int = 2) -> bfc_options:
    o = bfc_options()
    _check(_lib.bfc_autotune(g, stream, iters, ctypes.byref(o)), "bfc_autotune")
    return o


def bfc_server_config_init(**overrides) -> bfc_server_config:
    c = bfc_server_config()
    _lib.bfc_server_config_init(ctypes.byref(c))
    for k, v in overrides.items():
        setattr(c, k, v)
    return c


def bfc_server_create(cfg: bfc_server_config | None = None) -> int:
    h = c_void_p()
    _check(_lib.bfc_server_create(ctypes.byref(cfg) if cfg else None, ctypes.byref(h)),
           "bfc_server_create")
    return h.value


def bfc_server_submit(sv: int, num_u: int, num_l: int, num_edges: int, off_u_host: int,
                      adj_u_host: int) -> int:
    rid = c_uint64(0)
    _check(_lib.bfc_server_submit(sv, num_u, num_l, num_edges, off_u_host, adj_u_host,
                                  ctypes.byref(rid)), "bfc_server_submit")
    return int(rid.value)


def bfc_server_poll(sv: int, request_id: int, wait: bool = True):
    """Returns (status, total, latency_s); status -1 = still pending."""
    t = c_uint64(0)
    st = c_int(-1)
    lat = ctypes.c_double(0.0)
    _check(_lib.bfc_server_poll(sv, request_id, 1 if wait else 0, ctypes.byref(t), ctypes.byref(st),
                                ctypes.byref(lat)), "bfc_server_poll")
    return int(st.value), int(t.value), float(lat.value)


def bfc_server_get_stats(sv: int) -> dict:
    o = bfc_server_stats()
    _check(_lib.bfc_server_get_stats(sv, ctypes.byref(o)), "bfc_server_get_stats")
    return o.as_dict()


def bfc_server_destroy(sv: int):
    _lib.bfc_server_destroy(sv)


def bfc_count_small_noalloc(num_u: int, num_l: int, num_edges: int, off_u: int, adj_u: int,
                            stream: int, total_dev: int, status_dev: int | None = None):
    """Allocation-free count of a small graph (see include/bfc.h for the limits
    and the rules on overlapping calls)."""
    _check(_lib.bfc_count_small_noalloc(num_u, num_l, num_edges, off_u, adj_u, stream, total_dev,
                                        status_dev), "bfc_count_small_noalloc")


def bfc_release(g: int):
    _lib.bfc_release(g)


def bfc_status_string(status: int) -> str:
    return _lib.bfc_status_string(status).decode()


def bfc_last_error() -> str:
    return (_lib.bfc_last_error() or b"").decode()


def bfc_version() -> int:
    return int(_lib.bfc_version())


def bfc_caterpillars(g: int, stream: int, out_dev: int):
    _check(_lib.bfc_caterpillars(g, stream, out_dev), "bfc_caterpillars")


def bfc_clustering_coefficient(g: int, stream: int, butterflies_dev: int, caterpillars_dev: int,
                               coefficient_dev: int):
    _check(_lib.bfc_clustering_coefficient(g, stream, butterflies_dev, caterpillars_dev,
                                           coefficient_dev), "bfc_clustering_coefficient")


def bfc_kernel_launches() -> int:
    return int(_lib.bfc_kernel_launches())


def bfc_bench_smem_atomics(stream: int, iters: int) -> tuple[float, float]:
    """(increments per second, device ms) of the counter-operation microbenchmark."""
    rate, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(_lib.bfc_bench_smem_atomics(stream, iters, ctypes.byref(rate), ctypes.byref(ms)),
           "bfc_bench_smem_atomics")
    return rate.value, ms.value


def library():
    """The loaded ctypes library (for symbol checks)."""
    return _lib
