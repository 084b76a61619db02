"""Thin ctypes binding of libcompass (include/compass.h).

The entry points keep the C names (cmp_*).  This module only marshals arguments:
torch CUDA tensors are passed by data_ptr(), streams by their cudaStream_t handle, and
every status code other than CMP_OK raises CompassError.  All arithmetic of the path
runs in the library's kernels; there is no fallback when the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build_lib

CMP_OK, CMP_EINVAL, CMP_EUNSUPPORTED, CMP_EOVERFLOW, CMP_ECUDA, CMP_EWORKSPACE, CMP_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
CMP_I32, CMP_I64 = 0, 1
CMP_RANGE, CMP_EQ, CMP_IN_BITMAP = 0, 1, 2
CMP_EST_GENERIC_ONLY = 1
CMP_EST_CACHE_MESSAGES = 2
CMP_EST_STAR_LATTICE = 4
CMP_EST_NO_WIDE = 8
CMP_ABI_VERSION = 7
CMP_PART_MAX_AXES = 4
CMP_MAX_COLS, CMP_MAX_PREDS, CMP_MAX_SKETCHES, CMP_MAX_D = 32, 8, 16, 64


class CompassError(RuntimeError):
    def __init__(self, fn: str, status: int):
        super().__init__(f"{fn}: {status_str(status)} ({status})")
        self.status = status


CMP_COL_UNIQUE = 1
CMP_COL_DOMAIN = 2


class cmp_col(C.Structure):
    _fields_ = [("data", C.c_void_p), ("dtype", C.c_int32), ("flags", C.c_int32), ("dom_lo", C.c_int64),
                ("dom_hi", C.c_int64)]


class cmp_pred(C.Structure):
    _fields_ = [("col", C.c_int32), ("op", C.c_int32), ("lo", C.c_int64), ("hi", C.c_int64),
                ("bitmap", C.c_void_p), ("bitmap_nbits", C.c_int64)]


class cmp_hash(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("a", "b", "c0", "c1", "c2", "c3")]


class cmp_table(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("n_cols", C.c_int32), ("n_preds", C.c_int32), ("n_sketches", C.c_int32),
                ("reserved", C.c_int32), ("cols", C.POINTER(cmp_col)), ("preds", C.POINTER(cmp_pred)),
                ("key_col", C.POINTER(C.c_int32)), ("edge_id", C.POINTER(C.c_int32)),
                ("sample_seed", C.c_uint64), ("sample_rate", C.c_double)]


class cmp_build_cfg(C.Structure):
    _fields_ = [("mode", C.c_int32), ("pairs_per_slab", C.c_int32), ("threads", C.c_int32),
                ("tile_rows", C.c_int32), ("dedupe", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("aggregate", C.c_int32), ("unique", C.c_int32)]

    @classmethod
    def make(cls, mode=0, pairs_per_slab=0, threads=0, tile_rows=0, dedupe=-1, ctas_per_sm=0, aggregate=-1,
             unique=0):
        return cls(mode, pairs_per_slab, threads, tile_rows, dedupe, ctas_per_sm, aggregate, unique)


class cmp_build_plan_info(C.Structure):
    _fields_ = [("n_tables", C.c_int32), ("n_agg", C.c_int32), ("n_unique_slabs", C.c_int32),
                ("unique_grid", C.c_int32), ("n_unique_items", C.c_int64), ("row_grid", C.c_int64),
                ("ws_bytes", C.c_int64), ("launches", C.c_int32), ("n_presence", C.c_int32)]


class cmp_part_estimate_cfg(C.Structure):
    _fields_ = [("wait_polls", C.c_int32), ("reserved", C.c_int32)]


class cmp_estimate_plan_info(C.Structure):
    _fields_ = [("n_sub", C.c_int64), ("n_items", C.c_int64), ("n_ops", C.c_int64), ("n_jobs", C.c_int64),
                ("n_job_items", C.c_int64), ("n_tri", C.c_int64), ("n_levels", C.c_int32), ("grid", C.c_int32),
                ("n_star", C.c_int64), ("n_star_sub", C.c_int64), ("n_star_entries", C.c_int64)]


class cmp_estimate_cfg(C.Structure):
    _fields_ = [("threads", C.c_int32), ("ctas_per_sm", C.c_int32), ("cond_chunk", C.c_int32),
                ("flags", C.c_int32)]

    @classmethod
    def make(cls, threads=0, ctas_per_sm=0, cond_chunk=0, flags=0):
        return cls(threads, ctas_per_sm, cond_chunk, flags)


class cmp_graph(C.Structure):
    _fields_ = [("n_tables", C.c_int32), ("n_edges", C.c_int32), ("edge_u", C.POINTER(C.c_int32)),
                ("edge_v", C.POINTER(C.c_int32)), ("sketch", C.POINTER(C.c_void_p)),
                ("abs_sorted", C.POINTER(C.c_void_p)), ("perm", C.POINTER(C.c_void_p)),
                ("ranks", C.POINTER(C.c_void_p)), ("slot", C.POINTER(C.c_int32)), ("survivors_dev", C.c_void_p),
                ("sample_rate", C.POINTER(C.c_double))]


class cmp_enum_cfg(C.Structure):
    _fields_ = [("alpha", C.c_double), ("beta", C.c_double), ("max_plans", C.c_int64), ("max_nodes", C.c_int64)]

    @classmethod
    def make(cls, alpha=0.0, beta=0.0, max_plans=0, max_nodes=0):
        return cls(alpha, beta, max_plans, max_nodes)


class cmp_part_build_cfg(C.Structure):
    _fields_ = [("mode", C.c_int32), ("rows_per_cta", C.c_int32), ("threads", C.c_int32), ("tile_rows", C.c_int32),
                ("ctas_per_sm", C.c_int32), ("reserved", C.c_int32)]

    @classmethod
    def make(cls, mode=0, rows_per_cta=0, threads=0, tile_rows=0, ctas_per_sm=0):
        return cls(mode, rows_per_cta, threads, tile_rows, ctas_per_sm, 0)


class cmp_part_join(C.Structure):
    _fields_ = [("n_tables", C.c_int32), ("n_edges", C.c_int32), ("edge_u", C.POINTER(C.c_int32)),
                ("edge_v", C.POINTER(C.c_int32)), ("width", C.POINTER(C.c_int32)), ("n_axes", C.POINTER(C.c_int32)),
                ("axis_edge", C.POINTER(C.c_int32)), ("tensor", C.POINTER(C.c_void_p)),
                ("sample_rate", C.POINTER(C.c_double))]


_lib = None

_SIGS = {
    "cmp_abi_version": (C.c_int32, []),
    "cmp_status_str": (C.c_char_p, [C.c_int32]),
    "cmp_hash_params": (C.c_int32, [C.c_uint64, C.c_int32, C.c_int32, C.POINTER(cmp_hash)]),
    "cmp_sketch_build": (C.c_int32, [C.POINTER(cmp_table), C.c_int32, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.POINTER(cmp_build_cfg), C.c_void_p]),
    "cmp_build_plan_bytes": (C.c_int32, [C.POINTER(cmp_table), C.c_int32, C.c_int32, C.c_int32,
                                         C.POINTER(cmp_build_cfg), C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
    "cmp_build_plan_encode": (C.c_int32, [C.POINTER(cmp_table), C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                          C.POINTER(C.c_void_p), C.c_void_p, C.POINTER(cmp_build_cfg), C.c_void_p,
                                          C.c_size_t]),
    "cmp_sketch_build_batched": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t,
                                             C.c_void_p, C.c_void_p]),
    "cmp_presort_ws_bytes": (C.c_size_t, [C.c_int64, C.c_int32]),
    "cmp_presort": (C.c_int32, [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t,
                                C.c_void_p]),
    "cmp_cross_ranks": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32,
                                    C.POINTER(C.c_int32), C.c_void_p, C.c_void_p]),
    "cmp_cross_ranks_multi": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(C.c_int32),
                                          C.POINTER(C.c_int32), C.c_int32, C.c_int32, C.c_void_p, C.c_void_p]),
    "cmp_estimate_plan_bytes": (C.c_int32, [C.POINTER(cmp_graph), C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                            C.c_void_p, C.c_void_p, C.POINTER(cmp_estimate_cfg),
                                            C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
    "cmp_estimate_plan_encode": (C.c_int32, [C.POINTER(cmp_graph), C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                             C.c_void_p, C.c_void_p, C.POINTER(cmp_estimate_cfg), C.c_void_p,
                                             C.c_size_t]),
    "cmp_estimate": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p]),
    "cmp_estimate_plan_stats": (C.c_int32, [C.c_void_p, C.POINTER(cmp_estimate_plan_info)]),
    "cmp_enum_plan_bytes": (C.c_int32, [C.POINTER(cmp_graph), C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                        C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
    "cmp_enum_plan_encode": (C.c_int32, [C.POINTER(cmp_graph), C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_size_t]),
    "cmp_enumerate": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(cmp_enum_cfg), C.c_void_p,
                                  C.c_size_t, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "cmp_estimate_noalloc": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "cmp_build_plan_stats": (C.c_int32, [C.c_void_p, C.POINTER(cmp_build_plan_info)]),
    "cmp_part_estimate_ex": (C.c_int32, [C.POINTER(cmp_part_join), C.c_int32, C.c_void_p, C.c_size_t, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.POINTER(cmp_part_estimate_cfg), C.c_void_p]),
    "cmp_estimate_ex": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.c_void_p]),
    "cmp_mlp_combine_ex": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_void_p,
                                       C.c_void_p]),
    "cmp_microbench_cw": (C.c_int32, [C.c_void_p, C.c_int32, C.c_int64, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p]),
    "cmp_part_build": (C.c_int32, [C.POINTER(cmp_table), C.c_int32, C.POINTER(C.c_int32), C.c_void_p, C.c_int32,
                                   C.c_void_p, C.c_void_p, C.POINTER(cmp_part_build_cfg), C.c_void_p]),
    "cmp_part_estimate_ws_bytes": (C.c_int32, [C.POINTER(cmp_part_join), C.c_int32, C.POINTER(C.c_size_t)]),
    "cmp_part_estimate": (C.c_int32, [C.POINTER(cmp_part_join), C.c_int32, C.c_void_p, C.c_size_t, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p]),
    "cmp_mlp_param_count": (C.c_int64, [C.c_int32, C.c_int32]),
    "cmp_sketch_f2": (C.c_int32, [C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p]),
    "cmp_mlp_features": (C.c_int32, [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p]),
    "cmp_mlp_features_indexed": (C.c_int32, [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                             C.c_void_p]),
    "cmp_mlp_infer": (C.c_int32, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p,
                                  C.c_void_p]),
    "cmp_mlp_combine": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "cmp_mlp_train_ws_bytes": (C.c_size_t, [C.c_int32, C.c_int32, C.c_int64]),
    "cmp_mlp_train_step": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32,
                                       C.c_void_p, C.c_void_p, C.c_int64, C.c_float, C.c_float, C.c_int32,
                                       C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
}


def lib_path() -> str:
    return build_lib.LIB


def lib(build_if_missing: bool = True):
    """Load libcompass; raises if it is missing and cannot be built (no fallback)."""
    global _lib
    if _lib is None:
        path = build_lib.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"libcompass not built at {path}")
            build_lib.build()
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        if L.cmp_abi_version() != CMP_ABI_VERSION:
            raise RuntimeError(f"libcompass at {path} has interface version {L.cmp_abi_version()}, "
                               f"this binding needs {CMP_ABI_VERSION}: rebuild it")
        _lib = L
    return _lib


def exported_symbols() -> list:
    L = lib()
    return [n for n in _SIGS if getattr(L, n, None) is not None]


def status_str(s: int) -> str:
    return lib().cmp_status_str(int(s)).decode()


def _check(fn: str, st: int):
    if st != CMP_OK:
        raise CompassError(fn, st)


def stream_handle(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


# ------------------------------------------------------------------ entry points

def cmp_hash_params(seed: int, n_edges: int, d: int):
    arr = (cmp_hash * max(n_edges * d, 1))()
    _check("cmp_hash_params", lib().cmp_hash_params(C.c_uint64(seed), n_edges, d, arr))
    return arr


def hash_params_u64(seed: int, n_edges: int, d: int):
    """Hash parameters as a [n_edges, d, 6] numpy uint64 array (a, b, c0, c1, c2, c3)."""
    import numpy as np
    arr = cmp_hash_params(seed, n_edges, d)
    out = np.frombuffer(arr, dtype=np.uint64, count=max(n_edges * d, 1) * 6).copy()
    return out[: n_edges * d * 6].reshape(n_edges, d, 6)


def cmp_sketch_build(table: cmp_table, d: int, w: int, hash_dev: int, n_edges: int, counters_dev: int,
                     survivors_dev: int, status_dev: int, cfg: cmp_build_cfg | None, stream: int):
    _check("cmp_sketch_build",
           lib().cmp_sketch_build(C.byref(table), d, w, hash_dev, n_edges, counters_dev, survivors_dev, status_dev,
                                  C.byref(cfg) if cfg is not None else None, stream))


def cmp_build_plan_bytes(tables, d: int, w: int, cfg: cmp_build_cfg | None) -> tuple[int, int]:
    """(plan bytes, workspace bytes) of a batched build."""
    arr = (cmp_table * len(tables))(*tables)
    n, ws = C.c_size_t(0), C.c_size_t(0)
    _check("cmp_build_plan_bytes", lib().cmp_build_plan_bytes(arr, len(tables), d, w,
                                                              C.byref(cfg) if cfg is not None else None, C.byref(n),
                                                              C.byref(ws)))
    return n.value, ws.value


def cmp_build_plan_encode(tables, d: int, w: int, n_edges: int, counters_ptrs, survivors_dev: int,
                          cfg: cmp_build_cfg | None, plan_host: int, plan_bytes: int):
    arr = (cmp_table * len(tables))(*tables)
    cp = (C.c_void_p * len(tables))(*counters_ptrs)
    _check("cmp_build_plan_encode",
           lib().cmp_build_plan_encode(arr, len(tables), d, w, n_edges, cp, survivors_dev,
                                       C.byref(cfg) if cfg is not None else None, plan_host, plan_bytes))


def cmp_sketch_build_batched(plan_host: int, plan_dev: int, hash_dev: int, ws_dev: int, ws_bytes: int,
                             status_dev: int, stream: int):
    _check("cmp_sketch_build_batched", lib().cmp_sketch_build_batched(plan_host, plan_dev, hash_dev, ws_dev, ws_bytes,
                                                                      status_dev, stream))


def cmp_presort_ws_bytes(n_rows: int, w: int) -> int:
    return int(lib().cmp_presort_ws_bytes(n_rows, w))


def cmp_presort(counters_dev: int, n_rows: int, w: int, abs_sorted_dev: int, perm_dev: int, ws_dev: int,
                ws_bytes: int, stream: int):
    _check("cmp_presort", lib().cmp_presort(counters_dev, n_rows, w, abs_sorted_dev, perm_dev, ws_dev, ws_bytes,
                                            stream))


def cmp_cross_ranks(abs_dev: int, perm_dev: int, k: int, d: int, w: int, edge_ids, ranks_dev: int, stream: int):
    e = (C.c_int32 * max(k, 1))(*edge_ids)
    _check("cmp_cross_ranks", lib().cmp_cross_ranks(abs_dev, perm_dev, k, d, w, e, ranks_dev, stream))


def cmp_cross_ranks_multi(abs_dev: int, perm_dev: int, ks, edge_ids, d: int, w: int, ranks_dev: int, stream: int):
    kk = (C.c_int32 * max(len(ks), 1))(*ks)
    ee = (C.c_int32 * max(len(edge_ids), 1))(*edge_ids)
    _check("cmp_cross_ranks_multi",
           lib().cmp_cross_ranks_multi(abs_dev, perm_dev, len(ks), kk, ee, d, w, ranks_dev, stream))


def cmp_estimate_plan_bytes(graphs, d: int, w: int, sub_graph, sub_mask, cfg: cmp_estimate_cfg | None = None):
    import numpy as np
    g = (cmp_graph * len(graphs))(*graphs)
    sg = np.ascontiguousarray(sub_graph, np.int32)
    sm = np.ascontiguousarray(sub_mask, np.uint64)
    pb, wb = C.c_size_t(0), C.c_size_t(0)
    _check("cmp_estimate_plan_bytes",
           lib().cmp_estimate_plan_bytes(g, len(graphs), d, w, sg.size, sg.ctypes.data, sm.ctypes.data,
                                         C.byref(cfg) if cfg is not None else None, C.byref(pb), C.byref(wb)))
    return pb.value, wb.value


def cmp_estimate_plan_encode(graphs, d: int, w: int, sub_graph, sub_mask, plan_host: int, plan_bytes: int,
                             cfg: cmp_estimate_cfg | None = None):
    import numpy as np
    g = (cmp_graph * len(graphs))(*graphs)
    sg = np.ascontiguousarray(sub_graph, np.int32)
    sm = np.ascontiguousarray(sub_mask, np.uint64)
    _check("cmp_estimate_plan_encode",
           lib().cmp_estimate_plan_encode(g, len(graphs), d, w, sg.size, sg.ctypes.data, sm.ctypes.data,
                                          C.byref(cfg) if cfg is not None else None, plan_host, plan_bytes))


def cmp_estimate_plan_stats(plan_host: int) -> cmp_estimate_plan_info:
    info = cmp_estimate_plan_info()
    _check("cmp_estimate_plan_stats", lib().cmp_estimate_plan_stats(plan_host, C.byref(info)))
    return info


def cmp_estimate(plan_host: int, plan_dev: int, ws_dev: int, ws_bytes: int, est_dev: int, row_est_dev: int,
                 status_dev: int, stream: int):
    _check("cmp_estimate", lib().cmp_estimate(plan_host, plan_dev, ws_dev, ws_bytes, est_dev, row_est_dev,
                                              status_dev, stream))


CMP_NOALLOC_WS_BYTES = 32 << 20


def cmp_estimate_noalloc(plan_host: int, plan_dev: int, est_dev: int, row_est_dev: int, status_dev: int,
                         stream: int):
    _check("cmp_estimate_noalloc", lib().cmp_estimate_noalloc(plan_host, plan_dev, est_dev, row_est_dev, status_dev,
                                                              stream))


def cmp_build_plan_stats(plan_host: int) -> cmp_build_plan_info:
    info = cmp_build_plan_info()
    _check("cmp_build_plan_stats", lib().cmp_build_plan_stats(plan_host, C.byref(info)))
    return info


def cmp_estimate_ex(plan_host: int, plan_dev: int, ws_dev: int, ws_bytes: int, est_dev: int, row_est_dev: int,
                    wide_rows_dev: int, status_dev: int, stream: int):
    _check("cmp_estimate_ex", lib().cmp_estimate_ex(plan_host, plan_dev, ws_dev, ws_bytes, est_dev, row_est_dev,
                                                    wide_rows_dev, status_dev, stream))


def cmp_mlp_combine_ex(median_dev: int, y_dev: int, eligible_dev: int, n: int, use_median_at: float, est_dev: int,
                       stream: int):
    _check("cmp_mlp_combine_ex", lib().cmp_mlp_combine_ex(median_dev, y_dev, eligible_dev, n, use_median_at, est_dev,
                                                          stream))


def cmp_microbench_cw(hash_dev: int, n_pairs: int, n_keys: int, w: int, form: int, out_dev: int, stream: int):
    _check("cmp_microbench_cw", lib().cmp_microbench_cw(hash_dev, n_pairs, n_keys, w, form, out_dev, stream))


def cmp_enum_plan_bytes(graphs, sub_graph, sub_mask) -> tuple[int, int]:
    import numpy as np
    g = (cmp_graph * len(graphs))(*graphs)
    sg = np.ascontiguousarray(sub_graph, np.int32)
    sm = np.ascontiguousarray(sub_mask, np.uint64)
    pb, wb = C.c_size_t(0), C.c_size_t(0)
    _check("cmp_enum_plan_bytes", lib().cmp_enum_plan_bytes(g, len(graphs), sg.size, sg.ctypes.data, sm.ctypes.data,
                                                            C.byref(pb), C.byref(wb)))
    return pb.value, wb.value


def cmp_enum_plan_encode(graphs, sub_graph, sub_mask, plan_host: int, plan_bytes: int):
    import numpy as np
    g = (cmp_graph * len(graphs))(*graphs)
    sg = np.ascontiguousarray(sub_graph, np.int32)
    sm = np.ascontiguousarray(sub_mask, np.uint64)
    _check("cmp_enum_plan_encode", lib().cmp_enum_plan_encode(g, len(graphs), sg.size, sg.ctypes.data, sm.ctypes.data,
                                                              plan_host, plan_bytes))


def cmp_enumerate(plan_host: int, plan_dev: int, est_dev: int, cfg: cmp_enum_cfg | None, ws_dev: int, ws_bytes: int,
                  order_dev: int, cost_dev: int, stats_dev: int, status_dev: int, stream: int):
    _check("cmp_enumerate", lib().cmp_enumerate(plan_host, plan_dev, est_dev, C.byref(cfg) if cfg is not None else None,
                                                ws_dev, ws_bytes, order_dev, cost_dev, stats_dev, status_dev, stream))


def cmp_part_build(table: cmp_table, d: int, widths, hash_dev: int, n_edges: int, counters_dev: int,
                   survivors_dev: int, cfg: cmp_part_build_cfg | None, stream: int):
    wa = (C.c_int32 * max(len(widths), 1))(*widths)
    _check("cmp_part_build", lib().cmp_part_build(C.byref(table), d, wa, hash_dev, n_edges, counters_dev, survivors_dev,
                                                  C.byref(cfg) if cfg is not None else None, stream))


def part_join(edge_u, edge_v, width, axes, tensor_ptrs, sample_rate=None):
    """A cmp_part_join and the ctypes arrays it points into (keep both alive)."""
    ne, nt = len(edge_u), len(axes)
    keep = [(C.c_int32 * max(ne, 1))(*edge_u), (C.c_int32 * max(ne, 1))(*edge_v), (C.c_int32 * max(ne, 1))(*width),
            (C.c_int32 * max(nt, 1))(*[len(a) for a in axes]),
            (C.c_int32 * max(sum(len(a) for a in axes), 1))(*[e for a in axes for e in a]),
            (C.c_void_p * max(nt, 1))(*tensor_ptrs)]
    rates = (C.c_double * max(nt, 1))(*sample_rate) if sample_rate is not None else None
    return cmp_part_join(nt, ne, *keep, rates), keep + [rates]


def cmp_part_estimate_ws_bytes(join: cmp_part_join, d: int) -> int:
    n = C.c_size_t(0)
    _check("cmp_part_estimate_ws_bytes", lib().cmp_part_estimate_ws_bytes(C.byref(join), d, C.byref(n)))
    return n.value


def cmp_part_estimate(join: cmp_part_join, d: int, ws_dev: int, ws_bytes: int, est_dev: int, row_est_dev: int,
                      status_dev: int, stream: int):
    _check("cmp_part_estimate", lib().cmp_part_estimate(C.byref(join), d, ws_dev, ws_bytes, est_dev, row_est_dev,
                                                        status_dev, stream))


def cmp_part_estimate_ex(join: cmp_part_join, d: int, ws_dev: int, ws_bytes: int, est_dev: int, row_est_dev: int,
                         status_dev: int, wait_polls: int, stream: int):
    cfg = cmp_part_estimate_cfg(wait_polls, 0)
    _check("cmp_part_estimate_ex", lib().cmp_part_estimate_ex(C.byref(join), d, ws_dev, ws_bytes, est_dev, row_est_dev,
                                                              status_dev, C.byref(cfg), stream))


def cmp_mlp_param_count(nin: int, nh: int) -> int:
    return int(lib().cmp_mlp_param_count(nin, nh))


def cmp_sketch_f2(counters_dev: int, n_sketches: int, d: int, w: int, f2_dev: int, stream: int):
    _check("cmp_sketch_f2", lib().cmp_sketch_f2(counters_dev, n_sketches, d, w, f2_dev, stream))


def cmp_mlp_features(row_est_dev: int, n: int, d: int, f2a_dev: int, f2b_dev: int, feat_dev: int, stream: int):
    _check("cmp_mlp_features", lib().cmp_mlp_features(row_est_dev, n, d, f2a_dev, f2b_dev, feat_dev, stream))


def cmp_mlp_features_indexed(row_est_dev: int, n: int, d: int, f2_dev: int, f2_index_dev: int, feat_dev: int,
                             stream: int):
    _check("cmp_mlp_features_indexed",
           lib().cmp_mlp_features_indexed(row_est_dev, n, d, f2_dev, f2_index_dev, feat_dev, stream))


def cmp_mlp_infer(params_dev: int, nin: int, nh: int, skip: int, x_dev: int, n: int, y_dev: int, stream: int):
    _check("cmp_mlp_infer", lib().cmp_mlp_infer(params_dev, nin, nh, skip, x_dev, n, y_dev, stream))


def cmp_mlp_combine(median_dev: int, y_dev: int, n: int, est_dev: int, stream: int):
    _check("cmp_mlp_combine", lib().cmp_mlp_combine(median_dev, y_dev, n, est_dev, stream))


def cmp_mlp_train_ws_bytes(nin: int, nh: int, n: int) -> int:
    return int(lib().cmp_mlp_train_ws_bytes(nin, nh, n))


def cmp_mlp_train_step(params_dev: int, m_dev: int, v_dev: int, nin: int, nh: int, skip: int, x_dev: int, y_dev: int,
                       n: int, huber_delta: float, lr: float, step: int, loss_dev: int, grad_dev: int, ws_dev: int,
                       ws_bytes: int, stream: int):
    _check("cmp_mlp_train_step",
           lib().cmp_mlp_train_step(params_dev, m_dev, v_dev, nin, nh, skip, x_dev, y_dev, n, C.c_float(huber_delta),
                                    C.c_float(lr), step, loss_dev, grad_dev, ws_dev, ws_bytes, stream))
