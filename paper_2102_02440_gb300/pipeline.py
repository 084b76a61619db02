"""Device-side orchestration over the C ABI: uploads a workload's columns, keeps the C
descriptors alive, and calls the cmp_* entry points in the order of the hot path
(build -> presort -> estimate -> optional learned combiner).  Marshalling only: every
step of the path runs in libcompass kernels."""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import compass as K


def _dev(a: np.ndarray, device) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).to(device)


class DeviceTable:
    """One table's device columns, bitmaps, outputs and its cmp_table descriptor."""

    def __init__(self, t, d: int, w: int, device, upload: bool = True, cols_dev=None):
        self.name = t.name
        self.n_rows = t.n_rows
        self.k = len(t.key_col)
        self.cols = cols_dev if cols_dev is not None else [_dev(c, device) for c in t.cols]
        self.bitmaps = [(_dev(q.bitmap, device) if q.bitmap is not None else None) for q in t.preds]
        self.counters = torch.zeros((max(self.k, 1), d, w), dtype=torch.int32, device=device)
        ncols = len(self.cols)
        self._cols = (K.cmp_col * max(ncols, 1))(*[
            K.cmp_col(c.data_ptr(), K.CMP_I32 if c.dtype == torch.int32 else K.CMP_I64, 0) for c in self.cols])
        self._preds = (K.cmp_pred * max(len(t.preds), 1))(*[
            K.cmp_pred(q.col, q.op, int(q.lo), int(q.hi), bm.data_ptr() if bm is not None else None, int(q.nbits))
            for q, bm in zip(t.preds, self.bitmaps)])
        self._key = (C.c_int32 * max(self.k, 1))(*t.key_col)
        self._edge = (C.c_int32 * max(self.k, 1))(*t.edge_id)
        self.desc = K.cmp_table(self.n_rows, ncols, len(t.preds), self.k, 0, self._cols, self._preds, self._key,
                                self._edge)
        self.key_col = list(t.key_col)
        self.edge_id = list(t.edge_id)


class DeviceWorkload:
    def __init__(self, wl, device="cuda", hash_seed: int | None = None):
        self.wl = wl
        self.device = torch.device(device)
        self.d, self.w = wl.d, wl.w
        self.n_edges = wl.n_edges
        seed = wl.hash_seed if hash_seed is None else hash_seed
        self.hash_host = K.cmp_hash_params(seed, self.n_edges, self.d)
        hp = np.frombuffer(self.hash_host, dtype=np.uint64, count=max(self.n_edges * self.d, 1) * 6).copy()
        self.hash_u64 = hp[: self.n_edges * self.d * 6].reshape(self.n_edges, self.d, 6)
        self.hash_dev = torch.from_numpy(hp.view(np.int64)).to(self.device)
        self.tables = [DeviceTable(t, self.d, self.w, self.device) for t in wl.tables]
        self.survivors = torch.zeros(len(self.tables), dtype=torch.int64, device=self.device)
        self.status = torch.zeros(1, dtype=torch.int32, device=self.device)
        self._plan = None

    # --------------------------------------------------------------- build
    def build(self, cfg=None, stream=None):
        s = K.stream_handle(stream)
        for i, t in enumerate(self.tables):
            K.cmp_sketch_build(t.desc, self.d, self.w, self.hash_dev.data_ptr(), self.n_edges,
                               t.counters.data_ptr(), self.survivors.data_ptr() + 8 * i, self.status.data_ptr(), cfg,
                               s)

    def encode_batched(self, cfg=None):
        descs = [t.desc for t in self.tables]
        nb = K.cmp_build_plan_bytes(descs, self.d, self.w, cfg)
        host = np.zeros(nb, np.uint8)
        K.cmp_build_plan_encode(descs, self.d, self.w, self.n_edges, [t.counters.data_ptr() for t in self.tables],
                                self.survivors.data_ptr(), cfg, host.ctypes.data, nb)
        self._plan = (host, torch.from_numpy(host).to(self.device))
        return nb

    def build_batched(self, cfg=None, stream=None):
        if self._plan is None:
            self.encode_batched(cfg)
        host, dev = self._plan
        K.cmp_sketch_build_batched(host.ctypes.data, dev.data_ptr(), self.hash_dev.data_ptr(), self.status.data_ptr(),
                                   K.stream_handle(stream))

    def check_status(self):
        st = int(self.status.item())
        if st != 0:
            raise K.CompassError("device status", st)

    def sketch(self, e: int, end: int) -> torch.Tensor:
        t, s = self.wl.sketch_of(e, end)
        return self.tables[t].counters[s]
