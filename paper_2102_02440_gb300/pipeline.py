"""Device-side orchestration over the C ABI: uploads a workload's columns, keeps the C
descriptors alive, and calls the cmp_* entry points in the order of the hot path
(build -> presort -> estimate -> optional learned combiner).  Marshalling only: every
step of the path runs in libcompass kernels."""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import compass as K


def _dev(a, device) -> torch.Tensor:
    if isinstance(a, torch.Tensor):
        return a.to(device).contiguous()
    return torch.from_numpy(np.ascontiguousarray(a)).to(device)


class DeviceTable:
    """One table's device columns, bitmaps, outputs and its cmp_table descriptor."""

    def __init__(self, t, d: int, w: int, device, upload: bool = True, cols_dev=None, sample_seed: int = 0,
                 sample_rate: float = 0.0, hints: bool = True):
        self.name = t.name
        self.n_rows = t.n_rows
        self.k = len(t.key_col)
        self.cols = cols_dev if cols_dev is not None else [_dev(c, device) for c in t.cols]
        self.bitmaps = [(_dev(q.bitmap, device) if q.bitmap is not None else None) for q in t.preds]
        self.counters = torch.zeros((max(self.k, 1), d, w), dtype=torch.int32, device=device)
        ncols = len(self.cols)
        meta = list(getattr(t, "col_meta", None) or []) if hints else []
        meta += [None] * (ncols - len(meta))

        def col(c, m):
            dt = K.CMP_I32 if c.dtype == torch.int32 else K.CMP_I64
            if m is None:
                return K.cmp_col(c.data_ptr(), dt, 0, 0, 0)
            flags = K.CMP_COL_DOMAIN | (K.CMP_COL_UNIQUE if m[0] == "unique" else 0)
            return K.cmp_col(c.data_ptr(), dt, flags, int(m[1]), int(m[2]))
        self._cols = (K.cmp_col * max(ncols, 1))(*[col(c, m) for c, m in zip(self.cols, meta)])
        self._preds = (K.cmp_pred * max(len(t.preds), 1))(*[
            K.cmp_pred(q.col, q.op, int(q.lo), int(q.hi), bm.data_ptr() if bm is not None else None, int(q.nbits))
            for q, bm in zip(t.preds, self.bitmaps)])
        self._key = (C.c_int32 * max(self.k, 1))(*t.key_col)
        self._edge = (C.c_int32 * max(self.k, 1))(*t.edge_id)
        self.desc = K.cmp_table(self.n_rows, ncols, len(t.preds), self.k, 0, self._cols, self._preds, self._key,
                                self._edge, sample_seed, sample_rate)
        self.sample_rate = sample_rate
        self.key_col = list(t.key_col)
        self.edge_id = list(t.edge_id)


class DeviceWorkload:
    """A workload's tables on the device with their sketches.
    sample_rates: optional per-table row-sample rates (0 or 1 = every row; Sec. 2
      "Workflow"), table t sampled with seed sample_seed + t; the estimates scale back by
      the rates.
    hints: pass the tables' column metadata (unique keys, key domains) to the build; the
      sketches are the same either way, only the build's path changes.
    offline: tables without predicates whose sketches are built once by build_offline()
      and plugged into every query (Sec. 2 "Workflow"): build_batched() and presort() then
      cover only the other tables.  Counters, presort and cross-rank buffers hold the
      online tables first, so each of those steps stays one launch over a prefix."""

    def __init__(self, wl, device="cuda", hash_seed: int | None = None, cols_dev=None, sample_rates=None,
                 sample_seed: int = 0x5A3B1E, offline=None, hints: bool = True):
        self.wl = wl
        self.device = torch.device(device)
        self.d, self.w = wl.d, wl.w
        self.n_edges = wl.n_edges
        seed = wl.hash_seed if hash_seed is None else hash_seed
        self.hash_host = K.cmp_hash_params(seed, self.n_edges, self.d)
        hp = np.frombuffer(self.hash_host, dtype=np.uint64, count=max(self.n_edges * self.d, 1) * 6).copy()
        self.hash_u64 = hp[: self.n_edges * self.d * 6].reshape(self.n_edges, self.d, 6)
        self.hash_dev = torch.from_numpy(hp.view(np.int64)).to(self.device)
        self.sample_rates = [float(r) for r in sample_rates] if sample_rates is not None else None
        self.tables = [DeviceTable(t, self.d, self.w, self.device, cols_dev=cols_dev[i] if cols_dev else None,
                                   sample_seed=sample_seed + i,
                                   sample_rate=self.sample_rates[i] if self.sample_rates else 0.0, hints=hints)
                       for i, t in enumerate(wl.tables)]
        self.offline = sorted(set(int(t) for t in (offline or [])))
        for t in self.offline:
            if wl.tables[t].preds or (self.sample_rates and 0.0 < self.sample_rates[t] < 1.0):
                raise ValueError(f"table {t}: offline sketches serve tables without predicates or samples")
        n = len(self.tables)
        self.online = [t for t in range(n) if t not in self.offline]
        self.storage_order = self.online + self.offline
        # every table's counters as consecutive blocks of one buffer, online tables first
        # (tables without sketches keep their own): presort and cross ranks then take one
        # launch each for all online (or offline) tables
        total = sum(t.k for t in self.tables)
        self.counters_all = torch.zeros((max(total, 1), self.d, self.w), dtype=torch.int32, device=self.device)
        off = 0
        for i in self.storage_order:
            t = self.tables[i]
            if t.k:
                t.counters = self.counters_all[off:off + t.k]
                off += t.k
        self.survivors = torch.zeros(n, dtype=torch.int64, device=self.device)
        self.status = torch.zeros(1, dtype=torch.int32, device=self.device)
        self._plan = None
        self._plans = None
        self._offline_plans = None

    # --------------------------------------------------------------- build
    def build(self, cfg=None, stream=None):
        s = K.stream_handle(stream)
        for i, t in enumerate(self.tables):
            K.cmp_sketch_build(t.desc, self.d, self.w, self.hash_dev.data_ptr(), self.n_edges,
                               t.counters.data_ptr(), self.survivors.data_ptr() + 8 * i, self.status.data_ptr(), cfg,
                               s)

    @staticmethod
    def _runs(ids):
        """Maximal ranges [a, b) of consecutive table ids (one batched plan each: a plan's
        survivors are one array)."""
        runs = []
        for t in ids:
            if runs and runs[-1][1] == t:
                runs[-1][1] = t + 1
            else:
                runs.append([t, t + 1])
        return runs

    def _encode_runs(self, ids, cfg):
        plans = []
        for a, b in self._runs(ids):
            descs = [self.tables[t].desc for t in range(a, b)]
            nb, wb = K.cmp_build_plan_bytes(descs, self.d, self.w, cfg)
            host = np.zeros(nb, np.uint8)
            K.cmp_build_plan_encode(descs, self.d, self.w, self.n_edges,
                                    [self.tables[t].counters.data_ptr() for t in range(a, b)],
                                    self.survivors.data_ptr() + 8 * a, cfg, host.ctypes.data, nb)
            ws = getattr(self, "build_ws", None)
            if wb and (ws is None or ws.numel() < wb):
                self.build_ws = torch.empty(wb, dtype=torch.uint8, device=self.device)
            plans.append((host, torch.from_numpy(host).to(self.device), wb))
        return plans

    def _run_plans(self, plans, stream):
        for host, dev, wb in plans:
            ws = self.build_ws.data_ptr() if wb else 0
            K.cmp_sketch_build_batched(host.ctypes.data, dev.data_ptr(), self.hash_dev.data_ptr(), ws, wb,
                                       self.status.data_ptr(), K.stream_handle(stream))

    def encode_batched(self, cfg=None):
        """Batched build plans of the online tables (one per run of consecutive ids)."""
        self._plans = self._encode_runs(self.online, cfg)
        self._plan = self._plans[0] if len(self._plans) == 1 else None
        return sum(p[0].size for p in self._plans)

    def upload(self, host_cols, n_streams: int = 4, stream=None):
        """Copies every column from host memory (host_cols[t][c], ideally pinned, the shapes and
        dtypes of the device columns) into the device columns the build reads, each column cut
        into n_streams contiguous parts copied on as many side streams (the copy engines run
        them side by side); `stream` (default: the current one) waits for all of them."""
        main = stream if stream is not None else torch.cuda.current_stream(self.device)
        if getattr(self, "_up_streams", None) is None or len(self._up_streams) != n_streams:
            self._up_streams = [torch.cuda.Stream(self.device) for _ in range(n_streams)]
            self._up_events = [torch.cuda.Event() for _ in range(n_streams)]
        start = torch.cuda.Event()
        start.record(main)
        for i, st in enumerate(self._up_streams):
            st.wait_event(start)
            with torch.cuda.stream(st):
                for hc, t in zip(host_cols, self.tables):
                    for h, dcol in zip(hc, t.cols):
                        n = dcol.numel()
                        a, b = n * i // n_streams, n * (i + 1) // n_streams
                        if b > a:
                            dcol[a:b].copy_(h[a:b], non_blocking=True)
            self._up_events[i].record(st)
        for ev in self._up_events:
            main.wait_event(ev)

    def build_batched(self, cfg=None, stream=None):
        if self._plans is None or (self._plan is None and len(self._plans) == 1):
            self.encode_batched(cfg)
        self._run_plans(self._plans, stream)

    def build_offline(self, cfg=None, stream=None):
        """Sketches, presort and cross ranks of the offline tables (once, outside any query)."""
        if not self.offline:
            return
        if self._offline_plans is None:
            self._offline_plans = self._encode_runs(self.offline, cfg)
        self._run_plans(self._offline_plans, stream)
        _prep_tables(self)
        _presort_tables(self, K.stream_handle(stream), offline=True)

    def check_status(self):
        st = int(self.status.item())
        if st != 0:
            raise K.CompassError("device status", st)

    def sketch(self, e: int, end: int) -> torch.Tensor:
        t, s = self.wl.sketch_of(e, end)
        return self.tables[t].counters[s]


def _prep_tables(dw):
    """Presort and cross-rank buffers for every table of a DeviceWorkload (once): one
    buffer each for all tables, in the storage order of the counters, with per-table views."""
    if getattr(dw, "ranks", None) is None:
        dev, d, w = dw.device, dw.d, dw.w
        order = getattr(dw, "storage_order", list(range(len(dw.tables))))
        ks = [dw.tables[i].k for i in order]
        total, rtotal = sum(ks), sum(k * k for k in ks)
        dw.abs_all = torch.empty((max(total, 1), d, w), dtype=torch.int32, device=dev)
        dw.perm_all = torch.empty((max(total, 1), d, w), dtype=torch.int32, device=dev)
        dw.ranks_all = torch.empty((max(rtotal, 1), d, w), dtype=torch.int32, device=dev)
        n = len(dw.tables)
        dw.abs_sorted, dw.perm, dw.ranks = [None] * n, [None] * n, [None] * n
        off = roff = 0
        for i, k in zip(order, ks):
            if k:
                dw.abs_sorted[i] = dw.abs_all[off:off + k]
                dw.perm[i] = dw.perm_all[off:off + k]
                dw.ranks[i] = dw.ranks_all[roff:roff + k * k].view(k, k, d, w)
                off += k
                roff += k * k
            else:  # no sketch: never referenced by a graph
                dw.abs_sorted[i] = dw.abs_all[:0]
                dw.perm[i] = dw.perm_all[:0]
                dw.ranks[i] = dw.ranks_all[:0]


def sorted_tables(n_tables: int, edge_u, edge_v, masks) -> set:
    """Tables whose sorted sketch rows (presort, cross ranks) an estimate plan over `masks`
    reads: the root of every multi-table sub-plan (its lowest table id) and every table
    joined to two or more others in one.  A table that is only ever a leaf is read through
    its counters alone, in its neighbour's sorted order."""
    need = set()
    for m in masks:
        m = int(m)
        if m & (m - 1) == 0:
            continue  # one table: its survivor count
        need.add((m & -m).bit_length() - 1)
        deg = [0] * n_tables
        for u, v in zip(edge_u, edge_v):
            if (m >> u) & 1 and (m >> v) & 1:
                deg[u] += 1
                deg[v] += 1
        need.update(t for t in range(n_tables) if deg[t] >= 2)
    return need


def presort_runs(dw, offline: bool = False, only=None) -> list:
    """The runs of tables that _presort_tables sorts with one launch pair each: [(row
    offset, rank offset, [tables])], tables consecutive in the buffers."""
    order = getattr(dw, "storage_order", list(range(len(dw.tables))))
    n_on = len(getattr(dw, "online", order))
    lo = sum(dw.tables[i].k for i in order[:n_on]) if offline else 0
    rlo = sum(dw.tables[i].k ** 2 for i in order[:n_on]) if offline else 0
    tabs = order[n_on:] if offline else order[:n_on]
    runs, cur = [], None  # [(row offset, rank offset, tables)]
    for i in tabs:
        if only is None or i in only:
            if cur is None:
                cur = (lo, rlo, [])
                runs.append(cur)
            cur[2].append(i)
        else:
            cur = None
        lo += dw.tables[i].k
        rlo += dw.tables[i].k ** 2
    return runs


def _presort_tables(dw, s, offline: bool = False, only=None):
    """cmp_presort of every sketch row of the online (or the offline) tables (of those in
    `only`, when given), then cmp_cross_ranks_multi: one launch each per run of tables
    consecutive in the buffers."""
    for lo, rlo, run in presort_runs(dw, offline, only):
        total = sum(dw.tables[i].k for i in run)
        if total == 0:
            continue
        need = K.cmp_presort_ws_bytes(total * dw.d, dw.w)
        ws = getattr(dw, "presort_ws", None)
        if need and (ws is None or ws.numel() < need):
            ws = dw.presort_ws = torch.empty(need, dtype=torch.uint8, device=dw.device)
        K.cmp_presort(dw.counters_all[lo:].data_ptr(), total * dw.d, dw.w, dw.abs_all[lo:].data_ptr(),
                      dw.perm_all[lo:].data_ptr(), ws.data_ptr() if need else 0, need, s)
        K.cmp_cross_ranks_multi(dw.abs_all[lo:].data_ptr(), dw.perm_all[lo:].data_ptr(),
                                [dw.tables[i].k for i in run], [e for i in run for e in dw.tables[i].edge_id], dw.d,
                                dw.w, dw.ranks_all[rlo:].data_ptr(), s)


def _graph_struct(dw, g_tables, g_eu, g_ev, sketch_of, survivors_ptr, keep, sample_rates=None):
    """cmp_graph over tables of `dw`; sketch_of(e, end) -> (table index in dw, sketch index)."""
    ne = len(g_eu)
    eu = (C.c_int32 * max(ne, 1))(*g_eu)
    ev = (C.c_int32 * max(ne, 1))(*g_ev)
    sk, ab, pm, rk, sl = [], [], [], [], []
    for e in range(ne):
        for end in range(2):
            ti, si = sketch_of(e, end)
            sk.append(dw.tables[ti].counters[si].data_ptr())
            ab.append(dw.abs_sorted[ti][si].data_ptr())
            pm.append(dw.perm[ti][si].data_ptr())
            rk.append(dw.ranks[ti][si].data_ptr())
            sl.append(si)
    n2 = max(2 * ne, 1)
    arrs = [(C.c_void_p * n2)(*sk), (C.c_void_p * n2)(*ab), (C.c_void_p * n2)(*pm), (C.c_void_p * n2)(*rk),
            (C.c_int32 * n2)(*sl)]
    rates = (C.c_double * max(g_tables, 1))(*sample_rates) if sample_rates is not None else None
    keep += [eu, ev, rates] + arrs
    return K.cmp_graph(g_tables, ne, eu, ev, arrs[0], arrs[1], arrs[2], arrs[3], arrs[4], survivors_ptr, rates)


class DeviceEstimator:
    """Presorted sketches of a built DeviceWorkload plus an encoded estimate plan for a
    list of sub-plans (bit t = table t), replayable with one cmp_estimate call."""

    def __init__(self, dws, masks, graph_of=None, cfg=None):
        dws = dws if isinstance(dws, (list, tuple)) else [dws]
        self.dws = dws
        self.d, self.w = dws[0].d, dws[0].w
        self.device = dws[0].device
        self.graphs = []
        self._keep = []
        for dw in dws:
            _prep_tables(dw)
            self.graphs.append(_graph_struct(dw, len(dw.tables), dw.wl.edge_u, dw.wl.edge_v, dw.wl.sketch_of,
                                             dw.survivors.data_ptr(), self._keep, dw.sample_rates))
        self.masks = np.ascontiguousarray(masks, np.uint64)
        self.sub_graph = np.zeros(self.masks.size, np.int32) if graph_of is None else np.ascontiguousarray(graph_of,
                                                                                                          np.int32)
        pb, wb = K.cmp_estimate_plan_bytes(self.graphs, self.d, self.w, self.sub_graph, self.masks, cfg)
        self.plan_host = np.zeros(max(pb, 16), np.uint8)
        K.cmp_estimate_plan_encode(self.graphs, self.d, self.w, self.sub_graph, self.masks,
                                   self.plan_host.ctypes.data, pb, cfg)
        self.plan_dev = torch.from_numpy(self.plan_host).to(self.device)
        self.ws = torch.empty(max(wb, 16), dtype=torch.uint8, device=self.device)
        self.est = torch.empty(self.masks.size, dtype=torch.float64, device=self.device)
        self.row_est = torch.empty((self.masks.size, self.d, 2), dtype=torch.int64, device=self.device)

    def presort(self, stream=None):
        """Presort and cross ranks of the tables this plan reads sorted (sorted_tables)."""
        s = K.stream_handle(stream)
        for g, dw in enumerate(self.dws):
            _presort_tables(dw, s, only=self.sorted_tables(g))

    def sorted_tables(self, g: int = 0) -> set:
        dw = self.dws[g]
        return sorted_tables(len(dw.tables), dw.wl.edge_u, dw.wl.edge_v, self.masks[self.sub_graph == g])

    def estimate(self, stream=None, row_est=True):
        status = self.dws[0].status
        K.cmp_estimate(self.plan_host.ctypes.data, self.plan_dev.data_ptr(), self.ws.data_ptr(), self.ws.numel(),
                       self.est.data_ptr(), self.row_est.data_ptr() if row_est else 0, status.data_ptr(),
                       K.stream_handle(stream))

    def row_values(self):
        """Exact row estimates as Python ints, [n_sub][d]."""
        r = self.row_est.cpu().numpy()
        lo = r[..., 0].astype(np.uint64).astype(object)
        hi = r[..., 1].astype(object)
        return (hi * (1 << 64) + lo).tolist()

    def estimate_wide(self, stream=None):
        """cmp_estimate_ex: the estimate with every row also as a 1024-bit integer (the rows
        of sub-plans beyond int128 from the exact tier)."""
        if getattr(self, "wide_rows", None) is None:
            self.wide_rows = torch.empty((self.masks.size, self.d, 16), dtype=torch.int64, device=self.device)
        status = self.dws[0].status
        K.cmp_estimate_ex(self.plan_host.ctypes.data, self.plan_dev.data_ptr(), self.ws.data_ptr(), self.ws.numel(),
                          self.est.data_ptr(), self.row_est.data_ptr(), self.wide_rows.data_ptr(), status.data_ptr(),
                          K.stream_handle(stream))

    def wide_values(self):
        """The rows of the last estimate_wide as Python ints, [n_sub][d]."""
        r = self.wide_rows.cpu().numpy().astype(np.uint64)
        out = []
        for q in range(r.shape[0]):
            rows = []
            for i in range(r.shape[1]):
                v = 0
                for l in range(15, -1, -1):
                    v = (v << 64) | int(r[q, i, l])
                rows.append(v - (1 << 1024) if v >> 1023 else v)
            out.append(rows)
        return out


class Enumerator:
    """Algorithm 1 (join-order enumeration) over an estimate plan's sub-plans, for every
    graph of the plan in one launch: run(est) reads the estimates where cmp_estimate wrote
    them.  graphs: cmp_graph structs (edges and survivors_dev are what it uses)."""

    def __init__(self, graphs, sub_graph, sub_mask, device="cuda", cfg=None):
        self.graphs = list(graphs)
        self.cfg = cfg
        self.device = torch.device(device)
        self.sub_graph = np.ascontiguousarray(sub_graph, np.int32)
        self.sub_mask = np.ascontiguousarray(sub_mask, np.uint64)
        pb, wb = K.cmp_enum_plan_bytes(self.graphs, self.sub_graph, self.sub_mask)
        self.plan_host = np.zeros(max(pb, 16), np.uint8)
        K.cmp_enum_plan_encode(self.graphs, self.sub_graph, self.sub_mask, self.plan_host.ctypes.data, pb)
        self.plan_dev = torch.from_numpy(self.plan_host).to(self.device)
        self.ws = torch.empty(max(wb, 16), dtype=torch.uint8, device=self.device)
        ng = len(self.graphs)
        self.order = torch.empty((ng, 64), dtype=torch.int32, device=self.device)
        self.cost = torch.empty(ng, dtype=torch.float64, device=self.device)
        self.stats = torch.empty((ng, 3), dtype=torch.int64, device=self.device)
        self.status = torch.zeros(1, dtype=torch.int32, device=self.device)

    def run(self, est, stream=None):
        K.cmp_enumerate(self.plan_host.ctypes.data, self.plan_dev.data_ptr(), est.data_ptr(), self.cfg,
                        self.ws.data_ptr(), self.ws.numel(), self.order.data_ptr(), self.cost.data_ptr(),
                        self.stats.data_ptr(), self.status.data_ptr(), K.stream_handle(stream))

    def plans(self):
        """[(order tuple, cost, (plans, extensions, pruned))] per graph, on the host."""
        o, c, st = self.order.cpu().numpy(), self.cost.cpu().numpy(), self.stats.cpu().numpy()
        return [(tuple(int(x) for x in o[g] if x >= 0), float(c[g]), tuple(int(x) for x in st[g]))
                for g in range(len(self.graphs))]


class PartitionedJoin:
    """Partitioned sketches (Sec. 4.1) of one tree-shaped join of a workload on the device:
    each listed table gets one tensor over its edges of the join (cmp_part_build, hashed with
    the workload's per-edge parameters), and estimate() contracts them (cmp_part_estimate).
    tables: workload table indices, the first is the contraction's root; edges: workload edge
    ids forming a spanning tree of those tables; widths: buckets per listed edge.  A table's
    axes follow the order of its sketches in the workload.  cols_dev: optional uploaded
    columns per listed table (e.g. a DeviceWorkload's)."""

    def __init__(self, wl, tables, edges, widths, device="cuda", cols_dev=None, cfg=None, hash_dev=None,
                 sample_rates=None, sample_seed: int = 0x5A3B1E):
        from . import datagen as G
        self.wl = wl
        self.device = torch.device(device)
        self.d = wl.d
        self.cfg = cfg
        self.table_ids = list(tables)
        self.edge_ids = list(edges)
        self.widths = [int(x) for x in widths]
        if hash_dev is None:
            hp = K.hash_params_u64(wl.hash_seed, wl.n_edges, self.d)
            hash_dev = torch.from_numpy(np.ascontiguousarray(hp).reshape(-1).view(np.int64)).to(self.device)
        self.hash_dev = hash_dev
        pos = {t: i for i, t in enumerate(self.table_ids)}
        local = {e: i for i, e in enumerate(self.edge_ids)}
        eu = [pos[wl.edge_u[e]] for e in self.edge_ids]
        ev = [pos[wl.edge_v[e]] for e in self.edge_ids]
        self.tables, self.tensors, self.axes = [], [], []
        for i, t in enumerate(self.table_ids):
            src = wl.tables[t]
            sel = [s for s, e in enumerate(src.edge_id) if e in local]
            tt = G.Table(src.name, src.cols, src.preds, [src.key_col[s] for s in sel], [src.edge_id[s] for s in sel])
            self.tables.append(DeviceTable(tt, self.d, 1, self.device, cols_dev=cols_dev[i] if cols_dev else None,
                                           sample_seed=sample_seed + t,
                                           sample_rate=float(sample_rates[i]) if sample_rates is not None else 0.0))
            ax = [local[src.edge_id[s]] for s in sel]
            self.axes.append(ax)
            size = int(np.prod([self.widths[a] for a in ax])) if ax else 1
            self.tensors.append(torch.zeros((self.d, size), dtype=torch.int32, device=self.device))
        self.survivors = torch.zeros(len(self.tables), dtype=torch.int64, device=self.device)
        self.join, self._keep = K.part_join(eu, ev, self.widths, self.axes, [x.data_ptr() for x in self.tensors],
                                            sample_rates)
        nb = K.cmp_part_estimate_ws_bytes(self.join, self.d)
        self.ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=self.device)
        self.est = torch.empty(1, dtype=torch.float64, device=self.device)
        self.row_est = torch.empty((self.d, 2), dtype=torch.int64, device=self.device)
        self.status = torch.zeros(1, dtype=torch.int32, device=self.device)

    def table_widths(self, i: int) -> list:
        return [self.widths[a] for a in self.axes[i]]

    def build(self, stream=None):
        s = K.stream_handle(stream)
        for i, t in enumerate(self.tables):
            K.cmp_part_build(t.desc, self.d, self.table_widths(i), self.hash_dev.data_ptr(), self.wl.n_edges,
                             self.tensors[i].data_ptr(), self.survivors.data_ptr() + 8 * i, self.cfg, s)

    def estimate(self, stream=None, row_est=True):
        K.cmp_part_estimate(self.join, self.d, self.ws.data_ptr(), self.ws.numel(), self.est.data_ptr(),
                            self.row_est.data_ptr() if row_est else 0, self.status.data_ptr(),
                            K.stream_handle(stream))

    def row_values(self):
        r = self.row_est.cpu().numpy()
        lo = r[:, 0].astype(np.uint64).astype(object)
        hi = r[:, 1].astype(object)
        return (hi * (1 << 64) + lo).tolist()


class PairBatch:
    """N independent two-table joins R_i |x| S_i on a key: every sketch built in one
    batched launch, all N two-way estimates in one plan (one graph per pair), and the
    learned combiner's features over them."""

    def __init__(self, pairs, d: int, w: int, hash_seed: int, device="cuda", cfg=None, device_keys=None, offsets=None):
        """pairs: list of (keys_R, keys_S) host arrays; or device_keys (one int32 device
        tensor) with offsets (table t = device_keys[offsets[t]:offsets[t+1]], tables 2i
        and 2i+1 forming pair i)."""
        from . import datagen as G
        tables, eu, ev, cols_dev = [], [], [], None
        if device_keys is not None:
            n_pairs = (len(offsets) - 1) // 2
            cols_dev = []
            for t in range(2 * n_pairs):
                n = int(offsets[t + 1] - offsets[t])
                shape_only = np.lib.stride_tricks.as_strided(np.zeros(1, np.int32), shape=(n,), strides=(0,))
                tables.append(G.Table(f"T{t}", [shape_only], [], [0], [t // 2]))
                cols_dev.append([device_keys[int(offsets[t]):int(offsets[t + 1])]])
        else:
            n_pairs = len(pairs)
            for i, (a, b) in enumerate(pairs):
                tables += [G.Table(f"R{i}", [a], [], [0], [i]), G.Table(f"S{i}", [b], [], [0], [i])]
        for i in range(n_pairs):
            eu.append(2 * i)
            ev.append(2 * i + 1)
        self.n = n_pairs
        self.d, self.w = d, w
        self.dw = DeviceWorkload(G.Workload("pairs", tables, eu, ev, d, w, hash_seed, 0), device=device,
                                 cols_dev=cols_dev)
        self.device = self.dw.device
        self.cfg = cfg
        # the tables' counters are consecutive [d][w] blocks: presort and self-join sizes
        # take one launch each
        self.counters = self.dw.counters_all

    def build(self, stream=None):
        self.dw.build_batched(self.cfg, stream)

    def prepare_estimate(self):
        dw, d, w = self.dw, self.d, self.w
        self.abs = torch.empty((2 * self.n, d, w), dtype=torch.int32, device=self.device)
        self.perm = torch.empty_like(self.abs)
        self.ranks = torch.empty_like(self.abs)   # one sketch per table: the inverse permutations
        dw.abs_sorted = [self.abs[i:i + 1] for i in range(2 * self.n)]
        dw.perm = [self.perm[i:i + 1] for i in range(2 * self.n)]
        dw.ranks = [self.ranks[i:i + 1].unsqueeze(0) for i in range(2 * self.n)]
        self.graphs, self._keep = [], []
        for i in range(self.n):
            self.graphs.append(_graph_struct(dw, 2, [0], [1], lambda e, end, i=i: (2 * i + end, 0),
                                             dw.survivors.data_ptr() + 16 * i, self._keep))
        sub_graph = np.arange(self.n, dtype=np.int32)
        masks = np.full(self.n, 0b11, np.uint64)
        pb, wb = K.cmp_estimate_plan_bytes(self.graphs, d, w, sub_graph, masks)
        self.plan_host = np.zeros(max(pb, 16), np.uint8)
        K.cmp_estimate_plan_encode(self.graphs, d, w, sub_graph, masks, self.plan_host.ctypes.data, pb)
        self.plan_dev = torch.from_numpy(self.plan_host).to(self.device)
        self.ws = torch.empty(max(wb, 16), dtype=torch.uint8, device=self.device)
        self.est = torch.empty(self.n, dtype=torch.float64, device=self.device)
        self.row_est = torch.empty((self.n, d, 2), dtype=torch.int64, device=self.device)
        self.f2 = torch.empty(2 * self.n, dtype=torch.float64, device=self.device)
        self.feat = torch.empty((self.n, d + 2), dtype=torch.float32, device=self.device)

    def estimate(self, stream=None):
        s = K.stream_handle(stream)
        need = K.cmp_presort_ws_bytes(2 * self.n * self.d, self.w)   # rows longer than 16384: merged in memory
        if need and (getattr(self, "presort_ws", None) is None or self.presort_ws.numel() < need):
            self.presort_ws = torch.empty(need, dtype=torch.uint8, device=self.device)
        K.cmp_presort(self.counters.data_ptr(), 2 * self.n * self.d, self.w, self.abs.data_ptr(), self.perm.data_ptr(),
                      self.presort_ws.data_ptr() if need else 0, need, s)
        # k = 1 per table: the cross ranks are the inverse permutations, one call for all tables
        K.cmp_cross_ranks(self.abs.data_ptr(), self.perm.data_ptr(), 1, 2 * self.n * self.d, self.w, [0],
                          self.ranks.data_ptr(), s)
        K.cmp_estimate(self.plan_host.ctypes.data, self.plan_dev.data_ptr(), self.ws.data_ptr(), self.ws.numel(),
                       self.est.data_ptr(), self.row_est.data_ptr(), self.dw.status.data_ptr(), s)

    def features(self, stream=None):
        s = K.stream_handle(stream)
        K.cmp_sketch_f2(self.counters.data_ptr(), 2 * self.n, self.d, self.w, self.f2.data_ptr(), s)
        f2 = self.f2.view(self.n, 2)
        self.f2a = f2[:, 0].contiguous()
        self.f2b = f2[:, 1].contiguous()
        K.cmp_mlp_features(self.row_est.data_ptr(), self.n, self.d, self.f2a.data_ptr(), self.f2b.data_ptr(),
                           self.feat.data_ptr(), s)
        return self.feat


def build_plan_info(dw) -> dict:
    """Totals of cmp_build_plan_stats over a DeviceWorkload's encoded batched-build plans."""
    out = {"launches": 0, "n_agg": 0, "n_unique_slabs": 0, "n_presence": 0}
    for host, _dev, _wb in (dw._plans or []):
        info = K.cmp_build_plan_stats(host.ctypes.data)
        out["launches"] += int(info.launches)
        out["n_agg"] += int(info.n_agg)
        out["n_unique_slabs"] += int(info.n_unique_slabs)
        out["n_presence"] += int(info.n_presence)
    return out


CHECKPOINT_DIR = __import__("os").path.join(__import__("os").path.dirname(__import__("os").path.abspath(__file__)),
                                            "checkpoints")


class Combiner:
    """The learned combiner's parameters and Adam state on the device."""

    @classmethod
    def for_sketches(cls, d: int, w: int, device="cuda"):
        """The trained combiner for d-row sketches (checkpoints/combiner_d{d}.bin, written
        by Combiner.save after training on the GPU on w-bucket sketches), else an untrained
        one with seed-0 weights.  Returns (combiner, description)."""
        import os
        path = os.path.join(CHECKPOINT_DIR, f"combiner_d{d}.bin")
        if os.path.exists(path):
            c, hdr = cls.load(path, device=device)
            if int(hdr.get("w", w)) == w:
                return c, {"weights": f"checkpoints/combiner_d{d}.bin", **hdr}
        return cls(d + 2, 64, seed=0, device=device, skip=d // 2), {"weights": "untrained (seed 0)"}

    def __init__(self, nin: int, nh: int = 64, seed: int = 0, device="cuda", skip: int = -1, init_scale: float = 1.0):
        self.nin, self.nh, self.skip = nin, nh, skip
        npar = K.cmp_mlp_param_count(nin, nh)
        rng = np.random.default_rng(seed)
        p = np.zeros(npar, np.float32)
        p[: nh * nin] = rng.standard_normal(nh * nin) * np.sqrt(2.0 / nin)
        p[nh * nin + nh: nh * nin + 2 * nh] = rng.standard_normal(nh) * np.sqrt(1.0 / nh) * init_scale
        self.params = torch.from_numpy(p).to(device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = 0
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.grad = torch.zeros_like(self.params)
        self._ws = None

    _MAGIC = b"CMPMLP1\0"

    def save(self, path: str, meta: dict | None = None, seed: int = 0):
        """Checkpoint: magic, int32 nin, nh, skip, step, int64 seed, parameter count, uint32
        length of a JSON description, the JSON, then fp32 parameters, Adam m and Adam v."""
        import json
        import struct
        js = json.dumps(meta or {}, sort_keys=True).encode()
        p, m, v = (t.detach().cpu().numpy().astype(np.float32) for t in (self.params, self.m, self.v))
        with open(path, "wb") as f:
            f.write(self._MAGIC)
            f.write(struct.pack("<iiiiqqI", self.nin, self.nh, self.skip, self.step, seed, p.size, len(js)))
            f.write(js)
            for a in (p, m, v):
                f.write(a.tobytes())

    @classmethod
    def load(cls, path: str, device="cuda"):
        import json
        import struct
        with open(path, "rb") as f:
            if f.read(8) != cls._MAGIC:
                raise ValueError(f"{path}: not a combiner checkpoint")
            nin, nh, skip, step, seed, n, jl = struct.unpack("<iiiiqqI", f.read(36))
            meta = json.loads(f.read(jl).decode())
            arrs = [np.frombuffer(f.read(4 * n), np.float32).copy() for _ in range(3)]
        if n != K.cmp_mlp_param_count(nin, nh):
            raise ValueError(f"{path}: {n} parameters for a {nin}->{nh}->1 network")
        c = cls(nin, nh, seed=seed, device=device, skip=skip)
        c.params.copy_(torch.from_numpy(arrs[0]))
        c.m.copy_(torch.from_numpy(arrs[1]))
        c.v.copy_(torch.from_numpy(arrs[2]))
        c.step = step
        return c, {"nin": nin, "nh": nh, "skip": skip, "step": step, **meta}

    def train_step(self, x: torch.Tensor, t: torch.Tensor, lr: float, huber_delta: float = 0.0, stream=None):
        n = x.shape[0]
        need = K.cmp_mlp_train_ws_bytes(self.nin, self.nh, n)
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(max(need, 16), dtype=torch.uint8, device=x.device)
        self.step += 1
        K.cmp_mlp_train_step(self.params.data_ptr(), self.m.data_ptr(), self.v.data_ptr(), self.nin, self.nh, self.skip,
                             x.data_ptr(), t.data_ptr(), n, huber_delta, lr, self.step, self.loss.data_ptr(), self.grad.data_ptr(),
                             self._ws.data_ptr(), self._ws.numel(), K.stream_handle(stream))

    def combine(self, median: torch.Tensor, y: torch.Tensor, stream=None) -> torch.Tensor:
        out = torch.empty_like(median)
        K.cmp_mlp_combine(median.data_ptr(), y.data_ptr(), median.numel(), out.data_ptr(), K.stream_handle(stream))
        return out

    def infer(self, x: torch.Tensor, stream=None) -> torch.Tensor:
        y = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        K.cmp_mlp_infer(self.params.data_ptr(), self.nin, self.nh, self.skip, x.data_ptr(), x.shape[0], y.data_ptr(),
                        K.stream_handle(stream))
        return y


class GraphBatch:
    """Many join graphs handled together: every table of every graph in one batched build
    (edges renumbered globally, one hash-parameter array), and the estimates of any set of
    (graph, sub-plan) pairs in one plan."""

    def __init__(self, graphs, device="cuda", hash_seed: int = 0xC0FFEE + 2):
        from . import datagen as G
        self.graphs = graphs
        self.d, self.w = graphs[0].d, graphs[0].w
        tables, eu, ev = [], [], []
        self.table_off, self.edge_off = [], []
        for g in graphs:
            assert g.d == self.d and g.w == self.w
            toff, eoff = len(tables), len(eu)
            self.table_off.append(toff)
            self.edge_off.append(eoff)
            for t in g.tables:
                tables.append(G.Table(t.name, t.cols, t.preds, t.key_col, [e + eoff for e in t.edge_id],
                                      list(getattr(t, "col_meta", None) or [])))
            eu += [u + toff for u in g.edge_u]
            ev += [v + toff for v in g.edge_v]
        self.wl = G.Workload("graph batch", tables, eu, ev, self.d, self.w, hash_seed, 0)
        self.dw = DeviceWorkload(self.wl, device=device)
        self.device = self.dw.device
        self.total_rows = self.wl.total_rows

    def build_batched(self, cfg=None, stream=None):
        self.dw.build_batched(cfg, stream)

    def build_per_table(self, cfg=None, stream=None):
        self.dw.build(cfg, stream)

    def graph_structs(self):
        """cmp_graph per graph over the batch's device sketches (presort arrays allocated)."""
        dw = self.dw
        if not hasattr(self, "_graphs"):
            _prep_tables(dw)
            self._graphs, self._keep = [], []
            for gi, g in enumerate(self.graphs):
                toff, eoff = self.table_off[gi], self.edge_off[gi]
                self._graphs.append(_graph_struct(dw, len(g.tables), g.edge_u, g.edge_v,
                                                  lambda e, end, eoff=eoff: self.wl.sketch_of(e + eoff, end),
                                                  dw.survivors.data_ptr() + 8 * toff, self._keep))
        return self._graphs

    def presort(self, stream=None):
        s = K.stream_handle(stream)
        self.graph_structs()
        _presort_tables(self.dw, s)

    def plan(self, sub_graph, sub_mask, cfg=None):
        """An encoded estimate plan (host blob, device copy, workspace, outputs)."""
        graphs = self.graph_structs()
        sg = np.ascontiguousarray(sub_graph, np.int32)
        sm = np.ascontiguousarray(sub_mask, np.uint64)
        pb, wb = K.cmp_estimate_plan_bytes(graphs, self.d, self.w, sg, sm, cfg)
        host = np.zeros(max(pb, 16), np.uint8)
        K.cmp_estimate_plan_encode(graphs, self.d, self.w, sg, sm, host.ctypes.data, pb, cfg)
        return EstimatePlan(host, self.device, wb, sm.size, self.d, self.dw.status)


class EstimatePlan:
    def __init__(self, host, device, ws_bytes, n_sub, d, status):
        self.host = host
        self.dev = torch.from_numpy(host).to(device)
        self.ws = torch.empty(max(ws_bytes, 16), dtype=torch.uint8, device=device)
        self.est = torch.empty(n_sub, dtype=torch.float64, device=device)
        self.row_est = torch.empty((n_sub, d, 2), dtype=torch.int64, device=device)
        self.status = status

    def run(self, stream=None, row_est=True):
        K.cmp_estimate(self.host.ctypes.data, self.dev.data_ptr(), self.ws.data_ptr(), self.ws.numel(),
                       self.est.data_ptr(), self.row_est.data_ptr() if row_est else 0, self.status.data_ptr(),
                       K.stream_handle(stream))
