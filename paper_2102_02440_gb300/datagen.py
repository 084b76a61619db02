"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only draws data (columns, predicates, join graphs).  It contains none of
the method's arithmetic: no hashing, no sketch update, no estimate.  Both the CUDA path
and the oracle are fed the arrays it returns.

Distributions follow the paper's workload shape (JOB over IMDB, which is not available
here): Zipf-skewed foreign keys, primary keys that are permutations of their domain,
dictionary-coded string columns with point / subset predicates, integer range
predicates with a chosen selectivity.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

RANGE, EQ, IN = 0, 1, 2
INT64_MIN = -(1 << 63)


@dataclass
class Pred:
    col: int
    op: int
    lo: int = 0
    hi: int = 0
    bitmap: np.ndarray | None = None   # uint32 words, bit v of the set
    nbits: int = 0


@dataclass
class Table:
    name: str
    cols: list                                     # numpy int32 / int64 columns, equal length
    preds: list = field(default_factory=list)      # conjunction
    key_col: list = field(default_factory=list)    # per sketch: column index of its join key
    edge_id: list = field(default_factory=list)    # per sketch: join-graph edge
    # per column: None, or what a catalog knows about it: ("unique", lo, hi) for a primary key
    # holding distinct values in [lo, hi), ("domain", lo, hi) for a foreign key in [lo, hi)
    col_meta: list = field(default_factory=list)

    @property
    def n_rows(self) -> int:
        return int(self.cols[0].shape[0]) if self.cols else 0


@dataclass
class Workload:
    name: str
    tables: list
    edge_u: list
    edge_v: list
    d: int
    w: int
    hash_seed: int
    data_seed: int
    note: str = ""

    @property
    def n_edges(self) -> int:
        return len(self.edge_u)

    @property
    def total_rows(self) -> int:
        return sum(t.n_rows for t in self.tables)

    def column_bytes(self) -> int:
        return sum(c.nbytes for t in self.tables for c in t.cols)

    def sketch_of(self, e: int, end: int):
        """(table index, sketch index) holding endpoint `end` (0 = edge_u side) of edge e."""
        t = self.edge_u[e] if end == 0 else self.edge_v[e]
        return t, self.tables[t].edge_id.index(e)


# ---------------------------------------------------------------- Zipf sampler

def _expm1_over(t):
    t = np.asarray(t, np.float64)
    out = np.ones_like(t)
    big = np.abs(t) > 1e-8
    out[big] = np.expm1(t[big]) / t[big]
    small = ~big
    out[small] = 1.0 + t[small] / 2.0 + t[small] ** 2 / 6.0
    return out


def _log1p_over(t):
    t = np.asarray(t, np.float64)
    out = np.ones_like(t)
    big = np.abs(t) > 1e-8
    out[big] = np.log1p(t[big]) / t[big]
    small = ~big
    out[small] = 1.0 - t[small] / 2.0 + t[small] ** 2 / 3.0
    return out


def zipf_ranks(rng: np.random.Generator, n: int, N: int, s: float, chunk: int = 1 << 23) -> np.ndarray:
    """n ranks in [1, N] with P(k) proportional to k^-s, s > 0.

    Rejection-inversion (Hoermann & Derflinger, ACM TOMACS 1996): with h(x) = x^-s and
    its antiderivative H, draw U uniformly on [H(1.5) - h(1), H(N + 1/2)], set
    X = H^-1(U), K = nearest integer to X, and accept K iff U >= H(K + 1/2) - h(K).
    Each integer k owns an interval of length exactly h(k), so accepted K follow the
    Zipf law exactly.
    """
    one_minus_s = 1.0 - s

    def H(x):
        lx = np.log(x)
        return lx * _expm1_over(lx * one_minus_s)

    def Hinv(y):
        return np.exp(y * _log1p_over(y * one_minus_s))

    lo = float(H(np.array([1.5]))[0] - 1.0)
    hi = float(H(np.array([N + 0.5]))[0])
    out = np.empty(n, np.int64)
    filled = 0
    while filled < n:
        m = min(chunk, n - filled)
        need = m
        buf = np.empty(0, np.int64)
        while need > 0:
            u = lo + rng.random(int(need * 1.15) + 64) * (hi - lo)
            x = Hinv(u)
            k = np.clip(np.floor(x + 0.5), 1, N)
            acc = u >= H(k + 0.5) - k ** (-s)
            kk = k[acc].astype(np.int64)[:need]
            buf = np.concatenate([buf, kk])
            need = m - buf.size
        out[filled:filled + m] = buf
        filled += m
    return out


def affine_perm(rng: np.random.Generator, D: int):
    """A seeded permutation of [0, D): v -> (A v + B) mod D with gcd(A, D) = 1."""
    while True:
        A = int(rng.integers(1, max(D, 2)))
        if np.gcd(A, D) == 1:
            break
    B = int(rng.integers(0, max(D, 1)))
    return A, B


def zipf_keys(rng, n: int, D: int, s: float, dtype=np.int32) -> np.ndarray:
    """Zipf(s) foreign keys over [0, D); hot keys scattered by a seeded permutation."""
    A, B = affine_perm(rng, D)
    r = zipf_ranks(rng, n, D, s) - 1
    return ((A * r + B) % D).astype(dtype)


def pk_column(rng, n: int, dtype=np.int32) -> np.ndarray:
    """A primary key: a seeded permutation of [0, n)."""
    return rng.permutation(n).astype(dtype)


def uniform_col(rng, n: int, lo: int, hi: int, dtype=np.int32) -> np.ndarray:
    return rng.integers(lo, hi, size=n, dtype=np.int64).astype(dtype)


def bitmap_of(values, nbits: int) -> np.ndarray:
    words = np.zeros((nbits + 31) // 32, np.uint32)
    for v in values:
        words[v >> 5] |= np.uint32(1 << (v & 31))
    return words


# ---------------------------------------------------------------- workloads

def two_way(n_r: int = 100_000, n_s: int = 1_000_000, domain: int = 100_000, s: float = 1.0, d: int = 5,
            w: int = 1024, cut: int = 300, data_seed: int = 20210204, hash_seed: int = 0xC0FFEE) -> Workload:
    """R(key, p) join S(key, p) on key; Zipf(s) keys over [0, domain); p uniform on
    [0, 1000) filtered by p < cut on both sides; one edge, d x w sketches."""
    rng = np.random.default_rng(data_seed)
    tabs = []
    for name, n in (("R", n_r), ("S", n_s)):
        key = zipf_keys(rng, n, domain, s)
        p = uniform_col(rng, n, 0, 1000)
        tabs.append(Table(name, [key, p], [Pred(1, RANGE, INT64_MIN, cut)], [0], [0]))
    return Workload(f"two_way R{n_r} S{n_s} d{d} w{w}", tabs, [0], [1], d, w, hash_seed, data_seed)


def five_table(scale: float = 1.0, d: int = 11, w: int = 4096, d1_sel_pct: int = 20, s: float = 1.1,
               data_seed: int = 20210205, hash_seed: int = 0xC0FFEE + 1) -> Workload:
    """The 5-table cyclic join graph shaped like the paper's running example
    (Sec. 1 query, Fig. 1): fact tables F1 (cast_info-like, 36M) and F2
    (movie_keyword-like, 4.5M), dimensions D1 (title-like, 2.5M), D2 (keyword-like,
    134k) and D3 (name-like, 4M).  Edges, in id order:
      e0 D2-F2 (keyword), e1 D1-F2 (movie), e2 D1-F1 (movie), e3 F1-F2 (movie),
      e4 D3-F1 (person);  F1-F2-D1 is the triangle.
    Predicates: D2 point on a dictionary code, D3 subset (IN, ~1% of codes), D1 range
    on a uniform [0,1000) column at d1_sel_pct percent; F1, F2 none."""
    rng = np.random.default_rng(data_seed)
    n_f1, n_f2, n_d1, n_d2, n_d3 = (max(int(round(x * scale)), 16)
                                    for x in (36_000_000, 4_500_000, 2_500_000, 134_000, 4_000_000))
    movie_dom, kw_dom, person_dom = n_d1, n_d2, n_d3
    # tables: 0 F1, 1 F2, 2 D1, 3 D2, 4 D3
    f1 = Table("F1", [zipf_keys(rng, n_f1, movie_dom, s), zipf_keys(rng, n_f1, person_dom, s)], [],
               [0, 0, 1], [2, 3, 4], [("domain", 0, movie_dom), ("domain", 0, person_dom)])
    f2 = Table("F2", [zipf_keys(rng, n_f2, kw_dom, s), zipf_keys(rng, n_f2, movie_dom, s)], [],
               [0, 1, 1], [0, 1, 3], [("domain", 0, kw_dom), ("domain", 0, movie_dom)])
    d1 = Table("D1", [pk_column(rng, n_d1), uniform_col(rng, n_d1, 0, 1000)],
               [Pred(1, RANGE, 0, 10 * d1_sel_pct)], [0, 0], [1, 2], [("unique", 0, n_d1), None])
    codes2 = zipf_keys(rng, n_d2, 10_000, 1.0)
    point = int(codes2[rng.integers(0, n_d2)])
    d2 = Table("D2", [pk_column(rng, n_d2), codes2], [Pred(1, EQ, point, 0)], [0], [0], [("unique", 0, n_d2), None])
    code_dom = 100_000
    codes3 = zipf_keys(rng, n_d3, code_dom, 0.8)
    subset = rng.choice(code_dom, size=code_dom // 100, replace=False)
    d3 = Table("D3", [pk_column(rng, n_d3), codes3], [Pred(1, IN, 0, 0, bitmap_of(subset, code_dom), code_dom)],
               [0], [4], [("unique", 0, n_d3), None])
    return Workload(f"five_table scale={scale} d{d} w{w} D1sel={d1_sel_pct}%", [f1, f2, d1, d2, d3],
                    [3, 2, 2, 0, 4], [1, 1, 0, 1, 0], d, w, hash_seed, data_seed)


def five_table_device(scale: float = 1.0, d: int = 11, w: int = 4096, d1_sel_pct: int = 20, s: float = 1.1,
                      data_seed: int = 20210205, hash_seed: int = 0xC0FFEE + 1, device="cuda") -> Workload:
    """five_table's recipe drawn on the device (columns are device tensors; same tables,
    sizes, key distributions, predicates and edges; another random stream)."""
    import torch
    rng = np.random.default_rng(data_seed)
    gen = torch.Generator(device=device)
    gen.manual_seed(data_seed)
    n_f1, n_f2, n_d1, n_d2, n_d3 = (max(int(round(x * scale)), 16)
                                    for x in (36_000_000, 4_500_000, 2_500_000, 134_000, 4_000_000))
    movie_dom, kw_dom, person_dom = n_d1, n_d2, n_d3
    i32 = torch.int32

    def pk(n):
        return torch.randperm(n, generator=gen, device=device, dtype=torch.int64).to(i32)

    f1 = Table("F1", [zipf_keys_device(gen, n_f1, movie_dom, s, i32), zipf_keys_device(gen, n_f1, person_dom, s, i32)],
               [], [0, 0, 1], [2, 3, 4], [("domain", 0, movie_dom), ("domain", 0, person_dom)])
    f2 = Table("F2", [zipf_keys_device(gen, n_f2, kw_dom, s, i32), zipf_keys_device(gen, n_f2, movie_dom, s, i32)],
               [], [0, 1, 1], [0, 1, 3], [("domain", 0, kw_dom), ("domain", 0, movie_dom)])
    d1 = Table("D1", [pk(n_d1), torch.randint(0, 1000, (n_d1,), generator=gen, device=device, dtype=i32)],
               [Pred(1, RANGE, 0, 10 * d1_sel_pct)], [0, 0], [1, 2], [("unique", 0, n_d1), None])
    codes2 = zipf_keys_device(gen, n_d2, 10_000, 1.0, i32)
    point = int(codes2[int(rng.integers(0, n_d2))].item())
    d2 = Table("D2", [pk(n_d2), codes2], [Pred(1, EQ, point, 0)], [0], [0], [("unique", 0, n_d2), None])
    code_dom = 100_000
    codes3 = zipf_keys_device(gen, n_d3, code_dom, 0.8, i32)
    subset = rng.choice(code_dom, size=code_dom // 100, replace=False)
    d3 = Table("D3", [pk(n_d3), codes3], [Pred(1, IN, 0, 0, bitmap_of(subset, code_dom), code_dom)],
               [0], [4], [("unique", 0, n_d3), None])
    return Workload(f"five_table scale={scale} d{d} w{w} D1sel={d1_sel_pct}%", [f1, f2, d1, d2, d3],
                    [3, 2, 2, 0, 4], [1, 1, 0, 1, 0], d, w, hash_seed, data_seed)


def random_graph_workload(rng: np.random.Generator, n_tables: int, extra_edges: int, rows_lo: int, rows_hi: int,
                          domain: int, d: int, w: int, s_range=(0.5, 1.5), int64_keys: bool = False,
                          pred_prob: float = 0.5, hash_seed: int = 1) -> Workload:
    """Small random connected join graph (a random tree plus `extra_edges` more, parallel
    edges allowed); one key column per (table, edge), optional predicates."""
    eu, ev = [], []
    for t in range(1, n_tables):
        u = int(rng.integers(0, t))
        eu.append(u)
        ev.append(t)
    for _ in range(extra_edges):
        a, b = rng.choice(n_tables, size=2, replace=False)
        eu.append(int(a))
        ev.append(int(b))
    tabs = []
    kdt = np.int64 if int64_keys else np.int32
    for t in range(n_tables):
        n = int(rng.integers(rows_lo, rows_hi + 1))
        cols, key_col, edge_id = [], [], []
        for e in range(len(eu)):
            if eu[e] == t or ev[e] == t:
                s = float(rng.uniform(*s_range))
                cols.append(zipf_keys(rng, n, domain, s, kdt))
                key_col.append(len(cols) - 1)
                edge_id.append(e)
        preds = []
        if rng.random() < pred_prob:
            cols.append(uniform_col(rng, n, 0, 1000))
            kind = int(rng.integers(0, 3))
            c = len(cols) - 1
            if kind == 0:
                preds.append(Pred(c, RANGE, int(rng.integers(0, 500)), int(rng.integers(500, 1001))))
            elif kind == 1:
                preds.append(Pred(c, EQ, int(rng.integers(0, 1000))))
            else:
                sub = rng.choice(1000, size=int(rng.integers(1, 400)), replace=False)
                preds.append(Pred(c, IN, 0, 0, bitmap_of(sub, 1000), 1000))
        tabs.append(Table(f"T{t}", cols, preds, key_col, edge_id))
    return Workload(f"random n{n_tables}+{extra_edges}", tabs, eu, ev, d, w, hash_seed, 0)


def connected_subplans(n_tables: int, edge_u, edge_v, min_size: int = 1) -> list:
    """Every connected induced sub-plan (bit t = table t), ascending mask order."""
    adj = [0] * n_tables
    for u, v in zip(edge_u, edge_v):
        adj[u] |= 1 << v
        adj[v] |= 1 << u
    out = []
    for mask in range(1, 1 << n_tables):
        if bin(mask).count("1") < min_size:
            continue
        start = mask & -mask
        seen = start
        frontier = start
        while frontier:
            nxt = 0
            m = frontier
            while m:
                b = m & -m
                nxt |= adj[b.bit_length() - 1]
                m ^= b
            nxt &= mask & ~seen
            seen |= nxt
            frontier = nxt
        if seen == mask:
            out.append(mask)
    return out


def join_pairs(n_pairs: int, rows_lo: int = 10_000, rows_hi: int = 10_000_000, dom_lo: int = 1_000,
               dom_hi: int = 1_000_000, s_lo: float = 0.5, s_hi: float = 1.5, seed: int = 20210208):
    """Independent two-table joins for the learned combiner: per pair, row counts
    log-uniform in [rows_lo, rows_hi], one domain log-uniform in [dom_lo, dom_hi], and
    each side's keys Zipf(s) with s uniform in [s_lo, s_hi] (own permutation of the
    domain), no predicates.  Returns a list of (keys_R, keys_S) int32 arrays."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_pairs):
        dom = int(np.exp(rng.uniform(np.log(dom_lo), np.log(dom_hi))))
        pair = []
        for _side in range(2):
            n = int(np.exp(rng.uniform(np.log(rows_lo), np.log(rows_hi))))
            pair.append(zipf_keys(rng, n, dom, float(rng.uniform(s_lo, s_hi))))
        out.append(tuple(pair))
    return out


def zipf_ranks_device(gen, s, N):
    """Device version of zipf_ranks with one (s, N) per element: s, N are float64 torch
    tensors of equal length on the generator's device; returns int64 ranks in [1, N].
    Same rejection-inversion as zipf_ranks, with rejected elements redrawn."""
    import torch

    one_minus_s = 1.0 - s

    def expm1_over(t):
        small = t.abs() <= 1e-8
        return torch.where(small, 1.0 + t / 2.0 + t * t / 6.0, torch.expm1(t) / torch.where(small, 1.0, t))

    def log1p_over(t):
        small = t.abs() <= 1e-8
        return torch.where(small, 1.0 - t / 2.0 + t * t / 3.0, torch.log1p(t) / torch.where(small, 1.0, t))

    def H(x, oms):
        lx = torch.log(x)
        return lx * expm1_over(lx * oms)

    def Hinv(y, oms):
        return torch.exp(y * log1p_over(y * oms))

    lo = H(torch.full_like(s, 1.5), one_minus_s) - 1.0
    hi = H(N + 0.5, one_minus_s)
    out = torch.zeros_like(s, dtype=torch.int64)
    todo = torch.arange(s.numel(), device=s.device)
    while todo.numel():
        ss, oms, l, h, NN = s[todo], one_minus_s[todo], lo[todo], hi[todo], N[todo]
        u = l + torch.rand(todo.numel(), dtype=torch.float64, device=s.device, generator=gen) * (h - l)
        k = torch.clamp(torch.floor(Hinv(u, oms) + 0.5), min=1.0)
        k = torch.minimum(k, NN)
        acc = u >= H(k + 0.5, oms) - torch.pow(k, -ss)
        out[todo[acc]] = k[acc].to(torch.int64)
        todo = todo[~acc]
    return out


def join_pairs_device(n_pairs: int, rows_lo: int, rows_hi: int, dom_lo: int = 1_000, dom_hi: int = 1_000_000,
                      s_lo: float = 0.5, s_hi: float = 1.5, seed: int = 20210208, device="cuda"):
    """join_pairs drawn on the device, all tables at once.  Returns (keys, offsets, meta):
    keys int32 [total] on the device, offsets int64 [2 n_pairs + 1] (table t is
    keys[offsets[t]:offsets[t+1]]; tables 2i and 2i+1 form pair i), meta = numpy arrays
    (rows, domain, s) per table."""
    import torch

    rng = np.random.default_rng(seed)
    dom = np.exp(rng.uniform(np.log(dom_lo), np.log(dom_hi), n_pairs)).astype(np.int64)
    rows = np.exp(rng.uniform(np.log(rows_lo), np.log(rows_hi), 2 * n_pairs)).astype(np.int64)
    sk = rng.uniform(s_lo, s_hi, 2 * n_pairs)
    dom_t = np.repeat(dom, 2)
    A = np.empty(2 * n_pairs, np.int64)
    B = np.empty(2 * n_pairs, np.int64)
    for t in range(2 * n_pairs):
        A[t], B[t] = affine_perm(rng, int(dom_t[t]))
    offsets = np.concatenate([[0], np.cumsum(rows)])
    table_of = torch.repeat_interleave(torch.arange(2 * n_pairs, device=device), torch.from_numpy(rows).to(device))
    s_el = torch.from_numpy(sk).to(device)[table_of]
    N_el = torch.from_numpy(dom_t.astype(np.float64)).to(device)[table_of]
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    r = zipf_ranks_device(gen, s_el, N_el) - 1
    A_el = torch.from_numpy(A).to(device)[table_of]
    B_el = torch.from_numpy(B).to(device)[table_of]
    D_el = torch.from_numpy(dom_t).to(device)[table_of]
    keys = ((A_el * r + B_el) % D_el).to(torch.int32)
    return keys, offsets, {"rows": rows, "domain": dom_t, "s": sk}


def graph_batch(n_graphs: int = 64, n_lo: int = 4, n_hi: int = 17, rows_lo: int = 10_000, rows_hi: int = 100_000_000,
                domain: int = 100_000, d: int = 11, w: int = 1024, pred_prob: float = 0.5, seed: int = 20210206,
                kinds=("chain", "star", "cycle"), hash_seed: int = 0xC0FFEE + 2) -> list:
    """Synthetic join graphs for batched enumeration: type uniform over `kinds`, n tables
    uniform in [n_lo, n_hi], rows log-uniform in [rows_lo, rows_hi].  Every (table, edge)
    has its own key column, Zipf(s) over [0, domain) with s uniform in [0.5, 1.5]; with
    probability pred_prob a table gets a predicate: EQ on a Zipf(1.0) code over 1000 codes,
    or a RANGE on a uniform [0, 1000) column with selectivity uniform in [1%, 50%].
    Returns one Workload per graph (edges: chain i-(i+1); star 0-i; cycle = chain + (n-1)-0)."""
    rng = np.random.default_rng(seed)
    out = []
    for gi in range(n_graphs):
        kind = kinds[int(rng.integers(0, len(kinds)))]
        n = int(rng.integers(n_lo, n_hi + 1))
        if kind == "chain":
            edges = [(i, i + 1) for i in range(n - 1)]
        elif kind == "star":
            edges = [(0, i) for i in range(1, n)]
        else:
            edges = [(i, i + 1) for i in range(n - 1)] + [(0, n - 1)]
        tabs = []
        for t in range(n):
            rows = int(np.exp(rng.uniform(np.log(rows_lo), np.log(rows_hi))))
            cols, kc, ei = [], [], []
            for e, (u, v) in enumerate(edges):
                if t in (u, v):
                    cols.append(zipf_keys(rng, rows, domain, float(rng.uniform(0.5, 1.5))))
                    kc.append(len(cols) - 1)
                    ei.append(e)
            preds = []
            if rng.random() < pred_prob:
                if rng.random() < 0.5:
                    codes = zipf_keys(rng, rows, 1000, 1.0)
                    cols.append(codes)
                    preds.append(Pred(len(cols) - 1, EQ, int(codes[int(rng.integers(0, rows))])))
                else:
                    cols.append(uniform_col(rng, rows, 0, 1000))
                    preds.append(Pred(len(cols) - 1, RANGE, 0, int(1000 * rng.uniform(0.01, 0.5))))
            tabs.append(Table(f"G{gi}T{t}", cols, preds, kc, ei))
        out.append(Workload(f"{kind}{n}", tabs, [u for u, _ in edges], [v for _, v in edges], d, w,
                            hash_seed + gi, seed))
    return out


def graph_batch_device(n_graphs: int = 64, n_lo: int = 4, n_hi: int = 17, rows_lo: int = 10_000,
                       rows_hi: int = 100_000_000, domain: int = 100_000, d: int = 11, w: int = 1024,
                       pred_prob: float = 0.5, seed: int = 20210207, kinds=("chain", "star", "cycle"),
                       hash_seed: int = 0xC0FFEE + 2, device="cuda", rows_scale: float = 1.0) -> list:
    """graph_batch's recipe drawn on the device (columns are device tensors): graph kinds,
    table sizes, Zipf exponents and predicates come from a host generator seeded with
    `seed`, the columns from a device generator with the same seed.  rows_scale multiplies
    every table's row count (at least rows_lo / 10), for runs that must fit a time or memory
    budget.  Key columns carry their domain [0, domain) as a catalog declaration."""
    import torch
    rng = np.random.default_rng(seed)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    out = []
    for gi in range(n_graphs):
        kind = kinds[int(rng.integers(0, len(kinds)))]
        n = int(rng.integers(n_lo, n_hi + 1))
        if kind == "chain":
            edges = [(i, i + 1) for i in range(n - 1)]
        elif kind == "star":
            edges = [(0, i) for i in range(1, n)]
        else:
            edges = [(i, i + 1) for i in range(n - 1)] + [(0, n - 1)]
        tabs = []
        for t in range(n):
            rows = int(np.exp(rng.uniform(np.log(rows_lo), np.log(rows_hi))))
            rows = max(int(rows * rows_scale), max(rows_lo // 10, 16))
            cols, kc, ei, meta = [], [], [], []
            for e, (u, v) in enumerate(edges):
                if t in (u, v):
                    cols.append(zipf_keys_device(gen, rows, domain, float(rng.uniform(0.5, 1.5)), dtype=torch.int32))
                    kc.append(len(cols) - 1)
                    ei.append(e)
                    meta.append(("domain", 0, domain))
            preds = []
            if rng.random() < pred_prob:
                if rng.random() < 0.5:
                    codes = zipf_keys_device(gen, rows, 1000, 1.0, dtype=torch.int32)
                    cols.append(codes)
                    meta.append(None)
                    preds.append(Pred(len(cols) - 1, EQ, int(codes[int(rng.integers(0, rows))].item())))
                else:
                    cols.append(torch.randint(0, 1000, (rows,), generator=gen, device=device, dtype=torch.int32))
                    meta.append(None)
                    preds.append(Pred(len(cols) - 1, RANGE, 0, int(1000 * rng.uniform(0.01, 0.5))))
            tabs.append(Table(f"G{gi}T{t}", cols, preds, kc, ei, meta))
        out.append(Workload(f"{kind}{n}", tabs, [u for u, _ in edges], [v for _, v in edges], d, w,
                            hash_seed + gi, seed))
    return out


def zipf_keys_device(gen, n: int, D: int, s: float, dtype=None, chunk: int = 1 << 26):
    """n Zipf(s) keys over [0, D) drawn on the generator's device (chunked), hot keys
    scattered by a seeded affine permutation; int64 unless dtype is given."""
    import torch
    dev = gen.device
    dtype = dtype or torch.int64
    lo = int(torch.randint(1, max(D, 2), (1,), generator=gen, device=dev).item())
    A = lo
    while np.gcd(A, D) != 1:
        A = A % (D - 1) + 1 if D > 2 else 1
    B = int(torch.randint(0, max(D, 1), (1,), generator=gen, device=dev).item())
    out = torch.empty(n, dtype=dtype, device=dev)
    for c0 in range(0, n, chunk):
        m = min(chunk, n - c0)
        s_t = torch.full((m,), float(s), dtype=torch.float64, device=dev)
        N_t = torch.full((m,), float(D), dtype=torch.float64, device=dev)
        r = zipf_ranks_device(gen, s_t, N_t) - 1
        out[c0:c0 + m] = ((A * r + B) % D).to(dtype)
    return out


def scale_workload_device(n_fact: int = 1_000_000_000, n_d1: int = 100_000_000, n_d2: int = 1_000_000,
                          d: int = 15, w: int = 65536, seed: int = 20210209, device="cuda",
                          hash_seed: int = 0xC0FFEE + 4) -> Workload:
    """The scale configuration, drawn on the device: fact F (n_fact rows) with fk1 int64
    Zipf(1.2) over [0, n_d1), fk2 int64 Zipf(1.2) over [0, n_d2), p1 and p2 int32 uniform
    on [0, 1000) filtered by p1 < 250 and p2 < 400 (10% combined); dimensions D1 (n_d1)
    and D2 (n_d2) with int64 primary keys that are permutations.  Edges e0 D1-F, e1 D2-F.
    Columns are device tensors."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    fk1 = zipf_keys_device(gen, n_fact, n_d1, 1.2)
    fk2 = zipf_keys_device(gen, n_fact, n_d2, 1.2)
    p1 = torch.randint(0, 1000, (n_fact,), generator=gen, device=device, dtype=torch.int32)
    p2 = torch.randint(0, 1000, (n_fact,), generator=gen, device=device, dtype=torch.int32)
    pk1 = torch.randperm(n_d1, generator=gen, device=device, dtype=torch.int64)
    pk2 = torch.randperm(n_d2, generator=gen, device=device, dtype=torch.int64)
    F = Table("F", [fk1, fk2, p1, p2], [Pred(2, RANGE, INT64_MIN, 250), Pred(3, RANGE, INT64_MIN, 400)], [0, 1],
              [0, 1], [("domain", 0, n_d1), ("domain", 0, n_d2), None, None])
    D1 = Table("D1", [pk1], [], [0], [0], [("unique", 0, n_d1)])
    D2 = Table("D2", [pk2], [], [0], [1], [("unique", 0, n_d2)])
    # tables: 0 F, 1 D1, 2 D2
    return Workload(f"scale F{n_fact} D1 {n_d1} D2 {n_d2} d{d} w{w}", [F, D1, D2], [1, 2], [0, 0], d, w,
                    hash_seed, seed)
