"""Oracle (test infrastructure only; the product path never imports it): partitioned
Fast-AGMS sketches (Sec. 4.1, sketch partitioning), written from the paper's description.

A table that takes part in a multi-way join through edges e_1..e_k gets, per sketch row i,
one k-dimensional tensor of w_{e_1} x ... x w_{e_k} int32 counters (axis l for edge e_l,
row-major: the last axis is contiguous).  Every tuple that satisfies the table's selection
adds the product of its signs xi_{e_l,i}(key_l) to the counter at (h_{e_l,i}(key_l))_l.
The bucket and sign functions are the per-(edge, row) ones of the 1-D sketches, with the
edge's width w_e, which both endpoint tables of the edge use; a one-axis partitioned sketch
is therefore the 1-D sketch, and a zero-axis one holds the selected count.

The estimate of the join of a set of tables whose edges form a tree is, per row, the full
contraction of their tensors (every edge's bucket index summed once over [0, w_e), shared
by the two endpoint tensors), and the estimate is the median over rows (Sec. 3.2).  For the
3-table chain this is the paper's double sum over i, j of sk_k[i] sk_part(mk)[i, j] sk_t[j].

Exact range (this library's reading; the paper does not discuss it).  The device computes
the contraction in a fixed order with int128 values and reports NaN for a row where a value
of that order leaves the int128 range; `contract_seq` follows the same order with Python
integers and says which rows those are:
  - the tree is rooted at table 0; a table's message to its parent is its tensor with every
    other axis contracted, the root's value is its tensor with every axis contracted;
  - a table contracts its child axes one at a time, last axis first; contracting axis l
    multiplies every entry by the child's message entry at its index on l and sums over l;
  - a leaf's message is its own 1-D tensor;
  - a row is out of range if any single product or any entry after a contraction is
    outside [-2^127, 2^127).

Hashing is the oracle's CW evaluation (`oracle.hash_eval`); predicates, the index and
sign arithmetic, the counters and the contractions are plain Python / numpy.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import oracle as orc

LIM = 1 << 127


def selected(table) -> np.ndarray:
    """Rows satisfying the conjunction of the table's predicates (RANGE keeps lo <= v < hi,
    EQ keeps v == lo, IN keeps 0 <= v < nbits with bit v of the bitmap set)."""
    keep = np.ones(table.n_rows, bool)
    for q in table.preds:
        v = table.cols[q.col].astype(np.int64)
        if q.op == orc.RANGE:
            keep &= (q.lo <= v) & (v < q.hi)
        elif q.op == orc.EQ:
            keep &= v == q.lo
        else:
            inb = (v >= 0) & (v < q.nbits)
            vv = v[inb]
            words = np.asarray(q.bitmap, np.uint64)
            bit = np.zeros(table.n_rows, bool)
            bit[inb] = ((words[vv >> 5] >> (vv & 31).astype(np.uint64)) & np.uint64(1)) == 1
            keep &= bit
    return keep


def build_partitioned(table, hp, d: int, widths, row_begin: int = 0, row_end: int | None = None):
    """Partitioned sketch of `table` over rows [row_begin, row_end): axes = the table's
    sketches in order (edge table.edge_id[l], key column table.key_col[l]), widths[l]
    buckets each.  hp: [n_edges][d][6] hash parameters.  Returns ([d][prod widths] int32,
    selected count)."""
    end = table.n_rows if row_end is None else row_end
    keep = selected(table)[row_begin:end]
    size = 1
    for w in widths:
        size *= int(w)
    n = int(keep.sum())
    out = np.zeros((d, size), np.int64)
    for i in range(d):
        idx = np.zeros(n, np.int64)
        sgn = np.ones(n, np.int64)
        for c, e, w in zip(table.key_col, table.edge_id, widths):
            keys = table.cols[c][row_begin:end][keep].astype(np.int64)
            b, x = orc.hash_eval(hp[e][i], int(w), keys)
            idx = idx * int(w) + b.astype(np.int64)
            sgn = sgn * x.astype(np.int64)
        np.add.at(out[i], idx, sgn)
    wrapped = ((out + (1 << 31)) % (1 << 32)) - (1 << 31)  # int32 counters wrap exactly
    return wrapped.astype(np.int32), n


def _other(edge_u, edge_v, e, t):
    return edge_v[e] if edge_u[e] == t else edge_u[e]


def contract_brute(edge_u, edge_v, width, dims, tensors, d: int) -> list:
    """The definition: per row, the sum over every assignment of bucket indices to the
    edges of the product of the tables' entries.  dims[t]: table t's axes (edge ids);
    tensors[t]: [d][prod widths].  Small widths only."""
    edges = sorted({e for ax in dims for e in ax})
    rows = []
    for i in range(d):
        total = 0
        for assign in itertools.product(*[range(int(width[e])) for e in edges]):
            j = dict(zip(edges, assign))
            prod = 1
            for t, ax in enumerate(dims):
                flat = 0
                for e in ax:
                    flat = flat * int(width[e]) + j[e]
                prod *= int(tensors[t][i][flat])
                if prod == 0:
                    break
            total += prod
        rows.append(total)
    return rows


def contract_seq(edge_u, edge_v, width, dims, tensors, d: int):
    """The contraction in the order stated in the module docstring, exact.  Returns (rows,
    out_of_range) with out_of_range[i] True where a value of that order left int128."""
    rows, oor = [], []
    for i in range(d):
        flag = [False]

        def message(t, parent_edge):
            ax = list(dims[t])
            shape = [int(width[e]) for e in ax]
            x = np.asarray([int(v) for v in tensors[t][i]], dtype=object).reshape(shape)
            for l in range(len(ax) - 1, -1, -1):
                e = ax[l]
                if e == parent_edge:
                    continue
                v = message(_other(edge_u, edge_v, e, t), e)
                bshape = [1] * x.ndim
                bshape[l] = shape[l]
                prod = x * np.asarray(v, dtype=object).reshape(bshape)
                if any(not (-LIM <= int(p) < LIM) for p in prod.flat):
                    flag[0] = True
                x = prod.sum(axis=l)
                x = np.asarray(x, dtype=object)
                if any(not (-LIM <= int(p) < LIM) for p in np.asarray(x).flat):
                    flag[0] = True
                shape.pop(l)
            return x

        r = message(0, None)
        rows.append(int(np.asarray(r).reshape(())[()]))
        oor.append(flag[0])
    return rows, oor


def median_to_double(rows) -> float:
    """Median of the exact row values (middle one for odd d, mean of the two middle ones
    for even d), rounded once to double."""
    r = sorted(int(v) for v in rows)
    n = len(r)
    if n % 2:
        return orc.dec_to_double(r[n // 2])
    return orc.dec_to_double(r[n // 2 - 1] + r[n // 2]) / 2.0   # halving is exact


def check_tree(n_tables: int, edge_u, edge_v, dims) -> None:
    """The shape the estimate accepts: the edges form a spanning tree of the tables and
    table t's axes are exactly its incident edges, each once."""
    if len(edge_u) != n_tables - 1:
        raise ValueError("the edges must form a spanning tree")
    seen = {0}
    frontier = [0]
    while frontier:
        t = frontier.pop()
        for e in range(len(edge_u)):
            if t in (edge_u[e], edge_v[e]):
                o = _other(edge_u, edge_v, e, t)
                if o not in seen:
                    seen.add(o)
                    frontier.append(o)
    if len(seen) != n_tables:
        raise ValueError("the edges must connect every table")
    for t in range(n_tables):
        inc = sorted(e for e in range(len(edge_u)) if t in (edge_u[e], edge_v[e]))
        if sorted(dims[t]) != inc:
            raise ValueError(f"table {t}: axes must be its incident edges")
