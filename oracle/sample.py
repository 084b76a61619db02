"""Oracle (test infrastructure only; the product path never imports it): sketches over a
row sample (Sec. 2 "Workflow": the sketches may be built over a sample only, at a cost in
accuracy), written from the definition.

Sample.  At rate p in (0, 1), row r of a table is kept iff output r (0-based) of SplitMix64
(Steele, Lea & Flood 2014) seeded with the table's sample seed is below keep = floor(p 2^64):
a Bernoulli trial per row, independent across rows.  p = 0 or 1 means no sampling.  The generator is
counter-based: output r is the mix of seed + (r + 1) * gamma, so any row's trial is computed
on its own.  Thresholds are nested: a row kept at `keep` is kept at every larger threshold.

Estimate.  A sketch of the sample is the sketch of the sampled rows (the selection and the
sample are both row-local).  Because tables are sampled independently, the expected two-way
Fast-AGMS estimate over samples is p_u p_v times the one over the full tables, so the
estimate of a sub-plan over tables S is scaled by prod_{t in S} 1 / p_t (the selected count
of a single table by 1 / p_t).  The scale is computed in double: the reciprocals in
ascending table order, multiplied left to right, and the median (already rounded) is
multiplied by it once.  For the merged multi-way estimate, whose merge step is not linear in
the counters, the same scale is the natural extension rather than an unbiased correction.
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15


def splitmix64_at(seed: int, rows) -> np.ndarray:
    """SplitMix64 outputs number `rows` (array of 0-based positions) of the stream seeded
    with `seed`, as uint64 (numpy arithmetic wraps modulo 2^64)."""
    r = np.asarray(rows, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & (2 ** 64 - 1)) + (r + np.uint64(1)) * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def keep_threshold(rate: float) -> int:
    """The threshold of a sampling rate in [0, 1]: 0 (no sampling) for 0 and 1, else
    floor(rate * 2^64) (the product is exact in double), at least 1."""
    if not (0.0 <= rate <= 1.0):
        raise ValueError("rate must be in [0, 1]")
    if rate == 0.0 or rate == 1.0:
        return 0
    return max(1, int(rate * 2.0 ** 64))


def sample_mask(n_rows: int, seed: int, keep: int) -> np.ndarray:
    if keep == 0:
        return np.ones(n_rows, bool)
    return splitmix64_at(seed, np.arange(n_rows, dtype=np.uint64)) < np.uint64(keep)


def sampled_table(t, seed: int, rate: float):
    """The table restricted to its sampled rows at `rate` (row order kept; same predicates
    and sketches)."""
    m = sample_mask(t.n_rows, seed, keep_threshold(rate))
    return type(t)(t.name, [np.ascontiguousarray(c[m]) for c in t.cols], t.preds, list(t.key_col),
                   list(t.edge_id))


def scale_of(mask: int, rates) -> float:
    """prod over the tables of the sub-plan (bit t of mask), ascending, of 1 / rate_t (a
    rate of 0 or 1 means an unsampled table and contributes 1)."""
    s = 1.0
    for t, r in enumerate(rates):
        if (mask >> t) & 1 and 0.0 < r < 1.0:
            s = s * (1.0 / r)
    return s
