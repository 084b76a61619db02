"""Pins of the oracle's hash family (Sec. 3.1 / 3.2: 4-wise xi, per-row bucket hash h;
Carter-Wegman polynomials over the Mersenne prime 2^61 - 1 where the paper names no family)."""
import os

import numpy as np
import pytest

P = (1 << 61) - 1
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_splitmix64_published_values(orc):
    rows = _golden_lines("splitmix64_seed1234567.txt")
    seed = int(rows[0][1])
    want = [int(r[0]) for r in rows[1:]]
    assert orc.splitmix64(seed, len(want)) == want


def test_hash_params_range_and_determinism(orc):
    hp = orc.hash_params(7, 5, 11)
    assert hp.shape == (5, 11, 6)
    assert (hp < P).all()
    assert (hp[..., 0] != 0).all()
    assert np.array_equal(hp, orc.hash_params(7, 5, 11))
    assert not np.array_equal(hp, orc.hash_params(8, 5, 11))
    # fields come from consecutive generator outputs, top 61 bits each
    raw = orc.splitmix64(7, 6)
    assert [int(v) for v in hp[0, 0]] == [(r >> 3) % P or (1 if i == 0 else 0) for i, r in enumerate(raw)]


EDGE_KEYS = [0, 1, -1, 2, 7, -(1 << 31), (1 << 31) - 1, (1 << 63) - 1, -(1 << 63), P - 1, P, P + 1, -P, 12345678901]


def _py_hash(hp, w, key):
    x = key % P                        # mathematical residue in [0, p)
    a, b, c0, c1, c2, c3 = (int(v) for v in hp)
    bucket = ((a * x + b) % P) % w
    v = (c3 * x ** 3 + c2 * x ** 2 + c1 * x + c0) % P
    return bucket, (-1 if v & 1 else 1)


@pytest.mark.parametrize("w", [1, 2, 3, 1023, 1024, 4096, 65536])
def test_hash_eval_matches_python_bigints(orc, w):
    rng = np.random.default_rng(w)
    hp = orc.hash_params(99 + w, 3, 4)
    keys = EDGE_KEYS + [int(v) for v in rng.integers(-(1 << 63), (1 << 63) - 1, size=200, dtype=np.int64)]
    for e in range(3):
        for i in range(4):
            b, s = orc.hash_eval(hp[e, i], w, keys)
            for k, bb, ss in zip(keys, b, s):
                assert (int(bb), int(ss)) == _py_hash(hp[e, i], w, k)


def test_hash_eval_extreme_params(orc):
    # largest field elements everywhere: products reach 2^122, sums 2^124
    hp = np.array([P - 1] * 6, np.uint64)
    keys = EDGE_KEYS
    b, s = orc.hash_eval(hp, 1000, keys)
    for k, bb, ss in zip(keys, b, s):
        assert (int(bb), int(ss)) == _py_hash(hp, 1000, k)


def test_sign_is_balanced(orc):
    # 4-wise independent +-1 family: over many keys the mean sign is ~0
    hp = orc.hash_params(3, 1, 1)[0, 0]
    _, s = orc.hash_eval(hp, 64, np.arange(200_000))
    assert abs(s.mean()) < 0.01
