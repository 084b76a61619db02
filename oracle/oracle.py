"""ctypes wrapper of the COMPASS oracle (compass_oracle.cpp).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's CPU
baseline load it; the product path never does.  Every function takes and returns
numpy arrays / Python ints and forwards to the single-threaded C++ oracle.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "compass_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

P61 = (1 << 61) - 1
RANGE, EQ, IN = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with the host compiler (portable flags only)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.orc_estimate.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_int, C.c_int, C.c_uint64, C.c_int, C.c_char_p, C.c_void_p, C.c_void_p]
        _lib.orc_dec_to_double.restype = C.c_double
        _lib.orc_dec_to_double.argtypes = [C.c_char_p]
    return _lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


# --------------------------------------------------------------------------- hashing

def splitmix64(seed: int, n: int) -> list:
    out = np.zeros(n, np.uint64)
    lib().orc_splitmix64(C.c_uint64(seed), n, C.c_void_p(_p(out)))
    return [int(v) for v in out]


def hash_params(seed: int, n_edges: int, d: int) -> np.ndarray:
    """[n_edges, d, 6] uint64 (a, b, c0, c1, c2, c3)."""
    out = np.zeros((max(n_edges, 0), d, 6), dtype=np.uint64)
    rc = lib().orc_hash_params(C.c_uint64(seed), n_edges, d, C.c_void_p(_p(out)))
    assert rc == 0
    return out


def hash_eval(hp: np.ndarray, w: int, keys) -> tuple[np.ndarray, np.ndarray]:
    hp = np.ascontiguousarray(hp, dtype=np.uint64).reshape(6)
    keys = np.ascontiguousarray(np.asarray(keys, dtype=np.int64))
    b = np.zeros(keys.size, np.int32)
    s = np.zeros(keys.size, np.int32)
    rc = lib().orc_hash_eval(C.c_void_p(_p(hp)), w, C.c_int64(keys.size), C.c_void_p(_p(keys)),
                             C.c_void_p(_p(b)), C.c_void_p(_p(s)))
    assert rc == 0
    return b, s


# --------------------------------------------------------------------------- build

@dataclass
class Pred:
    col: int
    op: int
    lo: int = 0
    hi: int = 0
    bitmap: np.ndarray | None = None   # uint32 words
    nbits: int = 0


@dataclass
class Table:
    cols: list                      # numpy int32 / int64 arrays, equal length
    preds: list = field(default_factory=list)
    key_col: list = field(default_factory=list)   # per sketch
    edge_id: list = field(default_factory=list)   # per sketch

    @property
    def n_rows(self) -> int:
        return int(self.cols[0].shape[0]) if self.cols else 0


def build_sketch(t: Table, hash_all: np.ndarray, d: int, w: int,
                 row_begin: int = 0, row_end: int | None = None,
                 accumulate: tuple[np.ndarray, np.ndarray] | None = None):
    """Oracle build of one table over rows [row_begin, row_end).

    Returns (counters [k, d, w] int32, survivors int).  With `accumulate`, adds into
    the given (counters, survivors[1]) arrays instead (partitions merge by addition).
    """
    n = t.n_rows if row_end is None else row_end
    cols = [np.ascontiguousarray(c[row_begin:n]) for c in t.cols]
    for c in cols:
        assert c.dtype in (np.int32, np.int64)
    col_ptrs = (C.c_void_p * max(len(cols), 1))(*[_p(c) for c in cols])
    dt = np.array([0 if c.dtype == np.int32 else 1 for c in cols] or [0], np.int32)
    npred = len(t.preds)
    pc = np.array([q.col for q in t.preds] or [0], np.int32)
    po = np.array([q.op for q in t.preds] or [0], np.int32)
    plo = np.array([q.lo for q in t.preds] or [0], np.int64)
    phi = np.array([q.hi for q in t.preds] or [0], np.int64)
    bms = [np.ascontiguousarray(q.bitmap, np.uint32) if q.bitmap is not None else np.zeros(1, np.uint32)
           for q in t.preds]
    pbm = (C.c_void_p * max(npred, 1))(*[_p(b) for b in bms])
    pnb = np.array([q.nbits for q in t.preds] or [0], np.int64)
    k = len(t.key_col)
    kc = np.array(t.key_col or [0], np.int32)
    ei = np.array(t.edge_id or [0], np.int32)
    hash_all = np.ascontiguousarray(hash_all, dtype=np.uint64)
    n_edges = hash_all.shape[0]
    if accumulate is None:
        counters = np.zeros((k, d, w), np.int32)
        surv = np.zeros(1, np.int64)
        acc = 0
    else:
        counters, surv = accumulate
        acc = 1
    rc = lib().orc_build(C.c_int64(n - row_begin), len(cols), col_ptrs, C.c_void_p(_p(dt)), npred,
                         C.c_void_p(_p(pc)), C.c_void_p(_p(po)), C.c_void_p(_p(plo)), C.c_void_p(_p(phi)),
                         pbm, C.c_void_p(_p(pnb)), k, C.c_void_p(_p(kc)), C.c_void_p(_p(ei)), n_edges, d, w,
                         C.c_void_p(_p(hash_all)), acc, C.c_void_p(_p(counters)), C.c_void_p(_p(surv)))
    if rc != 0:
        raise ValueError(f"orc_build rejected its arguments (rc={rc})")
    return counters, int(surv[0])


# --------------------------------------------------------------------------- estimate

@dataclass
class Estimate:
    est: float
    rows: list          # exact row estimates (Python ints)
    rows_dbl: np.ndarray


def estimate(edge_u, edge_v, sketches, survivors, d: int, w: int, mask: int, brute: bool = False) -> Estimate:
    """Sketch-merging estimate of the sub-plan `mask` (bit t = table t).

    sketches[e] = (sketch of endpoint edge_u[e], sketch of endpoint edge_v[e]), each
    [d, w] int32.  survivors[t] = exact selected count of table t.
    """
    eu = np.ascontiguousarray(edge_u, np.int32)
    ev = np.ascontiguousarray(edge_v, np.int32)
    ne = eu.size
    nt = len(survivors)
    sk = []
    for e in range(ne):
        for end in range(2):
            a = np.ascontiguousarray(sketches[e][end], np.int32)
            assert a.shape == (d, w)
            sk.append(a)
    skp = (C.c_void_p * max(2 * ne, 1))(*[_p(a) for a in sk])
    sv = np.ascontiguousarray(survivors, np.int64)
    dec = C.create_string_buffer(d * 2048)
    dbl = np.zeros(d, np.float64)
    est = np.zeros(1, np.float64)
    rc = lib().orc_estimate(nt, ne, _p(eu) if ne else None, _p(ev) if ne else None, C.cast(skp, C.c_void_p),
                            _p(sv), d, w, C.c_uint64(mask), 1 if brute else 0, dec, _p(dbl), _p(est))
    if rc == -2:
        raise OverflowError("brute force enumeration too large")
    if rc != 0:
        raise ValueError(f"orc_estimate rejected the sub-plan (rc={rc})")
    raw = dec.raw
    rows = [int(raw[i * 2048:(i + 1) * 2048].split(b"\0", 1)[0].decode()) for i in range(d)]
    return Estimate(float(est[0]), rows, dbl)


def dec_to_double(v: int) -> float:
    return lib().orc_dec_to_double(str(int(v)).encode())


def join2(a, b) -> int:
    a = np.ascontiguousarray(a, np.int64)
    b = np.ascontiguousarray(b, np.int64)
    buf = C.create_string_buffer(64)
    dbl = np.zeros(1, np.float64)
    rc = lib().orc_join2(C.c_int64(a.size), C.c_void_p(_p(a)), C.c_int64(b.size), C.c_void_p(_p(b)), buf,
                         C.c_void_p(_p(dbl)))
    assert rc == 0
    return int(buf.value.decode())


def join2_dense(a, b, domain: int) -> int:
    """Exact two-way join size of int32 key arrays with every key in [0, domain): the dot
    product of the key histograms (O(n + domain)).  The C call releases the interpreter
    lock, so threads can label many joins at once."""
    a = np.ascontiguousarray(a, np.int32)
    b = np.ascontiguousarray(b, np.int32)
    lo = np.zeros(1, np.uint64)
    hi = np.zeros(1, np.uint64)
    rc = lib().orc_join2_dense(C.c_int64(a.size), C.c_void_p(_p(a)), C.c_int64(b.size), C.c_void_p(_p(b)),
                               C.c_int64(domain), C.c_void_p(_p(lo)), C.c_void_p(_p(hi)))
    if rc != 0:
        raise ValueError("a key lies outside [0, domain)")
    return (int(hi[0]) << 64) | int(lo[0])


def join_brute(edge_u, edge_v, n_rows, keys, mask: int) -> int:
    """keys[e] = (key column of endpoint u, key column of endpoint v), aligned with that table's tuples."""
    eu = np.ascontiguousarray(edge_u, np.int32)
    ev = np.ascontiguousarray(edge_v, np.int32)
    nr = np.ascontiguousarray(n_rows, np.int64)
    ks = []
    for e in range(eu.size):
        for end in range(2):
            ks.append(np.ascontiguousarray(keys[e][end], np.int64))
    kp = (C.c_void_p * max(len(ks), 1))(*[_p(a) for a in ks])
    buf = C.create_string_buffer(64)
    dbl = np.zeros(1, np.float64)
    rc = lib().orc_join_brute(len(nr), eu.size, C.c_void_p(_p(eu)), C.c_void_p(_p(ev)), C.c_void_p(_p(nr)), kp,
                              C.c_uint64(mask), buf, C.c_void_p(_p(dbl)))
    if rc != 0:
        raise OverflowError("brute-force join too large")
    return int(buf.value.decode())


# --------------------------------------------------------------------------- MLP

def bf16_round(a) -> np.ndarray:
    a = np.ascontiguousarray(a, np.float32)
    out = np.empty_like(a)
    lib().orc_bf16_round(C.c_int64(a.size), C.c_void_p(_p(a)), C.c_void_p(_p(out)))
    return out


def mlp_forward(nin: int, nh: int, params, x, skip: int = -1) -> np.ndarray:
    params = np.ascontiguousarray(params, np.float32)
    x = np.ascontiguousarray(x, np.float32)
    n = x.shape[0]
    y = np.zeros(n, np.float64)
    lib().orc_mlp_forward(nin, nh, skip, C.c_void_p(_p(params)), C.c_int64(n), C.c_void_p(_p(x)), C.c_void_p(_p(y)))
    return y


def mlp_loss_grad(nin: int, nh: int, params, x, t, skip: int = -1, huber_delta: float | None = None):
    params = np.ascontiguousarray(params, np.float32)
    x = np.ascontiguousarray(x, np.float32)
    t = np.ascontiguousarray(t, np.float32)
    g = np.zeros(params.size, np.float64)
    loss = np.zeros(1, np.float64)
    kind = 0 if huber_delta is None else 1
    lib().orc_mlp_loss_grad(nin, nh, skip, kind, C.c_double(huber_delta or 0.0), C.c_void_p(_p(params)),
                            C.c_int64(x.shape[0]), C.c_void_p(_p(x)), C.c_void_p(_p(t)), C.c_void_p(_p(loss)),
                            C.c_void_p(_p(g)))
    return float(loss[0]), g


def adam_step(params, m, v, grad, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, step=1):
    """In place on float32 params and float64 moments."""
    assert params.dtype == np.float32 and m.dtype == np.float64 and v.dtype == np.float64
    grad = np.ascontiguousarray(grad, np.float64)
    lib().orc_adam_step(C.c_int64(params.size), C.c_void_p(_p(params)), C.c_void_p(_p(m)), C.c_void_p(_p(v)),
                        C.c_void_p(_p(grad)), C.c_double(lr), C.c_double(b1), C.c_double(b2), C.c_double(eps),
                        step)
