"""FP64 CPU oracle for diagonal-GMM k-means + EM (arXiv 1707.09094).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product package.  It
shares no code with the CUDA library.  The arithmetic lives in
``gmm_oracle.c`` (plain C, FP64, no fused multiply-add); this module compiles
it with gcc on first use and wraps it with ctypes + numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gmm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libgmm_oracle.so")
_lock = threading.Lock()
_lib = None

DIST_EUCL, DIST_MAHA, DIST_PROB = 0, 1, 2
SEED_KEEP_EXISTING, SEED_RANDOM_SUBSET, SEED_STATIC_SUBSET, SEED_STATIC_SPREAD, SEED_RANDOM_SPREAD = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle to ``oracle/_build/libgmm_oracle.so`` (OpenMP on)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i32, i64, u64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            sig = {
                "orc_log_gauss": (f64, [P, P, P, i32]),
                "orc_log_add": (f64, [f64, f64]),
                "orc_log_p": (ctypes.c_int, [P, i64, i32, i32, P, P, P, i32, i32, P]),
                "orc_avg_log_p": (ctypes.c_int, [P, i64, i32, i32, P, P, P, i32, P]),
                "orc_posteriors": (ctypes.c_int, [P, i64, i32, i32, P, P, P, P]),
                "orc_global_stats": (ctypes.c_int, [P, i64, i32, P, P]),
                "orc_seed_random_subset": (ctypes.c_int, [i64, i32, u64, P]),
                "orc_seed_static_subset": (ctypes.c_int, [i64, i32, P]),
                "orc_seed_spread": (ctypes.c_int, [P, i64, i32, i32, P, i64, P]),
                "orc_km_dist": (f64, [P, P, P, i32]),
                "orc_km_assign": (ctypes.c_int, [P, i64, i32, i32, P, P, P, P, P]),
                "orc_kmeans": (ctypes.c_int, [P, i64, i32, i32, P, P, P, P, P, i32, f64, P]),
                "orc_em_iterate": (ctypes.c_int, [P, i64, i32, i32, P, P, P, i32, f64, f64, i32, P, P]),
                "orc_em_step_twopass": (ctypes.c_int, [P, i64, i32, i32, P, P, P, f64]),
                "orc_em_fp32_budget": (ctypes.c_int, [P, i64, i32, i32, P, P, P, f64, i32, i32, i32, f64, P, P,
                                                      P, P]),
                "orc_assign": (ctypes.c_int, [P, i64, i32, i32, P, P, P, i32, P]),
                "orc_learn": (ctypes.c_int, [P, i64, i32, i32, i32, i32, u64, i32, i32, f64, f64,
                                             i32, P, P, P, P, P]),
                "orc_log_p_fp32_bound": (ctypes.c_int, [P, i64, i32, i32, P, P, P, i32, P]),
                "orc_num_threads": (ctypes.c_int, []),
                "orc_set_threads": (None, [i32]),
                "orc_generate": (ctypes.c_int, [P, P, P, i32, i32, i64, u64, P, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _x(X):
    X = np.ascontiguousarray(X, dtype=np.float32)
    if X.ndim != 2:
        raise ValueError("X must be [N][D]")
    return X


def _params(means, dcovs, hefts):
    return (np.ascontiguousarray(means, dtype=np.float64),
            np.ascontiguousarray(dcovs, dtype=np.float64),
            np.ascontiguousarray(hefts, dtype=np.float64))


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("oracle %s failed with status %d" % (what, rc))


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_threads(n: int) -> None:
    """OpenMP threads of the MapReduce loops (the CPU-baseline timing only)."""
    _load().orc_set_threads(int(n))


def log_gauss(x, mu, dcov) -> float:
    x = np.ascontiguousarray(x, dtype=np.float32)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    dcov = np.ascontiguousarray(dcov, dtype=np.float64)
    return float(_load().orc_log_gauss(_p(x), _p(mu), _p(dcov), x.size))


def log_add(a: float, b: float) -> float:
    return float(_load().orc_log_add(a, b))


def log_p(X, means, dcovs, hefts, g: int = -1, maxsum: bool = False):
    X = _x(X)
    m, v, h = _params(means, dcovs, hefts)
    out = np.empty(X.shape[0], np.float64)
    _check(_load().orc_log_p(_p(X), X.shape[0], X.shape[1], m.shape[0], _p(m), _p(v), _p(h),
                             g, int(maxsum), _p(out)), "log_p")
    return out


def avg_log_p(X, means, dcovs, hefts, g: int = -1) -> float:
    X = _x(X)
    m, v, h = _params(means, dcovs, hefts)
    out = ctypes.c_double()
    _check(_load().orc_avg_log_p(_p(X), X.shape[0], X.shape[1], m.shape[0], _p(m), _p(v), _p(h),
                                 g, ctypes.byref(out)), "avg_log_p")
    return out.value


def posteriors(X, means, dcovs, hefts):
    X = _x(X)
    m, v, h = _params(means, dcovs, hefts)
    out = np.empty((X.shape[0], m.shape[0]), np.float64)
    _check(_load().orc_posteriors(_p(X), X.shape[0], X.shape[1], m.shape[0], _p(m), _p(v), _p(h),
                                  _p(out)), "posteriors")
    return out


def global_stats(X):
    X = _x(X)
    mean = np.empty(X.shape[1], np.float64)
    var = np.empty(X.shape[1], np.float64)
    _check(_load().orc_global_stats(_p(X), X.shape[0], X.shape[1], _p(mean), _p(var)), "global_stats")
    return mean, var


def seed_random_subset(N: int, G: int, seed: int):
    idx = np.empty(G, np.int64)
    _check(_load().orc_seed_random_subset(N, G, ctypes.c_uint64(seed & (2**64 - 1)), _p(idx)),
           "seed_random_subset")
    return idx


def seed_static_subset(N: int, G: int):
    idx = np.empty(G, np.int64)
    _check(_load().orc_seed_static_subset(N, G, _p(idx)), "seed_static_subset")
    return idx


def seed_spread(X, G: int, w, first: int):
    """Farthest-first traversal from sample `first` (static_spread / random_spread)."""
    X = _x(X)
    N, D = X.shape
    w = np.ascontiguousarray(w, dtype=np.float64)
    idx = np.empty(G, np.int64)
    _check(_load().orc_seed_spread(_p(X), N, D, G, _p(w), first, _p(idx)), "seed_spread")
    return idx


def generate(means, dcovs, hefts, N: int, seed: int = 0):
    """M.generate(N) of Sec. 4.1: (X float32 [N][D], labels int32 [N])."""
    means = np.ascontiguousarray(means, dtype=np.float64)
    dcovs = np.ascontiguousarray(dcovs, dtype=np.float64)
    hefts = np.ascontiguousarray(hefts, dtype=np.float64)
    G, D = means.shape
    X = np.empty((N, D), np.float32)
    lab = np.empty(N, np.int32)
    _check(_load().orc_generate(_p(means), _p(dcovs), _p(hefts), G, D, N, ctypes.c_uint64(seed & (2**64 - 1)),
                                _p(X), _p(lab)), "generate")
    return X, lab


def km_dist(x, mu, w) -> float:
    x = np.ascontiguousarray(x, dtype=np.float32)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    return float(_load().orc_km_dist(_p(x), _p(mu), _p(w), x.size))


def km_assign(X, means, w):
    X = _x(X)
    means = np.ascontiguousarray(means, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    N = X.shape[0]
    a = np.empty(N, np.int32)
    b1 = np.empty(N, np.float64)
    b2 = np.empty(N, np.float64)
    _check(_load().orc_km_assign(_p(X), N, X.shape[1], means.shape[0], _p(means), _p(w), _p(a),
                                 _p(b1), _p(b2)), "km_assign")
    return a, b1, b2


def kmeans(X, seeds_means, w, gvar_floored, km_iter: int, var_floor: float):
    X = _x(X)
    G, D = np.asarray(seeds_means).shape
    means = np.array(seeds_means, dtype=np.float64, order="C", copy=True)
    dcovs = np.empty((G, D), np.float64)
    hefts = np.empty(G, np.float64)
    a = np.empty(X.shape[0], np.int32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    gv = np.ascontiguousarray(gvar_floored, dtype=np.float64)
    _check(_load().orc_kmeans(_p(X), X.shape[0], D, G, _p(w), _p(gv), _p(means), _p(dcovs),
                              _p(hefts), km_iter, var_floor, _p(a)), "kmeans")
    return means, dcovs, hefts, a


def em_iterate(X, means, dcovs, hefts, em_iter: int, var_floor: float, em_tol: float = 0.0,
               n_chunks: int = 1):
    """Run em_iter EM iterations; returns (means, dcovs, hefts, ll_hist)."""
    X = _x(X)
    m = np.array(means, dtype=np.float64, order="C", copy=True)
    v = np.array(dcovs, dtype=np.float64, order="C", copy=True)
    h = np.array(hefts, dtype=np.float64, order="C", copy=True)
    ll = np.zeros(max(em_iter, 1), np.float64)
    nd = ctypes.c_int32()
    rc = _load().orc_em_iterate(_p(X), X.shape[0], X.shape[1], m.shape[0], _p(m), _p(v), _p(h),
                                em_iter, var_floor, em_tol, n_chunks, _p(ll), ctypes.byref(nd))
    _check(rc, "em_iterate")
    return m, v, h, ll[: nd.value]


def fp32_accumulations(N: int, chunk: int = 0) -> int:
    """Upper bound on the FP32 additions into one statistics accumulator of an
    EM pass over N samples: at least 128 sample chunks (one per SM or more)
    of 32-sample tiles, each tile first summed over up to 128 terms.  `chunk`
    > 0 bounds the samples of one chunk instead (the batched form's items)."""
    per_chunk = chunk if chunk > 0 else -(-N // 128)
    return -(-per_chunk // 32) + 128


def em_fp32_budget(X, means, dcovs, hefts, var_floor: float, n_acc: int = 0, n_lse: int = 0,
                   drop: float = 1e-9, n_chunks: int = 0):
    """One EM iteration from (means, dcovs, hefts) and the FP32 error budget of
    each new parameter (see orc_em_fp32_budget).  n_acc: FP32 additions into
    one statistics accumulator (default fp32_accumulations(N)); n_lse: the
    longest chain of FP32 additions in one log-sum-exp (default G + 8, any
    order).  Returns (means, dcovs, hefts, mean_ll, (b_means, b_dcovs, b_hefts))."""
    X = _x(X)
    N, D = X.shape
    m = np.array(means, dtype=np.float64, order="C", copy=True)
    v = np.array(dcovs, dtype=np.float64, order="C", copy=True)
    h = np.array(hefts, dtype=np.float64, order="C", copy=True)
    G = m.shape[0]
    bm = np.zeros((G, D), np.float64)
    bv = np.zeros((G, D), np.float64)
    bw = np.zeros(G, np.float64)
    ll = ctypes.c_double()
    if n_chunks <= 0:
        n_chunks = max(num_threads(), 1) * (4 if N >= 100_000 else 1)
    if n_acc <= 0:
        n_acc = fp32_accumulations(N)
    if n_lse <= 0:
        n_lse = G + 8
    _check(_load().orc_em_fp32_budget(_p(X), N, D, G, _p(m), _p(v), _p(h), var_floor, n_chunks, n_acc, n_lse, drop,
                                      ctypes.byref(ll), _p(bm), _p(bv), _p(bw)), "em_fp32_budget")
    return m, v, h, ll.value, (bm, bv, bw)


def log_p_fp32_bound(X, means, dcovs, hefts, n_lse: int = 0):
    """Per sample, the bound on |FP32 log p(x_i) - FP64 log p(x_i)| of
    orc_log_p_fp32_bound (a parity tolerance)."""
    X = _x(X)
    m, v, h = _params(means, dcovs, hefts)
    out = np.empty(X.shape[0], np.float64)
    _check(_load().orc_log_p_fp32_bound(_p(X), X.shape[0], X.shape[1], m.shape[0], _p(m), _p(v), _p(h),
                                        n_lse if n_lse > 0 else m.shape[0] + 8, _p(out)), "log_p_fp32_bound")
    return out


def em_step_twopass(X, means, dcovs, hefts, var_floor: float):
    X = _x(X)
    m = np.array(means, dtype=np.float64, order="C", copy=True)
    v = np.array(dcovs, dtype=np.float64, order="C", copy=True)
    h = np.array(hefts, dtype=np.float64, order="C", copy=True)
    _check(_load().orc_em_step_twopass(_p(X), X.shape[0], X.shape[1], m.shape[0], _p(m), _p(v),
                                       _p(h), var_floor), "em_step_twopass")
    return m, v, h


def assign(X, means, dcovs, hefts, mode: int):
    X = _x(X)
    m, v, h = _params(means, dcovs, hefts)
    out = np.empty(X.shape[0], np.int32)
    _check(_load().orc_assign(_p(X), X.shape[0], X.shape[1], m.shape[0], _p(m), _p(v), _p(h),
                              mode, _p(out)), "assign")
    return out


def learn(X, G: int, dist_mode: int = DIST_MAHA, seed_mode: int = SEED_RANDOM_SUBSET,
          seed: int = 0, km_iter: int = 10, em_iter: int = 10, var_floor: float = 1e-10,
          em_tol: float = 0.0, n_chunks: int = 1, init=None):
    """learn() of Sec. 4.1; returns (means, dcovs, hefts, ll_hist)."""
    X = _x(X)
    N, D = X.shape
    if init is not None:
        m, v, h = (np.array(a, dtype=np.float64, order="C", copy=True) for a in init)
    else:
        m = np.zeros((G, D), np.float64)
        v = np.ones((G, D), np.float64)
        h = np.full(G, 1.0 / G, np.float64)
    ll = np.zeros(max(em_iter, 1), np.float64)
    nd = ctypes.c_int32()
    rc = _load().orc_learn(_p(X), N, D, G, dist_mode, seed_mode, ctypes.c_uint64(seed & (2**64 - 1)),
                           km_iter, em_iter, var_floor, em_tol, n_chunks, _p(m), _p(v), _p(h),
                           _p(ll), ctypes.byref(nd))
    _check(rc, "learn")
    return m, v, h, ll[: nd.value]
