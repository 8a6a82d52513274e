"""ctypes wrapper of the C oracle (oracle/kscann_oracle.c).

TEST INFRASTRUCTURE: a plain CPU restatement of the KScaNN query path
(arXiv 2511.03298).  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline legs may call it; the product never does.

Functions and the passages they follow (parity pins live in
tests/test_oracle_pins.py):
  kmeans        Sec. 2.2 / Alg. 1 (IVF clustering, PQ codebooks)   pinned
  build_index   Alg. 1 with the mean-centroid residual of Sec. 4.6.1 pinned
  encode        Sec. 2.3 (nearest codeword per sub-vector)         pinned
  rank          Alg. 2 TopNClusters                                pinned
  adc64         Eq. 1 with residual tables                         pinned
  lut_q8        Sec. 2.5 / Sec. 4.5 8-bit LUT (FP32 rule)          pinned
  scan_topr     Alg. 3 scan + candidate pool                       pinned
  hybrid_topr   Sec. 4.4 / Alg. 3 graph branch                     pinned
  rerank        Alg. 2 exact re-rank                               pinned
  exact_knn     brute force (ground truth)                         pinned
  recall        Sec. 5.4 Recall@10                                 pinned
  eq2           Eq. 2                                              pinned
  reg_map       regression-head mapping (predictor variant)        pinned
  mlp_*         Sec. 4.2.1-4.2.2 predictor (MLP stand-in)          pinned
  prune_*       Sec. 4.2.3 / Table 4 cluster pruning, Alg. 2       pinned
  component_*   Sec. 4.3 component filtration, Alg. 1 / Alg. 2     pinned
"""
import ctypes as C
import os

import numpy as np

from .build import LIB, build

_lib = None

_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
_vp = C.c_void_p
_i32, _i64, _f64 = C.c_int32, C.c_int64, C.c_double

K = 16


def lib():
    global _lib
    if _lib is None:
        path = build()  # compiles only when the source is newer than the library
        L = C.CDLL(path)
        sig = {
            "orc_kmeans": (C.c_int, [_f32p, _i64, _i32, _i32, _i64p, _i64, _i32, _i32, _f64p, _vp]),
            "orc_build_index": (C.c_int, [_f32p, _i64, _i32, _i32, _i32, _i32, _i64p, _i32,
                                          _f32p, _f32p, _f32p, _u8p, _i32p]),
            "orc_encode": (C.c_int, [_f32p, _i64, _i32, _i32, _f32p, _u8p, _vp]),
            "orc_lists": (C.c_int, [_i32p, _i64, _i32, _i64p, _i32p]),
            "orc_rank": (C.c_int, [_f32p, _i32, _f32p, _i32, _i32, _i32, _i32p, _vp]),
            "orc_adc64": (C.c_double, [_f32p, _i32, _i32, _f32p, _f32p, _u8p, _i32]),
            "orc_lut_q8": (C.c_int, [_f32p, _i32, _i32, _f32p, _f32p, _i32, _i32p, _i32,
                                     _u8p, _i32p, _vp]),
            "orc_int_dist": (C.c_int32, [_u8p, _i32, _u8p, _i32]),
            "orc_scan_topr": (C.c_int64, [_u8p, _i32, _i64p, _i32p, _i32p, _i32, _u8p, _i32p,
                                          _i32, _u64p]),
            "orc_graph_search": (C.c_int32, [_u8p, _i32, _i32p, _i32, _u8p, _i32, _i32, _i64, _u64p]),
            "orc_hybrid_topr": (C.c_int64, [_u8p, _i32, _i64p, _i32p, _i64, _i32p, _i32p, _i32p,
                                            _i32, _u8p, _i32p, _i32, _i32, _i32, _i32, _u64p, _vp]),
            "orc_build_graph": (C.c_int, [_f32p, _i32, _i64p, _i32p, _i32, _f32p, _i32p, _i32p]),
            "orc_rerank": (C.c_int, [_f32p, _f32p, _i32, _i32, _i32p, _i64, _i32, _i64p, _f64p]),
            "orc_exact_knn": (C.c_int, [_f32p, _i64, _f32p, _i64, _i32, _i32, _i32, _i64p, _f64p, _i32]),
            "orc_search": (C.c_int, [_f32p, _i64, _i32, _i32, _i32, _i32, _i32,
                                     _f32p, _f32p, _f32p, _f32p, _u8p, _i64p, _i32p,
                                     _i32p, _i32p, _i32, _i64p, _f64p,
                                     _vp, _i32, _vp, _i32, _vp, _i32]),
            "orc_recall": (C.c_double, [_f32p, _i64, _f32p, _i32, _i32, _i64p, _i32, _f64p, _i32, _i32]),
            "orc_eq2": (C.c_int32, [_f64, _i32, _i32, _f64, _f64]),
            "orc_mlp_forward": (C.c_int, [_f64p, _i32, _i32, _i32, _f64p, _i64, _f64p]),
            "orc_mlp_grad": (C.c_double, [_f64p, _i32, _i32, _i32, _f64p, _f64p, _i64, _f64p]),
            "orc_adam_step": (C.c_int, [_f64p, _f64p, _f64p, _f64p, _i64, _i32, _f64, _f64, _f64, _f64]),
            "orc_prune_stats": (C.c_int, [_f32p, _i64, _i32, _f32p, _i32, _i32p, _i32, _f64p, _f64p]),
            "orc_prune_features": (C.c_int, [_f32p, _i64, _i32, _f32p, _i32, _i32p, _i32, _vp, _i32,
                                             _f64p, _f64p, _f64p]),
            "orc_component_stats": (C.c_int, [_f32p, _i64, _i32, _f64p, _f64p, _f64p]),
            "orc_reg_map": (C.c_int32, [_f64, _i32, _i32, _f64, _f64]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------- build side
def kmeans(X, sample, L, iters, col0=0, d=None):
    """Lloyd FP64 on X[sample] columns [col0, col0+d); init = first L sample rows."""
    X = _c(X, np.float32)
    d = X.shape[1] if d is None else d
    Cc = np.zeros((L, d), np.float64)
    obj = np.zeros(iters + 1, np.float64)
    rc = lib().orc_kmeans(X, X.shape[1], col0, d, _c(sample, np.int64), len(sample), L, iters,
                          Cc, _ptr(obj))
    assert rc == 0
    return Cc, obj


def build_index(X, L, M, spherical, perm, iters=20, ip=False):
    """Alg. 1 (without filtration/graph/ML): returns the FP32 index arrays."""
    X = _c(X, np.float32)
    n, d = X.shape
    c_rank = np.zeros((L, d), np.float32)
    c_mean = np.zeros((L, d), np.float32)
    cb = np.zeros((M, K, d // M), np.float32)
    codes = np.zeros((n, M), np.uint8)
    assign = np.zeros(n, np.int32)
    rc = lib().orc_build_index(X, n, d, L, M, int(spherical), _c(perm, np.int64), iters,
                               c_rank, c_mean, cb, codes, assign)
    assert rc == 0
    return make_index(X, c_rank, c_mean, cb, codes, assign, ip=ip, spherical=spherical)


def make_index(X, c_rank, c_mean, codebook, codes, assign, ip=False, spherical=False):
    X = _c(X, np.float32)
    L, d = c_rank.shape
    M = codebook.shape[0]
    lo, ids = lists(assign, L)
    return dict(X=X, c_rank=_c(c_rank, np.float32), c_mean=_c(c_mean, np.float32),
                codebook=_c(codebook, np.float32), codes=_c(codes, np.uint8),
                assign=_c(assign, np.int32), list_off=lo, list_ids=ids,
                n=X.shape[0], d=d, L=L, M=M, ip=bool(ip), spherical=bool(spherical or ip))


def encode(R, M, codebook):
    """Nearest codeword per sub-vector (FP64), and the gap to the second best."""
    R = _c(R, np.float32)
    n, d = R.shape
    codes = np.zeros((n, M), np.uint8)
    gap = np.zeros((n, M), np.float64)
    lib().orc_encode(R, n, d, M, _c(codebook, np.float32), codes, _ptr(gap))
    return codes, gap


def lists(assign, L):
    assign = _c(assign, np.int32)
    lo = np.zeros(L + 1, np.int64)
    ids = np.zeros(len(assign), np.int32)
    assert lib().orc_lists(assign, len(assign), L, lo, ids) == 0
    return lo, ids


# --------------------------------------------------------------- query side
def rank(q, c_rank, spherical, P):
    q = _c(q, np.float32)
    cr = _c(c_rank, np.float32)
    probes = np.zeros(P, np.int32)
    scores = np.zeros(P, np.float64)
    P = lib().orc_rank(q, len(q), cr, cr.shape[0], int(spherical), P, probes, _ptr(scores))
    return probes[:P], scores[:P]


def adc64(q, ix, p, code):
    return lib().orc_adc64(_c(q, np.float32), ix["d"], ix["M"], _c(ix["c_mean"][p], np.float32),
                           ix["codebook"], _c(code, np.uint8), int(ix["ip"]))


def lut_q8(q, ix, probes):
    probes = _c(probes, np.int32)
    P, M = len(probes), ix["M"]
    Q = np.zeros((P, M, K), np.uint8)
    bias = np.zeros(P, np.int32)
    a = C.c_float(0)
    lib().orc_lut_q8(_c(q, np.float32), ix["d"], M, ix["c_mean"], ix["codebook"], int(ix["ip"]),
                     probes, P, Q, bias, C.byref(a))
    return Q, bias, a.value


def int_dist(Qp, bias_p, code):
    return lib().orc_int_dist(_c(Qp, np.uint8), int(bias_p), _c(code, np.uint8), len(code))


def scan_topr(ix, probes, Q, bias, R):
    probes = _c(probes, np.int32)
    keys = np.zeros(max(R, 1), np.uint64)
    cnt = lib().orc_scan_topr(ix["codes"], ix["M"], ix["list_off"], ix["list_ids"], probes,
                              len(probes), _c(Q, np.uint8), _c(bias, np.int32), R, keys)
    return keys[:cnt]


def key_dist(keys):
    """Integer distance D carried in the high word of a candidate key."""
    return ((keys >> np.uint64(32)).astype(np.int64) - (1 << 31)).astype(np.int64)


def key_id(keys):
    return (keys & np.uint64(0xFFFFFFFF)).astype(np.int64)


def build_graph(ix):
    n = ix["n"]
    g = np.zeros((n, 32), np.int32)
    entry = np.zeros(ix["L"], np.int32)
    lib().orc_build_graph(ix["X"], ix["d"], ix["list_off"], ix["list_ids"], ix["L"],
                          ix["c_mean"], g, entry)
    return g, entry


def graph_search(ix, graph, entry_c, Qp, bias_p, efs):
    W = np.zeros(max(efs, 1), np.uint64)
    cnt = lib().orc_graph_search(ix["codes"], ix["M"], _c(graph, np.int32), int(entry_c),
                                 _c(Qp, np.uint8), int(bias_p), efs, ix["n"], W)
    return W[:cnt]


def hybrid_topr(ix, graph, entry, probes, Q, bias, R, n_near=2, efs=64, tau=8):
    probes = _c(probes, np.int32)
    keys = np.zeros(max(R, 1), np.uint64)
    nf = C.c_int32(0)
    cnt = lib().orc_hybrid_topr(ix["codes"], ix["M"], ix["list_off"], ix["list_ids"], ix["n"],
                                _c(graph, np.int32), _c(entry, np.int32), probes, len(probes),
                                _c(Q, np.uint8), _c(bias, np.int32), R, n_near, efs, tau, keys,
                                C.byref(nf))
    return keys[:cnt], nf.value


def rerank(q, ix, cand_ids, k):
    cand_ids = _c(cand_ids, np.int32)
    ids = np.zeros(k, np.int64)
    dd = np.zeros(k, np.float64)
    lib().orc_rerank(_c(q, np.float32), ix["X"], ix["d"], int(ix["ip"]), cand_ids, len(cand_ids),
                     k, ids, dd)
    return ids, dd


def exact_knn(Q, X, k, ip=False, nthreads=0):
    Q = _c(Q, np.float32)
    X = _c(X, np.float32)
    ids = np.zeros((Q.shape[0], k), np.int64)
    dd = np.zeros((Q.shape[0], k), np.float64)
    lib().orc_exact_knn(Q, Q.shape[0], X, X.shape[0], X.shape[1], int(ip), k, ids, dd, nthreads)
    return ids, dd


def search(ix, Q, nprobe, R, k, nthreads=0, want_probes=False, want_cands=False):
    """Alg. 2 (plain leaf scan): per-query nprobe / R may be scalars or arrays."""
    Q = _c(Q, np.float32)
    nq = Q.shape[0]
    npb = _c(np.broadcast_to(nprobe, (nq,)), np.int32)
    Rr = _c(np.broadcast_to(R, (nq,)), np.int32)
    ids = np.zeros((nq, k), np.int64)
    dd = np.zeros((nq, k), np.float64)
    pstride = int(npb.max()) if want_probes else 0
    rstride = int(max(Rr.max(), k)) if want_cands else 0
    probes = np.zeros((nq, max(pstride, 1)), np.int32) if want_probes else None
    cands = np.zeros((nq, max(rstride, 1)), np.uint64) if want_cands else None
    ncand = np.zeros(nq, np.int64) if want_cands else None
    lib().orc_search(Q, nq, ix["d"], ix["M"], ix["L"], int(ix["ip"]), int(ix["spherical"]),
                     ix["X"], ix["c_rank"], ix["c_mean"], ix["codebook"], ix["codes"],
                     ix["list_off"], ix["list_ids"], npb, Rr, k, ids, dd,
                     _ptr(probes), pstride, _ptr(cands), rstride, _ptr(ncand), nthreads)
    out = dict(ids=ids, dists=dd)
    if want_probes:
        out["probes"] = probes
    if want_cands:
        out["cands"], out["ncand"] = cands, ncand
    return out


def recall(Q, X, ids, true_d, k=10, ip=False):
    Q = _c(Q, np.float32)
    ids = _c(ids, np.int64)
    true_d = _c(true_d, np.float64)
    return lib().orc_recall(Q, Q.shape[0], _c(X, np.float32), Q.shape[1], int(ip), ids,
                            ids.shape[1], true_d, true_d.shape[1], k)


# -------------------------------------------------------------- learned part
def eq2(p, pmin, pmax, p0, p1):
    return lib().orc_eq2(float(p), int(pmin), int(pmax), float(p0), float(p1))


def reg_map(p, lo, hi, a=0.0, b=0.0):
    """Regression heads: p read as the normalised log of the setting."""
    return lib().orc_reg_map(float(p), int(lo), int(hi), float(a), float(b))


def reg_target(v, lo, hi):
    """Training target of a regression head: the normalised log of a label."""
    return (np.log(np.asarray(v, np.float64)) - np.log(lo)) / (np.log(hi) - np.log(lo))


def mlp_nparams(F, H1, H2):
    return H1 * F + H1 + H2 * H1 + H2 + 2 * H2 + 2


def mlp_forward(w, F, H1, H2, x):
    x = _c(x, np.float64)
    prob = np.zeros((x.shape[0], 2), np.float64)
    lib().orc_mlp_forward(_c(w, np.float64), F, H1, H2, x, x.shape[0], prob)
    return prob


def mlp_grad(w, F, H1, H2, x, y):
    x = _c(x, np.float64)
    g = np.zeros(mlp_nparams(F, H1, H2), np.float64)
    loss = lib().orc_mlp_grad(_c(w, np.float64), F, H1, H2, x, _c(y, np.float64), x.shape[0], g)
    return loss, g


def adam_step(w, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """In place on w, m, v (float64 arrays)."""
    lib().orc_adam_step(w, _c(g, np.float64), m, v, len(w), t, lr, beta1, beta2, eps)


# -------------------------------------------------------------- cluster pruning
PRUNE_NSTAT, PRUNE_NFEAT = 12, 16
PRUNE_H = 32  # hidden units of the pruning classifier (F -> 32 -> 32 -> 2, head 0 used)


def prune_stats(X, c_mean, assign, iters=30):
    """Per-list statistics [L x 12] and vectors [L x 3 x d] (Sec. 4.2.3, Table 4):
    size, radius, mean / std of the member distances to the mean centroid, the
    distance histogram (4 bins over [0, radius]), the outlier fraction (beyond
    mean + 2 std), the variances along the two principal axes; the axes and the
    mean outlier offset."""
    X = _c(X, np.float32)
    c_mean = _c(c_mean, np.float32)
    L, d = c_mean.shape
    st = np.zeros((L, PRUNE_NSTAT), np.float64)
    vec = np.zeros((L, 3, d), np.float64)
    lib().orc_prune_stats(X, X.shape[0], d, c_mean, L, _c(assign, np.int32), int(iters), st, vec)
    return st, vec


def prune_features(Q, c_mean, probes, stats, vecs, P=None, nprobe=None):
    """Features [nq x Pmax x 16] of every (query, probe rank < P_q) (Table 4)."""
    Q = _c(Q, np.float32)
    probes = _c(probes, np.int32)
    nq, Pmax = probes.shape
    c_mean = _c(c_mean, np.float32)
    npb = None if nprobe is None else _c(nprobe, np.int32)
    out = np.zeros((nq, Pmax, PRUNE_NFEAT), np.float64)
    lib().orc_prune_features(Q, nq, Q.shape[1], c_mean, c_mean.shape[0], probes, Pmax, _ptr(npb),
                             int(P if P is not None else Pmax), _c(stats, np.float64), _c(vecs, np.float64), out)
    return out


def prune_prob(feats, mu, sd, w):
    """Keep probability of every row: the classifier's head 0 on the
    standardised features (f - mu) / sd (Alg. 2 f_prune)."""
    F = feats.shape[-1]
    x = (np.asarray(feats, np.float64).reshape(-1, F) - mu) / sd
    return mlp_forward(w, F, PRUNE_H, PRUNE_H, x)[:, 0].reshape(feats.shape[:-1])


def prune_keep(prob, theta, P=None, nprobe=None):
    """Alg. 2: a probe is searched when f_prune > theta; the nearest probe
    (rank 0) is always searched.  Returns the kept probe ranks per query."""
    nq, Pmax = prob.shape
    out = []
    for q in range(nq):
        Pq = int(nprobe[q]) if nprobe is not None else int(P if P is not None else Pmax)
        Pq = min(max(Pq, 1), Pmax)
        out.append([r for r in range(Pq) if r == 0 or prob[q, r] > theta])
    return out


def prune_labels(ids, dists, kth, assign, probes, P, ip=False, tol=1e-5):
    """Training label of (query, probe rank): 1 when the list holds one of the
    query's true k nearest neighbours that the search returned (distance at
    most the true k-th, up to tol relative)."""
    nq, Pmax = probes.shape
    y = np.zeros((nq, Pmax), np.float64)
    for q in range(nq):
        t = kth[q]
        tl = tol * abs(t) + 1e-6
        lists = set()
        for i, dv in zip(ids[q], dists[q]):
            if i < 0:
                continue
            if (dv >= t - tl) if ip else (dv <= t + tl):
                lists.add(int(assign[i]))
        for r in range(min(P, Pmax)):
            y[q, r] = 1.0 if int(probes[q, r]) in lists else 0.0
    return y


# -------------------------------------------------------------- component filtration
def component_stats(X):
    """Per-dimension mean, std and the fraction of values that are 0 or within
    one std of the mean (Sec. 4.3), FP64."""
    X = _c(X, np.float32)
    n, d = X.shape
    mu, sd, fr = np.zeros(d), np.zeros(d), np.zeros(d)
    lib().orc_component_stats(X, n, d, mu, sd, fr)
    return mu, sd, fr


def component_keep(frac, threshold):
    """Dimensions kept by FilterComponents (Alg. 1): those whose fraction is
    at most the threshold, ascending."""
    return np.nonzero(np.asarray(frac) <= threshold)[0].astype(np.int32)


def component_dims(kept, M):
    """The kept dimensions followed by -1 (a zero dimension) up to a multiple
    of M, so that the M subspaces divide the filtered vectors."""
    kept = np.asarray(kept, np.int32)
    dp = -(-len(kept) // M) * M
    return np.concatenate([kept, -np.ones(dp - len(kept), np.int32)])


def filter_rows(A, dims):
    """A[:, dims] with zeros at the -1 entries."""
    A = np.asarray(A, np.float32)
    out = np.zeros((A.shape[0], len(dims)), np.float32)
    sel = dims >= 0
    out[:, sel] = A[:, dims[sel]]
    return out
