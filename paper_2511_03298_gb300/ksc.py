"""Thin ctypes binding of the CUDA library (include/kscann.h).

Argument marshalling only: every step of the search runs in the library's
kernels.  Device arrays are torch CUDA tensors (plumbing for memory and
streams); the calls run on torch's current stream.  Importing this module
does not load the library; the first call does, and fails loudly if the
library has not been built (`__graft_entry__.build()`).
"""
import ctypes as C
import os

import numpy as np

from .build_ext import LIB

_lib = None

KSC_L2, KSC_IP = 0, 1
STATUS_CAND_OVERFLOW = 1
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "EUNSUPPORTED", -5: "ETIMEOUT", -6: "ESTATE"}


class KscError(RuntimeError):
    """A non-zero ksc_status with the library's message (ksc_last_error)."""

    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class BuildOpts(C.Structure):
    """ksc_build_opts: k-means iterations, spherical ranking, build permutation,
    seed, intra-list graphs, component-filtration threshold (Alg. 1, Sec. 4.3)."""
    _fields_ = [("kmeans_iters", C.c_int32), ("spherical", C.c_int32), ("perm_host", C.c_void_p),
                ("seed", C.c_uint64), ("build_graph", C.c_int32), ("filter_threshold", C.c_float)]


class IndexArrays(C.Structure):
    """ksc_index_arrays: sizes and host pointers of an index's interchange arrays."""
    _fields_ = [("n", C.c_int64), ("d", C.c_int32), ("nlist", C.c_int32), ("M", C.c_int32),
                ("metric", C.c_int32), ("spherical", C.c_int32),
                ("X", C.c_void_p), ("c_rank", C.c_void_p), ("c_mean", C.c_void_p), ("codebook", C.c_void_p),
                ("codes", C.c_void_p), ("assign", C.c_void_p), ("graph", C.c_void_p), ("entry", C.c_void_p)]


class AdaptiveParams(C.Structure):
    """ksc_adaptive_params: Eq. 2's bounds and offsets for nprobe and rerank."""
    _fields_ = [("pmin", C.c_int32), ("pmax", C.c_int32), ("rmin", C.c_int32), ("rmax", C.c_int32),
                ("p0", C.c_float), ("p1", C.c_float), ("r0", C.c_float), ("r1", C.c_float),
                ("regression", C.c_int32)]


class TrainOpts(C.Structure):
    """ksc_train_opts: labels (k, target hits, label grids) and training schedule."""
    _fields_ = [("k", C.c_int32), ("target_hits", C.c_int32), ("rerank_label", C.c_int32), ("epochs", C.c_int32),
                ("batch", C.c_int32), ("lr", C.c_float), ("seed", C.c_uint64), ("grid_host", C.c_void_p),
                ("ngrid", C.c_int32), ("rgrid_host", C.c_void_p), ("nrgrid", C.c_int32), ("regression", C.c_int32)]


class SearchOpts(C.Structure):
    """ksc_search_opts (see search_opts() for the fields' meaning)."""
    _fields_ = [("lanes_per_query", C.c_int32), ("hybrid", C.c_int32), ("n_near", C.c_int32),
                ("efs", C.c_int32), ("tau", C.c_int32), ("cand_cap", C.c_int32), ("rank_fp32", C.c_int32),
                ("precision", C.c_int32), ("rerank_final", C.c_int32), ("tile_blocks", C.c_int32),
                ("scan_tc", C.c_int32), ("rank_fp8", C.c_int32), ("rerank_band", C.c_int32)]


_vp, _i32, _i64 = C.c_void_p, C.c_int32, C.c_int64
_SIGS = {
    "ksc_build_index": [_vp, _i64, _i32, _i32, _i32, _i32, _i32, _vp, _vp, _vp],
    "ksc_index_free": [_vp],
    "ksc_index_import": [_vp, _vp, _vp],
    "ksc_index_info": [_vp, _vp],
    "ksc_index_export": [_vp, _vp],
    "ksc_index_save": [_vp, C.c_char_p],
    "ksc_index_load": [C.c_char_p, _vp, _vp],
    "ksc_search": [_vp, _vp, _i64, _i32, _i32, _i32, _vp, _vp, _vp, _vp],
    "ksc_search_varprobe": [_vp, _vp, _i64, _i32, _vp, _i32, _vp, _i32, _vp, _vp, _vp, _vp],
    "ksc_search_with_probes": [_vp, _vp, _i64, _vp, _i32, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp],
    "ksc_rank_lists": [_vp, _vp, _i64, _i32, _vp, _vp, _vp],
    "ksc_compute_luts": [_vp, _vp, _i64, _vp, _i32, _vp, _vp, _vp, _vp],
    "ksc_list_scores": [_vp, _vp, _i64, _i32, _vp, _vp, _vp],
    "ksc_compute_luts_noalloc": [_vp, _vp, _i64, _vp, _i32, _vp, _vp, _vp, _vp],
    "ksc_last_status": [_vp, _vp],
    "ksc_search_stats": [_vp, _vp],
    "ksc_plan_create": [_vp, _i64, _i32, _i32, _i32, _i32, _vp, _vp, _vp],
    "ksc_plan_execute": [_vp, _vp, _vp, _vp, _vp],
    "ksc_plan_buffers": [_vp, _vp, _vp, _vp],
    "ksc_plan_free": [_vp],
    "ksc_autotune": [_vp, _vp, _i64, _i32, _i32, _i32, _vp, _vp, _vp],
    "ksc_pair_distances": [_vp, _vp, _i64, _vp, _i32, _i32, _vp, _vp],
    "ksc_profile_enable": [_vp, _i32],
    "ksc_profile_read": [_vp, _vp, _i32, _vp],
    "ksc_lut16_peak": [_vp, _vp],
    "ksc_train_predictor": [_vp, _vp, _i64, _vp, _vp, _vp, _vp],
    "ksc_predictor_params": [_vp, _vp],
    "ksc_predictor_weights": [_vp, _vp, _vp],
    "ksc_search_adaptive": [_vp, _vp, _i64, _i32, _vp, _vp, _vp, _vp, _vp, _vp],
    "ksc_query_features": [_vp, _vp, _i64, _vp, _vp],
    "ksc_mlp_grad": [_vp, _vp, _vp, _i64, _vp, _vp, _vp],
    "ksc_mlp_forward": [_vp, _vp, _i64, _vp, _vp],
    "ksc_pruner_stats": [_vp, _i32, _vp],
    "ksc_pruner_export": [_vp, _vp, _vp, _vp],
    "ksc_pruner_import_model": [_vp, _vp],
    "ksc_prune_probes": [_vp, _vp, _i64, _vp, _i32, _vp, _i32, C.c_float, _vp, _vp, _vp, _vp, _vp],
    "ksc_prune_labels": [_vp, _vp, _vp, _i64, _i32, _vp, _vp, _i32, _i32, _vp, _vp],
    "ksc_train_pruner": [_vp, _vp, _i64, _vp, _i32, _i32, _i32, _vp, _vp, _vp],
    "ksc_search_pruned": [_vp, _vp, _i64, _i32, _i32, _i32, C.c_float, _vp, _vp, _vp, _vp, _vp],
    "ksc_prune_mlp_grad": [_vp, _vp, _vp, _i64, _vp, _vp, _vp],
    "ksc_pruner_theta": [_vp, C.c_float],
    "ksc_index_dims": [_vp, _vp, _vp],
    "ksc_index_view": [_vp, _vp],
    "ksc_component_stats": [_vp, _i64, _i32, _vp, _vp, _vp, _vp],
    "ksc_index_import_shard": [_vp, _vp, _i32, _vp, _vp],
    "ksc_shard_candidates": [_vp, _vp, _i64, _i32, _i32, _i32, _vp, _vp, _vp],
    "ksc_shard_rerank": [_vp, _vp, _i64, _i32, _i32, _vp, _vp, _i32, _vp, _vp, _vp],
    "ksc_merge_topk": [_vp, _vp, _i64, _i32, _i32, _i32, _vp, _vp, _vp],
    "ksc_last_error": [],
    "ksc_version": [],
}


def lib_path():
    """Path of the in-tree shared library."""
    return LIB


def lib():
    """The loaded library (loaded once; raises if it is not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError("CUDA library %s is missing: run __graft_entry__.build() first" % LIB)
        L = C.CDLL(LIB)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int
        L.ksc_last_error.restype = C.c_char_p
        L.ksc_version.restype = C.c_char_p
        L.ksc_index_free.restype = None
        L.ksc_plan_free.restype = None
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise KscError(rc, lib().ksc_last_error().decode())


def _torch():
    import torch
    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dptr(t, dtype=None, name="tensor"):
    torch = _torch()
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise ValueError("%s must be a contiguous CUDA tensor" % name)
    if dtype is not None and t.dtype != dtype:
        raise ValueError("%s must have dtype %s" % (name, dtype))
    return C.c_void_p(t.data_ptr())


def _hptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def search_opts(lanes_per_query=0, hybrid=False, n_near=2, efs=64, tau=8, cand_cap=0, rank_fp32=False,
                precision=0, rerank_final=0, tile_blocks=0, scan_tc=False, rank_fp8=False, rerank_band=0):
    """precision: 0 FP32 re-rank; 1 BF16 / 2 FP8 first re-rank of the widened
    shortlist, then FP32 over the best rerank_final.  scan_tc: the scan on
    the tensor cores (same keys).  rank_fp8: list scores from FP8 operands
    (same ranking).  rerank_band: 1 the exact re-rank reads U8 rows (exact,
    when every coordinate is an integer in [0, 255]) or BF16 rows first and
    FP32 rows only where its bound cannot exclude a candidate (same results),
    -1 FP32 rows of every candidate, 0 auto (the band for L2)."""
    return SearchOpts(lanes_per_query, int(hybrid), n_near, efs, tau, cand_cap, int(rank_fp32), precision,
                      rerank_final, tile_blocks, int(scan_tc), int(rank_fp8), int(rerank_band))


class Index:
    """An index resident on the GPU (owned by the library)."""

    def __init__(self, handle):
        self._h = C.c_void_p(handle)

    def __del__(self):
        self.free()

    def free(self):
        """Release the index's device memory (ksc_index_free); idempotent."""
        if getattr(self, "_h", None) and self._h.value and _lib is not None:
            _lib.ksc_index_free(self._h)
        self._h = C.c_void_p(None)

    @property
    def handle(self):
        """The opaque ksc_index* as a ctypes pointer."""
        return self._h

    def info(self):
        """n, d, nlist, M, metric and spherical of the index (ksc_index_info)."""
        a = IndexArrays()
        _check(lib().ksc_index_info(self._h, C.byref(a)))
        return dict(n=a.n, d=a.d, nlist=a.nlist, M=a.M, metric=a.metric, spherical=a.spherical)

    def view(self):
        """Another handle on the same index data with its own workspace, for
        searches on another stream at the same time (freed before this one)."""
        h = C.c_void_p()
        _check(lib().ksc_index_view(self._h, C.byref(h)))
        v = Index(h.value)
        v._source = self  # keeps this handle alive until the view is freed
        return v

    def dims(self):
        """(query width d, working dimension list: the query dimension of each
        working one, -1 for a zero padding dimension)."""
        inf = self.info()
        dfull = C.c_int32(0)
        dims = np.zeros(inf["d"], np.int32)
        _check(lib().ksc_index_dims(self._h, _hptr(dims), C.byref(dfull)))
        return dfull.value, dims

    def export(self, with_graph=False, fields=None):
        """Copy the index's interchange arrays to the host; `fields` (a subset
        of X, c_rank, c_mean, codebook, codes, assign) limits the copy."""
        inf = self.info()
        n, d, L, M = inf["n"], inf["d"], inf["nlist"], inf["M"]
        shapes = dict(X=((n, d), np.float32), c_rank=((L, d), np.float32), c_mean=((L, d), np.float32),
                      codebook=((M, 16, d // M), np.float32), codes=((n, M), np.uint8), assign=((n,), np.int32))
        out = {k: np.zeros(*v) for k, v in shapes.items() if fields is None or k in fields}
        if with_graph:
            out["graph"] = np.zeros((n, 32), np.int32)
            out["entry"] = np.zeros(L, np.int32)
        a = IndexArrays(n, d, L, M, inf["metric"], inf["spherical"],
                        *[_hptr(out.get(k)) for k in ("X", "c_rank", "c_mean", "codebook", "codes", "assign",
                                                      "graph", "entry")])
        _check(lib().ksc_index_export(self._h, C.byref(a)))
        out.update(inf)
        return out

    def save(self, path):
        """Write the index (and its graph, models and filtration state) to a file."""
        _check(lib().ksc_index_save(self._h, os.fsencode(path)))

    def search(self, Q, k, nprobe, rerank, opts=None, out=None, stream=None):
        """Alg. 2 with a fixed nprobe (ksc_search): Q [nq x d] fp32 on the device;
        returns ids [nq x k] int64 and dists [nq x k] fp32 (into `out` if given)."""
        torch = _torch()
        nq = Q.shape[0]
        ids, dists = out if out is not None else (
            torch.empty((nq, k), dtype=torch.int64, device=Q.device),
            torch.empty((nq, k), dtype=torch.float32, device=Q.device))
        _check(lib().ksc_search(self._h, _dptr(Q, torch.float32, "Q"), nq, k, nprobe, rerank,
                                _dptr(ids), _dptr(dists), C.byref(opts) if opts else None, _stream(stream)))
        return ids, dists

    def search_varprobe(self, Q, k, nprobe, rerank, nprobe_max=None, rerank_max=None, opts=None, stream=None):
        """Alg. 2 with per-query nprobe / rerank (int32 device tensors [nq]),
        bounded by nprobe_max / rerank_max (ksc_search_varprobe)."""
        torch = _torch()
        nq = Q.shape[0]
        ids = torch.empty((nq, k), dtype=torch.int64, device=Q.device)
        dists = torch.empty((nq, k), dtype=torch.float32, device=Q.device)
        pm = int(nprobe.max().item()) if nprobe_max is None else nprobe_max
        rm = int(rerank.max().item()) if rerank_max is None else rerank_max
        _check(lib().ksc_search_varprobe(self._h, _dptr(Q, torch.float32, "Q"), nq, k,
                                         _dptr(nprobe, torch.int32, "nprobe"), pm,
                                         _dptr(rerank, torch.int32, "rerank"), rm,
                                         _dptr(ids), _dptr(dists), C.byref(opts) if opts else None,
                                         _stream(stream)))
        return ids, dists

    def search_with_probes(self, Q, probes, k, rerank, want_cands=True, opts=None, stream=None):
        """Steps a2-a6 on given probe lists (int32 [nq x P], ranked); also the
        candidate keys [nq x R] and their counts (ksc_search_with_probes)."""
        torch = _torch()
        nq, P = probes.shape
        R = max(rerank, k)
        ids = torch.empty((nq, k), dtype=torch.int64, device=Q.device)
        dists = torch.empty((nq, k), dtype=torch.float32, device=Q.device)
        cand = torch.empty((nq, R), dtype=torch.int64, device=Q.device) if want_cands else None
        ncand = torch.empty((nq,), dtype=torch.int32, device=Q.device) if want_cands else None
        _check(lib().ksc_search_with_probes(self._h, _dptr(Q, torch.float32, "Q"), nq,
                                            _dptr(probes, torch.int32, "probes"), P, k, rerank,
                                            _dptr(ids), _dptr(dists), _dptr(cand), _dptr(ncand),
                                            C.byref(opts) if opts else None, _stream(stream)))
        return ids, dists, cand, ncand

    def shard_candidates(self, Q, k, nprobe, rerank, opts=None, stream=None):
        """Shard step 1: the shard's R = max(rerank, k) smallest keys per
        query (global ids), [nq x R] int64 holding the uint64 keys."""
        torch = _torch()
        nq = Q.shape[0]
        keys = torch.empty((nq, max(rerank, k)), dtype=torch.int64, device=Q.device)
        _check(lib().ksc_shard_candidates(self._h, _dptr(Q, torch.float32, "Q"), nq, nprobe, rerank, k, _dptr(keys),
                                          C.byref(opts) if opts else None, _stream(stream)))
        return keys

    def shard_rerank(self, Q, k, rerank, own_keys, all_keys, stream=None):
        """Shard step 2: all_keys [parts x nq x R] from every shard; the
        shard's k best (global ids, distances) among the whole index's R
        best keys."""
        torch = _torch()
        nq = Q.shape[0]
        ids = torch.empty((nq, k), dtype=torch.int64, device=Q.device)
        dists = torch.empty((nq, k), dtype=torch.float32, device=Q.device)
        _check(lib().ksc_shard_rerank(self._h, _dptr(Q, torch.float32, "Q"), nq, k, rerank,
                                      _dptr(own_keys, torch.int64, "own_keys"), _dptr(all_keys, torch.int64, "all_keys"),
                                      all_keys.shape[0], _dptr(ids), _dptr(dists), _stream(stream)))
        return ids, dists

    def rank_lists(self, Q, P, want_scores=True, stream=None):
        """Alg. 2 TopNClusters: the P nearest lists per query, ranked, and their
        exact FP32 scores (ksc_rank_lists)."""
        torch = _torch()
        nq = Q.shape[0]
        probes = torch.empty((nq, P), dtype=torch.int32, device=Q.device)
        scores = torch.empty((nq, P), dtype=torch.float32, device=Q.device) if want_scores else None
        _check(lib().ksc_rank_lists(self._h, _dptr(Q, torch.float32, "Q"), nq, P, _dptr(probes),
                                    _dptr(scores), _stream(stream)))
        return probes, scores

    def list_scores(self, Q, tensor_cores=True, stream=None):
        """Raw step-a1 scores [nq x L] and their per-query error bound [nq];
        tensor_cores: 0 / False FP32 CUDA cores, 1 / True 16-bit, 2 FP8."""
        torch = _torch()
        nq = Q.shape[0]
        L = self.info()["nlist"]
        scores = torch.empty((nq, L), dtype=torch.float32, device=Q.device)
        err = torch.empty((nq,), dtype=torch.float32, device=Q.device)
        _check(lib().ksc_list_scores(self._h, _dptr(Q, torch.float32, "Q"), nq, int(tensor_cores), _dptr(scores),
                                     _dptr(err), _stream(stream)))
        return scores, err

    def compute_luts(self, Q, probes, stream=None):
        """Step a2: the 8-bit residual tables [nq x P x M x 16], biases and
        per-query scales of the given probes (Sec. 2.5, Sec. 4.6.1; ksc_compute_luts)."""
        torch = _torch()
        nq, P = probes.shape
        M = self.info()["M"]
        lut = torch.empty((nq, P, M, 16), dtype=torch.uint8, device=Q.device)
        bias = torch.empty((nq, P), dtype=torch.int32, device=Q.device)
        scale = torch.empty((nq,), dtype=torch.float32, device=Q.device)
        _check(lib().ksc_compute_luts(self._h, _dptr(Q, torch.float32, "Q"), nq,
                                      _dptr(probes, torch.int32, "probes"), P, _dptr(lut), _dptr(bias),
                                      _dptr(scale), _stream(stream)))
        return lut, bias, scale

    # ---------------------------------------------------------- learned predictor
    def train_predictor(self, Qtrain, kth, k=10, target_hits=9, rerank_label=200, epochs=8, batch=256, lr=1e-3,
                        seed=0, grid=None, rgrid=None, regression=False, stream=None):
        """Train the nprobe / rerank MLP on training queries and their true
        k-th neighbour distances (device tensors).  Returns the mean loss of
        the last epoch."""
        torch = _torch()
        g = None if grid is None else np.ascontiguousarray(grid, dtype=np.int32)
        r = None if rgrid is None else np.ascontiguousarray(rgrid, dtype=np.int32)
        opts = TrainOpts(k, target_hits, rerank_label, epochs, batch, lr, seed, _hptr(g),
                         0 if g is None else len(g), _hptr(r), 0 if r is None else len(r), int(regression))
        loss = C.c_float(0)
        _check(lib().ksc_train_predictor(self._h, _dptr(Qtrain, torch.float32, "Qtrain"), Qtrain.shape[0],
                                         _dptr(kth, torch.float32, "kth"), C.byref(opts), _stream(stream),
                                         C.byref(loss)))
        return loss.value

    def set_predictor_params(self, pmin, pmax, rmin, rmax, p0, p1, r0, r1, regression=False):
        """regression: the heads' outputs are normalised logs of the settings
        (a model trained with regression=True) instead of Eq. 2's input."""
        _check(lib().ksc_predictor_params(self._h, C.byref(AdaptiveParams(pmin, pmax, rmin, rmax, p0, p1, r0, r1,
                                                                           int(regression)))))

    def predictor_weights(self, set_to=None):
        """The learned predictor's FP32 parameters (8450 values): read them, or
        set them from `set_to` (ksc_predictor_weights)."""
        if set_to is not None:
            w = np.ascontiguousarray(set_to, dtype=np.float32)
            _check(lib().ksc_predictor_weights(self._h, None, _hptr(w)))
            return w
        w = np.zeros(8450, np.float32)
        _check(lib().ksc_predictor_weights(self._h, _hptr(w), None))
        return w

    def search_adaptive(self, Q, k, opts=None, stream=None):
        """Alg. 2 with nprobe and rerank per query from the learned predictor and
        Eq. 2; returns ids, dists and the settings used (ksc_search_adaptive)."""
        torch = _torch()
        nq = Q.shape[0]
        ids = torch.empty((nq, k), dtype=torch.int64, device=Q.device)
        dists = torch.empty((nq, k), dtype=torch.float32, device=Q.device)
        npb = torch.empty((nq,), dtype=torch.int32, device=Q.device)
        rr = torch.empty((nq,), dtype=torch.int32, device=Q.device)
        _check(lib().ksc_search_adaptive(self._h, _dptr(Q, torch.float32, "Q"), nq, k, _dptr(ids), _dptr(dists),
                                         _dptr(npb), _dptr(rr), C.byref(opts) if opts else None, _stream(stream)))
        return ids, dists, npb, rr

    def query_features(self, Q, stream=None):
        """The predictor's 64 input features per query [nq x 64] (ksc_query_features)."""
        torch = _torch()
        f = torch.empty((Q.shape[0], 64), dtype=torch.float32, device=Q.device)
        _check(lib().ksc_query_features(self._h, _dptr(Q, torch.float32, "Q"), Q.shape[0], _dptr(f),
                                        _stream(stream)))
        return f

    # ---------------------------------------------------------- cluster pruning (Sec. 4.2.3)
    PRUNE_STATS, PRUNE_FEATURES, PRUNE_NPARAMS = 12, 16, 1666
    PRUNE_MODEL = PRUNE_NPARAMS + 2 * PRUNE_FEATURES

    def pruner_stats(self, iters=30, stream=None):
        """Per-list statistics of the pruning features (build time)."""
        _check(lib().ksc_pruner_stats(self._h, iters, _stream(stream)))

    def pruner_export(self, model=True):
        """Statistics [L x 12], vectors [L x 3 x d] and, if trained, the model."""
        inf = self.info()
        st = np.zeros((inf["nlist"], self.PRUNE_STATS), np.float32)
        vec = np.zeros((inf["nlist"], 3, inf["d"]), np.float32)
        mdl = np.zeros(self.PRUNE_MODEL, np.float32) if model else None
        _check(lib().ksc_pruner_export(self._h, _hptr(st), _hptr(vec), _hptr(mdl)))
        return st, vec, mdl

    def pruner_model(self, set_to=None):
        """Set (set_to: weights, feature means, feature stds) or read the model."""
        if set_to is not None:
            m = np.ascontiguousarray(set_to, dtype=np.float32)
            assert m.size == self.PRUNE_MODEL
            _check(lib().ksc_pruner_import_model(self._h, _hptr(m)))
            return m
        m = np.zeros(self.PRUNE_MODEL, np.float32)
        _check(lib().ksc_pruner_export(self._h, None, None, _hptr(m)))
        return m

    def prune_probes(self, Q, probes, P=None, nprobe=None, theta=0.5, feats=False, prob=False, kept=True,
                     stream=None):
        """Features / keep probabilities / kept probes (rank order, -1 after)
        and their count for given probes [nq x Pmax]; returns a dict."""
        torch = _torch()
        nq, Pmax = probes.shape
        dev = Q.device
        out = {}
        if feats:
            out["feats"] = torch.empty((nq, Pmax, self.PRUNE_FEATURES), dtype=torch.float32, device=dev)
        if prob:
            out["prob"] = torch.empty((nq, Pmax), dtype=torch.float32, device=dev)
        if kept:
            out["probes"] = torch.empty((nq, Pmax), dtype=torch.int32, device=dev)
            out["nprobe"] = torch.empty((nq,), dtype=torch.int32, device=dev)
        _check(lib().ksc_prune_probes(self._h, _dptr(Q, torch.float32, "Q"), nq, _dptr(probes, torch.int32, "probes"),
                                      Pmax, _dptr(nprobe, torch.int32, "nprobe"), int(P or Pmax), float(theta),
                                      _dptr(out.get("feats")), _dptr(out.get("prob")), _dptr(out.get("probes")),
                                      _dptr(out.get("nprobe")), _stream(stream)))
        return out

    def prune_labels(self, ids, dists, kth, probes, P, stream=None):
        """Training labels of the pruning classifier per (query, probe rank): 1
        where the list holds a returned id whose distance is within the true
        k-th distance kth, else 0 (ksc_prune_labels)."""
        torch = _torch()
        nq, Pmax = probes.shape
        lab = torch.empty((nq, Pmax), dtype=torch.float32, device=ids.device)
        _check(lib().ksc_prune_labels(self._h, _dptr(ids, torch.int64, "ids"), _dptr(dists, torch.float32, "dists"),
                                      nq, ids.shape[1], _dptr(kth, torch.float32, "kth"),
                                      _dptr(probes, torch.int32, "probes"), Pmax, int(P), _dptr(lab),
                                      _stream(stream)))
        return lab

    def train_pruner(self, Qtrain, kth, k=10, P=16, R=200, epochs=4, batch=1024, lr=1e-3, seed=0, stream=None):
        """Train the pruning classifier on training queries and their true
        k-th neighbour distances (device tensors).  Returns the mean loss of
        the last epoch."""
        torch = _torch()
        opts = TrainOpts(k, 0, 0, epochs, batch, lr, seed, None, 0, None, 0)
        loss = C.c_float(0)
        _check(lib().ksc_train_pruner(self._h, _dptr(Qtrain, torch.float32, "Qtrain"), Qtrain.shape[0],
                                      _dptr(kth, torch.float32, "kth"), k, P, R, C.byref(opts), _stream(stream),
                                      C.byref(loss)))
        return loss.value

    def pruner_theta(self, theta):
        """Pruning threshold of the adaptive search (< 0: off)."""
        _check(lib().ksc_pruner_theta(self._h, float(theta)))

    def search_pruned(self, Q, k, nprobe, rerank, theta, opts=None, out=None, stream=None):
        """ksc_search with the lists the pruning model rejects at theta
        dropped; returns ids, dists and the lists searched per query."""
        torch = _torch()
        nq = Q.shape[0]
        ids, dists = out if out is not None else (
            torch.empty((nq, k), dtype=torch.int64, device=Q.device),
            torch.empty((nq, k), dtype=torch.float32, device=Q.device))
        npb = torch.empty((nq,), dtype=torch.int32, device=Q.device)
        _check(lib().ksc_search_pruned(self._h, _dptr(Q, torch.float32, "Q"), nq, k, nprobe, rerank, float(theta),
                                       _dptr(ids), _dptr(dists), _dptr(npb), C.byref(opts) if opts else None,
                                       _stream(stream)))
        return ids, dists, npb

    # ---------------------------------------------------------- plans, autotuner
    def plan(self, nq, k, nprobe=1, rerank=0, adaptive=False, opts=None, stream=None):
        """Capture a search of fixed shapes into a CUDA graph (see Plan)."""
        torch = _torch()
        st = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        _check(lib().ksc_plan_create(self._h, nq, k, nprobe, rerank, int(adaptive),
                                     C.byref(opts) if opts else None, C.c_void_p(st.cuda_stream), C.byref(h)))
        return Plan(h.value, self, nq, k)

    def autotune(self, Q, k, nprobe, rerank, opts=None, stream=None):
        """Fastest scan lanes-per-query / tile length for this batch: (opts, ms)."""
        torch = _torch()
        o = opts if opts is not None else search_opts()
        ms = C.c_float(0)
        _check(lib().ksc_autotune(self._h, _dptr(Q, torch.float32, "Q"), Q.shape[0], k, nprobe, rerank,
                                  C.byref(o), _stream(stream), C.byref(ms)))
        return o, ms.value

    STAGES = ("rank", "worklist", "lut", "near_scan", "scan", "select", "rerank")

    def profile(self, on=True):
        """Turn the per-stage CUDA-event timing of searches on or off."""
        _check(lib().ksc_profile_enable(self._h, int(on)))

    def profile_read(self):
        """Per-stage milliseconds of the last search (dict) and its kernel count."""
        ms = (C.c_float * 8)()
        n = C.c_int32(0)
        _check(lib().ksc_profile_read(self._h, ms, len(self.STAGES), C.byref(n)))
        return {k: ms[i] for i, k in enumerate(self.STAGES)}, n.value

    def pair_distances(self, Q, ids, precision, stream=None):
        """Distances of given (query, id) pairs [nq x m] from FP32, BF16 (1) or
        FP8 (2) rows (ksc_pair_distances)."""
        torch = _torch()
        out = torch.empty(ids.shape, dtype=torch.float32, device=Q.device)
        _check(lib().ksc_pair_distances(self._h, _dptr(Q, torch.float32, "Q"), Q.shape[0],
                                        _dptr(ids, torch.int64, "ids"), ids.shape[1], precision, _dptr(out),
                                        _stream(stream)))
        return out

    def search_stats(self):
        """Counters of the last search: overflowed queries, candidates kept, max per query."""
        v = (C.c_int64 * 4)()
        _check(lib().ksc_search_stats(self._h, v))
        return dict(overflow_queries=v[0], candidates=v[1], max_candidates=v[2])

    def last_status(self):
        """The device status word of the last search: 0 clean, else a bitwise OR
        of KSC_STATUS_* flags (1: a candidate store overflowed and was redone
        exactly); a blocking read (ksc_last_status)."""
        s = C.c_int32(0)
        _check(lib().ksc_last_status(self._h, C.byref(s)))
        return s.value


class Plan:
    """A captured search: execute() copies queries in, replays the graph and
    returns views of the plan's own result buffers."""

    def __init__(self, handle, index, nq, k):
        self._h = C.c_void_p(handle)
        self.index = index  # keeps the index alive
        self.nq, self.k = nq, k

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value and _lib is not None:
            _lib.ksc_plan_free(self._h)
        self._h = C.c_void_p(None)

    def execute(self, Q, ids=None, dists=None, stream=None):
        """Copy Q into the plan's input, replay the captured search and return its
        results (views of the plan's buffers unless ids / dists are given)."""
        torch = _torch()
        st = stream if stream is not None else torch.cuda.current_stream()
        if ids is None:
            ids = torch.empty((self.nq, self.k), dtype=torch.int64, device=Q.device)
        if dists is None:
            dists = torch.empty((self.nq, self.k), dtype=torch.float32, device=Q.device)
        _check(lib().ksc_plan_execute(self._h, _dptr(Q, torch.float32, "Q"), _dptr(ids), _dptr(dists),
                                      C.c_void_p(st.cuda_stream)))
        return ids, dists


def build_index(X, nlist, M, nbits=4, metric="l2", spherical=False, perm=None, iters=20, seed=0x5EED,
                build_graph=False, filter_threshold=0.0, stream=None):
    """filter_threshold > 0: component filtration (Sec. 4.3) before the build."""
    torch = _torch()
    n, d = X.shape
    perm_np = None if perm is None else np.ascontiguousarray(perm, dtype=np.int64)
    opts = BuildOpts(iters, int(spherical), _hptr(perm_np), seed, int(build_graph), float(filter_threshold))
    h = C.c_void_p()
    _check(lib().ksc_build_index(_dptr(X, torch.float32, "X"), n, d, nlist, M, nbits,
                                 KSC_IP if metric == "ip" else KSC_L2, C.byref(opts), _stream(stream),
                                 C.byref(h)))
    return Index(h.value)


def index_load(path, stream=None):
    """An index read from a file written by Index.save."""
    h = C.c_void_p()
    _check(lib().ksc_index_load(os.fsencode(path), _stream(stream), C.byref(h)))
    return Index(h.value)


def index_import(arrs, metric="l2", spherical=False, stream=None):
    """arrs: dict of numpy arrays X, c_rank, c_mean, codebook, codes, assign
    (and optionally graph, entry)."""
    keep = {k: np.ascontiguousarray(arrs[k]) for k in ("X", "c_rank", "c_mean", "codebook", "codes", "assign")}
    keep["X"] = keep["X"].astype(np.float32, copy=False)
    for k in ("graph", "entry"):
        if arrs.get(k) is not None:
            keep[k] = np.ascontiguousarray(arrs[k], dtype=np.int32)
    n, d = keep["X"].shape
    L = keep["c_rank"].shape[0]
    M = keep["codebook"].shape[0]
    a = IndexArrays(n, d, L, M, KSC_IP if metric == "ip" else KSC_L2, int(spherical),
                    *[_hptr(keep.get(k)) for k in ("X", "c_rank", "c_mean", "codebook", "codes", "assign",
                                                   "graph", "entry")])
    h = C.c_void_p()
    _check(lib().ksc_index_import(C.byref(a), _stream(stream), C.byref(h)))
    return Index(h.value)


def _index_arrays(arrs, metric, spherical):
    keep = {k: np.ascontiguousarray(arrs[k]) for k in ("X", "c_rank", "c_mean", "codebook", "codes", "assign")}
    keep["X"] = keep["X"].astype(np.float32, copy=False)
    n, d = keep["X"].shape
    a = IndexArrays(n, d, keep["c_rank"].shape[0], keep["codebook"].shape[0], KSC_IP if metric == "ip" else KSC_L2,
                    int(spherical), *[_hptr(keep.get(k)) for k in ("X", "c_rank", "c_mean", "codebook", "codes",
                                                                   "assign")], None, None)
    return a, keep


def index_import_shard(arrs, list_owner, shard, metric="l2", spherical=False, stream=None):
    """Shard `shard` of a list-partitioned index: the lists p with
    list_owner[p] == shard (their vectors in ascending row id), centroids and
    codebooks replicated (ksc_index_import_shard)."""
    a, keep = _index_arrays(arrs, metric, spherical)
    owner = np.ascontiguousarray(list_owner, dtype=np.int32)
    h = C.c_void_p()
    _check(lib().ksc_index_import_shard(C.byref(a), _hptr(owner), int(shard), _stream(stream), C.byref(h)))
    return Index(h.value)


def merge_topk(ids, dists, ip=False, stream=None):
    """ids / dists [parts x nq x k] -> the k best per query (ksc_merge_topk)."""
    torch = _torch()
    parts, nq, k = ids.shape
    out_i = torch.empty((nq, k), dtype=torch.int64, device=ids.device)
    out_d = torch.empty((nq, k), dtype=torch.float32, device=ids.device)
    _check(lib().ksc_merge_topk(_dptr(ids, torch.int64, "ids"), _dptr(dists, torch.float32, "dists"), nq, parts, k,
                                int(ip), _dptr(out_i), _dptr(out_d), _stream(stream)))
    return out_i, out_d


def prune_mlp_grad(w, x, y, stream=None):
    """Loss and gradient of the pruning MLP (16 -> 32 -> 32 -> 2) on device tensors."""
    torch = _torch()
    g = torch.empty(Index.PRUNE_NPARAMS, dtype=torch.float32, device=x.device)
    loss = torch.empty(1, dtype=torch.float32, device=x.device)
    _check(lib().ksc_prune_mlp_grad(_dptr(w, torch.float32, "w"), _dptr(x, torch.float32, "x"),
                                    _dptr(y, torch.float32, "y"), x.shape[0], _dptr(g), _dptr(loss), _stream(stream)))
    return loss, g


def component_stats(X, stream=None):
    """Per-dimension mean, std and fraction of zero or within-one-std values
    of a device matrix (FP64 device tensors)."""
    torch = _torch()
    n, d = X.shape
    out = [torch.empty(d, dtype=torch.float64, device=X.device) for _ in range(3)]
    _check(lib().ksc_component_stats(_dptr(X, torch.float32, "X"), n, d, *[_dptr(o) for o in out],
                                     _stream(stream)))
    return tuple(out)


def lut16_peak(stream=None):
    """Measured lookup rates (Glookup/s) of the scan's instruction sequences:
    (shared selectors, per-slot selectors)."""
    v = (C.c_double * 2)()
    _check(lib().ksc_lut16_peak(v, _stream(stream)))
    return v[0], v[1]


def version():
    """Library version and target architecture."""
    return lib().ksc_version().decode()
