"""The LUT16 scan on the tensor cores (k_scan_tc: one-hot codes x FP16 tables,
FP32 sums of integers) against the CPU oracle and against the byte-permute
scan, through the C ABI (needs a GB300).

Bit-exact: the candidate store (the R best (distance, id) keys) equals the
oracle's scan of the same probes, and every result equals that of the
byte-permute scan on the same inputs.  Index shapes: M = 32, 24, 50 (not a
multiple of the 4-subspace chunk), 64, 16 and 12; lists of 100 to 1000
vectors (partial 128-vector tiles, odd tile counts); with the 10k x 128
configuration more than 64 queries probe a list (several query groups per
list).
"""
import numpy as np
import pytest

import oracle
from paper_2511_03298_gb300 import synth

from test_gpu_parity import small_index, gpu_index, oracle_probes, check_results

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


@pytest.fixture(scope="module")
def ksc(torch):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2511_03298_gb300 import ksc as k
    return k


@pytest.mark.parametrize("kind", ["l2", "ip", "m50", "small", "ds4", "ds3ip"])
def test_tc_scan_candidates_bit_exact(torch, ksc, kind):
    ix, Q = small_index(kind)
    g = gpu_index(ksc, ix)
    P, R, k = (8, 100, 10) if kind == "small" else (5, 150, 10)
    probes = oracle_probes(ix, Q, P)
    opts = ksc.search_opts(scan_tc=True)
    ids, dists, cand, ncand = g.search_with_probes(torch.from_numpy(Q).cuda(), torch.from_numpy(probes).cuda(),
                                                   k, R, opts=opts)
    assert g.last_status() == 0
    cand = cand.cpu().numpy().view(np.uint64)
    ncand = ncand.cpu().numpy()
    ids, dists = ids.cpu().numpy(), dists.cpu().numpy()
    ref_ids = np.zeros_like(ids)
    ref_d = np.zeros(ids.shape, np.float64)
    for qi in range(len(Q)):
        Ql, b, _ = oracle.lut_q8(Q[qi], ix, probes[qi])
        ref = oracle.scan_topr(ix, probes[qi], Ql, b, R)
        assert ncand[qi] == len(ref)
        assert np.array_equal(cand[qi, :len(ref)], ref), qi
        ref_ids[qi], ref_d[qi] = oracle.rerank(Q[qi], ix, oracle.key_id(ref).astype(np.int32), k)
    check_results(ix, Q, ids, dists, ref_ids, ref_d, k)


def _same(a, b):
    return all(bool((x == y).all()) for x, y in zip(a, b))


@pytest.mark.parametrize("tile", [0, 4, 12])
def test_tc_scan_equals_byte_permute_scan(torch, ksc, tile):
    ix, Q = small_index("small")
    g = gpu_index(ksc, ix)
    Qd = torch.from_numpy(Q).cuda()
    base = g.search(Qd, 10, 12, 200)
    tc = g.search(Qd, 10, 12, 200, opts=ksc.search_opts(scan_tc=True, tile_blocks=tile))
    assert g.last_status() == 0
    assert _same(base, tc)
    # per-query nprobe and rerank
    rng = np.random.default_rng(3)
    npb = torch.from_numpy(rng.integers(1, 17, len(Q)).astype(np.int32)).cuda()
    rr = torch.from_numpy(rng.integers(10, 201, len(Q)).astype(np.int32)).cuda()
    v0 = g.search_varprobe(Qd, 10, npb, rr, nprobe_max=16, rerank_max=200)
    v1 = g.search_varprobe(Qd, 10, npb, rr, nprobe_max=16, rerank_max=200, opts=ksc.search_opts(scan_tc=True))
    assert _same(v0, v1)


def test_tc_scan_in_a_captured_plan(torch, ksc):
    ix, Q = small_index("small")
    g = gpu_index(ksc, ix)
    Qd = torch.from_numpy(Q).cuda()
    ref = g.search(Qd, 10, 8, 100)
    torch.cuda.synchronize()
    s_ = torch.cuda.Stream()
    with torch.cuda.stream(s_):
        pl = g.plan(len(Q), 10, nprobe=8, rerank=100, opts=ksc.search_opts(scan_tc=True))
        got = [[t.clone() for t in pl.execute(Qd)] for _ in range(3)]
    s_.synchronize()
    for r in got:
        assert _same(ref, r)
    assert g.last_status() == 0


def test_tc_scan_full_size_workload(torch, ksc):
    """1M x 128, 10k queries, nprobe 7, R 200 (the benchmark's operating point):
    the tensor-core scan's results equal the byte-permute scan's."""
    X = synth.base(2)
    Q = synth.queries(2)
    g = ksc.build_index(torch.from_numpy(X).cuda(), 1024, 64, perm=synth.build_perm(2, len(X)))
    Qd = torch.from_numpy(Q).cuda()
    base = g.search(Qd, 10, 7, 200)
    tc = g.search(Qd, 10, 7, 200, opts=ksc.search_opts(scan_tc=True))
    assert g.last_status() == 0
    assert _same(base, tc)
    # the candidate stores of given probes, too
    probes, _ = g.rank_lists(Qd, 7, want_scores=False)
    c0 = g.search_with_probes(Qd, probes, 10, 200)
    c1 = g.search_with_probes(Qd, probes, 10, 200, opts=ksc.search_opts(scan_tc=True))
    assert _same(c0, c1)
