"""The allocation-free LUT entry point (ksc_compute_luts_noalloc).

It serves callers that cannot let this library allocate device memory (their
memory is reserved by their own allocator, or they cannot take the device
synchronisation of cudaMalloc).  Its output must equal ksc_compute_luts's
bit for bit, on consecutive calls that reuse its fixed scratch array.  This
file is collected last so that a failing run has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2511_03298_gb300 import ksc
    rng = np.random.default_rng(77)
    centres = rng.uniform(-4, 4, size=(12, 32))
    X = (centres[rng.integers(0, 12, 4000)] + rng.normal(size=(4000, 32))).astype(np.float32)
    ix_o = oracle.build_index(X, 16, 16, False, rng.permutation(4000).astype(np.int64), iters=4)
    return torch, ksc, ix_o, ksc.index_import(ix_o), rng


def _luts(torch, ksc, ix, Q, probes, noalloc):
    nq, P = probes.shape
    M = ix.info()["M"]
    lut = torch.full((nq, P, M, 16), 7, dtype=torch.uint8, device="cuda")
    bias = torch.full((nq, P), -5, dtype=torch.int32, device="cuda")
    scale = torch.full((nq,), -1.0, dtype=torch.float32, device="cuda")
    fn = ksc.lib().ksc_compute_luts_noalloc if noalloc else ksc.lib().ksc_compute_luts
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = fn(ix.handle, C.c_void_p(Q.data_ptr()), nq, C.c_void_p(probes.data_ptr()), P,
            C.c_void_p(lut.data_ptr()), C.c_void_p(bias.data_ptr()), C.c_void_p(scale.data_ptr()), st)
    assert rc == 0, ksc.lib().ksc_last_error()
    torch.cuda.synchronize()
    return lut.cpu().numpy(), bias.cpu().numpy(), scale.cpu().numpy()


def test_noalloc_luts_equal_the_allocating_entry_point_on_consecutive_calls(env):
    torch, ksc, ix_o, ix, rng = env
    for call, (nq, P) in enumerate([(300, 6), (120, 9)]):
        Q = (ix_o["X"][rng.integers(0, 4000, nq)] + rng.normal(size=(nq, 32))).astype(np.float32)
        probes = np.stack([oracle.rank(q, ix_o["c_rank"], False, P)[0] for q in Q]).astype(np.int32)
        Qd = torch.from_numpy(Q).cuda()
        pd = torch.from_numpy(probes).cuda()
        ref = _luts(torch, ksc, ix, Qd, pd, noalloc=False)
        got = _luts(torch, ksc, ix, Qd, pd, noalloc=True)
        for r, g in zip(ref, got):
            assert np.array_equal(r, g), "call %d differs" % call


def test_noalloc_rejects_batches_beyond_its_scratch(env):
    torch, ksc, ix_o, ix, rng = env
    lib = ksc.lib()
    rc = lib.ksc_compute_luts_noalloc(ix.handle, C.c_void_p(16), 65537, C.c_void_p(16), 4, C.c_void_p(16),
                                      C.c_void_p(16), C.c_void_p(16), None)
    assert rc == -1 and b"exceeds the fixed scratch" in lib.ksc_last_error()


def test_noalloc_first_call_on_a_fresh_index_allocates_nothing(env):
    """A second index with sub-vectors of width 4 (d 32, M 8) runs the generic
    table kernels rather than the width-2 ones.  Its first table call goes
    through the allocation-free entry point, before the allocating one has
    given it any workspace: the device's free memory is the same before and
    after the call, and the tables equal the allocating entry point's
    afterwards.  The module holding the scratch array is already loaded by
    the first index's calls, so loading it does not count here."""
    torch, ksc, ix_o, ix, rng = env
    q0 = torch.from_numpy(ix_o["X"][:4].copy()).cuda()
    p0 = torch.zeros((4, 2), dtype=torch.int32, device="cuda")
    p0[:, 1] = 1
    _luts(torch, ksc, ix, q0, p0, noalloc=True)  # module and scratch address resolved
    X = ix_o["X"]
    ix_o8 = oracle.build_index(X, 16, 8, False, rng.permutation(len(X)).astype(np.int64), iters=4)
    ix8 = ksc.index_import(ix_o8)
    assert ix8.info()["M"] == 8 and ix8.info()["d"] // 8 == 4
    for nq, P in [(200, 5), (64, 11)]:
        Q = (X[rng.integers(0, len(X), nq)] + rng.normal(size=(nq, 32))).astype(np.float32)
        probes = np.stack([oracle.rank(q, ix_o8["c_rank"], False, P)[0] for q in Q]).astype(np.int32)
        Qd = torch.from_numpy(Q).cuda()
        pd = torch.from_numpy(probes).cuda()
        lut = torch.full((nq, P, 8, 16), 7, dtype=torch.uint8, device="cuda")
        bias = torch.full((nq, P), -5, dtype=torch.int32, device="cuda")
        scale = torch.full((nq,), -1.0, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        rc = ksc.lib().ksc_compute_luts_noalloc(ix8.handle, C.c_void_p(Qd.data_ptr()), nq, C.c_void_p(pd.data_ptr()),
                                                P, C.c_void_p(lut.data_ptr()), C.c_void_p(bias.data_ptr()),
                                                C.c_void_p(scale.data_ptr()), st)
        assert rc == 0, ksc.lib().ksc_last_error()
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        got = (lut.cpu().numpy(), bias.cpu().numpy(), scale.cpu().numpy())
        ref = _luts(torch, ksc, ix8, Qd, pd, noalloc=False)
        for r, g in zip(ref, got):
            assert np.array_equal(r, g)
        # and the oracle's tables for the first query (the generic path is
        # pinned independently of the allocating entry point)
        Qo, bo, _ = oracle.lut_q8(Q[0], ix_o8, probes[0])
        assert np.array_equal(got[0][0], Qo) and np.array_equal(got[1][0], bo)
