"""Multi-process host logic of the benchmark on CPU (gloo, world size 2).

The query path shards by batch: every process holds a replica of the index
and searches its own query batch, with no collective on the data path.  What
the processes do share is host logic: each draws an independent batch, they
agree on one operating point (the largest nprobe any of them needs), and the
whole-job throughput divides all batches by the slowest process's time.  The
test runs that logic in two spawned processes over gloo; a rank that fails is
reported by its exit code.
"""
import os
import socket

import pytest


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, own_nprobe, own_ms, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      KSC_BENCH_GLOO="1")
    import bench
    import torch.distributed as dist
    r, w = bench.dist_setup()
    q = bench.rank_queries(r, 32)
    ms = bench.max_over_ranks(own_ms[r], w)
    res = dict(rank=r, ws=w, q=q.tolist(), nprobe=bench.common_nprobe(own_nprobe[r], w), ms=ms,
               value=bench.weak_value(10_000, w, ms))
    bench.barrier(w)
    dist.destroy_process_group()
    out.put(res)


def _run(ws, own_nprobe, own_ms):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, ws, port, own_nprobe, own_ms, out)) for r in range(ws)]
    for p in ps:
        p.start()
    try:
        res = [out.get(timeout=240) for _ in range(ws)]
    finally:
        for p in ps:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in ps), [p.exitcode for p in ps]
    return sorted(res, key=lambda d: d["rank"])


def test_two_ranks_agree_on_operating_point_and_timing():
    res = _run(2, own_nprobe=[8, 12], own_ms=[1.9, 2.5])
    assert [d["rank"] for d in res] == [0, 1] and all(d["ws"] == 2 for d in res)
    # one operating point: the larger of the two choices
    assert res[0]["nprobe"] == res[1]["nprobe"] == 12
    # the slowest rank's time, and all queries of both ranks over it
    assert res[0]["ms"] == res[1]["ms"] == 2.5
    assert res[0]["value"] == res[1]["value"] == pytest.approx(2 * 10_000 / 2.5e-3)
    # each rank searches its own batch; rank 0's is the single-process batch
    import numpy as np
    from paper_2511_03298_gb300 import synth
    q0, q1 = np.array(res[0]["q"], np.float32), np.array(res[1]["q"], np.float32)
    assert not np.array_equal(q0, q1)
    assert np.array_equal(q0, synth.queries(2, 32))
