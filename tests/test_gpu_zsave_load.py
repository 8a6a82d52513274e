"""Index persistence (ksc_index_save / ksc_index_load) on the GPU: a saved and
reloaded index holds the same arrays, graph, models and filtration state,
and every search on it returns exactly what the original returns (needs a
GB300)."""
import numpy as np
import pytest

import oracle
from paper_2511_03298_gb300 import synth

from test_gpu_parity import small_index, gpu_index

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2511_03298_gb300 import ksc
    return torch, ksc


def _same(a, b):
    return all(bool((x == y).all()) for x, y in zip(a, b))


def _same_arrays(g, h, with_graph=False):
    e0, e1 = g.export(with_graph=with_graph), h.export(with_graph=with_graph)
    keys = ["X", "c_rank", "c_mean", "codebook", "codes", "assign"] + (["graph", "entry"] if with_graph else [])
    for key in keys:
        np.testing.assert_array_equal(e0[key], e1[key])
    assert g.info() == h.info()


def test_round_trip_with_predictor_and_pruner(env, tmp_path):
    torch, ksc = env
    ix, Q = small_index("small")
    g = gpu_index(ksc, ix)
    rng = np.random.default_rng(4)
    w = (rng.normal(size=8450) * 0.1).astype(np.float32)
    g.predictor_weights(set_to=w)
    g.set_predictor_params(2, 16, 50, 200, 0.2, 0.5, 0.1, 0.5)
    g.pruner_stats()
    model = np.concatenate([rng.normal(size=g.PRUNE_NPARAMS) * 0.2, np.zeros(16), np.ones(16)]).astype(np.float32)
    g.pruner_model(set_to=model)
    g.pruner_theta(0.3)
    path = str(tmp_path / "small.ksc")
    g.save(path)
    h = ksc.index_load(path)
    _same_arrays(g, h)
    np.testing.assert_array_equal(h.predictor_weights(), w)
    for a, b in zip(g.pruner_export(), h.pruner_export()):
        np.testing.assert_array_equal(a, b)
    Qd = torch.from_numpy(Q).cuda()
    assert _same(g.search(Qd, 10, 8, 100), h.search(Qd, 10, 8, 100))
    # the learned nprobe / reorder and the pruning at the saved threshold
    assert _same(g.search_adaptive(Qd, 10), h.search_adaptive(Qd, 10))
    assert g.last_status() == 0 and h.last_status() == 0
    # a view writes the index it came from
    p2 = str(tmp_path / "view.ksc")
    v = g.view()
    v.save(p2)
    v.free()
    assert open(p2, "rb").read() == open(path, "rb").read()


def test_round_trip_with_graph(env, tmp_path):
    torch, ksc = env
    ix, Q = small_index("l2")
    graph, entry = oracle.build_graph(ix)
    g = ksc.index_import(dict(ix, graph=graph, entry=entry))
    path = str(tmp_path / "graph.ksc")
    g.save(path)
    h = ksc.index_load(path)
    _same_arrays(g, h, with_graph=True)
    Qd = torch.from_numpy(Q).cuda()
    opts = ksc.search_opts(hybrid=True, n_near=2, efs=32, tau=4)
    assert _same(g.search(Qd, 10, 5, 100, opts=opts), h.search(Qd, 10, 5, 100, opts=opts))
    assert h.last_status() == 0


def test_round_trip_of_a_filtered_index(env, tmp_path):
    torch, ksc = env
    N = 6000
    X = synth.base(6, n=N)
    Q = synth.queries(6, 60)
    g = ksc.build_index(torch.from_numpy(X).cuda(), 32, 196, filter_threshold=0.99, iters=10,
                        perm=synth.build_perm(6, N))
    path = str(tmp_path / "filtered.ksc")
    g.save(path)
    h = ksc.index_load(path)
    _same_arrays(g, h)
    d0, dims0 = g.dims()
    d1, dims1 = h.dims()
    assert d0 == d1 == 784
    np.testing.assert_array_equal(dims0, dims1)
    Qd = torch.from_numpy(Q).cuda()
    assert _same(g.search(Qd, 10, 6, 50), h.search(Qd, 10, 6, 50))


def test_load_rejects_a_corrupt_file(env, tmp_path):
    torch, ksc = env
    ix, _ = small_index("ip")
    g = gpu_index(ksc, ix)
    path = tmp_path / "ip.ksc"
    g.save(str(path))
    data = bytearray(path.read_bytes())
    with pytest.raises(ksc.KscError):
        bad = tmp_path / "cut.ksc"
        bad.write_bytes(bytes(data[:-1]))
        ksc.index_load(str(bad))
    assert ksc.index_load(str(path)).info() == g.info()
