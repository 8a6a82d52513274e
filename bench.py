"""Benchmark: QPS at recall@10 >= 0.90 of the IVF-PQ query path on one GB300.

Workload (SIFT1M-shaped synthetic stand-in): 1,000,000 x 128 non-negative
integer vectors 0..255, 10,000 queries, nlist 1024, M 64 x 4-bit, k 10,
rerank 200; nprobe = the smallest of the grid 4..128 whose recall@10 (ties
counted, FP64 ground truth) reaches 0.90.  One step = one search of the
whole 10k-query batch (rank lists, LUTs, scan, select, rerank), inputs
resident in HBM.  L2 is flushed (256 MB write) before every timed step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun): every rank holds a replica of the index and searches
its own 10k-query batch (weak scaling, no collective on the data path).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CFG = dict(workload="ivfpq-sift1m-shape", n=1_000_000, d=128, nq=10_000, nlist=1024, M=64, nbits=4, k=10,
           rerank=200, metric="l2")
GRID = (4, 5, 6, 7, 8, 9, 10, 12, 14, 16, 20, 24, 32, 48, 64, 96, 128)
METRIC = "QPS at recall@10\u22650.90 (1M\u00d7128, 1 GB300) vs plain path; ADC-scan HBM GB/s vs peak"
TARGET_RECALL = 0.90
L2_FLUSH_BYTES = 256 << 20
# DRAM bytes (read + write) of k_scan's two launches in one plain search at the
# given nprobe, from ncu (profiles/k_scan_ivfpq_sift1m_nq10k_nprobe<P>.md)
SCAN_TRAFFIC_BYTES = {7: 186_770_944}
# the same for the streaming leg of the 10M x 96 index at batch 256, nprobe 256
# (profiles/k_scan_deep10m_b256_nprobe256.md)
DEEP_STREAM_TRAFFIC_BYTES = {(256, 256): 429_400_832}
HBM_NOMINAL_GBS = 7900.0  # GB300 HBM3e, nominal


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("KSC_BENCH_GLOO") is None else "gloo")
    return rank, ws


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, ws):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_queries(rank, nq):
    """This rank's own query batch: rank 0 the standard 10k, rank r > 0 an
    independent stream of the same distribution."""
    from paper_2511_03298_gb300 import synth
    return synth.queries(2, nq, stream=rank)


def common_nprobe(own, ws):
    """Operating point shared by all ranks: the largest of their own choices,
    so every rank's batch reaches the recall target."""
    return int(max_over_ranks(float(own), ws))


def weak_value(nq, ws, ms_max):
    """Whole-job queries/s: every rank's batch over the slowest rank's time."""
    return nq * ws / (ms_max * 1e-3)


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_index):
        self.dev = dev_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.p:
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                out, _ = self.p.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def exact_topk(torch, X, Q, k, chunk=512):
    """FP64 brute-force top-k (ground truth for recall; ties by id)."""
    Xd = X.double()
    xn = (Xd * Xd).sum(1)
    out_d, out_i = [], []
    for b in range(0, Q.shape[0], chunk):
        q = Q[b:b + chunk].double()
        D = (q * q).sum(1, keepdim=True) - 2.0 * (q @ Xd.T) + xn[None]
        d, i = torch.topk(D, k, dim=1, largest=False, sorted=True)
        out_d.append(d.cpu().numpy())
        out_i.append(i.cpu().numpy())
    return np.concatenate(out_i), np.concatenate(out_d)


def kth_fp32(torch, Xd, Q, k=10, chunk=4096):
    """True k-th neighbour distance per query, FP32 brute force on the GPU
    (training labels only; integer data keeps these exact up to ~1e-7)."""
    xn = (Xd * Xd).sum(1)
    out = []
    for b in range(0, Q.shape[0], chunk):
        q = Q[b:b + chunk]
        D = (q * q).sum(1, keepdim=True) - 2.0 * (q @ Xd.T) + xn[None]
        out.append(torch.topk(D, k, dim=1, largest=False).values[:, k - 1])
    return torch.cat(out).contiguous()


def recall_at_10(torch, X, Q, ids, true_d, k=10):
    """A returned id counts when its exact distance <= the true 10th distance."""
    idt = torch.as_tensor(ids, device=X.device)
    valid = idt >= 0
    rows = X[idt.clamp_min(0)].double()
    d = ((rows - Q.double()[:, None, :]) ** 2).sum(-1)
    kth = torch.as_tensor(true_d[:, k - 1], device=X.device)[:, None]
    hit = (d <= kth + 1e-9 * kth.abs().clamp_min(1.0)) & valid
    return float(hit[:, :k].sum(1).clamp_max(k).double().mean().item() / k)


def scan_work(ix_export_sizes, probes):
    """Sum over (query, probe) of list sizes -> lookups and code bytes."""
    sizes = ix_export_sizes[probes]
    return int(sizes.sum())


def run_ours(args, rank, ws):
    import torch
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    barrier(ws)
    from paper_2511_03298_gb300 import ksc, synth
    ksc.lib()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    X = synth.base(2)
    Qh = rank_queries(rank, CFG["nq"])
    Xd = torch.from_numpy(X).to(dev)
    Qd = torch.from_numpy(Qh).to(dev)
    t0 = time.time()
    ix = ksc.build_index(Xd, CFG["nlist"], CFG["M"], perm=synth.build_perm(2, len(X)))
    torch.cuda.synchronize()
    build_s = time.time() - t0
    k, R = CFG["k"], CFG["rerank"]
    sweep = {}
    if args.quick:
        # profiling mode: fixed nprobe, no ground truth, sweep, e2e or CPU leg
        nprobe, recall, true_d = args.nprobe or 8, None, None
    else:
        true_i, true_d = exact_topk(torch, Xd, Qd, k)
        # operating point: smallest nprobe of the grid with recall >= 0.90
        nprobe = GRID[-1]
        for P in GRID:
            ids, _ = ix.search(Qd, k, P, R)
            rec = recall_at_10(torch, Xd, Qd, ids, true_d, k)
            sweep[P] = round(rec, 4)
            if rec >= TARGET_RECALL:
                nprobe = P
                break
        agreed = common_nprobe(nprobe, ws)
        if agreed != nprobe:
            ids, _ = ix.search(Qd, k, agreed, R)
            sweep[agreed] = round(recall_at_10(torch, Xd, Qd, ids, true_d, k), 4)
            nprobe = agreed
        recall = sweep[nprobe]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()
    ids = torch.empty((CFG["nq"], k), dtype=torch.int64, device=dev)
    dists = torch.empty((CFG["nq"], k), dtype=torch.float32, device=dev)

    def timed(search, clk_dev=None):
        """W warm-up + K timed steps of `search` (L2 flushed before each);
        returns mean ms, per-stage ms, kernel launches, clocks."""
        ix.profile(True)
        for _ in range(args.warmup):
            search()
        torch.cuda.synchronize()
        stage = {s_: [] for s_ in ksc.Index.STAGES}
        times, nl_tot = [], 0
        barrier(ws)
        with Clocks(local) as clk:
            for _ in range(args.steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(st)
                search()
                e1.record(st)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
                prof, nl = ix.profile_read()
                nl_tot += nl
                for s_, v in prof.items():
                    stage[s_].append(v)
        torch.cuda.synchronize()
        barrier(ws)
        ix.profile(False)
        return statistics.mean(times), {s_: statistics.mean(v) for s_, v in stage.items()}, nl_tot, clk.summary()

    sopts = ksc.search_opts(lanes_per_query=args.lanes, tile_blocks=args.tile_blocks, scan_tc=args.scan_tc) \
        if (args.lanes or args.tile_blocks or args.scan_tc) else None
    plain_ms, plain_stage, plain_launches, plain_clk = timed(
        lambda: ix.search(Qd, k, nprobe, R, opts=sopts, out=(ids, dists)))
    stats = ix.search_stats()
    if args.quick:
        line = {"quick": True, "nprobe": nprobe, "ms_per_step": round(plain_ms, 4),
                "value": round(CFG["nq"] / (plain_ms * 1e-3), 1),
                "stage_ms": {s_: round(v, 4) for s_, v in plain_stage.items()}, "search_stats": stats}
        if args.quick_learned:
            # the adaptive search after a short training, at fixed Eq. 2
            # settings (no tuning): for profiling its kernels
            T = synth.train_queries(5, args.ntrain)
            Td = torch.from_numpy(T).to(dev)
            ix.train_predictor(Td, kth_fp32(torch, Xd, Td, k), epochs=4)
            ix.set_predictor_params(2, 16, 100, R, 0.0, 0.0, 0.0, 2.0)
            if args.profile_range:
                torch.cuda.synchronize()
                torch.cuda.profiler.start()  # a profiler started with --profile-from-start off records from here
            l_ms, l_stage, _, _ = timed(lambda: ix.search_adaptive(Qd, k, opts=sopts))
            if args.profile_range:
                torch.cuda.profiler.stop()
            line["learned"] = {"ms_per_step": round(l_ms, 4), "eq2": [2, 16, 100, R, 0.0, 0.0, 0.0, 2.0],
                               "stage_ms": {s_: round(v, 4) for s_, v in l_stage.items()}}
        if rank == 0:
            print(json.dumps(line))
        return None
    # learned nprobe (the paper's adaptive search module, an MLP here):
    # train on seeded training queries, tune Eq. 2 on a held-out split
    learned = None
    if not args.no_learned:
        TV = synth.train_queries(5, args.ntrain + 5000)
        Td = torch.from_numpy(TV[:args.ntrain]).to(dev)
        Vd = torch.from_numpy(TV[args.ntrain:]).to(dev)
        t0 = time.time()
        kth_t = kth_fp32(torch, Xd, Td, k)
        loss = ix.train_predictor(Td, kth_t, epochs=8)
        train_s = time.time() - t0
        _, vd_true = exact_topk(torch, Xd, Vd, k)
        best = None
        for pmax in (16, 32, 64):
            for pmin in (1, 2, 4):
                for p0 in (0.0, 0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7):
                    for p1 in (0.0, 0.5, 1.0, 2.0, 4.0):
                        ix.set_predictor_params(pmin, pmax, R, R, p0, p1, 0.0, 0.0)
                        vids, _, vnp, _ = ix.search_adaptive(Vd, k)
                        rec = recall_at_10(torch, Xd, Vd, vids, vd_true, k)
                        cost = float(vnp.double().mean().item())
                        if rec >= TARGET_RECALL + 0.005 and (best is None or cost < best[0]):
                            best = (cost, rec, pmin, pmax, p0, p1)
        if best is not None:
            # then the reorder head: the smallest mean R that keeps the target
            rbest = (float(R), best[1], R, 0.0, 0.0)
            for rmin in (50, 100, 150):
                for r0 in (0.0, 0.2, 0.4, 0.6):
                    for r1 in (0.0, 0.5, 1.0, 2.0):
                        ix.set_predictor_params(best[2], best[3], rmin, R, best[4], best[5], r0, r1)
                        vids, _, _, vr = ix.search_adaptive(Vd, k)
                        rec = recall_at_10(torch, Xd, Vd, vids, vd_true, k)
                        mr = float(vr.double().mean().item())
                        if rec >= TARGET_RECALL + 0.005 and mr < rbest[0]:
                            rbest = (mr, rec, rmin, r0, r1)
            ix.set_predictor_params(best[2], best[3], rbest[2], R, best[4], best[5], rbest[3], rbest[4])
            lids, _, lnp, lrr = ix.search_adaptive(Qd, k, opts=sopts)
            l_rec = recall_at_10(torch, Xd, Qd, lids, true_d, k)
            l_ms, l_stage, l_launches, l_clk = timed(lambda: ix.search_adaptive(Qd, k, opts=sopts))
            learned = dict(ms=l_ms, stage=l_stage, launches=l_launches, clk=l_clk, recall=l_rec,
                           mean_nprobe=float(lnp.double().mean().item()), nprobe_q=lnp.cpu().numpy(),
                           mean_rerank=float(lrr.double().mean().item()),
                           params=dict(pmin=best[2], pmax=best[3], p0=best[4], p1=best[5], rmin=rbest[2], rmax=R,
                                       r0=rbest[3], r1=rbest[4]),
                           train_loss=loss, train_s=round(train_s, 1), val_recall=rbest[1], stats=ix.search_stats())
    # predictive cluster pruning (Sec. 4.2.3) inside the learned search (Alg. 2
    # order): the classifier trained on the same training queries, its
    # threshold and the nprobe head's Eq. 2 parameters tuned together on the
    # validation split for the fewest lists searched at the target recall
    pruned = None
    learned_state = None
    if learned is not None and not args.no_prune:
        lp = learned["params"]
        learned_state = (lp["pmin"], lp["pmax"], lp["rmin"], lp["rmax"], lp["p0"], lp["p1"], lp["r0"], lp["r1"])
        t0 = time.time()
        ploss = ix.train_pruner(Td, kth_t, k=k, P=lp["pmax"], R=R, epochs=4)
        ptrain_s = time.time() - t0
        pb = None
        for th in (0.05, 0.1, 0.15, 0.2, 0.3):
            ix.pruner_theta(th)
            for p0 in (0.0, 0.1, 0.2, 0.3, 0.4, 0.5):
                for p1 in (0.0, 0.5, 1.0, 2.0, 4.0):
                    ix.set_predictor_params(lp["pmin"], lp["pmax"], lp["rmin"], lp["rmax"], p0, p1, lp["r0"], lp["r1"])
                    vids, _, vnp, _ = ix.search_adaptive(Vd, k)
                    rec = recall_at_10(torch, Xd, Vd, vids, vd_true, k)
                    cost = float(vnp.double().mean().item())
                    if rec >= TARGET_RECALL + 0.005 and (pb is None or cost < pb[0]):
                        pb = (cost, rec, th, p0, p1)
        if pb is not None:
            pruned_state = (lp["pmin"], lp["pmax"], lp["rmin"], lp["rmax"], pb[3], pb[4], lp["r0"], lp["r1"])
            ix.pruner_theta(pb[2])
            ix.set_predictor_params(*pruned_state)
            pids, _, pnp, prr = ix.search_adaptive(Qd, k, opts=sopts)
            p_rec = recall_at_10(torch, Xd, Qd, pids, true_d, k)
            p_ms, p_stage, p_launches, p_clk = timed(lambda: ix.search_adaptive(Qd, k, opts=sopts))
            pruned = dict(ms=p_ms, stage=p_stage, launches=p_launches, recall=p_rec, theta=pb[2], state=pruned_state,
                          mean_lists=float(pnp.double().mean().item()), mean_rerank=float(prr.double().mean().item()),
                          params=dict(pmin=lp["pmin"], pmax=lp["pmax"], p0=pb[3], p1=pb[4]), train_loss=ploss,
                          train_s=round(ptrain_s, 1), val_recall=pb[1], stats=ix.search_stats())
        ix.pruner_theta(-1.0)
        ix.set_predictor_params(*learned_state)
    # the same steps without per-stage events, and replayed from CUDA graphs
    # (ksc_plan: the whole search captured once)
    gst = torch.cuda.Stream()  # graph capture needs a stream of its own

    def timed_bare(fn, s_):
        """The same steps without per-stage events: mean ms, clocks."""
        with torch.cuda.stream(s_):
            for _ in range(args.warmup):
                fn()
            torch.cuda.synchronize()
            ts = []
            barrier(ws)
            with Clocks(local) as clk:
                for _ in range(args.steps):
                    flush.zero_()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(s_)
                    fn()
                    e1.record(s_)
                    e1.synchronize()
                    ts.append(e0.elapsed_time(e1))
            barrier(ws)
        return statistics.mean(ts), clk.summary()

    # every way to run a step: direct calls, or the whole search replayed from a
    # CUDA graph (ksc_plan); the learned path only if it reaches the target
    variants = {"plain direct": timed_bare(lambda: ix.search(Qd, k, nprobe, R, opts=sopts, out=(ids, dists)), st)}
    with torch.cuda.stream(gst):
        pplan = ix.plan(CFG["nq"], k, nprobe=nprobe, rerank=R, opts=sopts)
    variants["plain graph"] = timed_bare(lambda: pplan.execute(Qd, ids, dists), gst)
    lplan = None
    ok_learned = learned is not None and learned["recall"] >= TARGET_RECALL
    if -max_over_ranks(-float(ok_learned), ws) > 0.5:  # on every rank, or on none
        variants["learned direct"] = timed_bare(lambda: ix.search_adaptive(Qd, k, opts=sopts), st)
        with torch.cuda.stream(gst):
            lplan = ix.plan(CFG["nq"], k, adaptive=True, opts=sopts)
        variants["learned graph"] = timed_bare(lambda: lplan.execute(Qd, ids, dists), gst)
    prplan = None
    ok_pruned = pruned is not None and pruned["recall"] >= TARGET_RECALL
    if -max_over_ranks(-float(ok_pruned), ws) > 0.5:
        ix.pruner_theta(pruned["theta"])
        ix.set_predictor_params(*pruned["state"])
        variants["pruned direct"] = timed_bare(lambda: ix.search_adaptive(Qd, k, opts=sopts), st)
        with torch.cuda.stream(gst):
            prplan = ix.plan(CFG["nq"], k, adaptive=True, opts=sopts)
        variants["pruned graph"] = timed_bare(lambda: prplan.execute(Qd, ids, dists), gst)
    torch.cuda.synchronize()
    # headline: the fastest variant, the same choice on every rank (by the
    # slowest rank's time of each)
    names = sorted(variants)
    worst = [max_over_ranks(variants[n_][0], ws) for n_ in names]
    head = names[int(np.argmin(worst))]
    use_pruned = head.startswith("pruned")
    use_learned = head.startswith("learned") or use_pruned
    use_graph = head.endswith("graph")
    # the index state of the chosen path for the end-to-end leg (a plan
    # re-captures itself after a state change)
    if pruned is not None:
        if use_pruned:
            ix.pruner_theta(pruned["theta"])
            ix.set_predictor_params(*pruned["state"])
        elif learned_state is not None:
            ix.pruner_theta(-1.0)
            ix.set_predictor_params(*learned_state)
    ms_max = worst[names.index(head)]
    clocks = variants[head][1]
    value = weak_value(CFG["nq"], ws, ms_max)
    if use_pruned:
        stage_avg, launches, stats = pruned["stage"], pruned["launches"], pruned["stats"]
    elif use_learned:
        stage_avg, launches, stats = learned["stage"], learned["launches"], learned["stats"]
    else:
        stage_avg, launches, stats = plain_stage, plain_launches, stats
    stage_ms = {s_: [v] for s_, v in stage_avg.items()}
    # end to end through the same public API with host buffers
    Qpin = torch.from_numpy(Qh).pin_memory()
    ids_h = torch.empty((CFG["nq"], k), dtype=torch.int64).pin_memory()
    d_h = torch.empty((CFG["nq"], k), dtype=torch.float32).pin_memory()
    Qtmp = torch.empty_like(Qd)
    e2e_ms = []
    es = gst if use_graph else st
    with torch.cuda.stream(es):
        for it in range(args.warmup + args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(es)
            Qtmp.copy_(Qpin, non_blocking=True)
            if use_graph:
                r_ids, r_d = (prplan if use_pruned else (lplan if use_learned else pplan)).execute(Qtmp, ids, dists)
            elif use_learned:
                r_ids, r_d, _, _ = ix.search_adaptive(Qtmp, k)
            else:
                r_ids, r_d = ix.search(Qtmp, k, nprobe, R, opts=sopts, out=(ids, dists))
            ids_h.copy_(r_ids, non_blocking=True)
            d_h.copy_(r_d, non_blocking=True)
            e1.record(es)
            e1.synchronize()
            if it >= args.warmup:
                e2e_ms.append(e0.elapsed_time(e1))
    e2e = weak_value(CFG["nq"], ws, max_over_ranks(statistics.mean(e2e_ms), ws))
    # roofline of the dominant kernel (the LUT16 scan), taken on the plain
    # step of this run (same kernel; its DRAM traffic was captured with ncu on
    # that step): lookups per search
    probes, _ = ix.rank_lists(Qd, nprobe, want_scores=False)
    sizes = np.bincount(ix.export()["assign"], minlength=CFG["nlist"]) if rank == 0 else None
    out = None
    if rank == 0:
        pr = probes.cpu().numpy()
        pairs_vecs = int(sizes[pr].sum())
        lookups = pairs_vecs * CFG["M"]
        code_bytes = pairs_vecs * CFG["M"] // 2
        # the scan runs in two launches (nearest lists, then the rest); the
        # first stage also holds the threshold kernel between them
        scan_ms = plain_stage["scan"] + plain_stage["near_scan"]
        peak_gl, peak_slot_gl = ksc.lut16_peak()
        achieved_gl = lookups / (scan_ms * 1e-3) / 1e9
        peaks = measured_peaks()
        # streaming form of the scan (few queries, each list read once from
        # DRAM): 8 queries at nprobe 128, L2 flushed before each search; code
        # bytes of the probed lists over the time of the two scan stages
        Bs, Ps = 8, 128
        qs8 = Qd[:Bs].contiguous()
        sbytes = int(sizes[ix.rank_lists(qs8, Ps, want_scores=False)[0].cpu().numpy()].sum()) * CFG["M"] // 2
        ix.profile(True)
        st_ms = []
        for it in range(args.warmup + 5):
            flush.zero_()
            ix.search(qs8, k, Ps, R)
            pp, _ = ix.profile_read()
            if it >= args.warmup:
                st_ms.append(pp["scan"] + pp["near_scan"])
        ix.profile(False)
        sms = statistics.median(st_ms)
        stream = {"queries": Bs, "nprobe": Ps, "code_bytes": sbytes, "scan_ms": round(sms, 4),
                  "GBps": round(sbytes / (sms * 1e-3) / 1e9, 1),
                  "frac_of_hbm": round(sbytes / (sms * 1e-3) / 1e9 / peaks.get("hbm_gbs", 6800.0), 4),
                  "frac_of_nominal": round(sbytes / (sms * 1e-3) / 1e9 / HBM_NOMINAL_GBS, 4),
                  "l2": "flushed before each search"}
        # a read-only streaming rate of this run (a 2 GB reduction), the third
        # denominator of the streaming figure
        try:
            rbuf = torch.ones(1 << 29, dtype=torch.float32, device=Qd.device)
            rs = []
            for it in range(args.warmup + 5):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                rbuf.sum()
                e1.record()
                e1.synchronize()
                if it >= args.warmup:
                    rs.append(e0.elapsed_time(e1))
            read_gbs = rbuf.numel() * 4 / (statistics.median(rs) * 1e-3) / 1e9
            del rbuf
            stream["read_stream_GBps"] = round(read_gbs, 1)
            stream["frac_of_read_stream"] = round(sbytes / (sms * 1e-3) / 1e9 / read_gbs, 4)
        except Exception as ex:  # reported, never fatal
            stream["read_stream_error"] = str(ex)[:200]
        # the opt-in tensor-core scan on the plain step: its results against the
        # plain search's and its two scan stages (L2 flushed before each search)
        tcs = None
        if not args.scan_tc:
            try:
                to = ksc.search_opts(scan_tc=True)
                r0 = ix.search(Qd, k, nprobe, R)
                r1 = ix.search(Qd, k, nprobe, R, opts=to)
                same = bool(torch.equal(r0[0], r1[0]) and torch.equal(r0[1], r1[1]))
                ix.profile(True)
                tn, tsc = [], []
                for it in range(args.warmup + 5):
                    flush.zero_()
                    ix.search(Qd, k, nprobe, R, opts=to)
                    pp, _ = ix.profile_read()
                    if it >= args.warmup:
                        tn.append(pp["near_scan"])
                        tsc.append(pp["scan"])
                ix.profile(False)
                tcs = {"kernel": "k_scan_tc (opt-in: ksc_search_opts.scan_tc)", "results_equal_plain": same,
                       "status": ix.last_status(), "near_scan_ms": round(statistics.median(tn), 4),
                       "scan_ms": round(statistics.median(tsc), 4),
                       "plain_near_scan_ms": round(plain_stage["near_scan"], 4),
                       "plain_scan_ms": round(plain_stage["scan"], 4)}
            except Exception as ex:  # reported, never fatal to the benchmark line
                ix.profile(False)
                tcs = {"error": str(ex)[:200]}
        # a1 on the tensor cores: the list-score call (query conversion + the
        # tcgen05 GEMM, 2 nq L d flops) with 16-bit and with FP8 operands, and
        # the plain step with FP8 ranking (same probes: the band is re-scored)
        gemm = {}
        try:
            for mode, name in ((1, "16bit"), (2, "fp8_e4m3")):
                for _ in range(3):
                    ix.list_scores(Qd, tensor_cores=mode)
                ts = []
                for _ in range(10):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    ix.list_scores(Qd, tensor_cores=mode)
                    e1.record()
                    e1.synchronize()
                    ts.append(e0.elapsed_time(e1))
                gms = statistics.median(ts)
                fl = 2.0 * CFG["nq"] * CFG["nlist"] * CFG["d"]
                tf = fl / (gms * 1e-3) / 1e12
                pk = peaks["bf16_tflops_sustained"] * (2.0 if mode == 2 else 1.0)
                gemm[name] = {"ms": round(gms, 4), "flops": fl, "TFLOPs": round(tf, 1), "peak_TFLOPs": round(pk, 1),
                              "frac": round(tf / pk, 4),
                              "peak_source": "bf16 sustained of MEASURED_PEAKS.json" +
                                             (" x 2 (nominal fp8 / bf16 ratio)" if mode == 2 else "")}
            f8o = ksc.search_opts(rank_fp8=True)
            r8 = ix.search(Qd, k, nprobe, R, opts=f8o)
            r16 = ix.search(Qd, k, nprobe, R)
            stg8, ms8 = stage_median(ix, lambda: ix.search(Qd, k, nprobe, R, opts=f8o), flush, 3, 5)
            gemm["plain_step_fp8_ranking"] = {"ms": round(ms8, 4), "rank_ms": round(stg8["rank"], 4),
                                              "results_equal_16bit_ranking": bool(torch.equal(r8[0], r16[0]) and
                                                                                   torch.equal(r8[1], r16[1]))}
            gemm["note"] = "call time of ksc_list_scores (query conversion + GEMM); tensor-pipe share from ncu in profiles/"
        except Exception as ex:  # reported, never fatal
            gemm["error"] = str(ex)[:200]
        # re-rank of the plain step: algorithmic bytes (R gathered rows of d
        # floats per query) over the measured stage time; rows re-read by
        # several queries may come from L2, so this is an effective rate
        rr_bytes, rr_ms = CFG["nq"] * R * CFG["d"] * 4, plain_stage.get("rerank", 0.0)
        rr_rate = rr_bytes / (rr_ms * 1e-3) / 1e9 if rr_ms > 0 else None
        cpu = cpu_baseline(ix, X, Qh, nprobe, R, k, true_d) if (ws == 1 and not args.no_cpu) else None
        plain = {"value": round(CFG["nq"] / (plain_ms * 1e-3), 1), "ms_per_step": round(plain_ms, 4),
                 "nprobe": nprobe, "rerank": R, "recall@10": recall,
                 "stage_ms": {s_: round(v, 4) for s_, v in plain_stage.items()}}
        lrn = None if learned is None else {
            "value": round(CFG["nq"] / (learned["ms"] * 1e-3), 1), "ms_per_step": round(learned["ms"], 4),
            "recall@10": round(learned["recall"], 4), "mean_nprobe": round(learned["mean_nprobe"], 3),
            "mean_rerank": round(learned["mean_rerank"], 1),
            "eq2": learned["params"], "validation_recall@10": round(learned["val_recall"], 4),
            "train_queries": args.ntrain, "train_loss": round(learned["train_loss"], 4),
            "train_s": learned["train_s"], "vs_plain": round(plain_ms / learned["ms"], 3),
            "stage_ms": {s_: round(v, 4) for s_, v in learned["stage"].items()}}
        prn = None if pruned is None else {
            "value": round(CFG["nq"] / (pruned["ms"] * 1e-3), 1), "ms_per_step": round(pruned["ms"], 4),
            "recall@10": round(pruned["recall"], 4), "mean_lists_searched": round(pruned["mean_lists"], 3),
            "mean_rerank": round(pruned["mean_rerank"], 1), "theta": pruned["theta"], "eq2": pruned["params"],
            "validation_recall@10": round(pruned["val_recall"], 4), "train_loss": round(pruned["train_loss"], 4),
            "train_s": pruned["train_s"], "vs_learned": round(learned["ms"] / pruned["ms"], 3),
            "stage_ms": {s_: round(v, 4) for s_, v in pruned["stage"].items()}}
        out = {
            "metric": METRIC,
            "value": round(value, 1), "unit": "queries/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_max, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8 LUT / int32 ADC, fp32 rank+rerank",
            "data": "synthetic (seeded mixture, SIFT1M shape)",
            "config": {"workload": CFG["workload"], "n": CFG["n"], "d": CFG["d"], "nq": CFG["nq"],
                       "nlist": CFG["nlist"], "M": CFG["M"], "nbits": 4, "k": k, "rerank": R,
                       "nprobe": nprobe, "recall@10": recall, "nprobe_sweep": sweep,
                       "l2": "flushed (256 MB write) before every timed step", "parallelism": "replica x%d" % ws},
            "recall@10": round(pruned["recall"], 4) if use_pruned else (
                round(learned["recall"], 4) if use_learned else recall),
            "path": ("learned nprobe (MLP + Eq. 2) + predictive cluster pruning" if use_pruned else
                     ("learned nprobe (MLP + Eq. 2)" if use_learned else "plain fixed nprobe")) +
                    (", replayed from a CUDA graph (ksc_plan)" if use_graph else ", direct calls"),
            "variants_ms": {n_: round(w_, 4) for n_, w_ in zip(names, worst)},
            "plain": plain, "learned": lrn, "pruned": prn,
            "e2e": {"value": round(e2e, 1), "unit": "queries/s",
                    "h2d_bytes_per_step": int(Qh.nbytes), "d2h_bytes_per_step": int(ids_h.numel() * 12)},
            "gpu_launches": launches,
            "search_stats": stats,
            "stage_ms": {s_: round(statistics.mean(v), 4) for s_, v in stage_ms.items()},
            "roofline": {"bound": "alu", "kernel": "k_scan (LUT16 ADC scan)", "achieved": round(achieved_gl, 1),
                         "peak": round(peak_gl, 1), "unit": "Glookup/s", "frac": round(achieved_gl / peak_gl, 4),
                         "peak_source": "measured: ksc_lut16_peak, the scan's shared-selector lookup sequence "
                                        "with no global memory traffic",
                         "peak_per_slot_sequence": round(peak_slot_gl, 1),
                         # the chip's integer-issue bound of that sequence: 64 integer-ALU
                         # lane-operations per clock per SM, 1.156 ALU operations per lookup
                         # (16 byte permutes per 16 lookups + 2.5 selector operations shared by
                         # a warp's four query slots), at the maximum SM clock
                         "integer_issue_bound": round(64 * 152 * 2.07e9 / (18.5 / 16) / 1e9, 1),
                         "frac_of_integer_issue_bound": round(achieved_gl / (64 * 152 * 2.07e9 / (18.5 / 16) / 1e9), 4),
                         "lookups_per_launch": lookups,
                         # DRAM read + write of the scan's two launches per search, from the
                         # ncu capture of the plain step (profiles/k_scan_*.md)
                         "traffic": None if sopts else SCAN_TRAFFIC_BYTES.get(nprobe),
                         "step": "plain nprobe %d search of this run" % nprobe,
                         "code_bytes_per_launch": code_bytes,
                         "effective_code_GBps": round(code_bytes / (scan_ms * 1e-3) / 1e9, 1),
                         "hbm_peak_gbs": peaks.get("hbm_gbs"),
                         # the index's codes once; DRAM traffic above them is candidate keys
                         # and L2 misses of lists re-read by many queries
                         "unique_code_bytes": CFG["n"] * CFG["M"] // 2,
                         "traffic_over_unique_code_bytes": None if sopts or SCAN_TRAFFIC_BYTES.get(nprobe) is None
                         else round(SCAN_TRAFFIC_BYTES[nprobe] / (CFG["n"] * CFG["M"] / 2), 2)},
            # re-rank of the plain step: R gathered rows of d floats per query
            # (algorithmic bytes; an effective rate, some rows hit L2).  With
            # the band (the default for L2) every candidate is first read as
            # a low-precision row (U8 here: the rows are integers in
            # [0, 255], held exactly; else BF16), so the effective rate
            # exceeds the copy peak: the band's gain, not a bandwidth
            "rerank_hbm": {"algorithmic_bytes": rr_bytes, "ms": round(rr_ms, 4) if rr_ms > 0 else None,
                           "effective_GBps": None if rr_rate is None else round(rr_rate, 1),
                           "effective_frac_of_hbm": None if rr_rate is None else
                           round(rr_rate / peaks.get("hbm_gbs", 6800.0), 4),
                           "band": "u8 rows (exact) or bf16 rows, then fp32 rows of the candidates kept",
                           "bytes_note": "algorithmic = every candidate's FP32 row; the band reads U8 rows "
                                         "(d bytes) of all and FP32 rows of those its bound keeps"},
            "scan_stream": stream,
            "rank_gemm": gemm,
            "scan_tc": tcs,
            "clocks": clocks,
            "build_s": round(build_s, 2),
            "cpu_baseline": cpu,
        }
        if ws == 1 and not args.no_extra:
            # the other configurations, compact (not the headline): the 10M x 96
            # index (streaming scan, batches with per-query nprobe) and the
            # 1.2M x 100 inner-product index (re-rank precision variants)
            for name, fn in (("deep", lambda: deep_workload(torch, ksc, synth, dev, flush, args)),
                             ("glove", lambda: glove_workload(torch, ksc, synth, dev, flush))):
                try:
                    out[name] = fn()
                except Exception as ex:  # reported, never fatal to the headline line
                    out[name] = {"error": str(ex)[:300]}
    return out


def cpu_model():
    """The host CPU as /proc/cpuinfo names it (model name on x86, the
    implementer / part codes on Arm), or None."""
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return None
    fields = {}
    for line in info:
        if ":" in line:
            k_, v_ = line.split(":", 1)
            fields.setdefault(k_.strip(), v_.strip())
    if "model name" in fields:
        return fields["model name"]
    if "CPU part" in fields:
        return "Arm implementer %s part %s" % (fields.get("CPU implementer", "?"), fields["CPU part"])
    return None


def cpu_baseline(ix, X, Qh, nprobe, R, k, true_d, budget_s=12.0):
    """The CPU oracle (as it stands) on a bounded sample of the same queries,
    all host cores, on the same (exported) index."""
    import oracle
    e = ix.export()
    oix = oracle.make_index(X, e["c_rank"], e["c_mean"], e["codebook"], e["codes"], e["assign"])
    cores = os.cpu_count() or 1
    n = 64
    t0 = time.time()
    oracle.search(oix, Qh[:n], nprobe, R, k, nthreads=cores)
    dt = time.time() - t0
    n2 = int(min(len(Qh), max(n, n * budget_s / max(dt, 1e-3))))
    t0 = time.time()
    res = oracle.search(oix, Qh[:n2], nprobe, R, k, nthreads=cores)
    dt = time.time() - t0
    rec = oracle.recall(Qh[:n2], X, res["ids"], true_d[:n2], 10)
    # one core, for reference (a small sample)
    n1 = 32
    t0 = time.time()
    oracle.search(oix, Qh[:n1], nprobe, R, k, nthreads=1)
    one_core = n1 / (time.time() - t0)
    return {"value": round(n2 / dt, 1), "unit": "queries/s", "cores": cores, "kind": "oracle",
            "cpu": cpu_model(), "one_core_value": round(one_core, 1),
            "sample": "first %d of the 10k queries, same index / nprobe %d / rerank %d (OpenMP over queries)"
                      % (n2, nprobe, R), "recall@10": round(rec, 4), "seconds": round(dt, 2)}


def stage_median(ix, fn, flush, warm, reps):
    """Per-stage library times (median over `reps` calls, L2 flushed before
    each) and the median wall time of the call on the current stream."""
    import torch
    for _ in range(warm):
        fn()
    ix.profile(True)
    st, tot = [], []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        pp, _ = ix.profile_read()
        st.append(pp)
        tot.append(e0.elapsed_time(e1))
    ix.profile(False)
    return {k_: statistics.median([p_[k_] for p_ in st]) for k_ in st[0]}, statistics.median(tot)


def deep_workload(torch, ksc, synth, dev, flush, args, batches=(16, 1024, 16384), stream_batches=(16, 64, 256),
                  stream_reps=5, stream_nprobe=256):
    """The 10M x 96 configuration (unit-norm, Zipf(1.1) components, nlist 8192,
    M 48, k 100, rerank 1000), built on the GPU.

    stream: the scan where it streams its codes from DRAM (the 240 MB code
    array is larger than L2): batches of 16 .. 256 queries at nprobe 256, L2
    flushed before each search.  Per-(query, list) code bytes (each pair reads
    its list's n_p M / 2 bytes) over the time of the two scan stages, against
    the measured HBM copy peak; the unique code bytes those pairs touch (the
    DRAM bytes of an ideal cluster-major schedule) beside them.
    batches: per-query nprobe U{4..256}, the variable-nprobe path, autotuned
    from 256 queries up; recall@100 on a 1000-query sample."""
    c = synth.CONFIGS[4]
    out = {}
    t0 = time.time()
    X = synth.base(4)
    out["gen_s"] = round(time.time() - t0, 1)
    Xd = torch.from_numpy(X).to(dev)
    del X
    t0 = time.time()
    ix = ksc.build_index(Xd, c["L"], c["M"], spherical=True, perm=synth.build_perm(4, c["n"]))
    torch.cuda.synchronize()
    out["build_s"] = round(time.time() - t0, 1)
    k, R, M = c["k"], c["R"], c["M"]
    sizes = np.bincount(ix.export(fields=("assign",))["assign"], minlength=c["L"])
    peaks = measured_peaks()
    nq_max = max(list(batches) + list(stream_batches) + [1000])
    Qh = synth.queries(4, nq_max)
    Qd = torch.from_numpy(Qh).to(dev)
    stream = {}
    for B in stream_batches:
        q = Qd[:B].contiguous()
        pr = ix.rank_lists(q, stream_nprobe, want_scores=False)[0].cpu().numpy()
        cb = int(sizes[pr].sum()) * M // 2
        ub = int(sizes[np.unique(pr)].sum()) * M // 2
        stg, tot = stage_median(ix, lambda: ix.search(q, k, stream_nprobe, R), flush, 3, stream_reps)
        sms = stg["near_scan"] + stg["scan"]
        gbs = cb / (sms * 1e-3) / 1e9
        tr = DEEP_STREAM_TRAFFIC_BYTES.get((B, stream_nprobe))
        stream[str(B)] = {"nprobe": stream_nprobe, "code_bytes": cb, "unique_code_bytes": ub,
                          "dram_bytes_ncu": tr, "dram_over_unique": None if tr is None else round(tr / ub, 3),
                          "scan_ms": round(sms, 4), "search_ms": round(tot, 4), "GBps": round(gbs, 1),
                          "frac_of_hbm": round(gbs / peaks["hbm_gbs"], 4),
                          "frac_of_nominal": round(gbs / HBM_NOMINAL_GBS, 4),
                          "stage_ms": {k_: round(v_, 4) for k_, v_ in stg.items()}}
    if stream:
        out["scan_stream_deep"] = {"l2": "flushed (256 MB write) before each search", "rerank": R, "k": k,
                                   "batches": stream, "hbm_peak_gbs": peaks["hbm_gbs"],
                                   "peak_source": peaks.get("source")}
    if batches:
        npb = torch.from_numpy(synth.per_query_nprobe(4, nq_max)).to(dev)
        rr = torch.full((nq_max,), R, dtype=torch.int32, device=dev)
        ns = 1000
        ids, _ = ix.search_varprobe(Qd[:ns], k, npb[:ns], rr[:ns], nprobe_max=256, rerank_max=R)
        kth = kth_fp32(torch, Xd, Qd[:ns], k, chunk=64)
        d = ((Xd[ids.clamp_min(0)] - Qd[:ns, None, :]) ** 2).sum(-1)
        out["recall@100_sample1000"] = round(float(((d <= kth[:, None] + 1e-5) & (ids >= 0)).sum(1)
                                                 .clamp_max(k).double().mean() / k), 4)
        res = {}
        for B in batches:
            q, nb = Qd[:B], npb[:B]
            # tuned at the mean of the nprobe distribution
            o = ix.autotune(q, k, 130, R)[0] if B >= 256 else ksc.search_opts()
            fn = lambda: ix.search_varprobe(q, k, nb, rr[:B], nprobe_max=256, rerank_max=R, opts=o)
            stg, ms = stage_median(ix, fn, flush, 3, 5)
            sts = ix.search_stats()
            res[str(B)] = {"ms": round(ms, 4), "qps": round(B / (ms * 1e-3), 1),
                           "candidates_per_query": round(sts["candidates"] / B, 1),
                           "overflow_queries": sts["overflow_queries"],
                           "lanes_per_query": o.lanes_per_query, "tile_blocks": o.tile_blocks,
                           "stage_ms": {s_: round(v, 4) for s_, v in stg.items()}}
        out["batches"] = res
    del ix, Xd
    torch.cuda.empty_cache()
    return out


def glove_workload(torch, ksc, synth, dev, flush):
    """The 1.2M x 100 inner-product configuration (nlist 2048, M 50, k 10):
    FP32 re-rank of R = 200 against BF16 / FP8-e4m3 re-rank of a widened
    shortlist (400, 800) before the FP32 re-rank of the best 100, each at the
    smallest nprobe reaching recall@10 0.90."""
    c = synth.CONFIGS[3]
    X = synth.base(3)
    Xd = torch.from_numpy(X).to(dev)
    del X
    ix = ksc.build_index(Xd, c["L"], c["M"], metric="ip", spherical=True, perm=synth.build_perm(3, c["n"]))
    Qh = synth.queries(3)
    Qd = torch.from_numpy(Qh).to(dev)
    k = c["k"]
    sims = []
    for b in range(0, len(Qh), 2048):
        sims.append(torch.topk(Qd[b:b + 2048] @ Xd.T, k, dim=1).values[:, k - 1])
    kth = torch.cat(sims)
    res = {}
    for name, opts, Rw in (("fp32_R200", None, 200),
                           ("bf16_Rw400_Rf100", ksc.search_opts(precision=1, rerank_final=100), 400),
                           ("fp8_Rw800_Rf100", ksc.search_opts(precision=2, rerank_final=100), 800)):
        for P in (8, 12, 16, 24, 32, 48, 64):
            ids, dd = ix.search(Qd, k, P, Rw, opts=opts)
            sim = (Xd[ids.clamp_min(0)] * Qd[:, None, :]).sum(-1)
            rec = float(((sim >= kth[:, None] - 1e-5) & (ids >= 0)).sum(1).clamp_max(k).double().mean() / k)
            if rec >= TARGET_RECALL:
                break
        stg, ms = stage_median(ix, lambda: ix.search(Qd, k, P, Rw, opts=opts), flush, 3, 5)
        res[name] = {"nprobe": P, "recall@10": round(rec, 4), "ms": round(ms, 4), "qps": round(len(Qh) / (ms * 1e-3), 1),
                     "rerank_ms": round(stg["rerank"], 4)}
    del ix, Xd
    torch.cuda.empty_cache()
    return {"variants": res, "n": c["n"], "d": c["d"], "nlist": c["L"], "M": c["M"], "metric_space": "inner product"}


def measured_peaks():
    """Measured GB300 peaks (copy bandwidth, BF16 GEMM) from MEASURED_PEAKS.json,
    else fixed fallback figures."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        pk = json.load(open(path))
        pk["source"] = "measured (MEASURED_PEAKS.json)"
        return pk
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


def run_workload(args):
    """Secondary workloads (one JSON line each, not the headline):
    deep  -- 10M x 96 unit-norm, Zipf(1.1) components, nlist 8192, M 48,
             k 100, rerank 1000, per-query nprobe U{4..256}, batches 1..16384
             through the variable-nprobe path, plans (CUDA graphs) and the
             autotuner; recall on a 1000-query sample.
    glove -- 1.2M x 100 unit-norm, inner product, nlist 2048, M 50, k 10:
             FP32 re-rank of R = 200 vs BF16 / FP8-e4m3 re-rank of a widened
             shortlist (400, 800) before the FP32 re-rank of 100.
    fashion -- 60k x 784 image-like, L2, nlist 256, M 196, k 10, rerank 200:
             component filtration (Sec. 4.3) on vs off at recall@10 >= 0.99.
    latency -- the 1M x 128 index at nprobe 7, rerank 200: single-query
             searches replayed from CUDA graphs on 1, 2, 4, 8 streams, one
             index view per stream."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2511_03298_gb300 import ksc, synth
    dev = torch.device("cuda", 0)
    out = {"workload": args.workload, "data": "synthetic (seeded mixture)", "n_gpus": 1}
    st = torch.cuda.Stream()
    if args.workload in ("deep", "stream"):
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        out.update(deep_workload(torch, ksc, synth, dev, flush, args,
                                 batches=(1, 16, 256, 1024, 4096, 16384) if args.workload == "deep" else (),
                                 stream_batches=(16, 64, 256) if args.stream_batch == 0 else (args.stream_batch,),
                                 stream_reps=5 if args.workload == "deep" else args.steps))
        out["metric"] = "QPS per batch size (per-query nprobe U{4..256}, k 100, R 1000); streaming scan GB/s"
    elif args.workload == "glove":
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        out.update(glove_workload(torch, ksc, synth, dev, flush))
        out["metric"] = "QPS at recall@10>=0.90 per re-rank precision (1.2M x 100, inner product)"
    elif args.workload == "fashion":
        # component filtration (Sec. 4.3): the same 60k x 784 image-like data
        # indexed with all dimensions and with the background ones dropped
        # (threshold 0.99, sub-vector width 4 in both), each at the smallest
        # nprobe reaching recall@10 >= 0.99 (the recall of the paper's ablation)
        c = synth.CONFIGS[6]
        X = synth.base(6)
        Xd = torch.from_numpy(X).to(dev)
        Qh = synth.queries(6)
        Qd = torch.from_numpy(Qh).to(dev)
        k, R = c["k"], c["R"]
        kth = kth_fp32(torch, Xd, Qd, k)
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        res = {}
        for name, thr in (("unfiltered", 0.0), ("filtered", 0.99)):
            t0 = time.time()
            ix = ksc.build_index(Xd, c["L"], c["M"], filter_threshold=thr, perm=synth.build_perm(6, c["n"]))
            torch.cuda.synchronize()
            b_s = time.time() - t0
            _, dims = ix.dims()
            for P in (1, 2, 3, 4, 5, 6, 8, 10, 12, 16, 24, 32, 48, 64):
                ids, _ = ix.search(Qd, k, P, R)
                dd = ((Xd[ids.clamp_min(0)] - Qd[:, None, :]) ** 2).sum(-1)
                rec = float(((dd <= kth[:, None] * (1 + 1e-5) + 1e-3) & (ids >= 0)).sum(1).clamp_max(k).double().mean() / k)
                if rec >= 0.99:
                    break
            fn = lambda: ix.search(Qd, k, P, R)
            for _ in range(3):
                fn()
            times = []
            for _ in range(args.steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                fn()
                e1.record()
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
            ms = statistics.median(times)
            ix.profile(True)
            fn()
            stg, _ = ix.profile_read()
            ix.profile(False)
            inf = ix.info()
            res[name] = {"dims": int(inf["d"]), "kept": int((dims >= 0).sum()), "M": int(inf["M"]), "nprobe": P,
                         "recall@10": round(rec, 4), "ms": round(ms, 4), "qps": round(len(Qh) / (ms * 1e-3), 1),
                         "build_s": round(b_s, 2), "stage_ms": {a_: round(v_, 4) for a_, v_ in stg.items()}}
            del ix
        out["variants"] = res
        out["speedup"] = round(res["filtered"]["qps"] / res["unfiltered"]["qps"], 3)
        out["metric"] = "QPS at recall@10>=0.99 with and without component filtration (60k x 784, L2)"
    elif args.workload == "latency":
        # single-query searches (batch 1), each replayed from a CUDA graph
        # (ksc_plan), on S streams at once through S handles on one index
        # (ksc_index_view): per-query device time and the throughput of S
        # streams, on the 1M x 128 index at the plain operating point
        c = synth.CONFIGS[2]
        X = synth.base(2)
        Xd = torch.from_numpy(X).to(dev)
        ix = ksc.build_index(Xd, c["L"], c["M"], perm=synth.build_perm(2, c["n"]))
        k, R, P, nq = 10, 200, 7, 2000
        Qd = torch.from_numpy(synth.queries(2, nq)).to(dev)
        ids_all, _ = ix.search(Qd, k, P, R)
        kth = kth_fp32(torch, Xd, Qd, k)
        dd = ((Xd[ids_all.clamp_min(0)] - Qd[:, None, :]) ** 2).sum(-1)
        out["recall@10"] = round(float(((dd <= kth[:, None] * (1 + 1e-5) + 1e-3) & (ids_all >= 0)).sum(1)
                                       .clamp_max(k).double().mean() / k), 4)
        res = {}
        for S in (1, 2, 4, 8):
            hs = [ix] + [ix.view() for _ in range(S - 1)]
            sts = [torch.cuda.Stream() for _ in range(S)]
            pls = []
            for h, s_ in zip(hs, sts):
                with torch.cuda.stream(s_):
                    pls.append(h.plan(1, k, nprobe=P, rerank=R))
                    for j in range(3):
                        pls[-1].execute(Qd[j:j + 1])
            torch.cuda.synchronize()
            cur = torch.cuda.current_stream()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(cur)
            for s_ in sts:
                s_.wait_event(t0)
            ev = []
            h0 = time.time()
            for q in range(nq):
                i = q % S
                with torch.cuda.stream(sts[i]):
                    a_ = torch.cuda.Event(enable_timing=True)
                    b_ = torch.cuda.Event(enable_timing=True)
                    a_.record(sts[i])
                    pls[i].execute(Qd[q:q + 1])
                    b_.record(sts[i])
                    ev.append((a_, b_))
            host_s = time.time() - h0
            for s_ in sts:
                cur.wait_stream(s_)
            t1.record(cur)
            t1.synchronize()
            total = t0.elapsed_time(t1)
            lat = sorted(a_.elapsed_time(b_) for a_, b_ in ev)
            res[str(S)] = {"qps": round(nq / (total * 1e-3), 1), "p50_ms": round(lat[nq // 2], 4),
                           "p99_ms": round(lat[int(nq * 0.99)], 4), "mean_ms": round(statistics.mean(lat), 4),
                           "host_us_per_query": round(host_s / nq * 1e6, 1)}
            del pls
            del hs[1:]
        out["streams"] = res
        out["config"] = {"n": c["n"], "d": c["d"], "nlist": c["L"], "M": c["M"], "k": k, "nprobe": P, "rerank": R,
                         "queries": nq}
        out["metric"] = "single-query (batch 1) device time and throughput on S streams (1M x 128)"
    print(json.dumps(out))


def run_reference(args, rank, ws):
    """The CPU oracle as the reference arm (FP64 except the 8-bit LUT rule),
    timed on the host cores: its own index over the full 1M base (FP64 Lloyd,
    OpenMP over rows), nprobe chosen on a 200-query sample with FP64 ground
    truth, then each step searches a bounded sample of 256 queries."""
    if rank != 0:
        return None
    import oracle
    from paper_2511_03298_gb300 import synth
    oracle.lib()
    X = synth.base(2)
    Qh = synth.queries(2)
    cores = os.cpu_count() or 1
    t0 = time.time()
    ix = oracle.build_index(X, CFG["nlist"], CFG["M"], False, synth.build_perm(2, len(X)), iters=20)
    build_s = time.time() - t0
    k, R = CFG["k"], CFG["rerank"]
    ns = 200
    _, true_d = oracle.exact_knn(Qh[:ns], X, k, nthreads=cores)
    nprobe, sweep = GRID[-1], {}
    for P in GRID:
        res = oracle.search(ix, Qh[:ns], P, R, k, nthreads=cores)
        sweep[P] = round(oracle.recall(Qh[:ns], X, res["ids"], true_d, k), 4)
        if sweep[P] >= TARGET_RECALL:
            nprobe = P
            break
    per = 256
    times = []
    for it in range(args.warmup + args.steps):
        b0 = (it * per) % (len(Qh) - per)
        t0 = time.time()
        oracle.search(ix, Qh[b0:b0 + per], nprobe, R, k, nthreads=cores)
        if it >= args.warmup:
            times.append(time.time() - t0)
    v = per / statistics.mean(times)
    return {"impl": "reference", "metric": METRIC,
            "value": round(v, 1), "unit": "queries/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(statistics.mean(times) * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded mixture, SIFT1M shape)",
            "config": {"workload": CFG["workload"], "n": CFG["n"], "d": CFG["d"], "nlist": CFG["nlist"],
                       "M": CFG["M"], "k": k, "rerank": R, "nprobe": nprobe, "recall@10": sweep[nprobe],
                       "nprobe_sweep": sweep, "queries_per_step": per, "oracle_build_s": round(build_s, 1)},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": round(v, 1),
                             "sample": "%d queries per step of the 10k, full 1M index built by the oracle" % per},
            "e2e": {"value": round(v, 1), "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--quick", action="store_true", help="profiling mode: timed steps only, at --nprobe")
    ap.add_argument("--quick-learned", action="store_true",
                    help="with --quick: also train the predictor briefly and time the adaptive search")
    ap.add_argument("--profile-range", action="store_true",
                    help="with --quick-learned: mark the adaptive search's steps as the profiled range")
    ap.add_argument("--nprobe", type=int, default=0)
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-nprobe path")
    ap.add_argument("--no-prune", action="store_true", help="skip predictive cluster pruning")
    ap.add_argument("--ntrain", type=int, default=100_000)
    ap.add_argument("--lanes", type=int, default=0, help="scan lanes per query (0 auto; 4, 8, 16, 32)")
    ap.add_argument("--tile-blocks", type=int, default=0, help="scan tile length in blocks (0 auto)")
    ap.add_argument("--scan-tc", type=int, default=0, help="1: the scan on the tensor cores")
    ap.add_argument("--workload", default="sift", choices=["sift", "deep", "glove", "fashion", "latency", "stream"],
                    help="sift: the headline line; deep / glove / fashion / latency: secondary workloads; "
                         "stream: the streaming scan of the 10M x 96 index alone")
    ap.add_argument("--stream-batch", type=int, default=0, help="stream workload: one batch size (0: 16, 64, 256)")
    ap.add_argument("--no-extra", action="store_true",
                    help="headline line without the 10M x 96 and 1.2M x 100 summaries")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.workload != "sift":
        run_workload(args)
        return
    rank, ws = dist_setup()
    out = run_reference(args, rank, ws) if args.impl == "reference" else run_ours(args, rank, ws)
    if rank == 0 and out is not None:
        print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
