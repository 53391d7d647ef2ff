#!/usr/bin/env python
"""Benchmark: one encrypted softmax-regression training step of HETAL on a GB300.

Workload (the configuration the headline metric is quoted on): CKKS N = 2^16,
q_0 ~ 2^60 + 11 rescale primes ~ 2^50 + 2 special primes ~ 2^61 (dnum 6),
scale 2^50; X 1024 x 768 ~ N(0,1)/sqrt(768) (24 ciphertexts of 1024 x 32
blocks), 10 classes padded to c = 16, W-bar 16 x 768 tiled vertically.
A step is DiagABT (logits/8) -> degree-15 softmax stand-in -> - Y -> DiagATB
(gradient, PRotUp branch); one step = one DiagABT + DiagATB instance pair.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun: every rank runs its own independent step
(replicas; the method has no data-path exchange), value = all ranks' steps
over the slowest rank's time.  One JSON line is printed by rank 0.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DiagABT+DiagATB ops/s at N=2^16, batched vs plain; NTT % HBM peak; p99 ms"
UNIT = "instance-pairs/s"
WORKLOAD = ("one encrypted training step (DiagABT -> degree-15 softmax stand-in -> -Y -> DiagATB): "
            "X 1024x768 N(0,1)/sqrt(768), 10 classes (c=16), 1024x32 blocks, CKKS N=2^16, "
            "12 primes (60 + 11x50 bit) + 2 special (61 bit), dnum 6, scale 2^50")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--flags", default="hoist,lazy,radix,shared",
                    help="algorithm variants: hoist (shared ModUp), lazy (relinearise sums once), "
                         "radix (SumCols/SumRows in radix steps, one ModUp and ModDown per step), "
                         "shared (PRotUp with one RotUp(B, 1); RotLeft from hoisted rotations)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched workload (independent instances: plain vs batched) in the default line")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="leave the short serving run out of the default line")
    ap.add_argument("--no-graph", action="store_true", help="time the steps call by call only")
    ap.add_argument("--kernel", default="", help="kernel to time for the roofline (default: the largest)")
    ap.add_argument("--nvtx", action="store_true", help="mark the timed steps with the NVTX range hetal_step")
    ap.add_argument("--sweep", default="", choices=["", "ntt", "rot", "word"],
                    help="primitive sweep instead of the training step: one JSON line per configuration "
                         "(ntt: batched NTT/INTT; rot: hoisted rotation batches from one ciphertext; word: 64-bit "
                         "against 32-bit RNS words at equal modulus size)")
    ap.add_argument("--sweep-logn", default="14,15,16")
    ap.add_argument("--sweep-limbs", default="1,4,12,24")
    ap.add_argument("--sweep-polys", default="1,16,64")
    ap.add_argument("--sweep-iters", type=int, default=20)
    ap.add_argument("--sweep-row-group", default="1", help="polys per CTA of the NTT row passes (--sweep ntt)")
    ap.add_argument("--sweep-rot", default="16,32,64,128", help="rotation batch sizes of --sweep rot")
    ap.add_argument("--sweep-dnum", default="2,3", help="digit counts of --sweep rot (alpha = K = 12 / dnum)")
    ap.add_argument("--sweep-blocks", type=int, default=1, help="ciphertexts rotated together in --sweep rot")
    ap.add_argument("--batched", action="store_true",
                    help="independent uneven DiagABT+DiagATB instances: plain (one after another) vs batched workers")
    ap.add_argument("--table4", action="store_true",
                    help="the five shapes of Table tab:matmul_comp at s0 = a: counts against the paper, GPU seconds")
    ap.add_argument("--nag", action="store_true",
                    help="two NAG iterations of the training step and the validation logits on a 29-prime chain")
    ap.add_argument("--train-boot", action="store_true",
                    help="several NAG iterations with W and V refreshed by bootstrapping (N=2^16)")
    ap.add_argument("--iterations", type=int, default=4, help="NAG iterations of --train-boot")
    ap.add_argument("--epochs", type=int, default=0,
                    help="with --train-boot: Protocol 1's epochs over --batches mini-batches, validation-based "
                         "early stopping (patience 3)")
    ap.add_argument("--batches", type=int, default=4, help="mini-batches of 1024 rows per epoch (--epochs)")
    ap.add_argument("--boot-per-level", type=int, default=3,
                    help="butterfly stages merged into one level of bootstrapping's transforms")
    ap.add_argument("--tb-softmax", default="asoftmax", choices=["asoftmax", "poly"],
                    help="the softmax of --train-boot: Algorithm ASoftmax with refreshes, or the degree-15 stand-in")
    ap.add_argument("--alpha", type=int, default=6,
                    help="primes per key-switching digit (and special primes) of --asoftmax and --bootstrap, "
                         "lowered where the chain would exceed 128 moduli")
    ap.add_argument("--tb-alpha", type=int, default=6,
                    help="primes per key-switching digit (and special primes) of --train-boot")
    ap.add_argument("--bootstrap", action="store_true",
                    help="CKKS bootstrapping of a full-slot level-0 ciphertext at N = 2^12, 2^14, 2^16")
    ap.add_argument("--asoftmax", action="store_true",
                    help="Algorithm ASoftmax (App. A) on the training step's 1024 x 10 logits at N=2^16, 119 levels")
    ap.add_argument("--instances", type=int, default=64)
    ap.add_argument("--fixed-flags", action="store_true",
                    help="batched workload: every instance with --flags (default: the tuner picks tile and variant)")
    ap.add_argument("--workers", type=int, default=4)
    ap.add_argument("--serve", action="store_true", help="serving loop: clients, Poisson arrivals, p50/p99")
    ap.add_argument("--clients", type=int, default=32)
    ap.add_argument("--requests", type=int, default=48)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--loads", default="0.5,0.7,0.9")
    return ap.parse_args()


def run_serve(args, d):
    """Serving (serve_measure) with the command line's clients, requests, slots and loads."""
    line = dict(mode="serve", metric=METRIC,
                **serve_measure(d, args.clients, args.requests, args.slots, [float(x) for x in args.loads.split(",")]))
    if d.rank == 0:
        print(json.dumps(line), flush=True)


def serve_measure(d, n_clients, n_requests, slots, fractions):
    """Serving: `n_clients` clients, each with its own secret and resident evaluation keys (the
    +-2^u rotation keys, conjugation, relinearisation); requests DiagABT or DiagATB with equal
    probability, rows U{256..4096}, classes U{2..100} (padded to powers of two), 768 features, block
    shapes from the tile tuner.  Capacity is measured with every request queued at once; then
    Poisson arrivals at the given fractions of it; p50 / p99 of queueing + running time per request."""
    import threading
    import torch
    import paper_2403_14111_gb300.hetal as H
    from paper_2403_14111_gb300 import workloads as wl
    dev = d.local
    torch.cuda.set_device(dev)
    P = wl.PARAMS_N16
    ctx = H.hetal_ctx_create(P["log_n"], P["q0_bits"], P["n_rescale"], P["rescale_bits"], P["n_special"],
                             P["special_bits"], P["alpha"], scale=2.0 ** P["log_scale"], device=dev)
    N, L, K = H.hetal_ctx_info(ctx)
    S = N // 2
    top = L - 1
    delta = 2.0 ** P["log_scale"]
    pow2 = [1 << u for u in range(15)] + [-(1 << u) for u in range(15)]
    t0 = time.perf_counter()
    clients = []
    for ci in range(n_clients):
        seed = 5000 + ci
        sk = H.hetal_keygen(ctx, seed)
        clients.append((seed, sk, H.hetal_evk_create(ctx, sk, seed, pow2)))
    keygen_s = time.perf_counter() - t0
    rng = np.random.default_rng(5)
    reqs, keep = [], []
    for i in range(n_requests):
        cl = int(rng.integers(0, n_clients))
        seed, sk, evk = clients[cl]
        kind = int(rng.integers(0, 2))
        a, k, b = int(rng.integers(256, 4097)), int(rng.integers(2, 101)), 768
        c = wl.pad_pow2(k)
        s0 = H.hetal_tile_choose(ctx, evk, a, b, c)
        s1 = S // s0
        X = rng.standard_normal((a, b)) / np.sqrt(b)
        if kind == 0:
            W = np.zeros((c, b))
            W[:k] = rng.standard_normal((k, b)) * 0.01
            ha = H.hetal_encrypt(ctx, sk, seed, 10 * i + 1, X, s0, s1, H.TILE_NONE, 0, top, delta)
            hb = H.hetal_encrypt(ctx, sk, seed, 10 * i + 2, W, s0, s1, H.TILE_VERT, c, top, delta)
            t = 1.0
        else:
            A = rng.uniform(-0.5, 0.5, (a, k))
            ha = H.hetal_encrypt(ctx, sk, seed, 10 * i + 3, A, s0, s1, H.TILE_HORIZ, c, top - 3, delta)
            hb = H.hetal_encrypt(ctx, sk, seed, 10 * i + 4, X, s0, s1, H.TILE_NONE, 0, top - 2, delta)
            t = 1.0 / a
        keep += [ha, hb]
        reqs.append((cl, kind, ha, hb, c, t))
    flags = H.FLAG_HOIST | H.FLAG_LAZY_RELIN
    free_b, total_b = torch.cuda.mem_get_info(dev)
    budget = int(free_b * 0.8)

    def run(arrivals):
        srv = H.hetal_server_create(ctx, slots, budget)
        ids = [H.hetal_server_add_client(ctx, srv, cl[2]) for cl in clients]
        lat, tickets, outs = [], [], []
        done = threading.Event()

        def collect():
            for tk in iter(tickets_q.get, None):
                o, q, r = H.hetal_server_wait(ctx, srv, tk)
                lat.append((q + r, q, r))
                outs.append(o)
            done.set()

        import queue
        tickets_q = queue.Queue()
        th = threading.Thread(target=collect)
        th.start()
        start = time.perf_counter()
        for (cl, kind, ha, hb, c, t), at in zip(reqs, arrivals):
            wait = start + at - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            tickets_q.put(H.hetal_server_submit(ctx, srv, ids[cl], kind, ha, hb, c, t, flags))
        tickets_q.put(None)
        th.join()
        wall = time.perf_counter() - start
        st = H.hetal_server_stats(srv)
        for o in outs:
            H.hetal_mat_free(o)
        H.hetal_server_destroy(srv)
        ms = np.array([x[0] for x in lat])
        return {"requests": len(lat), "wall_s": wall, "throughput": len(lat) / wall,
                "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
                "queue_p50_ms": float(np.percentile([x[1] for x in lat], 50)),
                "run_p50_ms": float(np.percentile([x[2] for x in lat], 50)),
                "peak_inflight_gb": st["peak_inflight_bytes"] / 1e9, "resident_keys_gb": st["resident_bytes"] / 1e9}

    run([0.0] * len(reqs))                       # warm-up (per-slot tables and masks)
    cap = run([0.0] * len(reqs))                 # capacity: everything queued at once
    loads = []
    for f in fractions:
        lam = f * cap["throughput"]
        arr = np.cumsum(np.random.default_rng(55).exponential(1.0 / lam, len(reqs)))
        r = run(list(arr))
        r["load"] = f
        r["offered_per_s"] = lam
        loads.append(r)
    out = {"unit": "requests/s", "clients": n_clients, "requests": len(reqs), "slots": slots,
           "budget_gb": budget / 1e9, "keygen_s": keygen_s, "capacity": cap, "poisson": loads}
    for h in keep:
        H.hetal_mat_free(h)
    for seed, sk, evk in clients:
        H.hetal_evk_free(evk)
        H.hetal_sk_free(sk)
    H.hetal_ctx_destroy(ctx)
    return out


def config3(args, d):
    """Batched matrix products: `instances` independent DiagABT + DiagATB instances at N = 2^16
    (rows U{256..4096}, classes U{2..100} padded to powers of two, features {384, 768, 1024}, seed
    3); block shapes from the tile tuner; DiagATB from A three levels below the top and B two
    below (PRotUp branch).  Three runs of the same jobs on the same inputs, each timed with CUDA
    events on the context's stream:
      plain         one instance after another, one diagonal k at a time (every primitive of
                    every instance its own launch: the algorithms as written);
      per_instance  one instance after another, the instance's c/2 diagonals and blocks batched;
      batched       instances grouped by block shape, every primitive of a group one launch over
                    all its instances (hetal_run_pairs_batched), the whole batch replayed as one
                    CUDA graph.
    The outputs of the three runs are compared bit for bit, a sample is decrypted against FP64,
    and the batched run gets a roofline from the paper-counted work of every instance."""
    import torch
    import paper_2403_14111_gb300.hetal as H
    from paper_2403_14111_gb300 import workloads as wl
    from paper_2403_14111_gb300 import workmodel as wm
    from paper_2403_14111_gb300.step import step_rotations
    dev = d.local
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    P = wl.PARAMS_N16
    ctx = H.hetal_ctx_create(P["log_n"], P["q0_bits"], P["n_rescale"], P["rescale_bits"], P["n_special"],
                             P["special_bits"], P["alpha"], scale=2.0 ** P["log_scale"], device=dev,
                             stream=stream.cuda_stream)
    N, L, K = H.hetal_ctx_info(ctx)
    S = N // 2
    delta = 2.0 ** P["log_scale"]
    seed = 300 + d.rank
    sk = H.hetal_keygen(ctx, seed)
    inst = wl.batched_instances(args.instances, seed=3)
    evk0 = H.hetal_evk_create(ctx, sk, seed, [1], with_conj=False, with_relin=False)
    flags = parse_flags(args.flags)
    if args.fixed_flags:   # tile from the tuner, the variant from --flags for every instance
        plans = [(H.hetal_tile_choose(ctx, evk0, i["a"], i["b"], i["c"]), flags) for i in inst]
    else:                  # tile and variant from the tuner, per instance
        plans = [H.hetal_plan_choose(ctx, evk0, i["a"], i["b"], i["c"]) for i in inst]
    H.hetal_evk_free(evk0)
    tiles = [s0 for s0, _ in plans]
    rots = set()
    for i, (s0, f) in zip(inst, plans):
        rots |= set(step_rotations(s0, S // s0, i["c"], f))
    t0 = time.perf_counter()
    evk = H.hetal_evk_create(ctx, sk, seed, sorted(rots))
    keygen_s = time.perf_counter() - t0
    top = L - 1
    jobs, handles = [], []
    for idx, (i, s0) in enumerate(zip(inst, tiles)):
        s1 = S // s0
        hX = H.hetal_encrypt(ctx, sk, seed, 10000 * idx + 1, i["X"], s0, s1, H.TILE_NONE, 0, top, delta)
        hW = H.hetal_encrypt(ctx, sk, seed, 10000 * idx + 2000, i["W"], s0, s1, H.TILE_VERT, i["c"], top, delta)
        hA = H.hetal_encrypt(ctx, sk, seed, 10000 * idx + 4000, i["A"], s0, s1, H.TILE_HORIZ, i["c"], top - 3, delta)
        hB = H.hetal_mat_drop(ctx, hX, top - 2)
        handles += [hX, hW, hA, hB]
        jobs.append(dict(x=hX, wbar=hW, a_under=hA, b=hB, c=i["c"], t_abt=1.0, t_atb=1.0 / i["a"],
                         flags=plans[idx][1]))

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        l0 = H.hetal_launch_count(ctx)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1) / 1e3, H.hetal_launch_count(ctx) - l0

    res, launches, got = {}, {}, {}
    sample = list(range(0, len(jobs), max(1, len(jobs) // 16)))
    err = [0.0]

    def keep(name, outs):
        """Residues of the sampled instances' outputs (host copies), then every output freed;
        the batched run's sample is also decrypted against FP64."""
        got[name] = [(hashlib.sha256(H.hetal_mat_export(ctx, outs[0][i]).tobytes()).hexdigest(),
                      hashlib.sha256(H.hetal_mat_export(ctx, outs[1][i]).tobytes()).hexdigest()) for i in sample]
        if name == "batched":
            for i in sample[::4]:
                it, s0 = inst[i], tiles[i]
                s1 = S // s0
                abt = H.hetal_decrypt(ctx, sk, outs[0][i])[:it["a"], :s1]
                err[0] = max(err[0], float(np.max(np.abs(abt - np.tile(it["X"] @ it["W"].T, (1, s1 // it["c"]))))))
                atb = H.hetal_decrypt(ctx, sk, outs[1][i])[:s0, :it["b"]]
                Ap = np.zeros((it["a"], it["c"]))
                Ap[:, :it["classes"]] = it["A"]
                err[0] = max(err[0], float(np.max(np.abs(atb - np.tile(Ap.T @ it["X"] / it["a"],
                                                                        (s0 // it["c"], 1))))))
        for h in outs[0] + outs[1]:
            H.hetal_mat_free(h)

    # batched: one eager run (encodes every mask), then the batch recorded once and replayed
    outs, res["batched_eager"], launches["batched_eager"] = timed(
        lambda: H.hetal_run_pairs_batched(ctx, evk, jobs, flags))
    keep("batched_eager", outs)
    try:
        H.hetal_graph_begin(ctx)
        try:
            gout = H.hetal_run_pairs_batched(ctx, evk, jobs, flags)
        except H.HetalError:
            try:
                H.hetal_graph_end(ctx)
            except H.HetalError:
                pass
            raise
        graph = H.hetal_graph_end(ctx)   # runs it once
        try:
            H.hetal_ctx_sync(ctx)
            _, res["batched"], _ = timed(lambda: H.hetal_graph_launch(ctx, graph))
            launches["batched"] = H.hetal_graph_kernels(graph)
        finally:
            H.hetal_graph_free(graph)
        keep("batched", gout)
    except H.HetalError as ex:
        print("batched: graph recording failed (%s); the eager run is the batched figure" % ex, file=sys.stderr)
        res["batched"], launches["batched"], got["batched"] = res["batched_eager"], launches["batched_eager"], \
            got["batched_eager"]
    outs, res["per_instance"], launches["per_instance"] = timed(lambda: H.hetal_run_pairs(ctx, evk, jobs, 1, flags))
    keep("per_instance", outs)
    H.hetal_ctx_set_batch_bytes(ctx, 1 << 20)   # every chunk one diagonal, every hoisted pass one amount
    outs, res["plain"], launches["plain"] = timed(lambda: H.hetal_run_pairs(ctx, evk, jobs, 1, flags))
    H.hetal_ctx_set_batch_bytes(ctx, 8 << 30)
    keep("plain", outs)
    same = all(x[k] == y[k] for m in ("per_instance", "batched_eager", "batched")
               for x, y in zip(got["plain"], got[m]) for k in (0, 1))
    err = err[0]
    n = len(jobs)

    def work(C, f):   # f: the paper's method (HOIST) or None for each instance's own variant
        w = wm.Work()
        for it, (s0, fi) in zip(inst, plans):
            w.add(wm.instance_pair(C, it["a"], it["b"], it["c"], s0, S // s0, top, fi if f is None else f))
        return w

    roof = step_roofline(H, ctx, P, res["batched"] * 1e3, work, None, measured_peaks())
    out = {"workload": "%d independent DiagABT+DiagATB instances, N=2^16, rows 256-4096, classes 2-100, features "
                       "384/768/1024 (seed 3), tuned tiles" % n,
           "flags": args.flags, "unit": UNIT,
           "plain": n / res["plain"], "per_instance": n / res["per_instance"], "batched": n / res["batched"],
           "batched_eager": n / res["batched_eager"],
           "speedup": res["plain"] / res["batched"], "speedup_vs_per_instance": res["per_instance"] / res["batched"],
           "seconds": res, "gpu_launches": launches, "bit_identical": bool(same), "compared_instances": len(sample),
           "max_abs_err": err, "rotation_keys": len(rots), "keygen_s": keygen_s, "tiles": sorted(set(tiles)),
           "plans": "tuner (tile and variant per instance)" if not args.fixed_flags else "tuner tiles, --flags",
           "variants": {str(f): sum(1 for _, g in plans if g == f) for f in sorted(set(g for _, g in plans))},
           "roofline": roof}
    for h in handles:
        H.hetal_mat_free(h)
    H.hetal_evk_free(evk)
    H.hetal_sk_free(sk)
    H.hetal_ctx_destroy(ctx)
    return out


def run_batched(args, d):
    line = dict(config3(args, d), mode="batched", metric=METRIC)
    if d.rank == 0:
        print(json.dumps(line), flush=True)


def run_ntt_sweep(args, d):
    """Batched forward + inverse NTT of polys x limbs x N uint64 residues (uniform in [0, q_i)).
    Reports butterflies/s against the register-only butterfly rate and bytes/s (one read and one write
    of every word per transform) against the measured HBM copy bandwidth."""
    import torch
    import paper_2403_14111_gb300.hetal as H
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0) * 1e9
    dev = d.local
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    for logn, group in [(int(x), int(g)) for x in args.sweep_logn.split(",") for g in args.sweep_row_group.split(",")]:
        ctx = H.hetal_ctx_create(logn, 60, 23, 50, 1, 61, 2, scale=2.0 ** 50, device=dev, stream=stream.cuda_stream)
        H.hetal_ctx_set_row_group(ctx, group)
        N = 1 << logn
        mods = H.hetal_ctx_moduli(ctx)
        peak = H.hetal_probe_butterfly_rate(ctx, 20000)
        ceil = alu_ceiling(dev)
        for limbs in [int(x) for x in args.sweep_limbs.split(",")]:
            for polys in [int(x) for x in args.sweep_polys.split(",")]:
                rng = np.random.default_rng(limbs * 1000 + polys)
                host = np.stack([rng.integers(0, mods[l], (polys, N), dtype=np.uint64) for l in range(limbs)], 1)
                buf = torch.from_numpy(host.view(np.int64)).cuda()
                torch.cuda.synchronize()
                for _ in range(2):
                    H.hetal_ntt_forward(ctx, buf.data_ptr(), polys, limbs)
                    H.hetal_ntt_inverse(ctx, buf.data_ptr(), polys, limbs)
                res = {}
                for kind, fn in (("forward", H.hetal_ntt_forward), ("inverse", H.hetal_ntt_inverse)):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize()
                    e0.record(stream)
                    for _ in range(args.sweep_iters):
                        fn(ctx, buf.data_ptr(), polys, limbs)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    res[kind] = e0.elapsed_time(e1) / args.sweep_iters
                ok = np.array_equal(buf.cpu().numpy().view(np.uint64), host) if args.sweep_iters % 2 == 0 else None
                bfly = polys * limbs * (N // 2) * logn
                byts = 2.0 * polys * limbs * N * 8
                for kind, ms in res.items():
                    line = {"sweep": "ntt", "direction": kind, "log_n": logn, "limbs": limbs, "polys": polys,
                            "row_group": group,
                            "ms": ms, "gbutterfly_per_s": bfly / (ms * 1e-3) / 1e9,
                            "frac_of_butterfly_peak": bfly / (ms * 1e-3) / peak,
                            "frac_of_alu_ceiling": bfly / (ms * 1e-3) / ceil,
                            "gb_per_s": byts / (ms * 1e-3) / 1e9, "frac_of_hbm": byts / (ms * 1e-3) / hbm,
                            "roundtrip_identity": ok}
                    if d.rank == 0:
                        print(json.dumps(line), flush=True)
                del buf
        H.hetal_ctx_destroy(ctx)


def word_size(d, polys=64, iters=20):
    """The RNS word size by measurement, at N = 2^16 and equal modulus size: the step's 12
    ciphertext primes (64-bit words, 50-60-bit primes) against as many 30-bit primes as
    reach the same log2 q (32-bit words), `polys` polynomials per transform (inputs larger
    than L2), forward NTT timed with CUDA events; and each word's butterfly in a
    register-only loop.  The unit is polynomials of the whole modulus per second."""
    import math
    import torch
    import paper_2403_14111_gb300.hetal as H
    from paper_2403_14111_gb300 import workloads as wl
    dev = d.local
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    P = wl.PARAMS_N16
    ctx = H.hetal_ctx_create(P["log_n"], P["q0_bits"], P["n_rescale"], P["rescale_bits"], P["n_special"],
                             P["special_bits"], P["alpha"], scale=2.0 ** P["log_scale"], device=dev,
                             stream=stream.cuda_stream)
    try:
        N, L, K = H.hetal_ctx_info(ctx)
        m64 = H.hetal_ctx_moduli(ctx)[:L]
        bits = sum(math.log2(q) for q in m64)
        cand, _ = H.hetal_ntt32_moduli(ctx, 40)
        l32 = next(i + 1 for i in range(40) if sum(math.log2(q) for q in cand[:i + 1]) >= bits)
        m32, _ = H.hetal_ntt32_moduli(ctx, l32)
        rng = np.random.default_rng(17)
        out = {}
        for name, mods, dt, fwd in (("u64", m64, np.uint64, H.hetal_ntt_forward),
                                    ("u32", m32, np.uint32, H.hetal_ntt32_forward)):
            host = np.stack([rng.integers(0, q, (polys, N), dtype=dt) for q in mods], 1)
            buf = torch.from_numpy(host.view(np.int64 if dt == np.uint64 else np.int32).copy()).cuda()
            torch.cuda.synchronize()
            for _ in range(3):
                fwd(ctx, buf.data_ptr(), polys, len(mods))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(iters):
                fwd(ctx, buf.data_ptr(), polys, len(mods))
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / iters
            bfly = polys * len(mods) * (N // 2) * int(math.log2(N))
            out[name] = {"limbs": len(mods), "log2_q": sum(math.log2(q) for q in mods), "ms_per_transform": ms,
                         "polys_per_s": polys / (ms * 1e-3), "gbutterfly_per_s": bfly / (ms * 1e-3) / 1e9,
                         "bytes_per_poly": len(mods) * N * np.dtype(dt).itemsize}
            del buf
        out["u64"]["probe_gbutterfly_per_s"] = H.hetal_probe_butterfly_rate(ctx, 20000) / 1e9
        out["u32"]["probe_gbutterfly_per_s"] = H.hetal_probe_butterfly32_rate(ctx, 20000) / 1e9
        for k in ("u64", "u32"):
            out[k]["frac_of_probe"] = out[k]["gbutterfly_per_s"] / out[k]["probe_gbutterfly_per_s"]
        out["u32_over_u64_at_equal_log_q"] = out["u32"]["polys_per_s"] / out["u64"]["polys_per_s"]
        out["workload"] = ("forward NTT, N=2^16, %d polynomials of log2 q = %.0f bits: %d x 64-bit words against %d x "
                           "32-bit words" % (polys, bits, L, l32))
        return out
    finally:
        H.hetal_ctx_destroy(ctx)


# Table "tab:matmul_comp" (Sec. 5.3): shapes (a, b, c) and the paper's seconds on one A40 for
# DiagABT and DiagATB (context only: another GPU, library and parameter set).
TABLE4 = [((128, 128, 4), 0.0601, 0.0415), ((256, 256, 8), 0.1211, 0.1239), ((512, 769, 4), 0.1223, 0.3343),
          ((1024, 769, 8), 0.3710, 1.2558), ((2048, 769, 16), 1.2376, 4.9970)]
# Table "tab:matnum_fixed" (App. D): CMult, Mult, Rot of DiagABT, DiagATB RotLeft branch, PRotUp branch.
TABLE4_COUNTS = {(128, 128, 4): ((4, 2, 34), (4, 2, 18), (4, 2, 18)),
                 (256, 256, 8): ((8, 8, 64), (12, 8, 72), (15, 8, 75)),
                 (512, 769, 4): ((4, 26, 50), (28, 26, 238), (40, 26, 250)),
                 (1024, 769, 8): ((8, 100, 140), (104, 100, 1008), (176, 100, 1080)),
                 (2048, 769, 16): ((16, 392, 456), (400, 392, 4328), (736, 392, 4664))}


def run_table4(args, d):
    """The shapes of Table tab:matmul_comp at s0 = a (App. C.3) on N = 2^16 with 12 primes: DiagABT
    with both inputs at the top level, DiagATB in its RotLeft branch (both at the top, as the
    paper's inputs are) and its PRotUp branch (A one level lower).  With the paper's algorithms
    (flags hoist,lazy: hoisting and lazy relinearisation change no count) the CMult / Mult / Rot
    counts are asserted against Table tab:matnum_fixed; the same products are then timed with
    --flags.  U(-1, 1) inputs; decrypted errors against FP64; the paper's A40 seconds as context."""
    import torch
    import paper_2403_14111_gb300.hetal as H
    from paper_2403_14111_gb300 import workloads as wl
    from paper_2403_14111_gb300.step import step_rotations
    dev = d.local
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    P = wl.PARAMS_N16
    ctx = H.hetal_ctx_create(P["log_n"], P["q0_bits"], P["n_rescale"], P["rescale_bits"], P["n_special"],
                             P["special_bits"], P["alpha"], scale=2.0 ** P["log_scale"], device=dev,
                             stream=stream.cuda_stream)
    N, L, K = H.hetal_ctx_info(ctx)
    S, top, delta = N // 2, L - 1, 2.0 ** P["log_scale"]
    paper_flags = H.FLAG_HOIST | H.FLAG_LAZY_RELIN
    run_flags = parse_flags(args.flags)
    sk = H.hetal_keygen(ctx, 44)
    try:
        for (a, b, c), t_abt, t_atb in TABLE4:
            s0, s1 = a, S // a
            evk = H.hetal_evk_create(ctx, sk, 44, sorted(set(step_rotations(s0, s1, c, paper_flags) +
                                                             step_rotations(s0, s1, c, run_flags))))
            rng = np.random.default_rng(a + b + c)
            A, Bm = rng.uniform(-1, 1, (a, b)), rng.uniform(-1, 1, (c, b))     # DiagABT: A B^T
            U, V = rng.uniform(-1, 1, (a, c)), rng.uniform(-1, 1, (a, b))      # DiagATB: U^T V
            hA = H.hetal_encrypt(ctx, sk, 44, 1, A, s0, s1, H.TILE_NONE, 0, top, delta)
            hB = H.hetal_encrypt(ctx, sk, 44, 100, Bm, s0, s1, H.TILE_VERT, c, top, delta)
            hU = H.hetal_encrypt(ctx, sk, 44, 200, U, s0, s1, H.TILE_HORIZ, c, top, delta)
            hUl = H.hetal_mat_drop(ctx, hU, top - 1)
            hV = H.hetal_encrypt(ctx, sk, 44, 300, V, s0, s1, H.TILE_NONE, 0, top, delta)
            line = {"mode": "table4", "shape": [a, b, c], "s0": s0, "s1": s1, "flags": args.flags,
                    "paper_a40_seconds": {"DiagABT": t_abt, "DiagATB": t_atb}}
            for name, fn, idx, want in (
                    ("DiagABT", lambda f: H.hetal_diag_abt(ctx, evk, hA, hB, c, 1.0, None, f), 0,
                     lambda o: (H.hetal_decrypt(ctx, sk, o)[:a, :s1], np.tile(A @ Bm.T, (1, s1 // c)))),
                    ("DiagATB_rotleft", lambda f: H.hetal_diag_atb(ctx, evk, hU, hV, c, 1.0 / a, None, f), 1,
                     lambda o: (H.hetal_decrypt(ctx, sk, o)[:s0, :b], np.tile(U.T @ V / a, (s0 // c, 1)))),
                    ("DiagATB_protup", lambda f: H.hetal_diag_atb(ctx, evk, hUl, hV, c, 1.0 / a, None, f), 2,
                     lambda o: (H.hetal_decrypt(ctx, sk, o)[:s0, :b], np.tile(U.T @ V / a, (s0 // c, 1))))):
                H.hetal_counters_reset(ctx)
                out = fn(paper_flags)   # also the warm-up (masks, tables)
                cnt = H.hetal_counters_get(ctx)
                counts = (cnt["cmult"], cnt["mult"], cnt["rot"])
                H.hetal_mat_free(out)
                res = {"counts": list(counts), "counts_match_paper": counts == TABLE4_COUNTS[(a, b, c)][idx]}
                for tag, f in (("paper_algorithms", paper_flags), ("flags", run_flags)):
                    H.hetal_mat_free(fn(f))   # warm-up of this variant
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize()
                    e0.record(stream)
                    out = fn(f)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    got, ref = want(out)
                    res[tag] = {"seconds": e0.elapsed_time(e1) / 1e3, "max_abs_err": float(np.max(np.abs(got - ref)))}
                    H.hetal_mat_free(out)
                line[name] = res
            for h in (hA, hB, hU, hUl, hV):
                H.hetal_mat_free(h)
            H.hetal_evk_free(evk)
            if d.rank == 0:
                print(json.dumps(line), flush=True)
    finally:
        H.hetal_sk_free(sk)
        H.hetal_ctx_destroy(ctx)


def run_nag(args, d):
    """The training loop (Protocol 1, step 3): two NAG iterations (Sec. 2.1) of the training step's
    workload and the validation logits, without bootstrapping, on N = 2^16 with 29 ciphertext
    primes (60 + 28 x 50 bits) + 2 special primes: log2 q ~ 1520, near the paper's 1555 (Sec. 5.1).
    Each iteration is timed with CUDA events; the decrypted weights and validation logits are
    compared with the same loop on FP64 matrices."""
    import torch
    import paper_2403_14111_gb300.hetal as H
    from paper_2403_14111_gb300 import workloads as wl
    from paper_2403_14111_gb300.step import nag_gammas, step_rotations, train_step
    dev = d.local
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    P = wl.PARAMS_N16_NAG
    ctx = H.hetal_ctx_create(P["log_n"], P["q0_bits"], P["n_rescale"], P["rescale_bits"], P["n_special"],
                             P["special_bits"], P["alpha"], scale=2.0 ** P["log_scale"], device=dev,
                             stream=stream.cuda_stream)
    flags = parse_flags(args.flags)
    N, L, K = H.hetal_ctx_info(ctx)
    delta, top, s0, s1 = 2.0 ** P["log_scale"], L - 1, 1024, 32
    X, Y, W1, c = wl.training_step(seed=7)
    Xval = wl.features(1024, 768, 8)
    coeffs = wl.sigmoid_cheb15()
    valid = wl.valid_mask(1024, 10, c, s0, s1)
    lr = 1.0 / 1024
    sk = H.hetal_keygen(ctx, 7)
    t0 = time.perf_counter()
    evk = H.hetal_evk_create(ctx, sk, 7, step_rotations(s0, s1, c, flags))
    keygen_s = time.perf_counter() - t0
    hX = H.hetal_encrypt(ctx, sk, 7, 1000, X, s0, s1, H.TILE_NONE, 0, top, delta)
    hXv = H.hetal_encrypt(ctx, sk, 7, 5000, Xval, s0, s1, H.TILE_NONE, 0, top, delta)
    hW = H.hetal_encrypt(ctx, sk, 7, 2000, W1, s0, s1, H.TILE_VERT, c, top, delta)
    hY = H.hetal_encrypt(ctx, sk, 7, 3000, Y, s0, s1, H.TILE_HORIZ, c, top - 8, delta)
    W = V = hW
    owned, times, levels = [], [], []
    try:
        for rep in range(2):   # the first pass warms up (masks, tables); the second is timed
            W = V = hW
            for h in owned:
                H.hetal_mat_free(h)
            owned, times, levels = [], [], []
            for gamma in nag_gammas(2):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                G, inter = train_step(ctx, evk, hX, V, hY, coeffs, valid, c, lr, delta, flags)
                for h in inter:
                    H.hetal_mat_free(h)
                Gs = H.hetal_mul_const(ctx, G, 1.0, H.hetal_mat_desc_get(V).scale)
                Wn = H.hetal_sub(ctx, V, Gs)
                dd = H.hetal_sub(ctx, W, Wn)
                gd = H.hetal_mul_const(ctx, dd, gamma, H.hetal_mat_desc_get(Wn).scale)
                Vn = H.hetal_add(ctx, Wn, gd)
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
                for h in (G, Gs, dd, gd):
                    H.hetal_mat_free(h)
                owned += [Wn, Vn]
                W, V = Wn, Vn
                levels.append(H.hetal_mat_desc_get(Vn).level)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            Lg = H.hetal_diag_abt(ctx, evk, hXv, W, c, 1.0, None, flags)
            e1.record(stream)
            torch.cuda.synchronize()
            val_ms = e0.elapsed_time(e1)
            owned.append(Lg)
        Wm, Vm = W1.copy(), W1.copy()
        cls = (np.arange(c) < 10).astype(float)
        for gamma in nag_gammas(2):
            Pm = np.polynomial.polynomial.polyval(X @ Vm.T / 8.0, coeffs) * cls
            Wn = Vm - lr * (Pm - Y).T @ X
            Vm, Wm = Wn + gamma * (Wm - Wn), Wn
        errW = float(np.max(np.abs(H.hetal_decrypt(ctx, sk, W)[:c, :768] - Wm)))
        errL = float(np.max(np.abs(H.hetal_decrypt(ctx, sk, Lg)[:1024, :c] - Xval @ Wm.T)))
        cpu = None
        if d.rank == 0 and not args.no_cpu_baseline:
            cpu = oracle_nag_baseline(dev, stream, flags)
        line = {"mode": "nag", "metric": METRIC, "cpu_baseline": cpu,
                "workload": "two NAG iterations of the training step (X 1024x768, 10 classes, c=16) and the "
                            "validation logits (1024x768), N=2^16, 29 primes (60 + 28x50 bit) + 2 special, dnum 15",
                "flags": args.flags, "ms_per_iteration": times, "validation_logits_ms": val_ms,
                "levels_after_iterations": levels, "validation_logits_level": H.hetal_mat_desc_get(Lg).level,
                "max_abs_err_W": errW, "max_abs_err_logits": errL, "keygen_s": keygen_s}
    finally:
        for h in owned + [hX, hXv, hW, hY]:
            H.hetal_mat_free(h)
        H.hetal_evk_free(evk)
        H.hetal_sk_free(sk)
        H.hetal_ctx_destroy(ctx)
    if d.rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# The oracle timed beside the deep circuits (cpu_baseline legs of --bootstrap, --asoftmax,
# --nag): the same procedure on the same small configuration, the GPU run in the same
# process; the oracle's keys are made before its clock starts, like the library's.
# ---------------------------------------------------------------------------
def _oracle_threads():
    from oracle import ckks
    return ckks.set_threads(0)


def oracle_bootstrap_baseline(gpu_ms, log_n=12, alpha=2):
    """Bootstrapping of one full-slot level-0 ciphertext by the oracle (factored transforms,
    working scale 2^55) at N = 2^log_n, against the GPU's graph time at the same N."""
    from oracle import bootstrap as bt
    from oracle import ckks, softmax as sm
    threads = _oracle_threads()
    prm = bt.BootParams()
    N = 1 << log_n
    p = ckks.Params(log_n, 60, bt.depth(prm, N) + 3, 60, alpha, 61, alpha, log_delta=40)
    o = ckks.Oracle(p, seed=5)
    for r in bt.fft_rotations(N, prm):
        o.key(ckks.kid_rot(r))
    o.key(ckks.KID_RELIN)
    o.key(ckks.KID_CONJ)
    m = np.random.default_rng(log_n).uniform(-1, 1, p.slots)
    ct = o.encrypt_int(ckks.encode(m, 2.0 ** 50, N), 0, 2.0 ** 50, 7)
    ops = sm.ScaledOps(o, 2.0 ** 55, hoist=True)
    t0 = time.perf_counter()
    out = bt.bootstrap_raised(ops, o.mod_raise(ct, p.top), N, 2.0 ** 55, prm)
    secs = time.perf_counter() - t0
    res = ckks.Ct(out.data, out.lv, out.scale * 2.0 ** 50 / float(p.q[0]))
    err = float(np.max(np.abs(o.decrypt_slots(res) - m)))
    return {"kind": "oracle", "cores": threads, "value": secs * 1e3, "unit": "ms per bootstrapping",
            "sample": "one whole bootstrapping at N=2^%d (keys made beforehand)" % log_n,
            "max_abs_err": err, "gpu_ms_same_config": gpu_ms, "oracle_over_gpu": secs * 1e3 / gpu_ms}


def _asoftmax_small_inputs(c, s0, s1, seed):
    cp = 1 << max(1, int(np.ceil(np.log2(c))))
    X = np.random.default_rng(seed).uniform(-4, 4, (s0, c))
    blk = np.zeros((s0, cp))
    blk[:, :c] = X
    return X, np.tile(blk, (1, s1 // cp))


def oracle_asoftmax_baseline(dev, stream):
    """Algorithm ASoftmax by the oracle and by the GPU on the same small configuration:
    N = 2^12, 128 rows of 3 classes (c' = 4), 89 levels."""
    import torch
    import paper_2403_14111_gb300.hetal as H
    from paper_2403_14111_gb300 import asoftmax as A
    from paper_2403_14111_gb300 import circuit
    from paper_2403_14111_gb300 import workloads as wl
    from oracle import ckks, softmax as sm
    threads = _oracle_threads()
    P = wl.PARAMS_N12_SMX4
    c, s1 = 3, 16
    o = ckks.Oracle(ckks.Params(P["log_n"], P["q0_bits"], P["n_rescale"], P["rescale_bits"], P["n_special"],
                                P["special_bits"], P["alpha"], log_delta=P["log_scale"]), seed=3)
    p = o.p
    s0 = p.slots // s1
    X, tiled = _asoftmax_small_inputs(c, s0, s1, 3)
    for r in A.rotations(c, s1):
        o.key(ckks.kid_rot(r % p.slots))
    o.key(ckks.KID_RELIN)
    delta = 2.0 ** P["log_scale"]
    M = o.encrypt_int(ckks.encode(tiled.reshape(-1), delta, p.N), p.top, delta, 5)
    t0 = time.perf_counter()
    sm.asoftmax_block(sm.ScaledOps(o, delta), M, c, s0, s1, sm.Params())
    secs = time.perf_counter() - t0
    ctx = H.hetal_ctx_create(P["log_n"], P["q0_bits"], P["n_rescale"], P["rescale_bits"], P["n_special"],
                             P["special_bits"], P["alpha"], scale=delta, device=dev, stream=stream.cuda_stream)
    cache, times = {}, []
    try:
        sk = H.hetal_keygen(ctx, 3)
        evk = H.hetal_evk_create(ctx, sk, 3, A.rotations(c, s1), with_conj=False)
        hM = H.hetal_encrypt(ctx, sk, 3, 5, tiled, s0, s1, H.TILE_NONE, 0, p.top, delta)
        for rep in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            H.hetal_mat_free(A.asoftmax(ctx, evk, hM, c, s0, s1, delta, cache=cache))
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        H.hetal_mat_free(hM)
        circuit.free_plains(cache)
        H.hetal_evk_free(evk)
        H.hetal_sk_free(sk)
    finally:
        H.hetal_ctx_destroy(ctx)
    gpu_ms = min(times[1:])
    return {"kind": "oracle", "cores": threads, "value": secs * 1e3, "unit": "ms per block",
            "sample": "Algorithm ASoftmax on one block at N=2^12 (%d rows x 3 classes, 89 levels; keys made "
                      "beforehand)" % s0, "gpu_ms_same_config": gpu_ms, "oracle_over_gpu": secs * 1e3 / gpu_ms}


def oracle_nag_baseline(dev, stream, flags):
    """Two NAG iterations and the validation logits by the oracle and by the GPU on the same
    small configuration: N = 2^13, 28 levels, X 100 x 64 (one 128 x 32 block row), 4 classes."""
    import torch
    import paper_2403_14111_gb300.hetal as H
    from paper_2403_14111_gb300 import workloads as wl
    from paper_2403_14111_gb300.step import nag_train, step_rotations
    from oracle import ckks, matmul as mm
    threads = _oracle_threads()
    P = wl.PARAMS_N13_NAG
    o = ckks.Oracle(ckks.Params(P["log_n"], P["q0_bits"], P["n_rescale"], P["rescale_bits"], P["n_special"],
                                P["special_bits"], P["alpha"], log_delta=P["log_scale"]), seed=6)
    p = o.p
    s0, s1, c, a, b = 128, 32, 4, 100, 64
    rng = np.random.default_rng(3)
    X = rng.standard_normal((a, b)) / np.sqrt(b)
    Xval = rng.standard_normal((a, b)) / np.sqrt(b)
    Y = wl.one_hot(rng.integers(0, c, a), c)
    W1 = rng.standard_normal((c, b)) * 0.1
    coeffs, valid, lr, top = wl.sigmoid_cheb15(), wl.valid_mask(a, c, c, s0, s1), 0.5 / a, p.top
    for r in step_rotations(s0, s1, c, flags):
        o.key(ckks.kid_rot(r % p.slots))
    o.key(ckks.KID_RELIN)
    o.key(ckks.KID_CONJ)

    def enc(M, lv, nonce):
        return mm.EncMat([[o.encrypt_int(ckks.encode(bl, p.delta, p.N), lv, p.delta, nonce + 64 * r + j)
                           for j, bl in enumerate(row)] for r, row in enumerate(mm.block_split(M, s0, s1))],
                         M.shape[0], M.shape[1], s0, s1)
    EX, EXv = enc(X, top, 100), enc(Xval, top, 300)
    EW = enc(mm.tile_vertical(W1, c, s0), top, 500)
    EY = enc(mm.tile_horizontal(Y, c, s1), top - 8, 700)
    ops = mm.RnsOps(o, hoist=bool(flags & 1), lazy_relin=bool(flags & 2), radix_sum=bool(flags & 4),
                    shared_rot=bool(flags & 8))
    t0 = time.perf_counter()
    mm.nag_train(ops, EX, EW, EY, coeffs, valid, c, lr, p.delta, 2, EXv)
    secs = time.perf_counter() - t0
    ctx = H.hetal_ctx_create(P["log_n"], P["q0_bits"], P["n_rescale"], P["rescale_bits"], P["n_special"],
                             P["special_bits"], P["alpha"], scale=2.0 ** P["log_scale"], device=dev,
                             stream=stream.cuda_stream)
    times = []
    try:
        sk = H.hetal_keygen(ctx, 6)
        evk = H.hetal_evk_create(ctx, sk, 6, step_rotations(s0, s1, c, flags))
        d = p.delta
        hX = H.hetal_encrypt(ctx, sk, 6, 100, X, s0, s1, H.TILE_NONE, 0, top, d)
        hXv = H.hetal_encrypt(ctx, sk, 6, 300, Xval, s0, s1, H.TILE_NONE, 0, top, d)
        hW = H.hetal_encrypt(ctx, sk, 6, 500, W1, s0, s1, H.TILE_VERT, c, top, d)
        hY = H.hetal_encrypt(ctx, sk, 6, 700, Y, s0, s1, H.TILE_HORIZ, c, top - 8, d)
        for rep in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            outs = nag_train(ctx, evk, hX, hW, hY, coeffs, valid, c, lr, d, 2, hXv, flags)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            for h in outs:
                H.hetal_mat_free(h)
        for h in (hX, hXv, hW, hY):
            H.hetal_mat_free(h)
        H.hetal_evk_free(evk)
        H.hetal_sk_free(sk)
    finally:
        H.hetal_ctx_destroy(ctx)
    gpu_ms = min(times[1:])
    return {"kind": "oracle", "cores": threads, "value": secs * 1e3, "unit": "ms per loop",
            "sample": "two NAG iterations and the validation logits at N=2^13 (X 100x64, 4 classes, 28 levels; "
                      "keys made beforehand)", "gpu_ms_same_config": gpu_ms, "oracle_over_gpu": secs * 1e3 / gpu_ms}


def oracle_train_boot_baseline(dev, stream, flags, use_asm):
    """One bootstrapped NAG iteration (the update, W and V refreshed, the validation logits) by
    the oracle and by the GPU on the same small configuration: N = 2^10, 14 training primes
    (50 bits) under the bootstrapping's 60-bit primes, X 16 x 64; 4 classes with the
    stand-in softmax, 2 with Algorithm ASoftmax (use_asm: refreshed between its stages)."""
    import torch
    import paper_2403_14111_gb300.hetal as H
    from paper_2403_14111_gb300 import asoftmax as A
    from paper_2403_14111_gb300 import bootstrap as B
    from paper_2403_14111_gb300 import circuit
    from paper_2403_14111_gb300 import workloads as wl
    from paper_2403_14111_gb300.step import nag_train_boot, train_boot_rotations, train_step_asoftmax
    from oracle import bootstrap as bt
    from oracle import ckks, matmul as mm, softmax as sm
    threads = _oracle_threads()
    log_n, top = 10, 13
    N = 1 << log_n
    prm, bprm = bt.BootParams(), B.BootstrapParams()
    n_upper = bt.depth(prm, N)
    p = ckks.Params(log_n, 60, top + 1, 50, 2, 61, 2, log_delta=50, n_upper=n_upper, upper_bits=60)
    o = ckks.Oracle(p, seed=6)
    s1 = 32
    s0, c, b = p.slots // s1, (2 if use_asm else 4), 64
    a = s0
    d_sm = 2.0 ** 32
    rng = np.random.default_rng(3)
    X = rng.standard_normal((a, b)) / np.sqrt(b)
    Xval = rng.standard_normal((a, b)) / np.sqrt(b)
    Y = wl.one_hot(rng.integers(0, c, a), c)
    W1 = rng.standard_normal((c, b)) * 0.1
    coeffs, valid, lr = wl.sigmoid_cheb15(), wl.valid_mask(a, c, c, s0, s1), 0.5 / a
    y_scale = d_sm if use_asm else p.delta
    rots = train_boot_rotations(s0, s1, c, flags, bprm)
    if use_asm:
        rots = sorted(set(rots) | set(A.rotations(c, s1)))
    for r in rots:
        o.key(ckks.kid_rot(r % p.slots))
    o.key(ckks.KID_RELIN)
    o.key(ckks.KID_CONJ)

    def enc(M, lv, nonce, sc=p.delta):
        return mm.EncMat([[o.encrypt_int(ckks.encode(bl, sc, p.N), lv, sc, nonce + 64 * r + j)
                           for j, bl in enumerate(row)] for r, row in enumerate(mm.block_split(M, s0, s1))],
                         M.shape[0], M.shape[1], s0, s1)
    EX, EXv = enc(X, top, 100), enc(Xval, top, 300)
    EW, EY = enc(mm.tile_vertical(W1, c, s0), top, 500), enc(mm.tile_horizontal(Y, c, s1), top - 8, 700, y_scale)
    ops = mm.RnsOps(o, hoist=bool(flags & 1), lazy_relin=bool(flags & 2), radix_sum=bool(flags & 4),
                    shared_rot=bool(flags & 8))
    bops = sm.ScaledOps(o, 2.0 ** 55, hoist=True)
    grad = None
    if use_asm:
        sops = sm.ScaledOps(o, d_sm)
        sops.refresh = bt.Refresher(sops, bops, prm, 2.0 ** 55)

        def grad(V):
            return bt.train_step_asoftmax(ops, sops, EX, V, EY, c, c, valid, lr, p.delta, sm.Params())[0]
    t0 = time.perf_counter()
    bt.nag_train_boot(ops, bops, EX, EW, EY, coeffs, valid, c, lr, p.delta, 1, EXv, prm, 2.0 ** 55, grad=grad)
    secs = time.perf_counter() - t0
    ctx = H.hetal_ctx_create(log_n, 60, top + 1, 50, 2, 61, 2, scale=p.delta, n_upper=n_upper, upper_bits=60,
                             device=dev, stream=stream.cuda_stream)
    times, cache, sm_cache = [], {}, {}
    try:
        sk = H.hetal_keygen(ctx, 6)
        evk = H.hetal_evk_create(ctx, sk, 6, rots)
        hX = H.hetal_encrypt(ctx, sk, 6, 100, X, s0, s1, H.TILE_NONE, 0, top, p.delta)
        hXv = H.hetal_encrypt(ctx, sk, 6, 300, Xval, s0, s1, H.TILE_NONE, 0, top, p.delta)
        hW = H.hetal_encrypt(ctx, sk, 6, 500, W1, s0, s1, H.TILE_VERT, c, top, p.delta)
        hY = H.hetal_encrypt(ctx, sk, 6, 700, Y, s0, s1, H.TILE_HORIZ, c, top - 8, y_scale)
        ggrad = None
        if use_asm:
            refresher = B.Refresher(bprm, cache=cache)

            def ggrad(V):
                return train_step_asoftmax(ctx, evk, hX, V, hY, c, c, valid, lr, p.delta, d_sm, flags,
                                           cache=sm_cache, refresh=refresher)
        for rep in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            outs = nag_train_boot(ctx, evk, hX, hW, hY, coeffs, valid, c, lr, p.delta, 1, hXv, flags,
                                  boot_prm=bprm, boot_cache=cache, grad=ggrad)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            for h in outs:
                H.hetal_mat_free(h)
        circuit.free_plains(cache)
        circuit.free_plains(sm_cache)
        for h in (hX, hXv, hW, hY):
            H.hetal_mat_free(h)
        H.hetal_evk_free(evk)
        H.hetal_sk_free(sk)
    finally:
        H.hetal_ctx_destroy(ctx)
    gpu_ms = min(times[1:])
    return {"kind": "oracle", "cores": threads, "value": secs * 1e3, "unit": "ms per iteration",
            "sample": "one bootstrapped NAG iteration (%s) and the validation logits at N=2^10 (X 16x64, %d "
                      "classes, 14 training + %d bootstrapping primes; keys made beforehand)"
                      % ("Algorithm ASoftmax, refreshed" if use_asm else "degree-15 stand-in", c, n_upper),
            "gpu_ms_same_config": gpu_ms, "oracle_over_gpu": secs * 1e3 / gpu_ms}


def run_train_boot(args, d):
    """The training loop (Protocol 1, step 3) for several NAG iterations (Sec. 2.1) with W and V
    refreshed by bootstrapping (Sec. 2.2) after every update, so that the number of iterations
    is not bounded by the prime chain: N = 2^16, 15 training primes (60 + 14 x 50 bits) under
    the bootstrapping's 60-bit primes and 2 special primes, the training step's workload
    (X 1024x768, 10 classes padded to 16; W and V are 24 ciphertexts each, whose 16 distinct
    rows are packed into one ciphertext for the refresh).  The bootstrapping plaintexts are
    uploaded to the device in the first iteration and reused.  The softmax is Algorithm
    ASoftmax (App. A) at scale 2^32, refreshed between its stages (--tb-softmax asoftmax, Y
    then at 2^32), or the degree-15 stand-in (poly).  Each iteration is timed with CUDA
    events; the decrypted weights and validation logits are compared with the same loop on
    FP64 matrices (with the slot simulator's ASoftmax)."""
    import torch
    import paper_2403_14111_gb300.hetal as H
    from paper_2403_14111_gb300 import asoftmax as A
    from paper_2403_14111_gb300 import bootstrap as B
    from paper_2403_14111_gb300 import circuit
    from paper_2403_14111_gb300 import workloads as wl
    from paper_2403_14111_gb300.step import (nag_gammas, nag_train_boot, refresh_packed, train_boot_rotations,
                                             train_step_asoftmax)
    dev = d.local
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    log_n, n_train, steps = 16, 14, args.iterations
    N = 1 << log_n
    bprm = B.BootstrapParams(per_level=args.boot_per_level)
    n_upper = B.levels(N, bprm)
    delta, top, s0, s1 = 2.0 ** 50, n_train - 1, 1024, 32
    alpha = args.tb_alpha
    ctx = H.hetal_ctx_create(log_n, 60, n_train, 50, alpha, 61, alpha, scale=delta, n_upper=n_upper,
                             upper_bits=60, device=dev, stream=stream.cuda_stream)
    flags = parse_flags(args.flags)
    _, L, K = H.hetal_ctx_info(ctx)
    logq = float(sum(np.log2(np.array(H.hetal_ctx_moduli(ctx), dtype=float))))
    X, Y, W1, c = wl.training_step(seed=7)
    Xval = wl.features(1024, 768, 8)
    coeffs = wl.sigmoid_cheb15()
    valid = wl.valid_mask(1024, 10, c, s0, s1)
    lr = 1.0 / 1024
    use_asm = args.tb_softmax == "asoftmax"
    d_sm = 2.0 ** 32
    rots = train_boot_rotations(s0, s1, c, flags, bprm)
    if use_asm:
        rots = sorted(set(rots) | set(A.rotations(10, s1)))
    sk = H.hetal_keygen(ctx, 7)
    t0 = time.perf_counter()
    evk = H.hetal_evk_create(ctx, sk, 7, rots)
    keygen_s = time.perf_counter() - t0
    hX = H.hetal_encrypt(ctx, sk, 7, 1000, X, s0, s1, H.TILE_NONE, 0, top, delta)
    hXv = H.hetal_encrypt(ctx, sk, 7, 5000, Xval, s0, s1, H.TILE_NONE, 0, top, delta)
    hW = H.hetal_encrypt(ctx, sk, 7, 2000, W1, s0, s1, H.TILE_VERT, c, top, delta)
    hY = H.hetal_encrypt(ctx, sk, 7, 3000, Y, s0, s1, H.TILE_HORIZ, c, top - 8, d_sm if use_asm else delta)
    cache, sm_cache, outs, line = {}, {}, [], None
    refresher = B.Refresher(bprm, cache=cache)
    grad = None
    if use_asm:
        def grad(V):
            return train_step_asoftmax(ctx, evk, hX, V, hY, 10, c, valid, lr, delta, d_sm, flags,
                                       cache=sm_cache, refresh=refresher)
    try:
        marks = []

        def mark(t):
            e = torch.cuda.Event(enable_timing=True)
            e.record(stream)
            marks.append(e)
        start = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        start.record(stream)
        t0 = time.perf_counter()
        outs = nag_train_boot(ctx, evk, hX, hW, hY, coeffs, valid, c, lr, delta, steps, hXv, flags,
                              boot_prm=bprm, boot_cache=cache, on_iteration=mark, grad=grad)
        refreshes = refresher.calls
        end = torch.cuda.Event(enable_timing=True)
        end.record(stream)
        torch.cuda.synchronize()
        wall_s = time.perf_counter() - t0
        ev = [start] + marks
        iter_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(len(marks))]
        logits_ms = marks[-1].elapsed_time(end)
        W, V, Lg = outs
        dW, dL = H.hetal_mat_desc_get(W), H.hetal_mat_desc_get(Lg)
        # the refresh of W and V on its own (packed into one ciphertext; plaintexts on the device)
        ref_ms = []
        Vd = H.hetal_mat_drop(ctx, V, 1)
        Wd = H.hetal_mat_drop(ctx, W, 1)
        try:
            for rep in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                rs = refresh_packed(ctx, evk, [Wd, Vd], c * s1, s0 // c, delta, bprm, boot_cache=cache)
                e1.record(stream)
                torch.cuda.synchronize()
                ref_ms.append(e0.elapsed_time(e1))
                for r in rs:
                    H.hetal_mat_free(r)
        finally:
            H.hetal_mat_free(Vd)
            H.hetal_mat_free(Wd)
        # one more iteration (and the logits) with every kernel timed: where the time goes
        n0 = H.hetal_launch_count(ctx)
        H.hetal_profile_kernel(ctx, "*")
        for h in nag_train_boot(ctx, evk, hX, hW, hY, coeffs, valid, c, lr, delta, 1, hXv, flags, boot_prm=bprm,
                                boot_cache=cache, grad=grad):
            H.hetal_mat_free(h)
        H.hetal_ctx_sync(ctx)
        summary = H.hetal_profile_summary(ctx)
        H.hetal_profile_kernel(ctx, "")
        launches = H.hetal_launch_count(ctx) - n0
        kernel_ms = sum(v["ms"] for v in summary.values())
        roof = kernels_roofline(H, ctx, dev, summary, log_n, alpha)
        Wm, Vm = W1.copy(), W1.copy()
        cls = (np.arange(c) < 10).astype(float)
        for gamma in nag_gammas(steps):
            if use_asm:   # the exact softmax over the 10 classes (ASoftmax approximates it)
                Z = (X @ Vm.T)[:, :10]
                E = np.exp(Z - Z.max(axis=1, keepdims=True))
                Pm = np.zeros((X.shape[0], c))
                Pm[:, :10] = E / E.sum(axis=1, keepdims=True)
            else:
                Pm = np.polynomial.polynomial.polyval(X @ Vm.T / 8.0, coeffs) * cls
            Wn = Vm - lr * (Pm - Y).T @ X
            Vm, Wm = Wn + gamma * (Wm - Wn), Wn
        errW = float(np.max(np.abs(H.hetal_decrypt(ctx, sk, W)[:c, :768] - Wm)))
        errV = float(np.max(np.abs(H.hetal_decrypt(ctx, sk, V)[:c, :768] - Vm)))
        errL = float(np.max(np.abs(H.hetal_decrypt(ctx, sk, Lg)[:1024, :c] - Xval @ Wm.T)))
        nct = H.hetal_mat_desc_get(W).m * H.hetal_mat_desc_get(W).n
        cpu = None
        if d.rank == 0 and not args.no_cpu_baseline:
            cpu = oracle_train_boot_baseline(dev, stream, flags, use_asm)
        line = {"mode": "train_boot", "metric": METRIC, "cpu_baseline": cpu, "softmax": args.tb_softmax,
                "softmax_refreshes_per_iteration": refreshes / steps if use_asm else 0,
                "errors_against": ("the loop on FP64 matrices with the exact softmax" if use_asm else
                                   "the loop on FP64 matrices with the same polynomial"),
                "workload": "%d NAG iterations of the training step (X 1024x768, 10 classes, c=16), W and V "
                            "(%d ciphertexts each, their distinct rows packed into one ciphertext) bootstrapped "
                            "after every update, and the validation logits; "
                            "N=2^16, 60 + %dx50-bit training primes, %dx60-bit bootstrapping primes, %d special, "
                            "dnum %d" % (steps, nct, n_train, n_upper, K, -(-L // alpha)),
                "flags": args.flags, "primes": L, "special": K, "log2_PQ": round(logq, 1),
                "ms_per_iteration": iter_ms, "first_iteration_includes": "bootstrapping plaintexts encoded "
                "and uploaded", "validation_logits_ms": logits_ms, "wall_s": wall_s,
                "softmax_plaintexts": len(sm_cache),
                "refresh_ms_W_and_V": ref_ms,
                "one_iteration_and_logits": {"launches": launches, "kernel_ms": kernel_ms,
                                             "roofline_top_kernels": roof,
                                             "top_kernels": {k: round(v["ms"] / kernel_ms, 4) for k, v in
                                                             sorted(summary.items(), key=lambda kv: -kv[1]["ms"])[:10]}}, "bootstrap_plaintexts": len(cache),
                "rotation_keys": len(rots), "W_level_scale": [dW.level, dW.scale],
                "logits_level": dL.level, "max_abs_err_W": errW, "max_abs_err_V": errV,
                "max_abs_err_logits": errL, "keygen_s": keygen_s,
                "paper_a40_s_per_iteration": [4.29, 15.72]}
    finally:
        for h in list(outs) + [hX, hXv, hW, hY]:
            H.hetal_mat_free(h)
        circuit.free_plains(cache)
        circuit.free_plains(sm_cache)
        H.hetal_evk_free(evk)
        H.hetal_sk_free(sk)
        H.hetal_ctx_destroy(ctx)
    if d.rank == 0 and line is not None:
        print(json.dumps(line), flush=True)


def run_protocol(args, d):
    """Protocol 1, step 3 at N = 2^16 (the --train-boot chain, digits of --tb-alpha primes): up to
    --epochs epochs of NAG updates over --batches mini-batches of 1024 rows (768 features, 10
    classes, seeded class-dependent features standing in for the extracted ones), the softmax
    of --tb-softmax, W and V refreshed after every update; after each epoch the validation
    logits (1024 rows) go to the client, which decrypts them, computes the cross-entropy and
    stops the training after 3 epochs without improvement; the best W is kept.  Every update
    and every validation is timed with CUDA events; the client's losses and the best W are
    compared with the same protocol on FP64 matrices with the exact softmax."""
    import torch
    import paper_2403_14111_gb300.hetal as H
    from paper_2403_14111_gb300 import asoftmax as A
    from paper_2403_14111_gb300 import bootstrap as B
    from paper_2403_14111_gb300 import circuit
    from paper_2403_14111_gb300 import workloads as wl
    from paper_2403_14111_gb300.step import (ValidationClient, nag_gammas, train_boot_rotations, train_epochs,
                                             train_step, train_step_asoftmax)
    dev = d.local
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    log_n, n_train, s0, s1, c, k = 16, 14, 1024, 32, 16, 10
    N = 1 << log_n
    bprm = B.BootstrapParams(per_level=args.boot_per_level)
    n_upper = B.levels(N, bprm)
    delta, top, d_sm, alpha = 2.0 ** 50, n_train - 1, 2.0 ** 32, args.tb_alpha
    use_asm = args.tb_softmax == "asoftmax"
    ctx = H.hetal_ctx_create(log_n, 60, n_train, 50, alpha, 61, alpha, scale=delta, n_upper=n_upper,
                             upper_bits=60, device=dev, stream=stream.cuda_stream)
    flags = parse_flags(args.flags)
    train, (Xval, yval) = wl.classification_split(args.batches, s0, 768, k, seed=11)
    W1 = np.zeros((c, 768))
    lr = 1.0 / s0
    coeffs, valid = wl.sigmoid_cheb15(), wl.valid_mask(s0, k, c, s0, s1)
    rots = train_boot_rotations(s0, s1, c, flags, bprm)
    if use_asm:
        rots = sorted(set(rots) | set(A.rotations(k, s1)))
    sk = H.hetal_keygen(ctx, 7)
    evk = H.hetal_evk_create(ctx, sk, 7, rots)
    y_scale = d_sm if use_asm else delta
    hs = []
    for b, (X, y) in enumerate(train):
        hs.append((H.hetal_encrypt(ctx, sk, 7, 1000 + 10 * b, X, s0, s1, H.TILE_NONE, 0, top, delta),
                   H.hetal_encrypt(ctx, sk, 7, 1001 + 10 * b, wl.one_hot(y, c), s0, s1, H.TILE_HORIZ, c, top - 8,
                                   y_scale)))
    hXv = H.hetal_encrypt(ctx, sk, 7, 5000, Xval, s0, s1, H.TILE_NONE, 0, top, delta)
    hW = H.hetal_encrypt(ctx, sk, 7, 2000, W1, s0, s1, H.TILE_VERT, c, top, delta)
    cache, sm_cache, best, line = {}, {}, None, None
    refresher = B.Refresher(bprm, cache=cache)

    def grad_for(hX, hY):
        if use_asm:
            return lambda V: train_step_asoftmax(ctx, evk, hX, V, hY, k, c, valid, lr, delta, d_sm, flags,
                                                 cache=sm_cache, refresh=refresher)
        return lambda V: train_step(ctx, evk, hX, V, hY, coeffs, valid, c, lr, delta, flags)
    try:
        client = ValidationClient(ctx, sk, yval, k, patience=3)
        marks = []

        def mark(epoch, b):
            e = torch.cuda.Event(enable_timing=True)
            e.record(stream)
            marks.append((epoch, b, e))
        torch.cuda.synchronize()
        start = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        t0 = time.perf_counter()
        best, epochs = train_epochs(ctx, evk, hW, [grad_for(hX, hY) for hX, hY in hs], hXv, c, delta, args.epochs,
                                    client, flags, None, bprm, boot_cache=cache, on_update=mark)
        torch.cuda.synchronize()
        wall_s = time.perf_counter() - t0
        ev = [start] + [m[2] for m in marks]
        upd_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(len(marks))]
        per_epoch_s = wall_s / epochs
        # the same protocol on FP64 matrices with the exact softmax
        Wm, Vm = W1.copy(), W1.copy()
        gammas, t, f_losses, f_ws = nag_gammas(args.epochs * args.batches), 0, [], []
        for _ in range(epochs):
            for X, y in train:
                if use_asm:   # the exact softmax (ASoftmax approximates it)
                    Z = (X @ Vm.T)[:, :k]
                    E = np.exp(Z - Z.max(axis=1, keepdims=True))
                    Pm = np.zeros((s0, c))
                    Pm[:, :k] = E / E.sum(axis=1, keepdims=True)
                else:         # the same polynomial, valid classes only
                    Pm = np.polynomial.polynomial.polyval(X @ Vm.T / 8.0, coeffs) * (np.arange(c) < k)
                Wn = Vm - lr * (Pm - wl.one_hot(y, c)).T @ X
                Vm, Wm = Wn + gammas[t] * (Wm - Wn), Wn
                t += 1
            f_losses.append(client.loss(Xval @ Wm.T))
            f_ws.append(Wm)
        err_best = float(np.max(np.abs(H.hetal_decrypt(ctx, sk, best)[:c, :768] -
                                       f_ws[int(np.argmin(client.losses))])))
        line = {"mode": "protocol", "metric": METRIC, "softmax": args.tb_softmax, "alpha": alpha,
                "workload": "Protocol 1 step 3: up to %d epochs x %d mini-batches of 1024 rows (768 features, 10 "
                            "classes, class-dependent synthetic features), NAG with W and V bootstrapped after "
                            "every update, validation logits (1024 rows) decrypted by the client after each "
                            "epoch, early stopping with patience 3, N=2^16" % (args.epochs, args.batches),
                "epochs_run": epochs, "updates": len(upd_ms), "wall_s": wall_s, "s_per_epoch": per_epoch_s,
                "ms_per_update": upd_ms, "validation_losses": client.losses,
                "fp64_losses": f_losses,
                "fp64_protocol": ("the same epochs on FP64 matrices with the exact softmax" if use_asm else
                                  "the same epochs on FP64 matrices with the same polynomial"),
                "best_epoch": int(np.argmin(client.losses)) + 1,
                "max_abs_err_best_W_vs_fp64": err_best,
                "paper_a40_s_per_iteration": [4.29, 15.72]}
    finally:
        if best is not None:
            H.hetal_mat_free(best)
        for hX, hY in hs:
            H.hetal_mat_free(hX)
            H.hetal_mat_free(hY)
        H.hetal_mat_free(hXv)
        H.hetal_mat_free(hW)
        circuit.free_plains(cache)
        circuit.free_plains(sm_cache)
        H.hetal_evk_free(evk)
        H.hetal_sk_free(sk)
        H.hetal_ctx_destroy(ctx)
    if d.rank == 0 and line is not None:
        print(json.dumps(line), flush=True)


def run_bootstrap(args, d):
    """CKKS bootstrapping (Sec. 2.2; the paper reports 159 ms at N = 2^16 on an A40, Sec. 5.1)
    of one full-slot level-0 ciphertext (messages U(-1, 1) at scale 2^50), at N = 2^12, 2^14
    and 2^16, with the factored CoeffToSlot and SlotToCoeff (butterfly stages merged --boot-per-level to
    a level).  The plaintexts are encoded by the library and uploaded to the device once (an
    untimed first run) and reused; each timed run is the whole refresh with CUDA events,
    call by call (ms_eager) and as one CUDA graph launch of the recorded calls (ms_graph)."""
    import torch
    import paper_2403_14111_gb300.hetal as H
    from paper_2403_14111_gb300 import bootstrap as B
    from paper_2403_14111_gb300 import circuit
    dev = d.local
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    rows = []
    for log_n in (12, 14, 16):
        N = 1 << log_n
        bprm = B.BootstrapParams(per_level=args.boot_per_level)
        n_rescale = B.levels(N, bprm) + 3
        alpha = min(args.alpha, 127 - n_rescale)
        ctx = H.hetal_ctx_create(log_n, 60, n_rescale, 60, alpha, 61, alpha, scale=2.0 ** 40, device=dev,
                                 stream=stream.cuda_stream)
        sk = H.hetal_keygen(ctx, 5)
        t0 = time.perf_counter()
        evk = H.hetal_evk_create(ctx, sk, 5, B.rotations(N, bprm))
        keygen_s = time.perf_counter() - t0
        m = np.random.default_rng(log_n).uniform(-1, 1, N // 2)
        s1 = 16
        h = H.hetal_encrypt(ctx, sk, 5, 7, m.reshape(N // 2 // s1, s1), N // 2 // s1, s1, H.TILE_NONE, 0, 0,
                            2.0 ** 50)
        cache, times, out = {}, [], None
        try:
            t0 = time.perf_counter()
            out = B.bootstrap(ctx, evk, h, 2.0 ** 50, prm=bprm, cache=cache)   # encodes and uploads the plaintexts
            first_s = time.perf_counter() - t0
            for rep in range(3):
                H.hetal_mat_free(out)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                out = B.bootstrap(ctx, evk, h, 2.0 ** 50, prm=bprm, cache=cache)
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            dsc = H.hetal_mat_desc_get(out)
            err = float(np.max(np.abs(H.hetal_decrypt(ctx, sk, out).reshape(-1) - m)))
            # the same refresh recorded into one CUDA graph: no host work per launch
            g_times, g_kernels, same_bits, g_error = [], None, None, None
            H.hetal_graph_begin(ctx)
            try:
                g_out = B.bootstrap(ctx, evk, h, 2.0 ** 50, prm=bprm, cache=cache)
            except H.HetalError as e:   # a call that cannot be recorded: report it, keep the eager numbers
                g_error, g_out = str(e), None
                try:
                    H.hetal_graph_end(ctx)
                except H.HetalError:
                    pass
            if g_out is not None:
                graph = H.hetal_graph_end(ctx)   # runs it once
                for rep in range(5):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize()
                    e0.record(stream)
                    H.hetal_graph_launch(ctx, graph)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    g_times.append(e0.elapsed_time(e1))
                H.hetal_ctx_sync(ctx)
                same_bits = bool(np.array_equal(H.hetal_mat_export(ctx, g_out), H.hetal_mat_export(ctx, out)))
                g_kernels = H.hetal_graph_kernels(graph)
                H.hetal_mat_free(g_out)
                H.hetal_graph_free(graph)
            H.hetal_profile_kernel(ctx, "*")
            H.hetal_mat_free(B.bootstrap(ctx, evk, h, 2.0 ** 50, prm=bprm, cache=cache))
            summary = H.hetal_profile_summary(ctx)
            H.hetal_profile_kernel(ctx, "")
            kernel_ms = sum(v["ms"] for v in summary.values())
            roof = kernels_roofline(H, ctx, dev, summary, log_n, alpha)
            pts = cache
            rows.append({"log_n": log_n, "slots": N // 2, "primes": n_rescale + 1, "alpha_and_special": alpha,
                         "roofline_top_kernels": roof,
                         "levels_used": B.levels(N, bprm), "per_level": bprm.per_level,
                         "level_after": dsc.level, "ms_graph": g_times, "graph_kernels": g_kernels,
                         "graph_same_bits": same_bits, "graph_error": g_error, "ms_eager": times,
                         "first_run_s_with_encoding": first_s,
                         "max_abs_err": err, "plaintexts": len(pts), "rotation_keys": len(B.rotations(N, bprm)),
                         "kernel_ms": kernel_ms,
                         "top_kernels": {k: round(v["ms"] / kernel_ms, 4) for k, v in
                                         sorted(summary.items(), key=lambda kv: -kv[1]["ms"])[:8]},
                         "keygen_s": keygen_s})
        finally:
            if out is not None:
                H.hetal_mat_free(out)
            circuit.free_plains(cache)
            H.hetal_mat_free(h)
            H.hetal_evk_free(evk)
            H.hetal_sk_free(sk)
            H.hetal_ctx_destroy(ctx)
    cpu = None
    if d.rank == 0 and not args.no_cpu_baseline and rows and rows[0].get("ms_graph"):
        cpu = oracle_bootstrap_baseline(min(rows[0]["ms_graph"]), rows[0]["log_n"], rows[0]["alpha_and_special"])
    line = {"mode": "bootstrap", "metric": METRIC, "cpu_baseline": cpu,
            "workload": "bootstrapping one full-slot level-0 ciphertext, messages U(-1,1) at scale 2^50, "
                        "60-bit primes (q_0 ~ 2^60), working scale 2^55, factored transforms (per_level stages a level), "
                        "digits of alpha primes and alpha special primes, plaintexts uploaded once to the device",
            "paper_a40_ms_at_n16": 159, "rows": rows}
    if d.rank == 0:
        print(json.dumps(line), flush=True)


# Table tab:softmaxerr (App. A.3), row c = 10, R = 4: (max, average) of the per-row
# sup-norm error without and with the precise inverse of the extension.
PAPER_SOFTMAXERR_C10_R4 = {"extn": (0.0153, 0.0046), "extn+prec": (0.0040, 0.0006)}


def run_asoftmax(args, d):
    """Algorithm ASoftmax (App. A) with the paper's parameters (c' = 16 for 10 classes: four
    tournament rounds, L = 2, n = 5, AExp p_12(x/8)^8, AInv with R = 100 and 16 steps), without
    and with the precise inverse of the extension, on the training step's softmax input: one
    1024 x 32 block holding 1024 rows of 10 logits tiled twice, at N = 2^16 over 119 (123)
    levels of 60-bit primes (a stand-in for the levels bootstrapping would refresh).  Timed
    with CUDA events; the decryption's per-row sup-norm errors against the exact softmax are
    put beside Table tab:softmaxerr's row c = 10, R = 4 (inputs on [-4, 4]^10).  The plaintexts are
    uploaded to the device by the first run and reused; the circuit is also recorded into one
    CUDA graph and timed per launch (ms_graph)."""
    import torch
    import paper_2403_14111_gb300.hetal as H
    from paper_2403_14111_gb300 import asoftmax as A
    from paper_2403_14111_gb300 import circuit
    from paper_2403_14111_gb300 import workloads as wl
    dev = d.local
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    c, s0, s1 = 10, 1024, 32
    rng = np.random.default_rng(17)
    X = rng.uniform(-4, 4, (s0, c))
    cp = A.padded_classes(c)
    blk = np.zeros((s0, cp))
    blk[:, :c] = X
    tiled = np.tile(blk, (1, s1 // cp))
    Z = X - X.max(axis=1, keepdims=True)
    exact = np.exp(Z) / np.exp(Z).sum(axis=1, keepdims=True)
    variants = {}
    for name, precise, P in (("extn", False, wl.PARAMS_N16_SMX16), ("extn+prec", True, wl.PARAMS_N16_SMX16P)):
        prm = A.ASoftmaxParams(precise=precise)
        delta = 2.0 ** P["log_scale"]
        alpha = min(args.alpha, 127 - P["n_rescale"])   # a context holds at most 128 moduli
        ctx = H.hetal_ctx_create(P["log_n"], P["q0_bits"], P["n_rescale"], P["rescale_bits"], alpha,
                                 P["special_bits"], alpha, scale=delta, device=dev, stream=stream.cuda_stream)
        N, L, K = H.hetal_ctx_info(ctx)
        sk = H.hetal_keygen(ctx, 17)
        t0 = time.perf_counter()
        evk = H.hetal_evk_create(ctx, sk, 17, A.rotations(c, s1), with_conj=False)
        keygen_s = time.perf_counter() - t0
        hM = H.hetal_encrypt(ctx, sk, 17, 100, tiled, s0, s1, H.TILE_NONE, 0, L - 1, delta)
        times, out, cache = [], None, {}
        try:
            for rep in range(3):   # the first run warms up and uploads the plaintexts to the device
                if out is not None:
                    H.hetal_mat_free(out)
                H.hetal_counters_reset(ctx)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                out = A.asoftmax(ctx, evk, hM, c, s0, s1, delta, prm, cache=cache)
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            cnt = H.hetal_counters_get(ctx)   # one run's operations (the recording below counts again)
            # the same circuit recorded into one CUDA graph
            g_times, g_same = [], None
            H.hetal_graph_begin(ctx)
            try:
                g_out = A.asoftmax(ctx, evk, hM, c, s0, s1, delta, prm, cache=cache)
            except H.HetalError:
                g_out = None
                try:
                    H.hetal_graph_end(ctx)
                except H.HetalError:
                    pass
            if g_out is not None:
                graph = H.hetal_graph_end(ctx)
                for rep in range(3):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize()
                    e0.record(stream)
                    H.hetal_graph_launch(ctx, graph)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    g_times.append(e0.elapsed_time(e1))
                H.hetal_ctx_sync(ctx)
                g_same = bool(np.array_equal(H.hetal_mat_export(ctx, g_out), H.hetal_mat_export(ctx, out)))
                H.hetal_mat_free(g_out)
                H.hetal_graph_free(graph)
            err = np.max(np.abs(H.hetal_decrypt(ctx, sk, out)[:, :c] - exact), axis=1)
            # one more, untimed run with every launch timed: where the kernel time goes
            H.hetal_profile_kernel(ctx, "*")
            H.hetal_mat_free(A.asoftmax(ctx, evk, hM, c, s0, s1, delta, prm, cache=cache))
            summary = H.hetal_profile_summary(ctx)
            H.hetal_profile_kernel(ctx, "")
            kernel_ms = sum(v["ms"] for v in summary.values())
            variants[name] = {
                "primes": L, "special": K, "alpha": alpha, "levels": A.depth(c, prm), "ms": times[1:],
                "ms_first": times[0],
                "ms_graph": g_times, "graph_same_bits": g_same,
                "rows_per_s": s0 / (min(times[1:] + g_times) * 1e-3),
                "err_max": float(err.max()), "err_avg": float(err.mean()),
                "paper_table_max_avg": PAPER_SOFTMAXERR_C10_R4[name],
                "counts": {k: cnt[k] for k in ("mult", "cmult", "rot", "keyswitch", "rescale")},
                "kernel_ms": kernel_ms,
                "roofline_top_kernels": kernels_roofline(H, ctx, dev, summary, P["log_n"], alpha),
                "top_kernels": {k: round(v["ms"] / kernel_ms, 4) for k, v in
                                sorted(summary.items(), key=lambda kv: -kv[1]["ms"])[:8]},
                "keygen_s": keygen_s}
        finally:
            if out is not None:
                H.hetal_mat_free(out)
            circuit.free_plains(cache)
            H.hetal_mat_free(hM)
            H.hetal_evk_free(evk)
            H.hetal_sk_free(sk)
            H.hetal_ctx_destroy(ctx)
    cpu = None
    if d.rank == 0 and not args.no_cpu_baseline:
        cpu = oracle_asoftmax_baseline(dev, stream)
    line = {"mode": "asoftmax", "metric": METRIC, "cpu_baseline": cpu,
            "workload": "Algorithm ASoftmax, 1024 rows x 10 classes (c'=16) tiled in one 1024x32 block, inputs "
                        "U(-4,4)^10, N=2^16, 60-bit primes + as many special (61 bit) as primes per digit (the "
                        "variants' alpha), scale 2^40",
            "errors": "per-row sup-norm error against the exact softmax: max and average over the rows, as in "
                      "Table tab:softmaxerr", "variants": variants}
    if d.rank == 0:
        print(json.dumps(line), flush=True)


def e2e_graph(args, d, ctx, step, host_in, descs, g_host):
    """End to end through one CUDA graph per step: the recorded calls import the three
    matrices from pinned host memory, run the step and export the gradient's residues to
    pinned host memory; every timed step is one graph launch and a wait for it."""
    import torch
    import paper_2403_14111_gb300.hetal as H

    def calls():
        mats = [H.hetal_mat_import(ctx, a, dsc) for (_, a), dsc in zip(host_in, descs)]
        G = step(*mats)
        H.hetal_mat_export(ctx, G, g_host)
        H.hetal_mat_free(G)
        for m in mats:
            H.hetal_mat_free(m)

    calls()   # eager once: the same sequence, every table and plaintext cached
    H.hetal_ctx_sync(ctx)
    H.hetal_graph_begin(ctx)
    try:
        calls()
    except H.HetalError:
        try:   # close the void recording before the context is used again
            H.hetal_graph_end(ctx)
        except H.HetalError:
            pass
        raise
    graph = H.hetal_graph_end(ctx)   # instantiates and runs it once
    try:
        kernels = H.hetal_graph_kernels(graph)
        H.hetal_ctx_sync(ctx)
        d.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            H.hetal_graph_launch(ctx, graph)
            H.hetal_ctx_sync(ctx)   # the gradient's residues are in pinned host memory
        e2e_s = d.max(time.perf_counter() - t0)
    finally:
        H.hetal_graph_free(graph)
    return {"value": args.steps * d.world / e2e_s, "graph_kernels": kernels,
            "note": "one CUDA graph launch per step (hetal_graph_*): the recorded calls copy the step's inputs "
                    "(coefficient domain) from pinned host memory, run the step and copy the gradient to pinned "
                    "host memory; the host waits for each launch"}


def e2e_overlap(args, d, ctx, P, dev, stream, step, host_in, descs, g_words):
    """End to end with the copy-in of step i+1 overlapping step i: a second context on its
    own stream imports the step's ciphertexts from pinned host memory into one of two
    alternating device sets (an import graph per set), the step runs on the main stream
    from that set and exports the gradient to that set's pinned host buffer (a compute
    graph per set), and events order them: import(i+1) waits for step(i-1) to release its
    set, step(i) waits for import(i).  The host waits for each step's gradient."""
    import torch
    import paper_2403_14111_gb300.hetal as H
    s_in = torch.cuda.Stream(dev)
    ctx_in = H.hetal_ctx_create(P["log_n"], P["q0_bits"], P["n_rescale"], P["rescale_bits"], P["n_special"],
                                P["special_bits"], P["alpha"], scale=2.0 ** P["log_scale"], device=dev,
                                stream=s_in.cuda_stream)
    g_host = []
    for _ in range(2):
        t = torch.empty(g_words, dtype=torch.int64, pin_memory=True)
        g_host.append((t, t.numpy().view(np.uint64)))
    imports, computes, mats = [], [], []
    try:
        for k in range(2):
            # eager once (tables, masks), then recorded
            ms = [H.hetal_mat_import(ctx_in, a, dsc) for (_, a), dsc in zip(host_in, descs)]
            G = step(*ms)
            H.hetal_mat_export(ctx, G, g_host[k][1])
            H.hetal_mat_free(G)
            for m in ms:
                H.hetal_mat_free(m)
            H.hetal_ctx_sync(ctx)
            H.hetal_graph_begin(ctx_in)
            ms = [H.hetal_mat_import(ctx_in, a, dsc) for (_, a), dsc in zip(host_in, descs)]
            imports.append(H.hetal_graph_end(ctx_in))
            mats.append(ms)
            H.hetal_ctx_sync(ctx_in)
            H.hetal_graph_begin(ctx)
            G = step(*ms)
            H.hetal_mat_export(ctx, G, g_host[k][1])
            H.hetal_mat_free(G)
            computes.append(H.hetal_graph_end(ctx))
            H.hetal_ctx_sync(ctx)
        kernels = H.hetal_graph_kernels(computes[0]) + H.hetal_graph_kernels(imports[0])
        ready = [torch.cuda.Event() for _ in range(2)]
        done = [torch.cuda.Event() for _ in range(2)]
        d.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        H.hetal_graph_launch(ctx_in, imports[0])
        ready[0].record(s_in)
        for i in range(args.steps):
            k = i % 2
            stream.wait_event(ready[k])
            H.hetal_graph_launch(ctx, computes[k])
            done[k].record(stream)
            if i + 1 < args.steps:
                k1 = (i + 1) % 2
                if i >= 1:
                    s_in.wait_event(done[k1])   # step i-1 has finished reading set k1
                H.hetal_graph_launch(ctx_in, imports[k1])
                ready[k1].record(s_in)
            done[k].synchronize()                # step i's gradient is in pinned host memory
        e2e_s = d.max(time.perf_counter() - t0)
        torch.cuda.synchronize()
    finally:
        torch.cuda.synchronize()
        for g in imports + computes:
            H.hetal_graph_free(g)
        for ms in mats:
            for m in ms:
                H.hetal_mat_free(m)
        H.hetal_ctx_destroy(ctx_in)
    return {"value": args.steps * d.world / e2e_s, "graph_kernels": kernels,
            "note": "two alternating input sets: each step's ciphertexts (coefficient domain) are copied in from "
                    "pinned host memory by an import graph on a second stream while the previous step computes; "
                    "each step is one compute graph launch that exports the gradient to pinned host memory, and "
                    "the host waits for every step's gradient"}


def e2e_eager(args, d, ctx, P, dev, step, host_in, descs, g_host):
    """End to end without a graph: a second context (own CUDA stream) imports the next step's
    ciphertexts from pinned host memory while this one computes; each result is exported to
    pinned host memory."""
    import ctypes
    import queue
    import threading
    import torch
    import paper_2403_14111_gb300.hetal as H
    ctx_up = H.hetal_ctx_create(P["log_n"], P["q0_bits"], P["n_rescale"], P["rescale_bits"], P["n_special"],
                                P["special_bits"], P["alpha"], scale=2.0 ** P["log_scale"], device=dev)
    ready, done = queue.Queue(maxsize=1), queue.Queue()

    def uploader(n):
        for _ in range(n):
            ready.put([H.hetal_mat_import(ctx_up, a, dsc) for (_, a), dsc in zip(host_in, descs)])
            while not done.empty():
                for m in done.get():
                    H.hetal_mat_free(m)

    d.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    th = threading.Thread(target=uploader, args=(args.steps,))
    th.start()
    for _ in range(args.steps):
        mats = ready.get()
        G = step(*mats)
        H.lib().hetal_mat_export(ctx, G, g_host.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
        H.hetal_mat_free(G)
        done.put(mats)
    th.join()
    torch.cuda.synchronize()
    d.barrier()
    e2e_s = d.max(time.perf_counter() - t0)
    while not done.empty():
        for m in done.get():
            H.hetal_mat_free(m)
    H.hetal_ctx_destroy(ctx_up)
    return {"value": args.steps * d.world / e2e_s,
            "note": "inputs imported (coefficient domain, pinned host memory) on a second context's stream "
                    "while the previous step computes; the result exported to pinned host memory every step"}


def run_rot_sweep(args, d):
    """Hoisted rotation batches: one ciphertext at N = 2^16 with 12 primes (60 + 11 x 50 bit),
    rotated by steps 1..n sharing one ModUp, against n separate rotations, and the ciphertext
    plus the sum of those n rotations with one ModUp and one ModDown (kind "sum").  dnum digits of
    alpha = 12 / dnum primes and K = alpha special primes (61 bit).  Reports rotations/s, the
    counted modular multiplications per second against the register-only butterfly rate, and
    that every hoisted result decrypts to the rolled slot vector (max error)."""
    import torch
    import paper_2403_14111_gb300.hetal as H
    dev = d.local
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    batches = [int(x) for x in args.sweep_rot.split(",")]
    for dnum in [int(x) for x in args.sweep_dnum.split(",")]:
        alpha = 12 // dnum
        ctx = H.hetal_ctx_create(16, 60, 11, 50, alpha, 61, alpha, scale=2.0 ** 50, device=dev,
                                 stream=stream.cuda_stream)
        N, L, K = H.hetal_ctx_info(ctx)
        peak = H.hetal_probe_butterfly_rate(ctx, 20000)
        ceil = alu_ceiling(dev)
        nmax = max(batches)
        sk = H.hetal_keygen(ctx, 7)
        evk = H.hetal_evk_create(ctx, sk, 7, list(range(1, nmax + 1)), with_conj=False, with_relin=False)
        rng = np.random.default_rng(11)
        s0, s1, nb = 1024, N // 2 // 1024, args.sweep_blocks
        M = rng.uniform(-1, 1, (s0, s1 * nb))
        ct = H.hetal_encrypt(ctx, sk, 7, 1, M, s0, s1, H.TILE_NONE, 0, L - 1, 2.0 ** 50)
        for n in batches:
            steps = list(range(1, n + 1))
            res = {}
            for kind in ("hoisted", "separate", "sum"):
                def once():
                    if kind == "hoisted":
                        outs = H.hetal_rotate_hoisted(ctx, evk, ct, steps)
                    elif kind == "separate":
                        outs = [H.hetal_rotate(ctx, evk, ct, r) for r in steps]
                    else:   # ct + sum of the rotations, one ModUp and one ModDown
                        outs = [H.hetal_rotate_sum(ctx, evk, ct, steps)]
                    return outs
                for h in once():
                    H.hetal_mat_free(h)
                H.hetal_ctx_sync(ctx)
                H.hetal_counters_reset(ctx)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                outs = once()
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                mm = H.hetal_counters_get(ctx)["modmul"]
                err = 0.0
                if kind == "sum":
                    dec = H.hetal_decrypt(ctx, sk, outs[0])
                    for b in (0, nb - 1):
                        blk = slice(b * s1, (b + 1) * s1)
                        z = M[:, blk].reshape(-1)
                        want = z + sum(np.roll(z, -r) for r in steps)
                        err = max(err, float(np.max(np.abs(dec[:, blk].reshape(-1) - want))))
                for i in ((0, n // 2, n - 1) if kind != "sum" else ()):
                    dec = H.hetal_decrypt(ctx, sk, outs[i])
                    for b in (0, nb - 1):
                        blk = slice(b * s1, (b + 1) * s1)
                        err = max(err, float(np.max(np.abs(dec[:, blk].reshape(-1)
                                                           - np.roll(M[:, blk].reshape(-1), -steps[i])))))
                for h in outs:
                    H.hetal_mat_free(h)
                res[kind] = (ms, mm, err)
            for kind, (ms, mm, err) in res.items():
                line = {"sweep": "rot", "kind": kind, "log_n": 16, "levels": L, "dnum": dnum, "alpha": alpha,
                        "special": K, "blocks": nb, "rotations": n, "ms": ms,
                        "rotations_per_s": n * nb / (ms * 1e-3),
                        "gmodmul_per_s": mm / (ms * 1e-3) / 1e9, "frac_of_butterfly_peak": mm / (ms * 1e-3) / peak,
                        "frac_of_alu_ceiling": mm / (ms * 1e-3) / ceil,
                        "max_abs_err": err,
                        "speedup_vs_separate": res["separate"][0] / ms if kind != "separate" else None}
                if d.rank == 0:
                    print(json.dumps(line), flush=True)
        H.hetal_mat_free(ct)
        H.hetal_evk_free(evk)
        H.hetal_sk_free(sk)
        H.hetal_ctx_destroy(ctx)


class Dist:
    """The ranks of a torchrun launch (replicas: each runs its own steps; the only collectives are
    the barrier around the timed region and the max of the ranks' times).  NCCL on GPUs, gloo
    otherwise (the host-side tests)."""

    def __init__(self, backend=None):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        self.backend = None
        if self.world > 1:
            import torch.distributed as dist
            import torch
            if backend is None:
                backend = "nccl" if torch.cuda.is_available() else "gloo"
            if backend == "nccl":
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend)
            self.pg = dist
            self.backend = backend

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, v):
        if not self.pg:
            return v
        import torch
        t = torch.tensor([v], dtype=torch.float64, device="cuda" if self.backend == "nccl" else "cpu")
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def replica_value(d, steps, ms):
    """Whole-job throughput of the replicas: every rank's steps over the slowest rank's time."""
    ms_max = d.max(ms)
    return steps * d.world / (ms_max / 1e3), ms_max


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        rows = [ln.split(",") for ln in self.f.read().splitlines() if ln.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def parse_flags(text):
    import paper_2403_14111_gb300.hetal as H
    names = {"hoist": H.FLAG_HOIST, "lazy": H.FLAG_LAZY_RELIN, "radix": H.FLAG_RADIX_SUM, "shared": H.FLAG_SHARED_ROT}
    flags = 0
    for part in filter(None, (x.strip() for x in text.split(","))):
        if part not in names:
            raise SystemExit("unknown flag %r (hoist, lazy, radix, shared)" % part)
        flags |= names[part]
    return flags


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# FMA-heavy pipe cycles (per SM sub-partition) one warp-wide NTT butterfly occupies, measured with
# ncu on the register-only butterfly probe (the FMA-heavy pipe's busy cycles per warp-butterfly); the integer
# multiplies of the 64-bit Shoup
# product run on that pipe and it is the binding unit.
FMAHEAVY_CYCLES_PER_WARP_BUTTERFLY = 38.8


def alu_ceiling(dev):
    """Butterflies/s the FMA-heavy pipes allow: SMs x 4 pipes x max SM clock x 32 / cycles per warp-butterfly."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = measured_peaks().get("sm_max_mhz", 2070.0)
    return sms * 4 * mhz * 1e6 * 32 / FMAHEAVY_CYCLES_PER_WARP_BUTTERFLY


def kernels_roofline(H, ctx, dev, summary, log_n, na, top=3):
    """Roofline figures of the `top` kernels of a profile summary (hetal_profile_summary: per
    kernel launches, ms, and the algorithmic modular products and bytes its launches count).
    Transform passes against the derived butterfly ceiling (the fused conversion's na products
    per coefficient weighed as in the default line); key inner products against the measured
    multiply-accumulate rate; every kernel's algorithmic bytes against the measured HBM
    bandwidth.  `bound` names the larger of the two fractions (frac_of_bound)."""
    probe = H.hetal_probe_butterfly_rate(ctx, 20000)
    mac = H.hetal_probe_mac_rate(ctx, 20000)
    ceil = alu_ceiling(dev)
    hbm_peak = measured_peaks().get("hbm_gbs", 6800.0) * 1e9
    total = sum(v["ms"] for v in summary.values())
    out = []
    for name, v in sorted(summary.items(), key=lambda kv: -kv[1]["ms"])[:top]:
        sec = v["ms"] * 1e-3
        row = {"kernel": name, "share": round(v["ms"] / total, 4), "launches": v["launches"],
               "hbm_frac_of_measured": v["bytes"] / sec / hbm_peak}
        if name.startswith("ntt"):
            work = v["modmul"]
            if name == "ntt_fwd_cols_conv":
                bf = (log_n - 8) / 2.0
                work = work * (bf + probe / mac * na) / (bf + na)
            row.update({"bound": "alu", "unit": "Gbutterfly-eq/s", "achieved": work / sec / 1e9,
                        "peak": ceil / 1e9, "frac": work / sec / ceil, "frac_of_probe": work / sec / probe})
        elif name.startswith("kip"):
            row.update({"bound": "alu", "unit": "Gproduct/s", "achieved": v["modmul"] / sec / 1e9,
                        "peak": mac / 1e9, "peak_source": "measured: register-only multiply-accumulate probe",
                        "frac": v["modmul"] / sec / mac})
        hb = row["hbm_frac_of_measured"]
        if hb >= row.get("frac", 0.0):
            row["bound"] = "hbm"
        row["frac_of_bound"] = max(hb, row.get("frac", 0.0))
        out.append(row)
    return out


def step_roofline(H, ctx, P, ms_per_unit, work_fn, flags, peaks):
    """Whole-unit roofline (one training step, or one batch of instances): the algorithmic
    work of the unit -- operation counts x primitive costs of the algorithm variant that
    runs (paper_2403_14111_gb300/workmodel.py; no kernel counter is read) -- over its
    measured time, against the register-only butterfly probe's rate (butterflies count 1,
    the other modular products are weighed by the probe's butterfly / multiply-accumulate
    rate ratio), and its algorithmic bytes against the measured HBM bandwidth.  The same
    figure for the paper's method (hoisted rotations, nothing else) is given beside it."""
    from paper_2403_14111_gb300 import workmodel as wm
    costs = wm.Costs(1 << P["log_n"], P["n_special"], P["alpha"])
    bfly = H.hetal_probe_butterfly_rate(ctx, 20000)
    mac = H.hetal_probe_mac_rate(ctx, 20000)
    weight = bfly / mac
    t = ms_per_unit * 1e-3
    hbm = peaks.get("hbm_gbs", 6800.0) * 1e9

    def fig(f):
        w = wm.finish(work_fn(costs, f), costs)
        eq = w.equivalents(weight)
        alu_t, hbm_t = eq / bfly, w.nbytes / hbm
        return w, eq, {"bound": "alu" if alu_t >= hbm_t else "hbm", "achieved": eq / t / 1e9,
                       "frac": max(alu_t, hbm_t) / t, "roofline_ms": max(alu_t, hbm_t) * 1e3,
                       "butterfly_eq": eq, "butterflies": w.bfly, "products": w.mac, "bytes": w.nbytes,
                       "hbm_frac_of_measured": w.nbytes / t / hbm, "counts": w.counts}

    w, eq, run = fig(flags)
    _, _, paper = fig(wm.HOIST)
    out = {"bound": run["bound"], "achieved": run["achieved"], "peak": bfly / 1e9, "unit": "Gbutterfly-eq/s",
           "frac": run["frac"],
           "peak_source": "measured: register-only butterfly probe (hetal_probe_butterfly_rate)",
           "mac_weight": weight, "measured_ms": ms_per_unit, "variant": run,
           "paper_method": dict(paper, note="the paper's algorithms with hoisted rotations only; above 1 where "
                                            "the library's variants do less work than the paper's method"),
           "work_source": "operation counts x primitive costs of the variant that runs "
                          "(paper_2403_14111_gb300/workmodel.py)"}
    return out


def traffic_record(kernel, alg_bytes_per_launch):
    """DRAM bytes per launch of `kernel`: the ratio of DRAM bytes to algorithmic bytes that the
    committed ncu summary measured on a smaller case of the same kernel, times this run's
    algorithmic bytes per launch.  None when the summary has no line for the kernel or the kernel's
    source file changed since the counters were taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic_per_launch.txt")
    try:
        with open(path) as f:
            for ln in f:
                p = ln.split()
                if ln.startswith("#") or len(p) < 4 or p[0] != kernel:
                    continue
                src = os.path.join(ROOT, p[2])
                with open(src, "rb") as fs:
                    if hashlib.sha1(fs.read()).hexdigest() != p[3]:
                        return None
                return {"dram_bytes": float(p[1]) * alg_bytes_per_launch, "dram_per_algorithmic_byte": float(p[1]),
                        "source": "scaled from the ncu capture in profiles/traffic_per_launch.txt"}
    except OSError:
        pass
    return None


def cpu_baseline(flags_text):
    """The oracle as it stands, timed on this machine's host cores, with 1 thread and with one
    thread per core (the oracle splits independent limbs over threads):
      - config 1 (N = 2^13, X 128 x 32 by (16 x 32)^T, c = 16) DiagABT timed whole;
      - config 2 (the N = 2^16 training step) extrapolated from a bounded sample of timed
        operations (oracle/baseline.py), with the same model's error against config 1 timed.
    The line's value is the all-core extrapolation of the training step."""
    from oracle import baseline, ckks
    f = dict(hoist="hoist" in flags_text, lazy_relin="lazy" in flags_text, radix_sum="radix" in flags_text,
             shared_rot="shared" in flags_text)
    cores = os.cpu_count() or 1
    p13 = ckks.params_n13()
    runs = {}
    try:
        for T in sorted({1, cores}):
            ckks.set_threads(T)
            c1, c1_err = baseline.time_diag_abt(p13, 128, 32, 16, 128, 32, **f)
            hist = baseline.abt_operation_counts(128, 32, 16, 128, 32, p13.L, **f)
            c1_model = baseline.estimate_seconds(p13, hist)[0]
            sec, desc, _ = baseline.estimate_step_seconds(ckks.params_n16(), **f)
            runs[T] = {"threads": ckks.threads(), "step_seconds_extrapolated": sec, "sample": desc,
                       "config1_diag_abt_seconds_measured": c1, "config1_max_abs_err": c1_err,
                       "config1_diag_abt_seconds_model": c1_model, "model_error_on_config1": c1_model / c1 - 1.0}
    finally:
        ckks.set_threads(0)
    main = runs[cores]
    return {"value": 1.0 / main["step_seconds_extrapolated"], "unit": UNIT, "cores": main["threads"],
            "kind": "oracle",
            "sample": "training step extrapolated (labelled so): " + main["sample"] +
                      "; the model's error on config 1 timed whole: %+.1f%%" % (100 * main["model_error_on_config1"]),
            "seconds_per_step": main["step_seconds_extrapolated"], "extrapolated": True,
            "single_thread": runs[1], "all_cores": main}


def config1(d, flags_text):
    """Config 1 on the GPU: N = 2^13 (q0 ~ 2^60, 3 x ~2^40, 1 special), scale 2^40, X 128 x 32 and W 16 x 32
    U(-1,1), c = 16, 128 x 32 blocks: encrypt (from host FP64) -> DiagABT -> decrypt (to host FP64),
    latency over repeated runs after warm-up (host clock around the whole path; CUDA events around
    DiagABT alone), and its error against X W^T."""
    import torch
    import paper_2403_14111_gb300.hetal as H
    from paper_2403_14111_gb300 import workloads as wl
    from paper_2403_14111_gb300.step import step_rotations
    dev = d.local
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    P = wl.PARAMS_N13
    ctx = H.hetal_ctx_create(P["log_n"], P["q0_bits"], P["n_rescale"], P["rescale_bits"], P["n_special"],
                             P["special_bits"], P["alpha"], scale=2.0 ** P["log_scale"], device=dev,
                             stream=stream.cuda_stream)
    flags = parse_flags(flags_text)
    N, L, K = H.hetal_ctx_info(ctx)
    s0, s1, c = 128, 32, 16
    sk = H.hetal_keygen(ctx, 1)
    evk = H.hetal_evk_create(ctx, sk, 1, step_rotations(s0, s1, c, flags))
    X, W = wl.uniform_matrix(128, 32, 1), wl.uniform_matrix(16, 32, 2)
    delta = 2.0 ** P["log_scale"]

    def once(timing):
        hX = H.hetal_encrypt(ctx, sk, 1, 100, X, s0, s1, H.TILE_NONE, 0, L - 1, delta)
        hW = H.hetal_encrypt(ctx, sk, 1, 200, W, s0, s1, H.TILE_VERT, c, L - 1, delta)
        if timing is not None:
            timing[0].record(stream)
        out = H.hetal_diag_abt(ctx, evk, hX, hW, c, 1.0, None, flags)
        if timing is not None:
            timing[1].record(stream)
        dec = H.hetal_decrypt(ctx, sk, out)
        for h in (hX, hW, out):
            H.hetal_mat_free(h)
        return dec

    for _ in range(3):
        once(None)
    reps, e2e, abt = 20, [], []
    for _ in range(reps):
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dec = once(ev)
        e2e.append((time.perf_counter() - t0) * 1e3)
        abt.append(ev[0].elapsed_time(ev[1]))
    err = float(np.max(np.abs(dec[:128, :s1] - np.tile(X @ W.T, (1, s1 // c)))))
    H.hetal_evk_free(evk)
    H.hetal_sk_free(sk)
    H.hetal_ctx_destroy(ctx)
    return {"workload": "config 1: N=2^13, X 128x32 by (W 16x32)^T U(-1,1), c=16, 128x32 blocks, scale 2^40",
            "flags": flags_text, "repetitions": reps, "diag_abt_ms_median": float(np.median(abt)),
            "e2e_ms_median": float(np.median(e2e)), "e2e": "encrypt from host FP64, DiagABT, decrypt to host FP64",
            "max_abs_err": err}


def run_reference(args, d):
    """The reference arm: the oracle as it stands on this machine's host cores (one thread per
    core).  Each step is a bounded sample of the training step (its timed operations, about
    5-10 s of CPU work) extrapolated to the whole step; value is the median extrapolation,
    ms_per_step the sample's own measured time.  Under torchrun only rank 0 runs."""
    if d.rank != 0:
        return
    from oracle import baseline, ckks
    f = dict(hoist="hoist" in args.flags, lazy_relin="lazy" in args.flags, radix_sum="radix" in args.flags,
             shared_rot="shared" in args.flags)
    ckks.set_threads(0)
    cores = ckks.threads()
    for _ in range(args.warmup):
        baseline.estimate_step_seconds(ckks.params_n16(), **f)
    est, walls, desc = [], [], ""
    t_all = time.perf_counter()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        sec, desc, _ = baseline.estimate_step_seconds(ckks.params_n16(), **f)
        walls.append(time.perf_counter() - t0)
        est.append(sec)
    wall = time.perf_counter() - t_all
    sec = float(np.median(est))
    value = 1.0 / sec
    cb = {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "extrapolated": True,
          "sample": "each step: " + desc + "; value = 1 / median extrapolated seconds per training step over %d "
                    "steps" % args.steps,
          "seconds_per_step_extrapolated": sec, "wall_s": wall}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(walls)) * 1e3,
            "ms_per_step_is": "the measured time of one bounded sample (the step's value is extrapolated)",
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "flags": args.flags}, "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    d = Dist()
    if args.impl == "reference":
        run_reference(args, d)
        d.close()
        return
    if args.sweep == "ntt":
        run_ntt_sweep(args, d)
        d.close()
        return
    if args.sweep == "rot":
        run_rot_sweep(args, d)
        d.close()
        return
    if args.sweep == "word":
        line = dict(word_size(d), sweep="word")
        if d.rank == 0:
            print(json.dumps(line), flush=True)
        d.close()
        return
    if args.batched:
        run_batched(args, d)
        d.close()
        return
    if args.table4:
        run_table4(args, d)
        d.close()
        return
    if args.nag:
        run_nag(args, d)
        d.close()
        return
    if args.asoftmax:
        run_asoftmax(args, d)
        d.close()
        return
    if args.bootstrap:
        run_bootstrap(args, d)
        d.close()
        return
    if args.train_boot and args.epochs > 0:
        run_protocol(args, d)
        d.close()
        return
    if args.train_boot:
        run_train_boot(args, d)
        d.close()
        return
    if args.serve:
        run_serve(args, d)
        d.close()
        return
    import torch
    import paper_2403_14111_gb300.hetal as H
    from paper_2403_14111_gb300 import workloads as wl
    from paper_2403_14111_gb300.step import step_rotations, train_step
    from paper_2403_14111_gb300 import workmodel as wm

    dev = d.local
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    P = wl.PARAMS_N16
    ctx = H.hetal_ctx_create(P["log_n"], P["q0_bits"], P["n_rescale"], P["rescale_bits"], P["n_special"],
                             P["special_bits"], P["alpha"], scale=2.0 ** P["log_scale"], device=dev,
                             stream=stream.cuda_stream)
    flags = parse_flags(args.flags)
    N, L, K = H.hetal_ctx_info(ctx)
    delta = 2.0 ** P["log_scale"]
    s0, s1 = 1024, 32
    seed = 100 + d.rank
    X, Y, W, c = wl.training_step(seed=seed)
    coeffs = wl.sigmoid_cheb15()
    valid = wl.valid_mask(1024, 10, c, s0, s1)
    top = L - 1
    lvP = top - 3 - 5
    sk = H.hetal_keygen(ctx, seed)
    evk = H.hetal_evk_create(ctx, sk, seed, step_rotations(s0, s1, c, flags))
    hX = H.hetal_encrypt(ctx, sk, seed, 1000, X, s0, s1, H.TILE_NONE, 0, top, delta)
    hW = H.hetal_encrypt(ctx, sk, seed, 2000, W, s0, s1, H.TILE_VERT, c, top, delta)
    hY = H.hetal_encrypt(ctx, sk, seed, 3000, Y, s0, s1, H.TILE_HORIZ, c, lvP, delta)
    lr_n = 1.0 / 1024

    def step(x, w, y):
        G, inter = train_step(ctx, evk, x, w, y, coeffs, valid, c, lr_n, delta, flags)
        for h in inter:
            H.hetal_mat_free(h)
        return G

    for _ in range(args.warmup):
        H.hetal_mat_free(step(hX, hW, hY))
    H.hetal_ctx_sync(ctx)

    # one untimed step with every launch timed, to find the kernel that takes longest
    H.hetal_profile_kernel(ctx, "*")
    H.hetal_mat_free(step(hX, hW, hY))
    summary = H.hetal_profile_summary(ctx)
    H.hetal_profile_kernel(ctx, "")
    total_ms = sum(v["ms"] for v in summary.values())
    kernel = args.kernel or max(summary, key=lambda k: summary[k]["ms"])

    # Two timed regions of K steps each, on the same inputs.  First the steps run call by call
    # with every launch of the top kernel timed on the context's stream (the roofline's kernel
    # figures); then the step recorded once into a CUDA graph runs as K graph launches (value:
    # the same kernels, without the host's per-call work between them).
    clocks = Clocks(dev)
    clocks.start()
    H.hetal_profile_kernel(ctx, kernel)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    if args.nvtx:
        torch.cuda.nvtx.range_push("hetal_step")
    for _ in range(args.steps):
        H.hetal_mat_free(step(hX, hW, hY))
    if args.nvtx:
        torch.cuda.nvtx.range_pop()
    ev1.record(stream)
    torch.cuda.synchronize()
    d.barrier()
    ms_eager = ev0.elapsed_time(ev1)
    kstats = H.hetal_profile_read(ctx)
    H.hetal_profile_kernel(ctx, "")

    graph = None
    if not args.no_graph:
        try:
            H.hetal_graph_begin(ctx)
            try:
                H.hetal_mat_free(step(hX, hW, hY))
            except H.HetalError:
                try:   # close the void recording before the context is used again
                    H.hetal_graph_end(ctx)
                except H.HetalError:
                    pass
                raise
            graph = H.hetal_graph_end(ctx)   # instantiates and runs it once
            H.hetal_ctx_sync(ctx)
        except H.HetalError as ex:
            print("graph recording failed (%s); the timed steps run call by call" % ex, file=sys.stderr)
            graph = None
    launches0 = H.hetal_launch_count(ctx)
    d.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        if graph is not None:
            H.hetal_graph_launch(ctx, graph)
        else:
            H.hetal_mat_free(step(hX, hW, hY))
    ev1.record(stream)
    torch.cuda.synchronize()
    d.barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    launches = H.hetal_launch_count(ctx) - launches0
    if graph is not None:
        H.hetal_graph_free(graph)
    value, ms_max = replica_value(d, args.steps, ms)
    ms_eager_max = d.max(ms_eager)

    # end to end through the C ABI with host buffers: ciphertexts from pinned
    # host memory in, the gradient's residues back to pinned host memory
    e2e = None
    if not args.no_e2e:
        descs = [H.hetal_mat_desc_get(h) for h in (hX, hW, hY)]
        host_in = []
        for h in (hX, hW, hY):
            r = H.hetal_mat_export(ctx, h)
            t = torch.empty(r.size, dtype=torch.int64, pin_memory=True)
            a = t.numpy().view(np.uint64).reshape(r.shape)
            a[...] = r
            host_in.append((t, a))
        G0 = step(hX, hW, hY)
        Gd = H.hetal_mat_desc_get(G0)
        H.hetal_mat_free(G0)
        g_words = Gd.m * Gd.n * 2 * (Gd.level + 1) * N
        g_host_t = torch.empty(g_words, dtype=torch.int64, pin_memory=True)
        g_host = g_host_t.numpy().view(np.uint64)
        h2d = sum(a.nbytes for _, a in host_in)
        try:
            e2e = e2e_overlap(args, d, ctx, P, dev, stream, step, host_in, descs, g_words)
            e2e["serial_graph"] = e2e_graph(args, d, ctx, step, host_in, descs, g_host)["value"]
        except H.HetalError as ex:   # recording refused: the eager loop instead
            print("e2e: graph recording failed (%s); eager loop instead" % ex, file=sys.stderr)
            e2e = e2e_eager(args, d, ctx, P, dev, step, host_in, descs, g_host)
        e2e.update({"unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": int(g_words * 8)})

    peaks = measured_peaks()
    kms = kstats["ms"] / max(kstats["launches"], 1)
    if kernel.startswith("ntt"):
        probe = H.hetal_probe_butterfly_rate(ctx, 20000)
        ceil = alu_ceiling(dev)
        work = kstats["modmul"] / max(kstats["launches"], 1)
        unit, extra = "Gbutterfly/s", {}
        if kernel == "ntt_fwd_cols_conv":
            # the column pass with the fused base conversion: (log N - 8) / 2 butterflies and na
            # 128-bit products per coefficient, na = alpha (ModUp) = K (ModDown) here; a product
            # is weighed by the butterfly's rate over the multiply-accumulate's
            assert P["alpha"] == P["n_special"], "conversion width differs between ModUp and ModDown"
            na, bf = P["alpha"], (P["log_n"] - 8) / 2.0
            mac = H.hetal_probe_mac_rate(ctx, 20000)
            weight = probe / mac
            work = work * (bf + weight * na) / (bf + na)
            unit = "Gbutterfly-eq/s"
            extra = {"work": "butterflies plus the fused base conversion's %d products per coefficient, each "
                             "weighed as %.3f butterfly (measured butterfly rate / multiply-accumulate rate)"
                             % (na, weight),
                     "probe_mac_measured": mac / 1e9}
        achieved = work / (kms * 1e-3)
        roof = {"bound": "alu", "achieved": achieved / 1e9, "peak": ceil / 1e9, "unit": unit,
                "frac": achieved / ceil,
                "peak_source": "derived: SMs x 4 FMA-heavy pipes x max SM clock / %.1f pipe cycles per warp-butterfly "
                               "(ncu on the register-only butterfly probe)" % FMAHEAVY_CYCLES_PER_WARP_BUTTERFLY,
                "probe_measured": probe / 1e9, "frac_of_probe": achieved / probe}
        roof.update(extra)
        hbm = kstats["bytes"] / max(kstats["launches"], 1) / (kms * 1e-3)
        roof["hbm_frac_of_measured"] = hbm / (peaks.get("hbm_gbs", 6800.0) * 1e9)
    else:
        achieved = kstats["bytes"] / max(kstats["launches"], 1) / (kms * 1e-3)
        hp = peaks.get("hbm_gbs")
        roof = {"bound": "hbm", "achieved": achieved / 1e9, "peak": hp if hp else 6800.0, "unit": "GB/s",
                "frac": achieved / ((hp if hp else 6800.0) * 1e9),
                "peak_source": "MEASURED_PEAKS.json hbm_gbs" if hp else "fallback 6.8 TB/s"}
    tr = traffic_record(kernel, kstats["bytes"] / max(kstats["launches"], 1))
    roof.update({"kernel": kernel, "launches_timed": kstats["launches"], "avg_launch_us": kms * 1e3,
                 "timed_in": "the call-by-call timed region (each launch of the kernel between CUDA events on "
                             "the context's stream)",
                 "share_of_kernel_time": summary[kernel]["ms"] / total_ms if total_ms else None,
                 "traffic": tr["dram_bytes"] if tr else None,
                 "traffic_source": ("%s (%.3f DRAM bytes per algorithmic byte)" % (tr["source"], tr["dram_per_algorithmic_byte"])
                                    if tr else None)})

    step_roof = step_roofline(H, ctx, P, ms_max / args.steps,
                              lambda C, f: wm.training_step(C, 1024, 768, c, s0, s1, top, f), flags, peaks)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": d.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "flags": args.flags, "parallelism": "replicas" if d.world > 1 else "1 GPU",
                       "l2": "inputs larger than L2: 302 MB of X ciphertexts and 2.9 GB of keys per step"},
            "timed_path": "one CUDA graph launch per step" if graph is not None else "call by call",
            "ms_per_step_call_by_call": ms_eager_max / args.steps,
            "e2e": e2e, "gpu_launches": launches, "roofline": roof, "step_roofline": step_roof, "clocks": clk,
            # sum of the kernels' own durations in one step (each launch timed alone)
            "kernel_ms_per_step": total_ms,
            "top_kernels": {k: round(v["ms"] / total_ms, 4) for k, v in
                            sorted(summary.items(), key=lambda kv: -kv[1]["ms"])[:8]}}
    if d.rank == 0 and d.world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.flags)
    for h in (hX, hW, hY):
        H.hetal_mat_free(h)
    H.hetal_evk_free(evk)
    H.hetal_sk_free(sk)
    H.hetal_ctx_destroy(ctx)
    if d.world == 1:
        line["word_size"] = word_size(d)
        line["config1"] = config1(d, args.flags)
        if "cpu_baseline" in line:
            line["config1"]["oracle_seconds_measured"] = {
                "1 thread": line["cpu_baseline"]["single_thread"]["config1_diag_abt_seconds_measured"],
                "%d threads" % line["cpu_baseline"]["cores"]:
                    line["cpu_baseline"]["all_cores"]["config1_diag_abt_seconds_measured"]}
    if d.world == 1 and not args.no_batched:
        # the metric's batched-vs-plain half: the batched workload, measured after the step's
        # timed regions (its own context, keys and inputs)
        try:
            line["batched"] = config3(args, d)
        except Exception as ex:   # the training step's line still stands
            line["batched"] = {"error": "%s: %s" % (type(ex).__name__, ex)}
    if d.world == 1 and not args.no_serve:
        # the metric's latency half: a short serving run (its own context and clients), p50 / p99
        # at a Poisson load of 0.7 of the measured capacity
        try:
            line["serve"] = serve_measure(d, 8, 24, 4, [0.7])
        except Exception as ex:
            line["serve"] = {"error": "%s: %s" % (type(ex).__name__, ex)}
    if d.rank == 0:
        print(json.dumps(line), flush=True)
    d.close()


if __name__ == "__main__":
    main()
