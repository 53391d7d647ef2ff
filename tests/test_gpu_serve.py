"""Serving loop (hetal_server_*): two clients with their own keys (only the
+-2^u rotation keys, rotations composed from them), mixed DiagABT / DiagATB
requests.  Each result is the same bits alone (one slot, one request at a
time) and in the mix (three slots, all requests queued at once), and decrypts to
its FP64 product."""
import numpy as np
import pytest

import paper_2403_14111_gb300.hetal as H
from paper_2403_14111_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a visible GPU")
    P = wl.PARAMS_N13_DEEP
    ctx = H.hetal_ctx_create(P["log_n"], P["q0_bits"], P["n_rescale"], P["rescale_bits"], P["n_special"],
                             P["special_bits"], P["alpha"], scale=2.0 ** P["log_scale"])
    yield ctx
    H.hetal_ctx_destroy(ctx)


def test_results_same_alone_and_in_the_mix(env):
    ctx = env
    N, L, K = H.hetal_ctx_info(ctx)
    S = N // 2
    top = L - 1
    pow2 = [1 << u for u in range(12)] + [-(1 << u) for u in range(12)]
    clients = []
    for seed in (31, 32):
        sk = H.hetal_keygen(ctx, seed)
        clients.append((seed, sk, H.hetal_evk_create(ctx, sk, seed, pow2)))
    reqs, keep = [], []
    rng = np.random.default_rng(5)
    for i in range(6):
        cl = i % 2
        seed, sk, evk = clients[cl]
        a, b, k = int(rng.integers(64, 260)), int(rng.integers(20, 90)), int(rng.integers(2, 9))
        c = wl.pad_pow2(k)
        s0 = 128
        s1 = S // s0
        X = rng.standard_normal((a, b)) / np.sqrt(b)
        if i % 3 != 2:
            W = np.zeros((c, b))
            W[:k] = rng.standard_normal((k, b)) * 0.1
            hX = H.hetal_encrypt(ctx, sk, seed, 100 * i + 1, X, s0, s1, H.TILE_NONE, 0, top, 2.0 ** 40)
            hW = H.hetal_encrypt(ctx, sk, seed, 100 * i + 2, W, s0, s1, H.TILE_VERT, c, top, 2.0 ** 40)
            keep += [hX, hW]
            reqs.append(dict(cl=cl, kind=0, a=hX, b=hW, c=c, t=1.0,
                             want=np.tile(X @ W.T, (1, s1 // c)), rows=a, cols=s1))
        else:
            A = rng.uniform(-0.5, 0.5, (a, k))
            hA = H.hetal_encrypt(ctx, sk, seed, 100 * i + 3, A, s0, s1, H.TILE_HORIZ, c, top - 3, 2.0 ** 40)
            hX = H.hetal_encrypt(ctx, sk, seed, 100 * i + 4, X, s0, s1, H.TILE_NONE, 0, top - 2, 2.0 ** 40)
            keep += [hA, hX]
            Ap = np.zeros((a, c))
            Ap[:, :k] = A
            reqs.append(dict(cl=cl, kind=1, a=hA, b=hX, c=c, t=1.0 / a,
                             want=np.tile(Ap.T @ X / a, (s0 // c, 1)), rows=s0, cols=b))
    flags = H.FLAG_HOIST | H.FLAG_LAZY_RELIN
    results = {}
    for mode, slots in (("alone", 1), ("mix", 3)):
        srv = H.hetal_server_create(ctx, slots, 64 << 30)
        ids = [H.hetal_server_add_client(ctx, srv, cl[2]) for cl in clients]
        outs = []
        if mode == "alone":
            for r in reqs:
                t = H.hetal_server_submit(ctx, srv, ids[r["cl"]], r["kind"], r["a"], r["b"], r["c"], r["t"], flags)
                outs.append(H.hetal_server_wait(ctx, srv, t)[0])
        else:
            tickets = [H.hetal_server_submit(ctx, srv, ids[r["cl"]], r["kind"], r["a"], r["b"], r["c"], r["t"], flags)
                       for r in reqs]
            outs = [H.hetal_server_wait(ctx, srv, t)[0] for t in tickets]
        assert H.hetal_server_stats(srv)["completed"] == len(reqs)
        results[mode] = [H.hetal_mat_export(ctx, o) for o in outs]
        for r, o in zip(reqs, outs):
            sk = clients[r["cl"]][1]
            dec = H.hetal_decrypt(ctx, sk, o)[:r["rows"], :r["cols"]]
            assert np.max(np.abs(dec - r["want"])) <= 1e-4
        for o in outs:
            H.hetal_mat_free(o)
        with pytest.raises(H.HetalError):
            H.hetal_server_wait(ctx, srv, 999999)
        H.hetal_server_destroy(srv)
    for a, b in zip(results["alone"], results["mix"]):
        assert np.array_equal(a, b)
    for h in keep:
        H.hetal_mat_free(h)
    for seed, sk, evk in clients:
        H.hetal_evk_free(evk)
        H.hetal_sk_free(sk)


def test_admission_cancel_and_results_outliving_the_server(env):
    """Host-side checks of the serving loop: a request that can never fit the budget is
    refused at submission (HETAL_ERR_OOM); a request still queued can be withdrawn (its
    wait returns HETAL_ERR_CANCELLED) while the others run; a collected result belongs to
    the caller's context, so it can be used on the caller's stream and freed after the
    server is gone, and freeing it while the caller's stream still reads it is ordered
    after that read."""
    ctx = env
    N, L, K = H.hetal_ctx_info(ctx)
    top = L - 1
    s0, s1, c = 128, 32, 4
    sk = H.hetal_keygen(ctx, 41)
    evk = H.hetal_evk_create(ctx, sk, 41, [1 << u for u in range(12)] + [-(1 << u) for u in range(12)])
    rng = np.random.default_rng(9)
    X = rng.standard_normal((128, 32)) / np.sqrt(32)
    W = rng.standard_normal((c, 32)) * 0.1
    hX = H.hetal_encrypt(ctx, sk, 41, 1, X, s0, s1, H.TILE_NONE, 0, top, 2.0 ** 40)
    hW = H.hetal_encrypt(ctx, sk, 41, 2, W, s0, s1, H.TILE_VERT, c, top, 2.0 ** 40)
    want = np.tile(X @ W.T, (1, s1 // c))
    flags = H.FLAG_HOIST | H.FLAG_LAZY_RELIN
    # a budget below even the resident keys: every request is refused at submission
    tiny = H.hetal_server_create(ctx, 1, 1 << 20)
    cid = H.hetal_server_add_client(ctx, tiny, evk)
    with pytest.raises(H.HetalError) as ei:
        H.hetal_server_submit(ctx, tiny, cid, 0, hX, hW, c, 1.0, flags)
    assert ei.value.code == H.ERR_OOM
    H.hetal_server_destroy(tiny)
    # one slot: the first request runs, the later ones queue behind it; cancel the last one
    srv = H.hetal_server_create(ctx, 1, 64 << 30)
    cid = H.hetal_server_add_client(ctx, srv, evk)
    tickets = [H.hetal_server_submit(ctx, srv, cid, 0, hX, hW, c, 1.0, flags) for _ in range(4)]
    H.hetal_server_cancel(ctx, srv, tickets[-1])
    with pytest.raises(H.HetalError) as ei:
        H.hetal_server_cancel(ctx, srv, tickets[-1])   # no longer queued
    assert ei.value.code == H.ERR_INVALID_ARG
    outs = [H.hetal_server_wait(ctx, srv, t)[0] for t in tickets[:-1]]
    with pytest.raises(H.HetalError) as ei:
        H.hetal_server_wait(ctx, srv, tickets[-1])
    assert ei.value.code == H.ERR_CANCELLED
    assert H.hetal_server_stats(srv)["completed"] == 3
    # a parent-stream operation on a result, then the result freed while it may still run,
    # then another request: the freed memory is reused only after the read
    r0 = H.hetal_rotate(ctx, evk, outs[0], 1)
    H.hetal_mat_free(outs[0])
    t = H.hetal_server_submit(ctx, srv, cid, 0, hX, hW, c, 1.0, flags)
    outs.append(H.hetal_server_wait(ctx, srv, t)[0])
    H.hetal_server_destroy(srv)
    # the results outlive the server
    got = H.hetal_decrypt(ctx, sk, r0)[:128, :s1]
    assert np.max(np.abs(got - np.roll(want.reshape(-1), -1).reshape(128, s1))) <= 1e-4
    for o in outs[1:]:
        assert np.max(np.abs(H.hetal_decrypt(ctx, sk, o)[:128, :s1] - want)) <= 1e-4
        H.hetal_mat_free(o)
    for h in (r0, hX, hW):
        H.hetal_mat_free(h)
    H.hetal_evk_free(evk)
    H.hetal_sk_free(sk)


def test_import_rejects_non_canonical_residues(env):
    """hetal_mat_import refuses residues that are not below their limb's modulus."""
    ctx = env
    N, L, K = H.hetal_ctx_info(ctx)
    mods = H.hetal_ctx_moduli(ctx)
    lv = 2
    rng = np.random.default_rng(3)
    res = np.stack([np.stack([rng.integers(0, mods[l], N, dtype=np.uint64) for l in range(lv + 1)])
                    for _ in range(2)])[None]
    d = H.make_desc(1, 1, 128, 32, 128, 32, lv, 2.0 ** 40)
    ok = H.hetal_mat_import(ctx, res, d)
    assert np.array_equal(H.hetal_mat_export(ctx, ok), res)
    H.hetal_mat_free(ok)
    bad = res.copy()
    bad[0, 1, 2, 77] = np.uint64(mods[2])
    with pytest.raises(H.HetalError) as ei:
        H.hetal_mat_import(ctx, bad, d)
    assert ei.value.code == H.ERR_INVALID_ARG
