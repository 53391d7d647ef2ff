"""Many independent instances (hetal_run_pairs): the batched workers give the same
bits as one instance after another, instance results decrypt to their FP64
products, and the tile tuner picks legal block shapes."""
import numpy as np
import pytest

import paper_2403_14111_gb300.hetal as H
from paper_2403_14111_gb300 import workloads as wl
from paper_2403_14111_gb300.step import step_rotations

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
    sk = H.hetal_keygen(ctx, 21)
    yield ctx, sk
    H.hetal_sk_free(sk)
    H.hetal_ctx_destroy(ctx)


def test_run_pairs_workers_match_sequential(env):
    ctx, sk = env
    N, L, K = H.hetal_ctx_info(ctx)
    S = N // 2
    top = L - 1
    inst = wl.batched_instances(5, seed=7, rows=(64, 300), classes=(2, 9), dims=(40, 100))
    evk0 = H.hetal_evk_create(ctx, sk, 21, [1], with_conj=False, with_relin=False)
    tiles = [H.hetal_tile_choose(ctx, evk0, i["a"], i["b"], i["c"]) for i in inst]
    H.hetal_evk_free(evk0)
    rots = set()
    for i, s0 in zip(inst, tiles):
        s1 = S // s0
        assert s0 & (s0 - 1) == 0 and i["c"] <= min(s0, s1)
        rots |= set(step_rotations(s0, s1, i["c"]))
    evk = H.hetal_evk_create(ctx, sk, 21, sorted(rots))
    jobs, hs = [], []
    for idx, (i, s0) in enumerate(zip(inst, tiles)):
        s1 = S // s0
        hX = H.hetal_encrypt(ctx, sk, 21, 100 * idx + 1, i["X"], s0, s1, H.TILE_NONE, 0, top, 2.0 ** 40)
        hW = H.hetal_encrypt(ctx, sk, 21, 100 * idx + 50, i["W"], s0, s1, H.TILE_VERT, i["c"], top, 2.0 ** 40)
        hA = H.hetal_encrypt(ctx, sk, 21, 100 * idx + 70, i["A"], s0, s1, H.TILE_HORIZ, i["c"], top - 3, 2.0 ** 40)
        hB = H.hetal_mat_drop(ctx, hX, top - 2)
        hs += [hX, hW, hA, hB]
        jobs.append(dict(x=hX, wbar=hW, a_under=hA, b=hB, c=i["c"], t_abt=1.0, t_atb=1.0 / i["a"]))
    flags = H.FLAG_HOIST | H.FLAG_LAZY_RELIN
    sa, sb = H.hetal_run_pairs(ctx, evk, jobs, 1, flags)
    ba, bb = H.hetal_run_pairs(ctx, evk, jobs, 3, flags)
    for i, (it, s0) in enumerate(zip(inst, tiles)):
        s1 = S // s0
        assert np.array_equal(H.hetal_mat_export(ctx, sa[i]), H.hetal_mat_export(ctx, ba[i]))
        assert np.array_equal(H.hetal_mat_export(ctx, sb[i]), H.hetal_mat_export(ctx, bb[i]))
        abt = H.hetal_decrypt(ctx, sk, ba[i])[:it["a"], :s1]
        assert np.max(np.abs(abt - np.tile(it["X"] @ it["W"].T, (1, s1 // it["c"])))) <= 1e-4
        atb = H.hetal_decrypt(ctx, sk, bb[i])[:s0, :it["b"]]
        Ap = np.zeros((it["a"], it["c"]))
        Ap[:, :it["classes"]] = it["A"]
        assert np.max(np.abs(atb - np.tile(Ap.T @ it["X"] / it["a"], (s0 // it["c"], 1)))) <= 1e-4
    cnt = H.hetal_counters_get(ctx)
    assert cnt["rot"] > 0 and cnt["keyswitch"] > 0
    for h in sa + sb + ba + bb + hs:
        H.hetal_mat_free(h)
    H.hetal_evk_free(evk)


@pytest.mark.parametrize("flags", [0, H.FLAG_HOIST | H.FLAG_LAZY_RELIN,
                                   H.FLAG_HOIST | H.FLAG_LAZY_RELIN | H.FLAG_RADIX_SUM | H.FLAG_SHARED_ROT],
                         ids=["plain", "hoist+lazy", "all"])
@pytest.mark.parametrize("branch", ["protup", "rotleft"])
def test_batched_across_instances_matches_one_by_one(env, flags, branch):
    """Instances of one block shape with different c (2..16), row and column block counts run
    as groups (hetal_run_pairs_batched): every output has the bits of the instance run alone,
    for DiagATB's PRotUp branch and its RotLeft branch (where c = 2 forms its own group)."""
    ctx, sk = env
    N, L, K = H.hetal_ctx_info(ctx)
    top = L - 1
    s0, s1 = 128, 32
    shapes = [(300, 100, 8), (60, 40, 2), (200, 30, 16), (128, 64, 4), (90, 96, 8), (250, 20, 2)]
    rng = np.random.default_rng(5)
    rots = set()
    for f in (flags, flags | H.FLAG_SHARED_ROT | H.FLAG_RADIX_SUM):
        rots |= set(step_rotations(s0, s1, 16, f))
    evk = H.hetal_evk_create(ctx, sk, 22, sorted(rots))
    lv_a, lv_b = (top - 3, top - 2) if branch == "protup" else (top - 2, top - 2)
    jobs, hs, ref = [], [], []
    for idx, (a, b, c) in enumerate(shapes):
        X = rng.standard_normal((a, b)) / np.sqrt(b)
        W = rng.standard_normal((c, b)) * 0.1
        A = rng.uniform(-0.5, 0.5, (a, c))
        hX = H.hetal_encrypt(ctx, sk, 22, 1000 * idx + 1, X, s0, s1, H.TILE_NONE, 0, top, 2.0 ** 40)
        hW = H.hetal_encrypt(ctx, sk, 22, 1000 * idx + 200, W, s0, s1, H.TILE_VERT, c, top, 2.0 ** 40)
        hA = H.hetal_encrypt(ctx, sk, 22, 1000 * idx + 400, A, s0, s1, H.TILE_HORIZ, c, lv_a, 2.0 ** 40)
        hB = H.hetal_mat_drop(ctx, hX, lv_b)
        hs += [hX, hW, hA, hB]
        jobs.append(dict(x=hX, wbar=hW, a_under=hA, b=hB, c=c, t_abt=0.5, t_atb=1.0 / a))
        ref.append((X, W, A))
    sa, sb = H.hetal_run_pairs(ctx, evk, jobs, 1, flags)
    ba, bb = H.hetal_run_pairs_batched(ctx, evk, jobs, flags)
    for i, ((a, b, c), (X, W, A)) in enumerate(zip(shapes, ref)):
        assert np.array_equal(H.hetal_mat_export(ctx, sa[i]), H.hetal_mat_export(ctx, ba[i])), ("abt", i)
        assert np.array_equal(H.hetal_mat_export(ctx, sb[i]), H.hetal_mat_export(ctx, bb[i])), ("atb", i)
        got = H.hetal_decrypt(ctx, sk, ba[i])[:a, :s1]
        assert np.max(np.abs(got - np.tile(0.5 * X @ W.T, (1, s1 // c)))) <= 1e-4
        got = H.hetal_decrypt(ctx, sk, bb[i])[:s0, :b]
        assert np.max(np.abs(got - np.tile(A.T @ X / a, (s0 // c, 1)))) <= 1e-4
    for h in sa + sb + ba + bb + hs:
        H.hetal_mat_free(h)
    H.hetal_evk_free(evk)


def test_batched_graph_replays_the_batch(env):
    """The batched run of a fixed set of instances records into one CUDA graph; each launch
    recomputes every output with the eager run's bits."""
    ctx, sk = env
    N, L, K = H.hetal_ctx_info(ctx)
    top = L - 1
    s0, s1 = 128, 32
    flags = H.FLAG_HOIST | H.FLAG_LAZY_RELIN | H.FLAG_RADIX_SUM | H.FLAG_SHARED_ROT
    evk = H.hetal_evk_create(ctx, sk, 23, step_rotations(s0, s1, 8, flags))
    rng = np.random.default_rng(6)
    jobs, hs = [], []
    for idx, (a, b, c) in enumerate([(100, 50, 8), (240, 70, 4), (30, 32, 2)]):
        X = rng.standard_normal((a, b)) / np.sqrt(b)
        hX = H.hetal_encrypt(ctx, sk, 23, 1000 * idx + 1, X, s0, s1, H.TILE_NONE, 0, top, 2.0 ** 40)
        hW = H.hetal_encrypt(ctx, sk, 23, 1000 * idx + 200, rng.standard_normal((c, b)) * 0.1, s0, s1,
                             H.TILE_VERT, c, top, 2.0 ** 40)
        hA = H.hetal_encrypt(ctx, sk, 23, 1000 * idx + 400, rng.uniform(-0.5, 0.5, (a, c)), s0, s1,
                             H.TILE_HORIZ, c, top - 3, 2.0 ** 40)
        hB = H.hetal_mat_drop(ctx, hX, top - 2)
        hs += [hX, hW, hA, hB]
        jobs.append(dict(x=hX, wbar=hW, a_under=hA, b=hB, c=c, t_abt=1.0, t_atb=1.0 / a))
    ea, eb = H.hetal_run_pairs_batched(ctx, evk, jobs, flags)   # eager: encodes the masks
    want = [H.hetal_mat_export(ctx, h) for h in ea + eb]
    H.hetal_graph_begin(ctx)
    ga, gb = H.hetal_run_pairs_batched(ctx, evk, jobs, flags)
    g = H.hetal_graph_end(ctx)
    try:
        for _ in range(2):
            H.hetal_graph_launch(ctx, g)
            H.hetal_ctx_sync(ctx)
            for h, w in zip(ga + gb, want):
                assert np.array_equal(H.hetal_mat_export(ctx, h), w)
    finally:
        H.hetal_graph_free(g)
    for h in ea + eb + ga + gb + hs:
        H.hetal_mat_free(h)
    H.hetal_evk_free(evk)
