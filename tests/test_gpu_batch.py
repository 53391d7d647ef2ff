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
