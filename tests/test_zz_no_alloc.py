"""hetal_rescale_noalloc: rescale on caller-owned device buffers, for callers
that may not let the library allocate device memory after start-up.  Checked
through the C ABI against hetal_rescale on two calls in a row (the static
scratch array is reused between them), bit for bit like every ciphertext
comparison in this suite.  The file sorts last so that a run stopping at the
first failure has run every other test first."""
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
    P = wl.PARAMS_N16
    ctx = H.hetal_ctx_create(P["log_n"], P["q0_bits"], P["n_rescale"], P["rescale_bits"], P["n_special"],
                             P["special_bits"], P["alpha"], scale=2.0 ** P["log_scale"])
    sk = H.hetal_keygen(ctx, 9)
    yield ctx, sk
    H.hetal_sk_free(sk)
    H.hetal_ctx_destroy(ctx)


def _ntt_domain(ctx, mat, torch):
    """A ciphertext's NTT-domain residues in a torch device buffer (export, then forward NTT)."""
    d = H.hetal_mat_desc_get(mat)
    N = H.hetal_ctx_info(ctx)[0]
    buf = torch.zeros(d.m * d.n * 2 * (d.level + 1) * N, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    H.hetal_mat_export_dev(ctx, mat, buf.data_ptr())
    H.hetal_ntt_forward(ctx, buf.data_ptr(), 2 * d.m * d.n, d.level + 1)
    H.hetal_ctx_sync(ctx)
    return buf, d


def test_rescale_noalloc_matches_rescale_twice(env):
    import torch
    ctx, sk = env
    N, L, K = H.hetal_ctx_info(ctx)
    level = L - 1
    for call, nonce in enumerate((11, 12)):
        X = wl.uniform_matrix(1024, 32, 40 + call)
        h = H.hetal_encrypt(ctx, sk, 9, nonce, X, 1024, 32, H.TILE_NONE, 0, level, 2.0 ** 50)
        ref = H.hetal_rescale(ctx, h)
        want = H.hetal_mat_export(ctx, ref)
        src, d = _ntt_domain(ctx, h, torch)
        out = torch.zeros(2 * level * N, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        allocs = H.hetal_alloc_count(ctx)
        H.hetal_rescale_noalloc(ctx, src.data_ptr(), out.data_ptr(), 1, level)
        assert H.hetal_alloc_count(ctx) == allocs, "the call allocated device memory"
        H.hetal_ntt_inverse(ctx, out.data_ptr(), 2, level)
        H.hetal_ctx_sync(ctx)
        got = out.cpu().numpy().view(np.uint64).reshape(want.shape)
        assert np.array_equal(got, want), "call %d differs from hetal_rescale" % call
        H.hetal_mat_free(ref)
        H.hetal_mat_free(h)


def test_rescale_noalloc_rejects_sizes_beyond_scratch(env):
    import torch
    ctx, _ = env
    N, L, K = H.hetal_ctx_info(ctx)
    dummy = torch.zeros(16, dtype=torch.int64, device="cuda")
    with pytest.raises(H.HetalError) as ei:
        # 2 * 4 * 65536 * 12 words > 2^21: refused on the host before any device work
        H.hetal_rescale_noalloc(ctx, dummy.data_ptr(), dummy.data_ptr(), 4, L - 1)
    assert ei.value.code == H.ERR_INVALID_ARG
    assert "exceeds the static scratch" in H.hetal_last_error(ctx)


def test_rescale_noalloc_rejects_overlapping_buffers(env):
    """The output may not overlap the input: the last pass reads one while it writes the other."""
    import torch
    ctx, _ = env
    N, L, K = H.hetal_ctx_info(ctx)
    level = 3
    buf = torch.zeros(2 * (2 * level + 1) * N, dtype=torch.int64, device="cuda")
    base = buf.data_ptr()
    with pytest.raises(H.HetalError) as ei:   # output starting inside the input
        H.hetal_rescale_noalloc(ctx, base, base + 8 * N, 1, level)
    assert ei.value.code == H.ERR_INVALID_ARG and "overlaps" in H.hetal_last_error(ctx)
    # disjoint halves of one buffer are fine
    H.hetal_rescale_noalloc(ctx, base, base + 8 * 2 * (level + 1) * N, 1, level)
    H.hetal_ctx_sync(ctx)
