"""Host logic of Protocol 1's epochs (paper_2403_14111_gb300/step.py train_epochs) against the
fake C ABI: the client's answers decide the epochs run and the best weight, every handle the
loop makes is released (on success and when a step fails), and the gamma sequence runs on
across batches.  No GPU."""
import pytest

from paper_2403_14111_gb300 import bootstrap as B
from paper_2403_14111_gb300 import circuit, step

from fake_abi import FakeABI, chain


def _fake(monkeypatch):
    N, s0, s1, c = 2 ** 16, 1024, 32, 16
    top = 14 + B.levels(N)
    fake = FakeABI(N, chain(top), step.train_boot_rotations(s0, s1, c))
    for mod in (B, circuit, step):
        monkeypatch.setattr(mod, "H", fake)
    return fake, c


def test_epochs_best_weight_and_handles(monkeypatch):
    fake, c = _fake(monkeypatch)
    S = 2.0 ** 50
    Wbar, Xval = fake._new(13, S, 24), fake._new(13, S)
    calls = []

    def grad(V):
        calls.append(fake._get(V))
        return fake._new(2, S * (1 + 1e-7), 24), (fake._new(5, S), fake._new(7, S))
    answers = iter([(False, True), (False, False), (True, False)])
    seen = []

    def client(logits):
        seen.append(fake._get(logits))
        return next(answers)
    gammas = []
    real = step.nag_update_refresh
    monkeypatch.setattr(step, "nag_update_refresh", lambda *a, **k: (gammas.append(a[5]), real(*a, **k))[1])
    best, epochs = step.train_epochs(None, None, Wbar, [grad, grad], Xval, c, S, 10, client)
    assert epochs == 3 and len(seen) == 3 and len(calls) == 6
    assert gammas == step.nag_gammas(20)[:6]          # one NAG sequence across batches and epochs
    assert fake._get(best) == (13, S) and fake._blocks(best) == 24
    assert all(lv == 10 for lv, _ in seen)            # the logits of a refreshed W (13) and X_val (13)
    for h in (best, Wbar, Xval):
        fake.hetal_mat_free(h)
    assert not fake.live, "%d handles leaked" % len(fake.live)


def test_a_failing_step_releases_everything(monkeypatch):
    fake, c = _fake(monkeypatch)
    S = 2.0 ** 50
    Wbar, Xval = fake._new(13, S, 24), fake._new(13, S)
    n = [0]

    def grad(V):
        n[0] += 1
        if n[0] == 4:
            raise RuntimeError("the fourth step fails")
        return fake._new(2, S, 24), ()
    with pytest.raises(RuntimeError):
        step.train_epochs(None, None, Wbar, [grad], Xval, c, S, 10, lambda logits: (False, True))
    assert sorted(fake.live) == sorted([Wbar, Xval])


def test_validation_client_loss_and_patience(monkeypatch):
    """The client's cross-entropy equals scipy's log-softmax form and the oracle's independently
    written client; patience counts epochs without a new minimum."""
    import numpy as np
    from scipy.special import log_softmax
    from oracle import bootstrap as bt
    rng = np.random.default_rng(3)
    labels = rng.integers(0, 10, 64)
    Ls = [rng.normal(0, s, (64, 16)) for s in (1.0, 0.5, 2.0, 3.0, 0.4)]
    monkeypatch.setattr(step.H, "hetal_decrypt", lambda ctx, sk, h: h)   # the "handle" is the plaintext
    client = step.ValidationClient(None, None, labels, 10, patience=2)
    answers = [client(L) for L in Ls]
    want = [float(-log_softmax(L[:, :10], axis=1)[np.arange(64), labels].mean()) for L in Ls]
    assert np.allclose(client.losses, want, rtol=0, atol=1e-12)
    best, bad, expect = np.inf, 0, []
    for x in want:
        if x < best:
            best, bad = x, 0
            expect.append((False, True))
        else:
            bad += 1
            expect.append((bad >= 2, False))
    assert answers == expect

    class Plain:   # the oracle's client reads decrypted blocks: a stand-in oracle returning slots
        def decrypt_slots(self, ct):
            return ct
    oc = bt.ValidationClient(Plain(), labels, 10, patience=2)
    from types import SimpleNamespace
    for L in Ls:
        blk = np.zeros((64, 32), dtype=complex)
        blk[:, :16] = L
        oc(SimpleNamespace(blocks=[[blk.reshape(-1)]], s0=64, s1=32))
    assert np.allclose(oc.losses, client.losses, rtol=0, atol=1e-12)
