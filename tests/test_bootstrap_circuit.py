"""Host logic of the bootstrapping circuit (paper_2403_14111_gb300/bootstrap.py) against
the fake C ABI: handles, levels, keys, and every addition meeting two equal scales without
a relabel (EvalMod's double-angle steps would amplify a relabel's error 4^r times).  No GPU."""
import math

import numpy as np
import pytest

from paper_2403_14111_gb300 import bootstrap as B
from paper_2403_14111_gb300 import circuit

from fake_abi import FakeABI, chain


@pytest.mark.parametrize("log_n,fft", [(10, True), (13, True), (16, True), (10, False), (13, False)])
def test_bootstrap_circuit(monkeypatch, log_n, fft):
    N = 1 << log_n
    prm = B.BootstrapParams(fft=fft)
    top = B.levels(N, prm) + 3
    fake = FakeABI(N, chain(top), B.rotations(N, prm))
    monkeypatch.setattr(B, "H", fake)
    monkeypatch.setattr(circuit, "H", fake)
    d_in = 2.0 ** 50
    a = fake._new(0, d_in)
    out = B.bootstrap(None, None, a, d_in, 2.0 ** 50, prm)
    lv, sc = fake._get(out)
    assert lv == top - B.levels(N, prm)
    assert abs(math.log2(sc) - 40) < 1e-3
    assert fake.relabels == 0                     # no addition needed a relabel
    assert fake.max_coeff < 2.0 ** 63
    n = N // 2
    if fft:
        diags = sum(len(M) for inv in (True, False) for M in B._factored(N, inv, prm.per_level))
    else:
        diags = 2 * n
        n1 = 1 << int(round(math.log2(n) / 2))
        assert len(B.rotations(N, prm)) == (n1 - 1) + (n // n1 - 1)
    # two transforms (one summed product per level or giant step), two EvalMods (14 each)
    assert fake.calls.get("cmult_terms", 0) == diags
    sums = (2 * B.transform_levels(N, prm)) if fft else 2 * (n // (1 << int(round(math.log2(n) / 2))))
    assert fake.calls["cmult"] == sums + 2 * (1 + 12 + 1)
    assert fake.calls["conj"] == 1
    fake.hetal_mat_free(out)
    fake.hetal_mat_free(a)
    assert not fake.live, "%d handles leaked" % len(fake.live)


def test_diagonals_are_those_of_the_embedding():
    from oracle import bootstrap as bt   # the oracle's dense matrices, small N only
    N = 64
    U = bt.encoding_matrix(N)
    Ui = U.conj().T / N
    for k in (0, 1, 7, 31):
        assert np.max(np.abs(B.embedding_diagonal(N, k, False) - bt.diagonal(U, k))) < 1e-12
        assert np.max(np.abs(B.embedding_diagonal(N, k, True) - bt.diagonal(Ui, k))) < 1e-12


def test_device_plaintext_cache_is_filled_once_and_reused(monkeypatch):
    N = 1 << 12
    top = B.levels(N) + 3
    fake = FakeABI(N, chain(top), B.rotations(N))
    monkeypatch.setattr(B, "H", fake)
    monkeypatch.setattr(circuit, "H", fake)
    a = fake._new(0, 2.0 ** 50)
    cache = {}
    out1 = B.bootstrap(None, None, a, 2.0 ** 50, cache=cache)
    uploads, encodes = fake.calls["upload"], fake.calls["encode"]
    assert uploads == len(cache) and encodes == uploads
    out2 = B.bootstrap(None, None, a, 2.0 ** 50, cache=cache)
    assert fake.calls["upload"] == uploads and fake.calls["encode"] == encodes   # nothing new
    assert fake._get(out1) == fake._get(out2)
    for h in (out1, out2, a):
        fake.hetal_mat_free(h)
    circuit.free_plains(cache)
    assert not fake.live and not fake.plains


def test_refuses_a_raised_input_and_a_short_chain(monkeypatch):
    N = 1 << 10
    fake = FakeABI(N, chain(B.levels(N)), B.rotations(N))
    monkeypatch.setattr(B, "H", fake)
    monkeypatch.setattr(circuit, "H", fake)
    with pytest.raises(ValueError):
        B.bootstrap(None, None, fake._new(0, 2.0 ** 50), 2.0 ** 50)   # not enough levels
    fake2 = FakeABI(N, chain(B.levels(N) + 3), B.rotations(N))
    monkeypatch.setattr(B, "H", fake2)
    monkeypatch.setattr(circuit, "H", fake2)
    with pytest.raises(ValueError):
        B.bootstrap(None, None, fake2._new(2, 2.0 ** 50), 2.0 ** 50)  # not level 0
