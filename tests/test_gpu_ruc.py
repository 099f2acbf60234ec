"""Relaxed uniqueness checks (Section 5): cache admission on a 63-bit key
(a hash of the matrix, or the first-k-percent map of Section 7), optionally
with masked key bits (the masking experiment of Section 7).

Which of two matrices with equal keys is kept depends on timing, so a lossy
run is checked by what holds for every outcome:
* soundness: a returned formula separates, under the oracle's semantics, and
  has the reported size; no separator is smaller than the exact minimum;
* the cache holds distinct matrices of formulae of size <= k, so its size
  after level k is at most the exact enumeration's, and at most the number
  of distinct keys (2^(63 - masked bits));
* the candidate space of each level is the closed form of the unique counts
  the run itself admitted.
Where the key holds the whole matrix, or a 63-bit hash meets no collision at
these sizes, the relaxed check is exact and the run equals the oracle.
"""
import random

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import ltl_ref as R
from oracle import oracle as O
from paper_2402_12373_gb300 import _lib as L
from paper_2402_12373_gb300 import synth


@pytest.fixture(scope="module")
def ws():
    assert torch.cuda.is_available()
    return L.default_workspace(2 << 30)


def _exactly_equal(g, o):
    assert g["status"] == o["status"], (g, o)
    assert g["size"] == o["size"]
    d = g["levels_done"]
    assert d == o["levels_done"]
    assert g["unique"][1:d + 1] == o["unique"][1:d + 1]
    assert g["candidates"][1:d + 1] == o["candidates"][1:d + 1]


def _mixed(seed, n):
    rng = random.Random(seed)
    out = []
    for i in range(n):
        n_props = rng.choice([1, 2, 3])
        nt = rng.choice([8, 40, 150, 600])
        maxlen = rng.choice([6, 20, 45, 90])
        tr = [[rng.randrange(1 << n_props) for _ in range(rng.randrange(1, maxlen + 1))] for _ in range(nt)]
        h = rng.randrange(1, nt)
        out.append((synth.TraceSet.from_list(tr[:h]), synth.TraceSet.from_list(tr[h:]), n_props, 5))
    return out


@pytest.mark.parametrize("stop", [L.STOP_LEVEL, L.STOP_NONE])
def test_hash_without_mask_equals_exact(ws, stop):
    """A 63-bit hashed key meets no collision at these sizes (about 1e5
    entries), so hashed admission reproduces the exact enumeration."""
    probs = [(synth.plain_single(seed=s).P, synth.plain_single(seed=s).N, 2, 7) for s in range(3)] + _mixed(3, 8)
    with L.Context(workspace=ws, stop=stop, ruc=L.RUC_HASH) as ctx:
        for P, N, n_props, K in probs:
            g = ctx.learn(P, N, n_props, max_size=K)
            o = O.learn(P, N, n_props, max_size=K, stop_mode=2 if stop == L.STOP_LEVEL else 0)
            _exactly_equal(g, o)


def test_fkp_exact_when_key_holds_the_matrix(ws):
    """With n traces of length at most 63 // n, the first-k-percent key is the
    whole matrix: no information is lost and the run equals the oracle."""
    rng = random.Random(11)
    for n_traces, n_props in [(2, 1), (3, 2), (5, 2), (7, 1), (9, 3)]:
        b = 63 // n_traces
        tr = [[rng.randrange(1 << n_props) for _ in range(rng.randrange(1, b + 1))] for _ in range(n_traces)]
        h = max(1, n_traces // 2)
        P, N = synth.TraceSet.from_list(tr[:h]), synth.TraceSet.from_list(tr[h:])
        for stop, sm in [(L.STOP_LEVEL, 2), (L.STOP_NONE, 0)]:
            with L.Context(workspace=ws, stop=stop, ruc=L.RUC_FKP) as ctx:
                g = ctx.learn(P, N, n_props, max_size=6)
            _exactly_equal(g, O.learn(P, N, n_props, max_size=6, stop_mode=sm))


def _lossy_properties(g, exact, P, N, n_props, K, key_bits):
    d = g["levels_done"]
    assert d >= 1
    cum_g = np.cumsum(g["unique"][1:d + 1])
    cum_o = np.cumsum(exact["unique"][1:d + 1])
    assert (cum_g <= cum_o).all(), (g["unique"], exact["unique"])
    assert cum_g[-1] <= 2 ** key_bits
    cf = R.candidate_counts(g["unique"], L.ALL, d)
    assert g["candidates"][2:d + 1] == cf[2:d + 1]
    if g["status"] == "found":
        assert O.separates(g["formula"], P, N, n_props), g["formula"]
        assert O.size(g["formula"]) == g["size"]
        assert exact["size"] is not None and g["size"] >= exact["size"]


@pytest.mark.parametrize("mode,mask", [(L.RUC_HASH, 40), (L.RUC_HASH, 52), (L.RUC_HASH, 58), (L.RUC_HASH, 61),
                                       (L.RUC_FKP, 0), (L.RUC_FKP, 30), (L.RUC_FKP, 55)])
def test_lossy_admission_properties(ws, mode, mask):
    s = synth.single_large(n_each=128)
    P, N, n_props, K = s.P, s.N, 3, 6
    exact = O.learn(P, N, n_props, max_size=K, stop_mode=0)
    runs = {}
    for stop in (L.STOP_NONE, L.STOP_LEVEL):
        with L.Context(workspace=ws, stop=stop, ruc=mode, ruc_mask_bits=mask) as ctx:
            runs[stop] = g = ctx.learn(P, N, n_props, max_size=K)
        _lossy_properties(g, exact, P, N, n_props, K, 63 - mask)
    if mode == L.RUC_HASH and mask >= 52:
        # a key space of 2^11 or fewer values holds fewer matrices than exist
        g = runs[L.STOP_NONE]
        assert g["levels_done"] == K
        assert sum(g["unique"][1:K + 1]) < sum(exact["unique"][1:K + 1])


def test_lossy_batch_and_streaming(ws):
    """Batched problems under FKP; the chunk-group (streaming) kernel under
    hashed (masked and unmasked) and FKP admission."""
    probs = _mixed(7, 10)
    res = L.learn_batch([p[:3] + (L.ALL, p[3]) for p in probs], stop=L.STOP_NONE, workspace=ws, ruc=L.RUC_FKP)
    for (P, N, n_props, K), g in zip(probs, res):
        exact = O.learn(P, N, n_props, max_size=K, stop_mode=0)
        _lossy_properties(g, exact, P, N, n_props, K, 63)
    s = synth.single_large(n_each=3000)
    exact = O.learn(s.P, s.N, 3, max_size=4, stop_mode=0)
    for mode, mask in [(L.RUC_HASH, 50), (L.RUC_FKP, 0), (L.RUC_HASH, 0)]:
        with L.Context(workspace=ws, stop=L.STOP_NONE, ruc=mode, ruc_mask_bits=mask) as ctx:
            g = ctx.learn(s.P, s.N, 3, max_size=4)
        assert g["chunk_groups"] > 1
        _lossy_properties(g, exact, s.P, s.N, 3, 4, 63 - mask)
        if mode == L.RUC_HASH and mask == 0:
            _exactly_equal(g, exact)


def test_invalid_ruc_rejected(ws):
    with pytest.raises(L.LtlError):
        L.Context(workspace=ws, ruc=3)
    with pytest.raises(L.LtlError):
        L.Context(workspace=ws, ruc=L.RUC_HASH, ruc_mask_bits=63)
