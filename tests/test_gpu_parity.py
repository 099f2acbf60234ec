"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer work, so the bar is bit-exactness: characteristic sequences equal
bit for bit, the same minimal size, the same number of unique
characteristic matrices at every completed size level, the same candidate
counts, and a returned formula that separates under the oracle's semantics
(several minimal separators can exist; any one is correct).
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

ALL = L.ALL


@pytest.fixture(scope="module")
def ws():
    assert torch.cuda.is_available()
    return L.default_workspace(2 << 30)


def _ts(traces):
    return synth.TraceSet.from_list(traces)


def _pack(bits_per_trace, W):
    out = np.zeros((len(bits_per_trace), W), dtype=np.uint64)
    for t, v in enumerate(bits_per_trace):
        for i, b in enumerate(v):
            if b:
                out[t, i // 64] |= np.uint64(1) << np.uint64(i % 64)
    return out


def _oracle_words(formula, traces, n_props, W):
    return _pack(O.evaluate_traces(formula, traces, n_props), W)


def _rand_formula(rng, size, n_props):
    if size == 1:
        return ("p", rng.randrange(n_props))
    if size == 2 or rng.random() < 0.45:
        return (rng.choice(R.UNARY), _rand_formula(rng, size - 1, n_props))
    i = rng.randrange(1, size - 1)
    return (rng.choice(R.BINARY), _rand_formula(rng, i, n_props), _rand_formula(rng, size - 1 - i, n_props))


# ------------------------------------------------------------------ ltl_eval

def _trace_sets():
    yield "plain_single", synth.plain_single().P, 2
    s = synth.single_large(n_each=200)
    yield "single_large", s.N, 3
    rng = random.Random(7)
    for lo, hi in ((0, 3), (60, 70), (120, 136), (190, 260), (500, 520), (1000, 1024)):
        tr = [[rng.randrange(4) for _ in range(rng.randrange(lo, hi + 1))] for _ in range(37)]
        yield "len_%d_%d" % (lo, hi), _ts(tr), 2


@pytest.mark.parametrize("name,traces,n_props", list(_trace_sets()), ids=lambda x: x if isinstance(x, str) else "")
def test_eval_matches_oracle(name, traces, n_props):
    rng = random.Random(hash(name) & 0xffff)
    lens = traces.lengths()
    W = max(1, (int(lens.max()) + 63) // 64) if len(lens) else 1
    for _ in range(25):
        f = R.to_str(_rand_formula(rng, rng.randrange(1, 13), n_props))
        got = L.evaluate(f, traces, n_props)
        assert got.shape == (traces.n, W)
        want = _oracle_words(f, traces, n_props, W)
        assert np.array_equal(got, want), f


def test_eval_worked_example_and_wider_output():
    # Section 4: a over abcaa is 10011 (position 0 leftmost), X a is 00110
    abcaa = _ts([[1, 2, 4, 1, 1]])
    assert int(L.evaluate("p0", abcaa, 3)[0, 0]) == 0b11001
    assert int(L.evaluate("X p0", abcaa, 3)[0, 0]) == 0b01100
    assert int(L.evaluate("!p0", abcaa, 3)[0, 0]) == 0b00110
    out = L.evaluate("F p1", abcaa, 3, words_per_trace=3)
    assert out.shape == (1, 3) and int(out[0, 0]) == 0b00011 and int(out[0, 1]) == 0 and int(out[0, 2]) == 0


def test_eval_empty_traces():
    ts = _ts([[], [1], []])
    got = L.evaluate("!p0", ts, 1)
    assert [int(x) for x in got[:, 0]] == [0, 0, 0]
    assert [int(x) for x in L.evaluate("G p0", ts, 1)[:, 0]] == [0, 1, 0]


# ------------------------------------------------------------------ ltl_learn

def _compare(spec_P, spec_N, n_props, ws, ops=ALL, K=7, mode=L.STOP_LEVEL):
    with L.Context(workspace=ws, stop=mode) as ctx:
        got = ctx.learn(spec_P, spec_N, n_props, ops=ops, max_size=K)
    want = O.learn(spec_P, spec_N, n_props, ops=ops, max_size=K, stop_mode=mode)
    assert got["status"] == want["status"], (got, want)
    assert got["size"] == want["size"]
    done = min(got["levels_done"], want["levels_done"])
    assert got["levels_done"] == want["levels_done"]
    assert got["unique"][1:done + 1] == want["unique"][1:done + 1]
    assert got["candidates"][1:done + 1] == want["candidates"][1:done + 1]
    if got["status"] == "found":
        assert O.separates(got["formula"], spec_P, spec_N, n_props), got["formula"]
        assert O.size(got["formula"]) == got["size"]
    return got, want


def test_learn_plain_single_all_modes(ws):
    s = synth.plain_single()
    got, want = _compare(s.P, s.N, 2, ws, K=7, mode=L.STOP_LEVEL)
    assert got["size"] == 5
    got, want = _compare(s.P, s.N, 2, ws, K=7, mode=L.STOP_NONE)
    assert got["levels_done"] == 7
    with L.Context(workspace=ws, stop=L.STOP_FIRST) as ctx:
        g = ctx.learn(s.P, s.N, 2, max_size=7)
    assert g["size"] == 5 and O.separates(g["formula"], s.P, s.N, 2)
    assert g["unique"][1:5] == want["unique"][1:5]


def test_learn_single_large_levels_1_to_6(ws):
    s = synth.single_large()
    got, want = _compare(s.P, s.N, 3, ws, K=6, mode=L.STOP_NONE)
    assert got["levels_done"] == 6
    # candidates follow the closed form of the stated candidate space
    cc = R.candidate_counts(got["unique"], ALL, 6)
    assert got["candidates"][2:7] == cc[2:7]


def _random_specs(n, seed):
    rng = random.Random(seed)
    for i in range(n):
        n_props = rng.choice([1, 2, 2, 3, 4])
        nt = rng.randrange(1, 24)
        maxlen = rng.choice([3, 6, 10, 40, 70, 130])
        tr = [[rng.randrange(1 << n_props) for _ in range(rng.randrange(0, maxlen + 1))] for _ in range(nt)]
        h = rng.randrange(0, nt + 1)
        ops = ALL if rng.random() < 0.6 else rng.randrange(1, 128)
        yield tr[:h], tr[h:], n_props, ops


@pytest.mark.parametrize("case", list(range(60)))
def test_learn_random_specs(ws, case):
    P, N, n_props, ops = list(_random_specs(60, 11))[case]
    K = 5 if n_props >= 3 else 6
    _compare(_ts(P), _ts(N), n_props, ws, ops=ops, K=K, mode=L.STOP_LEVEL)


def test_learn_edge_cases(ws):
    # P and N intersect: unsolvable
    same = [[1, 2, 3]]
    _compare(_ts(same + [[0]]), _ts(same), 2, ws, K=5)
    # empty P, empty N, all-empty traces
    _compare(_ts([]), _ts([[1, 0]]), 1, ws, K=3)
    _compare(_ts([[1]]), _ts([]), 1, ws, K=3)
    _compare(_ts([[], []]), _ts([[]]), 1, ws, K=4)
    # max size 1 and a single proposition
    _compare(_ts([[1, 0]]), _ts([[0, 1]]), 1, ws, K=1)
    # only negation / only U
    _compare(_ts([[0]]), _ts([[1]]), 1, ws, ops=L.NOT, K=3)
    _compare(_ts([[1, 2]]), _ts([[2, 1]]), 2, ws, ops=L.U, K=4)


@pytest.mark.parametrize("L_len", [63, 64, 65, 127, 128, 129, 255, 256, 257, 511, 512])
def test_learn_word_boundaries(ws, L_len):
    rng = random.Random(L_len)
    P = [[rng.randrange(4) for _ in range(L_len)] for _ in range(5)]
    N = [[rng.randrange(4) for _ in range(rng.randrange(L_len - 3, L_len + 1))] for _ in range(5)]
    P[0][-1] |= 2
    _compare(_ts(P), _ts(N), 2, ws, K=4, mode=L.STOP_NONE)


def test_learn_chunk_groups_streaming_path(ws):
    """More traces than one CTA keeps in registers: the two-pass path."""
    s = synth.single_large(n_each=3000)
    with L.Context(workspace=ws, stop=L.STOP_NONE) as ctx:
        got = ctx.learn(s.P, s.N, 3, max_size=5)
    assert got["chunk_groups"] > 1
    want = O.learn(s.P, s.N, 3, max_size=5, stop_mode=0)
    assert got["unique"][1:6] == want["unique"][1:6]
    assert got["candidates"][1:6] == want["candidates"][1:6]


def test_learn_device_input_matches_host_input(ws):
    s = synth.plain_single(seed=2)
    letters = np.concatenate([s.P.letters, s.N.letters]).astype(np.int32)
    offs = np.concatenate([s.P.offsets, s.N.offsets[1:] + s.P.offsets[-1]]).astype(np.int64)
    dl = torch.from_numpy(letters).cuda()
    do = torch.from_numpy(offs).cuda()
    with L.Context(workspace=ws, stop=L.STOP_NONE) as ctx:
        a = ctx.learn(s.P, s.N, 2, max_size=6)
        b = ctx.learn_device(dl, do, s.P.n, s.N.n, s.max_len(), 2, max_size=6)
    assert a["unique"] == b["unique"] and a["candidates"] == b["candidates"] and a["size"] == b["size"]


def test_learn_device_input_with_bad_offsets_is_rejected(ws):
    """Device-resident offsets that decrease, or that do not start at 0: the
    pack kernel packs such a trace as empty (it reads none of its letters) and
    flags the input, the call returns LTL_ERR_INVALID, and the same context
    then learns a valid input exactly.  Every offset stays inside the letter
    buffer."""
    s = synth.plain_single(seed=2)
    letters = np.concatenate([s.P.letters, s.N.letters]).astype(np.int32)
    offs = np.concatenate([s.P.offsets, s.N.offsets[1:] + s.P.offsets[-1]]).astype(np.int64)
    dl = torch.from_numpy(letters).cuda()
    decreasing = offs.copy()
    decreasing[3] = decreasing[4] + 1          # offsets[3] > offsets[4]
    shifted = offs.copy()
    shifted[0] = 1                             # the first trace does not start at 0
    with L.Context(workspace=ws, stop=L.STOP_NONE) as ctx:
        for bad in (decreasing, shifted):
            assert bad.max() <= len(letters)
            with pytest.raises(L.LtlError) as e:
                ctx.learn_device(dl, torch.from_numpy(bad).cuda(), s.P.n, s.N.n, s.max_len(), 2, max_size=6)
            assert e.value.status == L.LTL_ERR_INVALID
            assert "offsets decrease" in str(e.value)
        got = ctx.learn_device(dl, torch.from_numpy(offs).cuda(), s.P.n, s.N.n, s.max_len(), 2, max_size=6)
    want = O.learn(s.P, s.N, 2, max_size=6, stop_mode=0)
    assert got["unique"][1:7] == want["unique"][1:7]
    assert got["candidates"][1:7] == want["candidates"][1:7]


def test_cache_entries_are_their_formulas_and_distinct(ws):
    """Every sampled cache entry: its rebuilt formula has the level's size and
    the oracle's characteristic matrix of that formula is the stored one; all
    entries of the cache are pairwise distinct."""
    s = synth.plain_single()
    T = s.n_traces
    both = synth.TraceSet.from_list(s.P.to_list() + s.N.to_list())
    rng = random.Random(3)
    with L.Context(workspace=ws, stop=L.STOP_NONE) as ctx:
        got = ctx.learn(s.P, s.N, 2, max_size=6)
        W = got["words_per_trace"]
        seen = set()
        for k in range(1, 7):
            b, c = ctx.level_range(k)
            assert c == got["unique"][k]
            for idx in range(b, b + c):
                f, cs = ctx.entry(idx, T, W)
                key = cs.tobytes()
                assert key not in seen
                seen.add(key)
                if rng.random() < 0.15 or k <= 2:
                    assert O.size(f) == k, f
                    assert np.array_equal(cs, _oracle_words(f, both, 2, W)), f


def test_cap_reached_with_small_budget(ws):
    s = synth.single_large(n_each=256)
    with L.Context(workspace=ws, stop=L.STOP_NONE, mem_budget=64 << 20) as ctx:
        got = ctx.learn(s.P, s.N, 3, max_size=9)
    assert got["status"] in ("cap", "found")
    assert got["entries"] <= got["max_entries"]
    want = O.learn(s.P, s.N, 3, max_size=got["levels_done"], stop_mode=0)
    d = got["levels_done"]
    assert got["unique"][1:d + 1] == want["unique"][1:d + 1]


def test_streaming_cache_fills_during_a_level(ws):
    """Matrices larger than a CTA (the two-pass streaming kernel) with a cache
    that fills during a level: the candidates after that are only tested for
    separation (no fingerprint, probe or second pass).  Completed levels,
    the capped level's candidate count, the status and a found size equal the
    oracle's with the same capacity."""
    s = synth.single_large(n_each=3000)
    with L.Context(workspace=ws, stop=L.STOP_NONE, mem_budget=64 << 20, level_kernel=L.KERNEL_FUSED) as ctx:
        got = ctx.learn(s.P, s.N, 3, max_size=8)
    assert got["chunk_groups"] > 1
    assert got["status"] in ("cap", "found")
    d = got["levels_done"]
    assert got["candidates"][d + 1] > 0 and got["entries"] == got["max_entries"]   # filled during level d + 1
    want = O.learn(s.P, s.N, 3, max_size=8, stop_mode=0, max_entries=got["max_entries"])
    assert want["levels_done"] == d
    assert got["status"] == want["status"]
    assert got["unique"][1:d + 1] == want["unique"][1:d + 1]
    assert got["candidates"][1:d + 2] == want["candidates"][1:d + 2]
    if got["status"] == "found":
        assert got["size"] == want["size"]
        assert O.separates(got["formula"], s.P, s.N, 3)


def _long_traces(seed, n_each, lo, hi, n_props=2):
    rng = random.Random(seed)
    mk = lambda: [rng.randrange(1 << n_props) for _ in range(rng.randrange(lo, hi + 1))]
    return _ts([mk() for _ in range(n_each)]), _ts([mk() for _ in range(n_each)])


@pytest.mark.parametrize("max_chunks", [0, 1, 2, 4, 8])
def test_launch_shapes_narrow_and_wide(ws, max_chunks):
    """Every launch shape the planner can pick gives the oracle's counts:
    narrow (traces <= 32) and wide (33..64) layouts, CTAs of 32..256 threads,
    fused and two-pass."""
    s = synth.single_large(n_each=2048)                 # 4096 traces, narrow
    P2, N2 = _long_traces(5, 2048, 33, 64)               # 4096 traces, wide W = 1
    for (P, N, n_props, K) in ((s.P, s.N, 3, 4), (P2, N2, 2, 4)):
        with L.Context(workspace=ws, stop=L.STOP_NONE, max_chunks=max_chunks) as ctx:
            got = ctx.learn(P, N, n_props, max_size=K)
        want = _oracle_cached(P, N, n_props, K)
        assert got["unique"][1:K + 1] == want["unique"][1:K + 1], (max_chunks, got["threads_per_cta"])
        assert got["candidates"][1:K + 1] == want["candidates"][1:K + 1]


_ORACLE_CACHE = {}


def _oracle_cached(P, N, n_props, K):
    key = (P.letters.tobytes(), P.offsets.tobytes(), N.letters.tobytes(), N.offsets.tobytes(), n_props, K)
    if key not in _ORACLE_CACHE:
        _ORACLE_CACHE[key] = O.learn(P, N, n_props, max_size=K, stop_mode=0)
    return _ORACLE_CACHE[key]


def test_context_reuse_across_shapes(ws):
    """One context, problems of different launch shapes in turn (the same
    kernel with more, then less, then more shared memory per CTA)."""
    big = _long_traces(8, 2048, 33, 64)      # wide, 256 threads, 96 KiB of operand slots
    small = _long_traces(9, 1024, 33, 64)    # wide, 128 threads, 48 KiB
    with L.Context(workspace=ws, stop=L.STOP_NONE) as ctx:
        for P, N in (big, small, big, small):
            got = ctx.learn(P, N, 2, max_size=3)
            want = _oracle_cached(P, N, 2, 3)
            assert got["unique"][1:4] == want["unique"][1:4]
