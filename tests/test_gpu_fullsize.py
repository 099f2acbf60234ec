"""Parity at the full sizes of the benchmark workloads, in the launch
configuration bench.py times (a context over a torch workspace, every level
enumerated).  The checks are (a) every level's unique and candidate counts
equal to the oracle's, read from the JSON files that
tests/golden/make_fullsize_levels.py writes by running the oracle alone on
the same seeded inputs (an input digest ties each file to the generator's
output); (b) sampled outputs the oracle computes one by one: cache entries of
every level, rebuilt into formulas whose characteristic matrices the oracle
evaluates and which must equal the stored ones, and the returned separator;
(c) properties that hold at any size: candidate counts follow the closed form
of the unique counts, every entry of a level has that level's size, sampled
entries are pairwise distinct.
"""
import hashlib
import json
import os
import random

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import ltl_ref as R
from oracle import oracle as O
from paper_2402_12373_gb300 import _lib as L
from paper_2402_12373_gb300 import synth


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden_levels(name, spec):
    """The oracle's per-level counts for workload `name`, after checking that
    they were computed on exactly these inputs."""
    with open(os.path.join(GOLDEN, "%s_levels.json" % name)) as f:
        g = json.load(f)
    h = hashlib.sha256()
    for ts in (spec.P, spec.N):
        h.update(np.ascontiguousarray(ts.letters, dtype=np.uint32).tobytes())
        h.update(np.ascontiguousarray(ts.offsets, dtype=np.uint64).tobytes())
    assert h.hexdigest() == g["input_sha256"], "generated inputs differ from the golden file's"
    return g


def _oracle_words(formula, traces, n_props, W):
    v = O.evaluate_traces(formula, traces, n_props)
    out = np.zeros((len(v), W), dtype=np.uint64)
    for t, bits in enumerate(v):
        idx = np.nonzero(bits)[0]
        for i in idx:
            out[t, i // 64] |= np.uint64(1) << np.uint64(i % 64)
    return out


def _check_sampled_entries(ctx, got, both, n_props, K, per_level, seed):
    rng = random.Random(seed)
    T, W = both.n, got["words_per_trace"]
    seen = set()
    for k in range(1, K + 1):
        b, c = ctx.level_range(k)
        assert c == got["unique"][k]
        for idx in rng.sample(range(b, b + c), min(per_level, c)):
            f, cs = ctx.entry(idx, T, W)
            assert O.size(f) == k, f
            assert np.array_equal(cs, _oracle_words(f, both, n_props, W)), f
            key = cs.tobytes()
            assert key not in seen
            seen.add(key)


def test_single_large_full_size():
    """The bench workload: 2048 traces, sizes 1..9, every level."""
    s = synth.single_large()
    ws = L.default_workspace(24 << 30)
    with L.Context(workspace=ws, stop=L.STOP_NONE) as ctx:
        got = ctx.learn(s.P, s.N, 3, max_size=9)
        assert got["levels_done"] == 9 and got["status"] == "found" and got["size"] == 8
        assert O.separates(got["formula"], s.P, s.N, 3)
        want = _golden_levels("single_large", s)      # the oracle, every level 1..9
        assert want["max_size"] == 9 and want["levels_done"] == 9 and want["size"] == 8
        assert got["unique"][1:10] == want["unique"][1:10]
        assert got["candidates"][1:10] == want["candidates"][1:10]
        cc = R.candidate_counts(got["unique"], L.ALL, 9)
        assert got["candidates"][2:10] == cc[2:10]
        both = synth.TraceSet.from_list(s.P.to_list() + s.N.to_list())
        _check_sampled_entries(ctx, got, both, 3, 9, 12, 1)


def test_single_large_full_size_time_to_learn_mode():
    s = synth.single_large()
    ws = L.default_workspace(8 << 30)
    with L.Context(workspace=ws, stop=L.STOP_FIRST) as ctx:
        got = ctx.learn(s.P, s.N, 3, max_size=9)
    assert got["status"] == "found" and got["size"] == 8
    assert O.separates(got["formula"], s.P, s.N, 3)
    # minimality below 8: the full enumeration found no separator at sizes <= 7
    assert got["levels_done"] == 7


def test_trace_scaling_full_size():
    """65536 traces of length 33..128 (two words, two-pass streaming kernel)."""
    s = synth.trace_scaling()
    want = _golden_levels("trace_scaling", s)         # the oracle, every level 1..K
    K = want["max_size"]
    ws = L.default_workspace(24 << 30)
    with L.Context(workspace=ws, stop=L.STOP_NONE) as ctx:
        got = ctx.learn(s.P, s.N, 4, max_size=K)
        assert got["words_per_trace"] == 2 and got["chunk_groups"] > 1
        assert got["levels_done"] == want["levels_done"] == K
        assert got["unique"][1:K + 1] == want["unique"][1:K + 1]
        assert got["candidates"][1:K + 1] == want["candidates"][1:K + 1]
        cc = R.candidate_counts(got["unique"], L.ALL, K)
        assert got["candidates"][2:K + 1] == cc[2:K + 1]
        assert got["status"] == want["status"] == "found" and got["size"] == want["size"] == 3
        assert O.separates(got["formula"], s.P, s.N, 4)
        both = synth.TraceSet.from_list(s.P.to_list() + s.N.to_list())
        _check_sampled_entries(ctx, got, both, 4, K, 2, 2)
