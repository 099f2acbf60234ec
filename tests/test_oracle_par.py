"""The multi-core oracle (oracle_learn_par) is the serial oracle with each
block of a level's candidates built on several host cores and admitted in
enumeration order: every count, the status, the first separator's size and its
formula text must equal the serial oracle's, whatever the thread count or
block size (a block of 1 candidate, or of one level's whole candidate list)."""
import random

import pytest

from oracle import oracle as O
from paper_2402_12373_gb300 import synth


def _same(a, b):
    for key in ("status", "size", "formula", "levels_done", "unique", "candidates"):
        assert a[key] == b[key], (key, a[key], b[key])


def _random_spec(seed):
    rng = random.Random(seed)
    n_props = rng.choice([1, 2, 3])
    tr = [[rng.randrange(1 << n_props) for _ in range(rng.randrange(0, 9))] for _ in range(rng.randrange(2, 14))]
    h = rng.randrange(1, len(tr))
    return synth.TraceSet.from_list(tr[:h]), synth.TraceSet.from_list(tr[h:]), n_props, rng.randrange(1, 128)


@pytest.mark.parametrize("stop_mode", [0, 1, 2])
def test_par_equals_serial_plain_single(stop_mode):
    s = synth.plain_single()
    want = O.learn(s.P, s.N, 2, max_size=7, stop_mode=stop_mode)
    for threads, block in ((1, 0), (3, 0), (0, 1), (0, 0), (4, 5000)):
        _same(O.learn_par(s.P, s.N, 2, max_size=7, stop_mode=stop_mode, threads=threads, block_bytes=block), want)


@pytest.mark.parametrize("seed", range(12))
def test_par_equals_serial_random_specs(seed):
    P, N, n_props, ops = _random_spec(seed)
    for stop_mode in (0, 1):
        want = O.learn(P, N, n_props, ops=ops, max_size=5, stop_mode=stop_mode)
        _same(O.learn_par(P, N, n_props, ops=ops, max_size=5, stop_mode=stop_mode, threads=4, block_bytes=300), want)


def test_par_equals_serial_with_a_full_cache():
    s = synth.plain_single(seed=3)
    for cap in (5, 40, 300):
        want = O.learn(s.P, s.N, 2, max_size=7, stop_mode=0, max_entries=cap)
        got = O.learn_par(s.P, s.N, 2, max_size=7, stop_mode=0, max_entries=cap, threads=4, block_bytes=2000)
        _same(got, want)


def test_par_equals_serial_on_large_traces():
    s = synth.single_large(n_each=48)
    want = O.learn(s.P, s.N, 3, max_size=6, stop_mode=2)
    got = O.learn_par(s.P, s.N, 3, max_size=6, stop_mode=2)
    _same(got, want)
    assert got["threads"] >= 1
