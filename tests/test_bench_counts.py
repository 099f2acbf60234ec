"""The candidate counts bench.py's roofline uses (algorithmic bytes and
operations per launch = per-connective candidates x per-candidate figures)
are the oracle's: summed over the connectives, the closed form of the
candidate space gives every level's candidate count of the oracle's
enumeration, on the bench's own traces and on other specifications."""
import os
import random
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2402_12373_gb300 import synth  # noqa: E402


def _check(spec, n_props, K):
    want = O.learn(spec.P, spec.N, n_props, max_size=K, stop_mode=0)
    for k in range(1, want["levels_done"] + 1):
        got = sum(bench.op_candidates(want["unique"], k, op, n_props) for op in range(8))
        assert got == want["candidates"][k], (k, got, want["candidates"][k])


def test_op_candidates_equal_the_oracle_on_the_bench_traces():
    _check(synth.single_large(), 3, 5)


def test_op_candidates_equal_the_oracle_on_other_specs():
    _check(synth.plain_single(), 2, 6)
    rng = random.Random(11)
    for n_props in (1, 2, 3):
        P = [[rng.randrange(1 << n_props) for _ in range(rng.randrange(1, 7))] for _ in range(5)]
        N = [[rng.randrange(1 << n_props) for _ in range(rng.randrange(1, 7))] for _ in range(5)]
        spec = synth.Spec(P=synth.TraceSet.from_list(P), N=synth.TraceSet.from_list(N), n_props=n_props)
        _check(spec, n_props, 5)


def test_integer_operation_counts():
    n = 5   # log steps for traces of at most 32 positions
    log = {op: bench.int_ops_per_candidate_trace(op, n, carry=False) for op in range(8)}
    carry = {op: bench.int_ops_per_candidate_trace(op, n, carry=True) for op in range(8)}
    # log steps: F a shift and an OR per step, G two more, U 4n - 2; plus 3
    assert log[5] == 2 * n + 3 and log[6] == 2 * n + 5 and log[7] == 4 * n + 1
    # the carry chain does not depend on the step count and is cheaper for F, G, U
    assert all(carry[op] == bench.int_ops_per_candidate_trace(op, 7, carry=True) for op in range(8))
    assert all(carry[op] < log[op] for op in (5, 6, 7))
    assert all(carry[op] == log[op] for op in (0, 1, 2, 3, 4))
