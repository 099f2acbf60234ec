"""CPU checks of the Hamming workload (Section 7) and of the divide-and-conquer
algebra of Section 6, with the oracle as the enumerator.

`dc_reference` restates detSplit and randSplit on index sets in plain Python
(the oracle learns each part, the oracle's evaluator decides membership); the
tests check that every combined formula separates its specification, which is
what the combination (f11 & f12) | (f21 & f22) must guarantee under the
readings taken (the first disjunct's language is L(f11) & L(f12)).
"""
import itertools
import math
import random

import pytest

from oracle import oracle as O
from paper_2402_12373_gb300 import synth


# ------------------------------------------------------------------ Hamming

@pytest.mark.parametrize("l,delta,n_props", [(3, 1, 2), (6, 2, 2), (9, 1, 1), (12, 2, 1), (48, 2, 2)])
def test_hamming_is_the_exact_distance_shell(l, delta, n_props):
    s = synth.hamming(l, delta, n_props=n_props, seed=7)
    assert s.P.n == 1 and s.N.n == math.comb(l * n_props, delta)
    tr = s.P.to_list()[0]
    assert len(tr) == l and all(0 <= x < (1 << n_props) for x in tr)
    seen = set()
    for t in s.N.to_list():
        assert len(t) == l
        d = sum(bin(a ^ b).count("1") for a, b in zip(tr, t))
        assert d == delta
        seen.add(tuple(t))
    assert len(seen) == s.N.n and tuple(tr) not in seen


def test_hamming_is_seeded():
    a, b, c = synth.hamming(20, 1, seed=1), synth.hamming(20, 1, seed=1), synth.hamming(20, 1, seed=2)
    assert a.P.to_list() == b.P.to_list() and a.N.to_list() == b.N.to_list()
    assert a.P.to_list() != c.P.to_list()


def test_hamming_48_2_has_4560_negatives():
    """Section 7 reports up to 4560 negatives at length 48: C(2 * 48, 2)."""
    assert synth.hamming(48, 2).N.n == 4560


# ------------------------------------------------------------------ D&C algebra

TRUE, FALSE = "T", "F"


def _and(a, b):
    if FALSE in (a, b):
        return FALSE
    return b if a == TRUE else a if b == TRUE else "(%s & %s)" % (a, b)


def _or(a, b):
    if TRUE in (a, b):
        return TRUE
    return b if a == FALSE else a if b == FALSE else "(%s | %s)" % (a, b)


class _Spec:
    def __init__(self, spec):
        self.traces = spec.P.to_list() + spec.N.to_list()
        self.nP = spec.P.n
        self.n_props = spec.n_props

    def ts(self, idx):
        return synth.TraceSet.from_list([self.traces[i] for i in idx])

    def member(self, f, idx):
        if f in (TRUE, FALSE):
            return {i for i in idx if f == TRUE}
        v = O.evaluate_traces(f, self.ts(idx), self.n_props)
        return {i for i, x in zip(idx, v) if len(x) and x[0]}


def dc_reference(spec, mode, window, K=5, seed=0):
    S = _Spec(spec)
    rng = random.Random(seed)

    def enum(P, N):
        r = O.learn(S.ts(P), S.ts(N), S.n_props, max_size=K, stop_mode=1)
        if r["status"] == "found":
            return r["formula"]
        assert len(P) + len(N) > 2, "tiny parts are solvable at these sizes"
        return None

    def det(P, N, win):
        if not N:
            return TRUE
        if not P:
            return FALSE
        if len(P) + len(N) <= win:
            f = enum(P, N)
            if f is not None:
                return f
            return det(P, N, max(2, min(win, len(P) + len(N)) // 2))
        hp, hn = (len(P) + 1) // 2, (len(N) + 1) // 2
        P1, P2, N1, N2 = P[:hp], P[hp:], N[:hn], N[hn:]
        f11 = det(P1, N1, win)
        L11 = S.member(f11, N2 + P2)
        f12 = det(P1, [t for t in N2 if t in L11], win)
        L12 = S.member(f12, P2)
        P2r = [t for t in P2 if not (t in L11 and t in L12)]
        f21 = det(P2r, N1, win)
        L21 = S.member(f21, N2)
        f22 = det(P2r, [t for t in N2 if t in L21], win)
        return _or(_and(f11, f12), _and(f21, f22))

    def rand(P, N, win):
        if not N:
            return TRUE
        if not P:
            return FALSE
        m = min(win, len(P) + len(N))
        while True:
            kp = min(len(P), (m + 1) // 2)
            kn = min(len(N), m - kp)
            kp = min(len(P), m - kn)
            P0, N0 = sorted(rng.sample(P, kp)), sorted(rng.sample(N, kn))
            f11 = enum(P0, N0)
            if f11 is not None:
                break
            m = max(2, m // 2)
        L = S.member(f11, P + N)
        Pin, Pout = [t for t in P if t in L], [t for t in P if t not in L]
        Nin, Nout = [t for t in N if t in L], [t for t in N if t not in L]
        return _or(_and(f11, rand(Pin, Nin, win)), _and(rand(Pout, Nout, win), rand(Pout, Nin, win)))

    P = list(range(S.nP))
    N = list(range(S.nP, len(S.traces)))
    return (det if mode == "det" else rand)(P, N, window)


@pytest.mark.parametrize("mode", ["det", "rand"])
@pytest.mark.parametrize("case", [("hamming", 5, 1, 8), ("hamming", 6, 2, 16), ("small", 40, 0, 8),
                                  ("small", 60, 1, 16)])
def test_dc_reference_combination_separates(mode, case):
    kind, a, b, window = case
    if kind == "hamming":
        spec = synth.hamming(a, b, n_props=2, seed=3)
    else:
        spec = synth.random_small(seed=b, n_traces=a, n_props=2, lo=3, hi=7)
        # drop traces that occur in both classes (no formula separates them)
        pos = {tuple(t) for t in spec.P.to_list()}
        spec = synth.Spec(spec.P, synth.TraceSet.from_list([t for t in spec.N.to_list() if tuple(t) not in pos]),
                          spec.n_props)
    f = dc_reference(spec, mode, window, K=5, seed=11)
    assert f not in (TRUE, FALSE)
    assert O.separates(f, spec.P, spec.N, spec.n_props), f
