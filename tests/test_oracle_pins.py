"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test would fail on a plausible mistake in the oracle: a wrong shift
direction or a weak next (worked examples), a dropped clause or an off-by-one
in F/G/U (brute force over every trace of length <= 6 against the
exponential-propagation algorithms), a wrong candidate space or a broken dedup
(brute force over all syntax trees), a non-minimal answer (exhaustive search
below the returned size).
"""
import itertools
import os
import random

import numpy as np
import pytest

import ltl_ref as R
from oracle import oracle as O
from paper_2402_12373_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _ts(traces):
    return synth.TraceSet.from_list(traces)


def _oracle_truth(formula, traces, n_props):
    return [list(map(int, v)) for v in O.evaluate_traces(formula, _ts(traces), n_props)]


# ------------------------------------------------------------ worked examples

def _read_worked_examples():
    cases = []
    word = None
    for line in open(os.path.join(GOLDEN, "worked_examples.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("word "):
            parts = line.split()
            letters = dict(kv.split("=") for kv in parts[2:])
            word = [1 << int(letters[ch][1:]) for ch in parts[1]]
            n_props = 1 + max(int(v[1:]) for v in letters.values())
            continue
        f, bits = [x.strip() for x in line.rsplit("=", 1)]
        cases.append((word, n_props, f, [int(c) for c in bits]))
    return cases


WORKED = _read_worked_examples()


@pytest.mark.parametrize("word,n_props,formula,bits", WORKED,
                         ids=[c[2] for c in WORKED])
def test_worked_examples(word, n_props, formula, bits):
    assert len(bits) == len(word)
    assert _oracle_truth(formula, [word], n_props) == [bits]
    # the independent pointwise reference agrees as well
    assert R.truth(R.parse(formula), word) == bits


def _lsb(s):          # paper string (position 0 leftmost) -> integer, bit i = position i
    return R.bits_of([int(c) for c in s])


def test_logstep_F_worked_example_and_lemma1():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "logstep_F_16.txt"))
            if l.strip() and not l.startswith("#")]
    L = int(rows[0][1])
    init = _lsb(rows[1][1])
    states = R.logstep_F(init, L)
    want = [_lsb(r[1]) for r in rows[2:]]
    assert states[1:1 + len(want)] == want
    # Lemma 1: after step i, position j holds iff the input holds somewhere in [j, j + 2^i)
    for i, st in enumerate(states):
        for j in range(L):
            assert ((st >> j) & 1) == int(any((init >> k) & 1 for k in range(j, min(j + (1 << i), L))))
    # ... and the oracle's F on a 16-long trace is the final state
    tr = [(init >> j) & 1 for j in range(L)]
    assert R.bits_of(_oracle_truth("F p0", [tr], 1)[0]) == states[-1]


def test_logstep_U_worked_example_and_lemma2():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "logstep_U_8.txt"))
            if l.strip() and not l.startswith("#")]
    L = int(rows[0][1])
    c1, c2 = _lsb(rows[1][1]), _lsb(rows[1][2])
    states = R.logstep_U(c1, c2, L)
    # rows come in (cs2, cs1) pairs per iteration
    it = 0
    for r in rows[2:]:
        var, shift, s1, s2 = r[0], int(r[1]), _lsb(r[2]), _lsb(r[3])
        k = shift.bit_length()          # iteration index after which this holds
        if var == "cs2":
            assert states[k][1] == s2
        else:
            assert states[k][0] == s1
    # Lemma 2 invariants at every step
    for i, (g, u) in enumerate(states):
        p = 1 << i
        for j in range(L):
            G_ok = all((c1 >> k) & 1 for k in range(j, min(j + p, L)))
            U_ok = any(((c2 >> k) & 1) and all((c1 >> m) & 1 for m in range(j, k))
                       for k in range(j, min(j + p, L)))
            assert ((g >> j) & 1) == int(G_ok) and ((u >> j) & 1) == int(U_ok)
    tr = [((c1 >> j) & 1) | (((c2 >> j) & 1) << 1) for j in range(L)]
    assert R.bits_of(_oracle_truth("(p0 U p1)", [tr], 2)[0]) == states[-1][1] == R.mask(L)


# ------------------------------------------------ brute force: all short traces

def _all_traces(max_len, n_props):
    out = []
    for L in range(max_len + 1):
        out += [list(t) for t in itertools.product(range(1 << n_props), repeat=L)]
    return out


ALL6 = _all_traces(6, 2)   # 5461 traces: every CS pair (p0, p1) of length <= 6


def test_all_short_traces_count():
    assert len(ALL6) == sum(4 ** L for L in range(7))


@pytest.mark.parametrize("formula", ["p0", "!p0", "X p0", "F p0", "G p0", "(p0 & p1)",
                                     "(p0 | p1)", "(p0 U p1)", "(p1 U p0)"])
def test_oracle_vs_logstep_every_trace_len_le_6(formula):
    """Naive semantics (oracle) == exponential propagation on every CS pair."""
    got = _oracle_truth(formula, ALL6, 2)
    for tr, g in zip(ALL6, got):
        L = len(tr)
        a = R.bits_of([t & 1 for t in tr])
        b = R.bits_of([(t >> 1) & 1 for t in tr])
        m = R.mask(L)
        want = {
            "p0": a, "!p0": m & ~a, "X p0": a >> 1, "F p0": R.logstep_F(a, L)[-1],
            "G p0": R.logstep_G(a, L), "(p0 & p1)": a & b, "(p0 | p1)": a | b,
            "(p0 U p1)": R.logstep_U(a, b, L)[-1][1], "(p1 U p0)": R.logstep_U(b, a, L)[-1][1],
        }[formula]
        assert R.bits_of(g) == want, (tr, formula)


def _random_formula(rng, size, n_props):
    if size == 1:
        return ("p", rng.randrange(n_props))
    if size == 2 or rng.random() < 0.45:
        return (rng.choice(R.UNARY), _random_formula(rng, size - 1, n_props))
    i = rng.randrange(1, size - 1)
    return (rng.choice(R.BINARY), _random_formula(rng, i, n_props),
            _random_formula(rng, size - 1 - i, n_props))


def test_oracle_vs_pointwise_nested_formulae():
    rng = random.Random(1)
    traces = ALL6[::7]
    for _ in range(60):
        f = _random_formula(rng, rng.randrange(1, 9), 2)
        got = _oracle_truth(R.to_str(f), traces, 2)
        want = [R.truth(f, tr) for tr in traces]
        assert got == want, R.to_str(f)


# ------------------------------------------------------------- closed forms

def test_closed_forms_F_G_X():
    """F f holds at i iff i <= last position of f (the footnote's 'round up to
    a power of two minus one' in the paper's bit order); G f holds at i iff
    i > last position where f fails; X f at i is f at i+1, false at the end."""
    rng = random.Random(2)
    traces = [[rng.randrange(2) for _ in range(rng.randrange(0, 40))] for _ in range(300)]
    F = _oracle_truth("F p0", traces, 1)
    G = _oracle_truth("G p0", traces, 1)
    X = _oracle_truth("X p0", traces, 1)
    for tr, f, g, x in zip(traces, F, G, X):
        L = len(tr)
        last1 = max([i for i in range(L) if tr[i]], default=-1)
        last0 = max([i for i in range(L) if not tr[i]], default=-1)
        assert f == [int(i <= last1) for i in range(L)]
        assert g == [int(i > last0) for i in range(L)]
        assert x == [tr[i + 1] if i + 1 < L else 0 for i in range(L)]
        a = R.bits_of(tr)
        # on one integer: F = 2^(msb+1) - 1 (bit i = position i)
        assert R.bits_of(f) == ((1 << a.bit_length()) - 1 if a else 0)


IDENTITIES = [
    ("F F p0", "F p0"),
    ("G p0", "!F !p0"),
    ("F p0", "((p1 | !p1) U p0)"),
    ("(p0 U p1)", "(p1 | (p0 & X (p0 U p1)))"),
    ("!!p0", "p0"),
    ("!(p0 & p1)", "(!p0 | !p1)"),
    ("G G p0", "G p0"),
    ("F (p0 | p1)", "(F p0 | F p1)"),
    ("G (p0 & p1)", "(G p0 & G p1)"),
    ("X (p0 & p1)", "(X p0 & X p1)"),
]


@pytest.mark.parametrize("lhs,rhs", IDENTITIES)
def test_identities(lhs, rhs):
    rng = random.Random(3)
    traces = [[rng.randrange(4) for _ in range(rng.randrange(0, 30))] for _ in range(200)]
    assert _oracle_truth(lhs, traces, 2) == _oracle_truth(rhs, traces, 2)


def test_empty_trace_never_satisfies():
    for f in ["p0", "!p0", "G p0", "F p0", "(p0 U p1)", "!X p0"]:
        assert _oracle_truth(f, [[]], 2) == [[]]
    P, N = _ts([[]]), _ts([[1]])
    assert not O.separates("!p0", P, N, 1)      # false at i >= |tr|, negation included
    assert O.separates("!p0", _ts([[0]]), _ts([[]]), 1)


def test_parse_errors_and_sizes():
    with pytest.raises(ValueError):
        O.evaluate("(p0 &", np.zeros(1, np.uint32), np.array([0, 1], np.uint64), 1)
    with pytest.raises(ValueError):
        O.evaluate("p3", np.zeros(1, np.uint32), np.array([0, 1], np.uint64), 2)
    assert O.size("F (p0 & X p1)") == 5
    assert O.size("(G (!p0 | F p1) | p2)") == 8
    assert O.size("((p0))") == 1


# ------------------------------------------------ enumeration vs brute force

def _tiny_specs():
    specs = []
    for seed in range(6):
        rng = random.Random(100 + seed)
        n_props = 1 + seed % 2
        n = rng.randrange(2, 9)
        traces = [[rng.randrange(1 << n_props) for _ in range(rng.randrange(0, 6))] for _ in range(n)]
        h = max(1, n // 2)
        specs.append((traces[:h], traces[h:], n_props))
    return specs


@pytest.mark.parametrize("spec", _tiny_specs())
def test_enumeration_equals_brute_force(spec):
    P, N, n_props = spec
    K = 6 if n_props == 1 else 5
    bf = R.brute_force(P, N, n_props, 127, K)
    r = O.learn(_ts(P), _ts(N), n_props, max_size=K, stop_mode=0)
    assert r["unique"][1:] == bf["unique"][1:]
    assert r["size"] == bf["min_size"]
    # the candidate counts follow the stated candidate space
    cc = R.candidate_counts(r["unique"], 127, K)
    assert r["candidates"][2:] == cc[2:]
    assert r["candidates"][1] == n_props


@pytest.mark.parametrize("ops", [R.OPBIT["F"] | R.OPBIT["&"] | R.OPBIT["!"],
                                 R.OPBIT["U"] | R.OPBIT["X"],
                                 R.OPBIT["G"] | R.OPBIT["|"]])
def test_enumeration_ops_mask_equals_brute_force(ops):
    P, N, n_props = _tiny_specs()[1]
    bf = R.brute_force(P, N, n_props, ops, 6)
    r = O.learn(_ts(P), _ts(N), n_props, ops=ops, max_size=6, stop_mode=0)
    assert r["unique"][1:] == bf["unique"][1:]
    assert r["size"] == bf["min_size"]


def test_minimality_on_plain_single():
    """No syntax tree below the returned size separates (exhaustive)."""
    s = synth.plain_single()
    r = O.learn(s.P, s.N, s.n_props, max_size=7)
    assert r["status"] == "found" and r["size"] == 5
    assert O.separates(r["formula"], s.P, s.N, 2)
    assert O.size(r["formula"]) == 5
    P, N = s.P.to_list(), s.N.to_list()
    trees = R.all_trees(2, 127, r["size"] - 1)
    for k in range(1, r["size"]):
        for t in trees[k]:
            assert not (all(R.holds(t, tr, 0) for tr in P) and not any(R.holds(t, tr, 0) for tr in N))


def test_stop_modes_agree():
    s = synth.plain_single()
    r1 = O.learn(s.P, s.N, 2, max_size=7, stop_mode=1)
    r2 = O.learn(s.P, s.N, 2, max_size=7, stop_mode=2)
    r0 = O.learn(s.P, s.N, 2, max_size=7, stop_mode=0)
    assert r1["size"] == r2["size"] == r0["size"] == 5
    assert r1["unique"][:5] == r2["unique"][:5] == r0["unique"][:5]
    assert r2["unique"][5] == r0["unique"][5]
    assert r0["levels_done"] == 7 and r2["levels_done"] == 5 and r1["levels_done"] == 4


# ---------------------------------------------------------------- metamorphic

def _min_and_counts(P, N, n_props, K):
    r = O.learn(_ts(P), _ts(N), n_props, max_size=K, stop_mode=2)
    return r["size"], r["unique"][: (r["size"] or K + 1)]


def test_metamorphic_permutation_and_renaming():
    s = synth.plain_single(seed=3)
    P, N = s.P.to_list(), s.N.to_list()
    base = _min_and_counts(P, N, 2, 7)
    rng = random.Random(5)
    P2, N2 = P[:], N[:]
    rng.shuffle(P2); rng.shuffle(N2)
    assert _min_and_counts(P2, N2, 2, 7) == base
    swap = lambda tr: [((x & 1) << 1) | ((x >> 1) & 1) for x in tr]
    assert _min_and_counts([swap(t) for t in P], [swap(t) for t in N], 2, 7) == base


def test_metamorphic_conservative_extension():
    """If phi is minimal for (P, N) and phi |= (P', N'), then (P u P', N u N')
    has the same minimal cost (Section 2)."""
    s = synth.plain_single(seed=1)
    r = O.learn(s.P, s.N, 2, max_size=7)
    phi = R.parse(r["formula"])
    rng = random.Random(9)
    extra = [[rng.randrange(4) for _ in range(rng.randrange(1, 9))] for _ in range(40)]
    P2 = s.P.to_list() + [t for t in extra if R.holds(phi, t, 0)]
    N2 = s.N.to_list() + [t for t in extra if not R.holds(phi, t, 0)]
    r2 = O.learn(_ts(P2), _ts(N2), 2, max_size=7)
    assert r2["size"] == r["size"]


def test_metamorphic_swap_classes():
    """Swapping P and N changes the minimal size by at most one (negation)."""
    for seed in range(3):
        s = synth.plain_single(seed=seed)
        a = O.learn(s.P, s.N, 2, max_size=7)["size"]
        b = O.learn(s.N, s.P, 2, max_size=7)["size"]
        assert a is not None and b is not None and abs(a - b) <= 1


def test_planted_formulae_separate_generated_specs():
    for f in (synth.plain_single, lambda: synth.single_large(n_each=64)):
        s = f()
        assert O.separates(s.planted, s.P, s.N, s.n_props)
        assert O.size(s.planted) == s.planted_size


def test_unsolvable_and_cap():
    same = [[1, 2, 3]]
    r = O.learn(_ts(same), _ts(same), 2, max_size=4)
    assert r["status"] == "not_found"
    s = synth.plain_single()
    r = O.learn(s.P, s.N, 2, max_size=7, stop_mode=0, max_entries=50)
    assert r["status"] in ("cap", "found")


# ------------------------------------------------ costs, NNF, noisy learning

VARIANTS = [
    dict(costs=[1, 1, 1, 1, 1, 1, 1, 1], nnf=False, max_errors=0),
    dict(costs=[1, 2, 1, 1, 1, 1, 1, 1], nnf=False, max_errors=0),
    dict(costs=[2, 1, 3, 1, 2, 1, 2, 3], nnf=False, max_errors=0),
    dict(costs=[1, 1, 1, 1, 1, 1, 1, 1], nnf=True, max_errors=0),
    dict(costs=[1, 1, 2, 2, 1, 1, 1, 9], nnf=True, max_errors=0),
    dict(costs=[1, 1, 1, 1, 1, 1, 1, 1], nnf=False, max_errors=1),
    dict(costs=[1, 1, 1, 1, 1, 1, 1, 1], nnf=False, max_errors=2),
]


@pytest.mark.parametrize("variant", VARIANTS, ids=lambda v: "c%s_nnf%d_e%d" % ("".join(map(str, v["costs"])), v["nnf"], v["max_errors"]))
@pytest.mark.parametrize("spec", _tiny_specs()[:4])
def test_variants_equal_brute_force(spec, variant):
    """Cost homomorphism (levels = costs), negation normal form and noisy
    learning, against every syntax tree of cost <= K."""
    P, N, n_props = spec
    K = 6 if n_props == 1 else 5
    bf = R.brute_force(P, N, n_props, 127, K, **variant)
    r = O.learn(_ts(P), _ts(N), n_props, max_size=K, stop_mode=0, **variant)
    assert r["unique"][1:] == bf["unique"][1:]
    assert r["size"] == bf["min_size"]
    if r["formula"] is not None:
        f = R.parse(r["formula"])
        assert R.cost(f, variant["costs"]) == r["size"]
        assert R.errors(f, P, N) <= variant["max_errors"]
        if variant["nnf"]:
            def nnf_ok(t):
                if t[0] == "!":
                    return t[1][0] == "p"
                return all(nnf_ok(c) for c in t[1:] if isinstance(c, tuple))
            assert nnf_ok(f)


def test_high_cost_bans_a_connective():
    """Section 2: a connective of cost above the budget is never used."""
    s = synth.plain_single()
    r = O.learn(s.P, s.N, 2, max_size=7, costs=[1, 1, 1, 1, 1, 50, 1, 1])   # F banned
    assert r["status"] == "found" and "F" not in r["formula"]
    assert r["size"] >= 5
