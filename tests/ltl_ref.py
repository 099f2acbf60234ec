"""Independent pure-Python references used to pin the oracle.

Nothing here is imported by the library or by the oracle.  Three things:

* `holds(f, tr, i)`: the satisfaction relation of Section 2, written
  pointwise and recursively straight from its clauses (no tables, no
  shifts).
* `logstep_*`: the exponential-propagation algorithms of Section 4 and
  Appendix B on Python integers, returning every intermediate state so that
  the invariants of Lemma 1 and Lemma 2 and the worked examples of Appendix A
  can be checked step by step.  Bit i of an integer is position i (the paper
  writes position 0 leftmost and uses a left shift for X; with position 0 as
  the least significant bit the same step is a right shift).
* `brute_force`: every syntax tree up to a size, evaluated with `holds`, no
  cache and no dedup; gives the per-size unique counts and the minimal
  separating size by definition.
"""
from __future__ import annotations

import itertools
from typing import Dict, Iterable, List, Optional, Sequence, Tuple

UNARY = ("!", "X", "F", "G")
BINARY = ("&", "|", "U")
OPBIT = {"!": 1, "&": 2, "|": 4, "X": 8, "F": 16, "G": 32, "U": 64}

# ---------------------------------------------------------------- parsing

def parse(s: str):
    """Formula text -> AST tuple.  Grammar: f := !f | Xf | Ff | Gf | p<n> |
    (f) | (f & f) | (f | f) | (f U f)."""
    pos = [0]

    def ws():
        while pos[0] < len(s) and s[pos[0]] in " \t\n":
            pos[0] += 1

    def f():
        ws()
        c = s[pos[0]]
        if c in "!XFG":
            pos[0] += 1
            return (c, f())
        if c == "p":
            pos[0] += 1
            j = pos[0]
            while pos[0] < len(s) and s[pos[0]].isdigit():
                pos[0] += 1
            return ("p", int(s[j:pos[0]]))
        if c == "(":
            pos[0] += 1
            a = f()
            ws()
            o = s[pos[0]]
            pos[0] += 1
            if o == ")":
                return a
            b = f()
            ws()
            assert s[pos[0]] == ")", s
            pos[0] += 1
            return (o, a, b)
        raise ValueError("bad formula %r at %d" % (s, pos[0]))

    t = f()
    ws()
    assert pos[0] == len(s), s
    return t


def to_str(f) -> str:
    k = f[0]
    if k == "p":
        return "p%d" % f[1]
    if k == "!":
        return "!" + to_str(f[1])
    if k in "XFG":
        return "%s %s" % (k, to_str(f[1]))
    return "(%s %s %s)" % (to_str(f[1]), k, to_str(f[2]))


def size(f) -> int:
    return 1 if f[0] == "p" else 1 + sum(size(c) for c in f[1:])


# ---------------------------------------------------------------- semantics

def holds(f, tr: Sequence[int], i: int) -> bool:
    """tr, i |= f (Section 2).  False whenever i >= |tr|."""
    n = len(tr)
    if i >= n:
        return False
    k = f[0]
    if k == "p":
        return bool((tr[i] >> f[1]) & 1)
    if k == "!":
        return not holds(f[1], tr, i)
    if k == "&":
        return holds(f[1], tr, i) and holds(f[2], tr, i)
    if k == "|":
        return holds(f[1], tr, i) or holds(f[2], tr, i)
    if k == "X":
        return holds(f[1], tr, i + 1)
    if k == "F":
        return any(holds(f[1], tr, j) for j in range(i, n))
    if k == "G":
        return all(holds(f[1], tr, j) for j in range(i, n))
    if k == "U":
        return any(holds(f[2], tr, j) and all(holds(f[1], tr, m) for m in range(i, j))
                   for j in range(i, n))
    raise ValueError(k)


def truth(f, tr) -> List[int]:
    return [int(holds(f, tr, i)) for i in range(len(tr))]


# ---------------------------------------------------------------- log-step

def mask(L: int) -> int:
    return (1 << L) - 1


def n_steps(L: int) -> int:
    """Shifts 1, 2, 4, ... until the reach covers distance L-1."""
    k = 0
    while (1 << k) < L:
        k += 1
    return k


def logstep_F(cs: int, L: int) -> List[int]:
    """States cs_0 .. cs_k of exponential propagation for F (Lemma 1)."""
    out = [cs]
    for i in range(n_steps(L)):
        cs = cs | (cs >> (1 << i))
        out.append(cs)
    return out


def logstep_U(cs1: int, cs2: int, L: int) -> List[Tuple[int, int]]:
    """States (cs1_i, cs2_i) of exponential propagation for U (Lemma 2)."""
    out = [(cs1, cs2)]
    for i in range(n_steps(L)):
        s = 1 << i
        cs2 = cs2 | (cs1 & (cs2 >> s))
        cs1 = cs1 & (cs1 >> s)
        out.append((cs1, cs2))
    return out


def logstep_G(cs: int, L: int) -> int:
    """G f = not F not f, restricted to the trace (reading of the paper's G)."""
    m = mask(L)
    return m & ~logstep_F(m & ~cs, L)[-1]


def bits_of(v: Sequence[int]) -> int:
    return sum(int(b) << i for i, b in enumerate(v))


def from_bits(x: int, L: int) -> List[int]:
    return [(x >> i) & 1 for i in range(L)]


# ---------------------------------------------------------------- brute force

def all_trees(n_props: int, ops: int, max_size: int) -> Dict[int, List]:
    trees: Dict[int, List] = {1: [("p", p) for p in range(n_props)]}
    un = [o for o in UNARY if ops & OPBIT[o]]
    bi = [o for o in BINARY if ops & OPBIT[o]]
    for s in range(2, max_size + 1):
        cur = [(o, t) for o in un for t in trees[s - 1]]
        for i in range(1, s - 1):
            j = s - 1 - i
            cur += [(o, a, b) for o in bi for a in trees[i] for b in trees[j]]
        trees[s] = cur
    return trees


COST_INDEX = {"p": 0, "!": 1, "&": 2, "|": 3, "X": 4, "F": 5, "G": 6, "U": 7}


def cost(f, costs) -> int:
    """Cost of a syntax tree under a cost homomorphism (Section 2)."""
    return costs[COST_INDEX[f[0]]] + sum(cost(c, costs) for c in f[1:] if isinstance(c, tuple))


def trees_by_cost(n_props: int, ops: int, max_cost: int, costs, nnf: bool = False) -> Dict[int, List]:
    """Every syntax tree of cost <= max_cost, by cost (NNF: ! over atoms only)."""
    out: Dict[int, List] = {c: [] for c in range(1, max_cost + 1)}
    if costs[0] <= max_cost:
        out[costs[0]] = [("p", p) for p in range(n_props)]
    un = [o for o in UNARY if ops & OPBIT[o]]
    bi = [o for o in BINARY if ops & OPBIT[o]]
    for c in range(1, max_cost + 1):
        for o in un:
            r = c - costs[COST_INDEX[o]]
            if r >= 1:
                src = out[r] if not (nnf and o == "!") else [t for t in out[r] if t[0] == "p"]
                out[c] += [(o, t) for t in src]
        for o in bi:
            r = c - costs[COST_INDEX[o]]
            for i in range(1, r):
                out[c] += [(o, a, b) for a in out[i] for b in out[r - i]]
    return out


def errors(f, P, N) -> int:
    return sum(1 for tr in P if not holds(f, tr, 0)) + sum(1 for tr in N if holds(f, tr, 0))


def brute_force(P: List[List[int]], N: List[List[int]], n_props: int, ops: int,
                max_size: int, costs=None, nnf: bool = False, max_errors: int = 0) -> Dict:
    """Unique characteristic matrices per cost level and the minimal cost of a
    formula misclassifying at most max_errors traces, from every syntax tree
    (no cache, no dedup, no compositional shortcut)."""
    costs = list(costs) if costs is not None else [1] * 8
    traces = list(P) + list(N)
    trees = trees_by_cost(n_props, ops, max_size, costs, nnf)
    seen = set()
    unique = [0] * (max_size + 1)
    min_size: Optional[int] = None
    for s in range(1, max_size + 1):
        new = set()
        for t in trees[s]:
            cm = tuple(tuple(truth(t, tr)) for tr in traces)
            if cm not in seen:
                new.add(cm)
            if min_size is None and errors(t, P, N) <= max_errors:
                min_size = s
        unique[s] = len(new)
        seen |= new
    return {"unique": unique, "min_size": min_size}


def candidate_counts(unique: Sequence[int], ops: int, max_size: int) -> List[int]:
    """Closed form of the candidate space from the unique counts (one reading
    of Section 3's handleOp): unary ops over level k-1; And/Or over splits
    i <= j (pairs a < b when i == j); U over ordered splits and pairs."""
    c = [0] * (max_size + 1)
    if max_size >= 1:
        c[1] = None  # atoms: one per proposition, filled by caller
    n_un = sum(1 for o in UNARY if ops & OPBIT[o])
    n_sym = sum(1 for o in "&|" if ops & OPBIT[o])
    has_u = bool(ops & OPBIT["U"])
    for k in range(2, max_size + 1):
        v = n_un * unique[k - 1]
        for i in range(1, k - 1):
            j = k - 1 - i
            if has_u:
                v += unique[i] * unique[j]
            if i < j:
                v += n_sym * unique[i] * unique[j]
            elif i == j:
                v += n_sym * unique[i] * (unique[i] - 1) // 2
        c[k] = v
    return c
