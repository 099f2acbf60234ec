"""Seeded synthetic learning problems (P, N) for the enumerative LTL learner.

This module only *generates inputs*. It holds none of the learner's
arithmetic (no characteristic sequences, no shifts, no enumeration, no
dedup); both the CUDA path and the CPU oracle take its traces as plain
input.  To label traces by a planted formula it carries its own small
evaluator (a backward recurrence over positions, numpy over a batch of
traces); the labels are inputs, and parity never depends on them being the
labels of any particular formula.

Traces follow the paper's model (Section 2): a trace is a finite string over
the powerset of the alphabet {p0 .. p(n-1)}; one position is stored as a
uint32 bit mask (bit p set iff proposition p holds there).  A trace set is the
pair (letters, offsets): the concatenated positions of all traces, and
n_traces+1 prefix offsets into them.

Random numbers come from a counter-based SplitMix64 (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): the i-th
output of the stream with seed s is the SplitMix64 output function applied
to s + (i+1)*0x9E3779B97F4A7C15 (mod 2^64), so any bit of any trace attempt is
a pure function of (seed, attempt, position, proposition).

Workload shapes follow the paper's benchmark families (Section 7: BenchBase
style uniform random traces with short lengths and small alphabets, labelled
by a separating formula):

* ``plain_single``   2 props, length U{4..10}, Bernoulli(0.5), F(p0 & X p1),
                      16 + 16 traces.
* ``single_large``   3 props, length U{16..32}, Bernoulli(0.3),
                      (G(!p0 | F p1) | p2), 1024 + 1024 traces.
* ``trace_scaling``  4 props, length U{33..128}, Bernoulli(0.25),
                      (((p0 U p1) & G !p3) & F p2), 32768 + 32768 traces.
* ``batched``        problem i: props U{2..5}, |P|=|N| log-uniform 16..4096,
                      length U{8..64}, Bernoulli(0.3), a planted formula drawn
                      uniformly among syntax trees of size U{3..9}.
* ``planted_large``  the plain-single shape with 1024 + 1024 traces (divide
                      and conquer with parts the enumerator solves).
"""
from __future__ import annotations

import dataclasses
import itertools
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_LEN_COUNTER = np.uint64(1 << 40)   # counter slot reserved for a trace's length draw
_AUX_COUNTER = np.uint64(1 << 41)   # counter slots for other per-attempt draws


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea & Flood 2014), vectorised."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def splitmix64(seed, counter) -> np.ndarray:
    """Counter-th output of the SplitMix64 stream seeded with ``seed``."""
    seed = np.asarray(seed, dtype=np.uint64)
    counter = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(seed + (counter + np.uint64(1)) * GOLDEN)


def _uniform01(u: np.ndarray) -> np.ndarray:
    return (u >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def _bernoulli(u: np.ndarray, p: float) -> np.ndarray:
    return (u >> np.uint64(11)) < np.uint64(int(p * (1 << 53)))


def _uniform_int(u: np.ndarray, lo: int, hi: int) -> np.ndarray:
    return lo + (u % np.uint64(hi - lo + 1)).astype(np.int64)


# --------------------------------------------------------------------------
# Trace sets
# --------------------------------------------------------------------------

@dataclasses.dataclass
class TraceSet:
    letters: np.ndarray   # uint32 [total positions]
    offsets: np.ndarray   # uint64 [n_traces + 1]

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0]) - 1

    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets).astype(np.int64)

    def trace(self, i: int) -> np.ndarray:
        return self.letters[int(self.offsets[i]):int(self.offsets[i + 1])]

    @staticmethod
    def from_list(traces: Sequence[Sequence[int]]) -> "TraceSet":
        lens = [len(t) for t in traces]
        off = np.zeros(len(traces) + 1, dtype=np.uint64)
        off[1:] = np.cumsum(lens, dtype=np.uint64) if lens else []
        let = np.array([x for t in traces for x in t], dtype=np.uint32)
        return TraceSet(let, off)

    @staticmethod
    def from_dense(bits: np.ndarray, lengths: np.ndarray) -> "TraceSet":
        """bits: uint32 [n, Lmax] letter masks; lengths: [n]."""
        n = bits.shape[0]
        lengths = np.asarray(lengths, dtype=np.int64)
        keep = np.arange(bits.shape[1])[None, :] < lengths[:, None]
        off = np.zeros(n + 1, dtype=np.uint64)
        off[1:] = np.cumsum(lengths).astype(np.uint64)
        return TraceSet(np.ascontiguousarray(bits[keep]).astype(np.uint32), off)

    def to_list(self) -> List[List[int]]:
        return [self.trace(i).tolist() for i in range(self.n)]


@dataclasses.dataclass
class Spec:
    """A learning problem: positive traces P, negative traces N, n_props."""
    P: TraceSet
    N: TraceSet
    n_props: int
    planted: Optional[str] = None
    planted_size: Optional[int] = None
    name: str = ""

    @property
    def n_traces(self) -> int:
        return self.P.n + self.N.n

    def max_len(self) -> int:
        m = 0
        for s in (self.P, self.N):
            if s.n:
                m = max(m, int(s.lengths().max()))
        return m


# --------------------------------------------------------------------------
# Planted formulae: a tiny AST and the generator's own labelling evaluator
# --------------------------------------------------------------------------
# AST nodes are tuples: ("p", i) | ("!", f) | ("X", f) | ("F", f) | ("G", f)
#                      | ("&", f, g) | ("|", f, g) | ("U", f, g)

def ast_size(f) -> int:
    if f[0] == "p":
        return 1
    return 1 + sum(ast_size(c) for c in f[1:])


def ast_str(f) -> str:
    k = f[0]
    if k == "p":
        return "p%d" % f[1]
    if k == "!":
        return "!" + ast_str(f[1])
    if k in "XFG":
        return "%s %s" % (k, ast_str(f[1]))
    return "(%s %s %s)" % (ast_str(f[1]), k, ast_str(f[2]))


def _label_eval(f, props: np.ndarray, lengths: np.ndarray) -> np.ndarray:
    """Truth of f at every position of a batch of traces.

    props: bool [n_props, n, Lmax]; lengths: int [n].  Returns bool [n, Lmax],
    false at positions >= length (finite-trace semantics, Section 2).
    """
    n, L = props.shape[1], props.shape[2]
    inside = np.arange(L)[None, :] < lengths[:, None]
    k = f[0]
    if k == "p":
        return props[f[1]] & inside
    if k == "!":
        return ~_label_eval(f[1], props, lengths) & inside
    if k in "&|":
        a = _label_eval(f[1], props, lengths)
        b = _label_eval(f[2], props, lengths)
        return (a & b) if k == "&" else (a | b)
    a = _label_eval(f[1], props, lengths)
    out = np.zeros((n, L), dtype=bool)
    if k == "X":
        out[:, :-1] = a[:, 1:]
        return out & inside
    if k == "F":
        acc = np.zeros(n, dtype=bool)
        for i in range(L - 1, -1, -1):
            acc = acc | a[:, i]
            out[:, i] = acc
        return out & inside
    if k == "G":
        acc = np.ones(n, dtype=bool)
        for i in range(L - 1, -1, -1):
            acc = np.where(inside[:, i], acc & a[:, i], True)
            out[:, i] = acc
        return out & inside
    if k == "U":
        b = _label_eval(f[2], props, lengths)
        acc = np.zeros(n, dtype=bool)
        for i in range(L - 1, -1, -1):
            acc = b[:, i] | (a[:, i] & acc)
            out[:, i] = acc
        return out & inside
    raise ValueError("bad node %r" % (k,))


def label_at_zero(f, bits: np.ndarray, lengths: np.ndarray, n_props: int) -> np.ndarray:
    """tr |= f for each trace of a dense batch (bits uint32 [n, Lmax])."""
    if bits.shape[1] == 0:
        return np.zeros(bits.shape[0], dtype=bool)
    props = np.stack([((bits >> np.uint32(p)) & np.uint32(1)).astype(bool)
                      for p in range(max(n_props, 1))])
    return _label_eval(f, props, np.asarray(lengths))[:, 0] & (np.asarray(lengths) > 0)


# --------------------------------------------------------------------------
# Random trace attempts
# --------------------------------------------------------------------------

def _attempts(seed: int, first: int, count: int, n_props: int, lo: int, hi: int,
              p_bit: float) -> Tuple[np.ndarray, np.ndarray]:
    """Trace attempts first..first+count-1: (bits uint32 [count, hi], lengths)."""
    att = np.arange(first, first + count, dtype=np.uint64)
    tseed = splitmix64(np.uint64(seed), att)                      # per-attempt stream
    lengths = _uniform_int(splitmix64(tseed, _LEN_COUNTER), lo, hi)
    pos = np.arange(hi, dtype=np.uint64)
    bits = np.zeros((count, hi), dtype=np.uint32)
    for p in range(n_props):
        ctr = pos * np.uint64(32) + np.uint64(p)
        u = splitmix64(tseed[:, None], ctr[None, :])
        bits |= (_bernoulli(u, p_bit).astype(np.uint32) << np.uint32(p))
    bits[np.arange(hi)[None, :] >= lengths[:, None]] = 0
    return bits, lengths


def rejection_fill(seed: int, formula, n_pos: int, n_neg: int, n_props: int,
                   lo: int, hi: int, p_bit: float, batch: int = 4096,
                   max_attempts: int = 1 << 26) -> Tuple[TraceSet, TraceSet, int]:
    """Draw attempts in counter order; each goes to P if the planted formula holds
    at position 0 and to N otherwise, until both classes are full."""
    pos_b, pos_l, neg_b, neg_l = [], [], [], []
    npos = nneg = 0
    first = 0
    while (npos < n_pos or nneg < n_neg) and first < max_attempts:
        bits, lens = _attempts(seed, first, batch, n_props, lo, hi, p_bit)
        lab = label_at_zero(formula, bits, lens, n_props)
        for want, sink_b, sink_l, have, cap in ((True, pos_b, pos_l, npos, n_pos),
                                                (False, neg_b, neg_l, nneg, n_neg)):
            idx = np.nonzero(lab == want)[0][: max(cap - have, 0)]
            sink_b.append(bits[idx]); sink_l.append(lens[idx])
        npos = sum(len(x) for x in pos_l); nneg = sum(len(x) for x in neg_l)
        first += batch
    if npos < n_pos or nneg < n_neg:
        raise RuntimeError("rejection sampling did not fill both classes")
    P = TraceSet.from_dense(np.concatenate(pos_b), np.concatenate(pos_l))
    N = TraceSet.from_dense(np.concatenate(neg_b), np.concatenate(neg_l))
    return P, N, first


# --------------------------------------------------------------------------
# The named workloads
# --------------------------------------------------------------------------

F_PLAIN = ("F", ("&", ("p", 0), ("X", ("p", 1))))                          # size 5
F_LARGE = ("|", ("G", ("|", ("!", ("p", 0)), ("F", ("p", 1)))), ("p", 2))   # size 8
F_SCALE = ("&", ("&", ("U", ("p", 0), ("p", 1)), ("G", ("!", ("p", 3)))),
           ("F", ("p", 2)))                                                  # size 10


def plain_single(seed: int = 0) -> Spec:
    """2 props, 16 + 16 traces of length U{4..10}, Bernoulli(0.5), F(p0 & X p1)."""
    P, N, _ = rejection_fill(seed, F_PLAIN, 16, 16, 2, 4, 10, 0.5, batch=256)
    return Spec(P, N, 2, ast_str(F_PLAIN), ast_size(F_PLAIN), "plain_single")


def single_large(seed: int = 0, n_each: int = 1024) -> Spec:
    """3 props, 1024 + 1024 traces of length U{16..32}, Bernoulli(0.3),
    (G(!p0 | F p1) | p2)."""
    P, N, _ = rejection_fill(seed, F_LARGE, n_each, n_each, 3, 16, 32, 0.3)
    return Spec(P, N, 3, ast_str(F_LARGE), ast_size(F_LARGE), "single_large")


def trace_scaling(seed: int = 0, n_each: int = 32768) -> Spec:
    """4 props, 32768 + 32768 traces of length U{33..128}, Bernoulli(0.25),
    (((p0 U p1) & G !p3) & F p2).

    Literal rejection sampling accepts a positive about once per 10^6 attempts
    (G !p3 must hold on every position).  Positives are therefore drawn from
    the same conditional law directly: since G !p3 forces p3 = 0 everywhere,
    P(length = L | accepted) is proportional to 0.75^L * P(rest | L); we draw
    L with weight 0.75^L, draw p0..p2 Bernoulli(0.25), and restart from the
    length draw whenever (p0 U p1) & F p2 fails.  Negatives are plain
    rejection sampling (almost every attempt is negative).
    """
    lo, hi, pb, n_props = 33, 128, 0.25, 4
    # negatives: ordinary counter-order attempts
    neg_b, neg_l, nneg, first = [], [], 0, 0
    while nneg < n_each:
        bits, lens = _attempts(seed, first, 8192, n_props, lo, hi, pb)
        lab = label_at_zero(F_SCALE, bits, lens, n_props)
        idx = np.nonzero(~lab)[0][: n_each - nneg]
        neg_b.append(bits[idx]); neg_l.append(lens[idx]); nneg += len(idx)
        first += 8192
    # positives: conditional sampler on a second stream
    Ls = np.arange(lo, hi + 1)
    w = 0.75 ** (Ls - lo)
    cdf = np.cumsum(w) / w.sum()
    rest = ("&", ("U", ("p", 0), ("p", 1)), ("F", ("p", 2)))
    pseed = int(splitmix64(np.uint64(seed), _AUX_COUNTER))
    pos_b, pos_l, npos, first = [], [], 0, 0
    while npos < n_each:
        cnt = 8192
        att = np.arange(first, first + cnt, dtype=np.uint64)
        tseed = splitmix64(np.uint64(pseed), att)
        lens = Ls[np.searchsorted(cdf, _uniform01(splitmix64(tseed, _LEN_COUNTER)), side="right")
                  .clip(0, len(Ls) - 1)]
        pos = np.arange(hi, dtype=np.uint64)
        bits = np.zeros((cnt, hi), dtype=np.uint32)
        for p in range(3):
            u = splitmix64(tseed[:, None], (pos * np.uint64(32) + np.uint64(p))[None, :])
            bits |= (_bernoulli(u, pb).astype(np.uint32) << np.uint32(p))
        bits[np.arange(hi)[None, :] >= lens[:, None]] = 0
        ok = label_at_zero(rest, bits, lens, n_props)
        idx = np.nonzero(ok)[0][: n_each - npos]
        pos_b.append(bits[idx]); pos_l.append(lens[idx]); npos += len(idx)
        first += cnt
    P = TraceSet.from_dense(np.concatenate(pos_b), np.concatenate(pos_l))
    N = TraceSet.from_dense(np.concatenate(neg_b), np.concatenate(neg_l))
    return Spec(P, N, n_props, ast_str(F_SCALE), ast_size(F_SCALE), "trace_scaling")


def planted_large(seed: int = 0, n_each: int = 1024) -> Spec:
    """The plain-single shape at divide-and-conquer scale: 2 props, n_each +
    n_each traces of length U{4..10}, Bernoulli(0.5), labelled by F(p0 & X p1)
    (size 5, U-free and in negation normal form, so every part of a split
    has a separator within the parts' size limit)."""
    P, N, _ = rejection_fill(seed, F_PLAIN, n_each, n_each, 2, 4, 10, 0.5)
    return Spec(P, N, 2, ast_str(F_PLAIN), ast_size(F_PLAIN), "planted_large_%d" % n_each)


# ---- uniform random syntax trees (for the batched workload) --------------

_UNARY = ["!", "X", "F", "G"]
_BINARY = ["&", "|", "U"]


def _tree_counts(n_props: int, max_size: int) -> List[int]:
    """c[s] = number of syntax trees of size s over n_props atoms and the 7 ops."""
    c = [0] * (max_size + 1)
    for s in range(1, max_size + 1):
        v = n_props if s == 1 else 4 * c[s - 1]
        for i in range(1, s - 1):
            v += 3 * c[i] * c[s - 1 - i]
        c[s] = v
    return c


def _unrank(rank: int, size: int, n_props: int, c: List[int]):
    if size == 1:
        return ("p", rank)
    block = c[size - 1]
    for op in _UNARY:
        if rank < block:
            return (op, _unrank(rank, size - 1, n_props, c))
        rank -= block
    for op in _BINARY:
        for i in range(1, size - 1):
            j = size - 1 - i
            blk = c[i] * c[j]
            if rank < blk:
                return (op, _unrank(rank // c[j], i, n_props, c),
                        _unrank(rank % c[j], j, n_props, c))
            rank -= blk
    raise AssertionError("rank out of range")


def random_tree(seed: int, counter: int, size: int, n_props: int):
    """A syntax tree drawn uniformly among all trees of the given size."""
    c = _tree_counts(n_props, size)
    total = c[size]
    # 128 random bits -> rank (bias below 2^-60 for totals under 2^64)
    hi = int(splitmix64(np.uint64(seed), np.uint64(2 * counter)))
    lo = int(splitmix64(np.uint64(seed), np.uint64(2 * counter + 1)))
    return _unrank(((hi << 64) | lo) % total, size, n_props, c)


def batched_problem(i: int, base_seed: int = 0, max_len_each: int = 4096, min_class_rate: float = 0.01) -> Spec:
    """Problem i of the batched workload (seed base_seed + i): props U{2..5},
    |P| = |N| = round(2^(4 + 8u)) (log-uniform 16..4096), length U{8..64},
    Bernoulli(0.3) bits, a planted formula drawn uniformly among all syntax
    trees of size U{3..9}.  A formula is redrawn when, on a probe of 4096
    attempts, either class is accepted at a rate below `min_class_rate` (the
    rejection fill would otherwise need millions of attempts)."""
    seed = base_seed + i
    s = np.uint64(seed)
    u = [splitmix64(s, _AUX_COUNTER + np.uint64(k)) for k in range(4)]
    n_props = int(_uniform_int(u[0], 2, 5))
    n_each = int(round(2 ** (4 + 8 * float(_uniform01(u[1])))))
    n_each = max(16, min(n_each, max_len_each))
    size = int(_uniform_int(u[2], 3, 9))
    for tries in range(1000):
        f = random_tree(int(u[3]) + tries, 0, size, n_props)
        bits, lens = _attempts(seed * 1000003 + tries, 0, 4096, n_props, 8, 64, 0.3)
        frac = float(label_at_zero(f, bits, lens, n_props).mean())
        if min_class_rate <= frac <= 1.0 - min_class_rate:
            P, N, _ = rejection_fill(seed * 1000003 + 7919 * (tries + 1), f, n_each, n_each, n_props,
                                     8, 64, 0.3, batch=8192, max_attempts=1 << 24)
            return Spec(P, N, n_props, ast_str(f), size, "batched_%d" % i)
    raise RuntimeError("could not plant a formula for problem %d" % i)


def batched_workload(n: int = 256, base_seed: int = 0, processes: int = 0) -> List[Spec]:
    """The n problems of the batched workload, generated in a spawn-started
    process pool when processes > 1."""
    if processes and processes > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(processes) as pool:
            return pool.starmap(batched_problem, [(i, base_seed) for i in range(n)])
    return [batched_problem(i, base_seed) for i in range(n)]


def random_small(seed: int, n_traces: int, n_props: int, lo: int, hi: int,
                 p_bit: float = 0.5) -> Spec:
    """Unlabelled random traces split half/half into P and N (BenchBase style)."""
    bits, lens = _attempts(seed, 0, n_traces, n_props, lo, hi, p_bit)
    h = n_traces // 2
    return Spec(TraceSet.from_dense(bits[:h], lens[:h]),
                TraceSet.from_dense(bits[h:], lens[h:]), n_props, None, None,
                "random_small_%d" % seed)


def hamming(l: int, delta: int, n_props: int = 2, seed: int = 0) -> Spec:
    """Hamming(B, l, delta) of Section 7: P = {tr} with tr uniform among the
    traces of length l (each position a letter of n_props propositions, one
    fair bit each), N = every trace of length l whose bits differ from tr's in
    exactly delta places (|N| = C(l * n_props, delta); with 2 propositions and
    l = 48, delta = 2 that is 4560)."""
    if l < 1 or delta < 1 or delta > l * n_props:
        raise ValueError("need 1 <= delta <= l * n_props")
    u = splitmix64(np.uint64(seed), _AUX_COUNTER + np.uint64(1 << 20) + np.arange(l * n_props, dtype=np.uint64))
    bits = (u >> np.uint64(63)).astype(np.uint32)          # one fair bit per (position, proposition)
    tr = [int(sum(int(bits[i * n_props + q]) << q for q in range(n_props))) for i in range(l)]
    neg = []
    for flips in itertools.combinations(range(l * n_props), delta):
        t = list(tr)
        for b in flips:
            t[b // n_props] ^= 1 << (b % n_props)
        neg.append(t)
    return Spec(TraceSet.from_list([tr]), TraceSet.from_list(neg), n_props, None, None,
                "hamming_%d_%d" % (l, delta))
