"""Parity of the learning variants (cost homomorphism, negation normal form,
noisy learning; Sections 2 and 3) between the CUDA path and the oracle.

Integer work, so the comparison is exact: status, minimal cost, completed
cost levels, unique and candidate counts per level.  The returned formula
has the reported cost and misclassifies at most max_errors traces under the
oracle's semantics (several minimal formulae can exist; any one is correct).
"""
import random

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import ltl_ref as R
from oracle import oracle as O
from paper_2402_12373_gb300 import _lib as L
from paper_2402_12373_gb300 import synth

VARIANTS = [
    dict(costs=[1, 2, 1, 1, 1, 1, 1, 1], nnf=False, max_errors=0),
    dict(costs=[2, 1, 3, 1, 2, 1, 2, 3], nnf=False, max_errors=0),
    dict(costs=[1, 1, 1, 1, 1, 1, 1, 1], nnf=True, max_errors=0),
    dict(costs=[1, 1, 2, 2, 1, 1, 1, 9], nnf=True, max_errors=0),
    dict(costs=[1, 1, 1, 1, 1, 1, 1, 1], nnf=False, max_errors=1),
    dict(costs=[1, 1, 1, 1, 1, 1, 1, 1], nnf=False, max_errors=3),
    dict(costs=[1, 3, 2, 2, 1, 2, 2, 2], nnf=True, max_errors=2),
]
EXTRA = [0, 4, 0, 1, 0, 0, 2]   # extra cost levels so that heavier costs still reach separators
VID = ["c%s_nnf%d_e%d" % ("".join(map(str, v["costs"])), v["nnf"], v["max_errors"]) for v in VARIANTS]


@pytest.fixture(scope="module")
def ws():
    assert torch.cuda.is_available()
    return L.default_workspace(2 << 30)


def _problems():
    """Narrow (length <= 32) and wide layouts, a few props, uneven classes."""
    out = []
    for s in range(3):
        p = synth.plain_single(seed=s)
        out.append(("plain%d" % s, p.P, p.N, 2, 6))
    rng = random.Random(5)
    for i, (n_props, nt, maxlen) in enumerate([(1, 12, 9), (3, 40, 30), (2, 90, 70), (3, 300, 130)]):
        tr = [[rng.randrange(1 << n_props) for _ in range(rng.randrange(1, maxlen + 1))] for _ in range(nt)]
        h = nt // 3 + 1
        out.append(("rand%d" % i, synth.TraceSet.from_list(tr[:h]), synth.TraceSet.from_list(tr[h:]), n_props, 5))
    return out


PROBLEMS = _problems()


def _errors(formula, P, N, n_props):
    vp = O.evaluate_traces(formula, P, n_props)
    vn = O.evaluate_traces(formula, N, n_props)
    return sum(1 for v in vp if not (len(v) and v[0])) + sum(1 for v in vn if len(v) and v[0])


def _check(g, o, variant, P, N, n_props):
    assert g["status"] == o["status"], (g, o)
    assert g["size"] == o["size"]
    d = g["levels_done"]
    assert d == o["levels_done"]
    assert g["unique"][1:d + 1] == o["unique"][1:d + 1]
    assert g["candidates"][1:d + 1] == o["candidates"][1:d + 1]
    if g["status"] == "found":
        assert R.cost(R.parse(g["formula"]), variant["costs"]) == g["size"], g["formula"]
        assert _errors(g["formula"], P, N, n_props) <= variant["max_errors"], g["formula"]
        if variant["nnf"]:
            f = g["formula"].replace(" ", "")
            assert all(f[i + 1] == "p" for i, c in enumerate(f) if c == "!"), f


def _ops(variant):
    return L.ALL | (L.NNF if variant["nnf"] else 0)


@pytest.mark.parametrize("vi", range(len(VARIANTS)), ids=VID)
@pytest.mark.parametrize("stop", [L.STOP_LEVEL, L.STOP_NONE])
def test_variant_matches_oracle(ws, vi, stop):
    variant = VARIANTS[vi]
    with L.Context(workspace=ws, stop=stop, costs=variant["costs"], max_errors=variant["max_errors"]) as ctx:
        for name, P, N, n_props, K in PROBLEMS:
            K += EXTRA[vi]
            g = ctx.learn(P, N, n_props, ops=_ops(variant), max_size=K)
            o = O.learn(P, N, n_props, max_size=K, stop_mode=2 if stop == L.STOP_LEVEL else 0, **variant)
            _check(g, o, variant, P, N, n_props)


@pytest.mark.parametrize("variant", VARIANTS[1:6:2], ids=VID[1:6:2])
def test_variant_streaming_shapes(ws, variant):
    """The same counts with the CM spread over chunk groups (streaming kernel)
    and with the smallest fused tiles."""
    name, P, N, n_props, K = PROBLEMS[-1]
    o = O.learn(P, N, n_props, max_size=K, stop_mode=2, **variant)
    for mc in (1, 2, 8):
        with L.Context(workspace=ws, stop=L.STOP_LEVEL, max_chunks=mc, costs=variant["costs"],
                       max_errors=variant["max_errors"]) as ctx:
            g = ctx.learn(P, N, n_props, ops=_ops(variant), max_size=K)
        _check(g, o, variant, P, N, n_props)


def test_variant_batch(ws):
    """Batched learning carries the context's costs and error budget."""
    v = VARIANTS[6]
    probs = [(P, N, n_props, _ops(v), K) for _, P, N, n_props, K in PROBLEMS]
    res = L.learn_batch(probs, stop=L.STOP_LEVEL, workspace=ws, costs=v["costs"], max_errors=v["max_errors"])
    for (name, P, N, n_props, K), g in zip(PROBLEMS, res):
        o = O.learn(P, N, n_props, max_size=K, stop_mode=2, **v)
        _check(g, o, v, P, N, n_props)


@pytest.mark.parametrize("max_errors", [26, 60, 100])
def test_noisy_large(ws, max_errors):
    """Noisy learning on 512 traces with error budgets of 5% (no separator up
    to size 6), 12% (size 6) and 20% (size 5)."""
    s = synth.single_large(n_each=256)
    v = dict(costs=[1] * 8, nnf=False, max_errors=max_errors)
    with L.Context(workspace=ws, stop=L.STOP_LEVEL, max_errors=max_errors) as ctx:
        g = ctx.learn(s.P, s.N, 3, max_size=6)
    o = O.learn(s.P, s.N, 3, max_size=6, stop_mode=2, **v)
    _check(g, o, v, s.P, s.N, 3)


def test_invalid_costs_rejected(ws):
    with pytest.raises(ValueError):
        L.Context(workspace=ws, costs=[1, 1, 1])
    with pytest.raises(ValueError):
        L.Context(workspace=ws, costs=[0, 1, 1, 1, 1, 1, 1, 1])
