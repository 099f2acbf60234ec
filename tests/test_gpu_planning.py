"""Device planning of small size levels (ltl_opts.level_planning).

With LTL_PLAN_AUTO a single problem's small levels are planned by a device
kernel and run back to back, with one read-back for the whole chain; with
LTL_PLAN_HOST every level is planned on the host after reading back the level
before.  Integer work, so both must give exactly the same status, minimal
size, completed levels and unique and candidate counts per level, and both
must match the oracle; any returned formula separates (or misclassifies at
most max_errors traces) under the oracle's semantics.  That the chain path
ran is seen in the read-back bytes: one level log per level instead of one
control block per level.
"""
import random

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


def _problems():
    out = []
    for s in range(3):
        p = synth.plain_single(seed=s)
        out.append(("plain%d" % s, p.P, p.N, 2, 7))
    rng = random.Random(11)
    for i, (n_props, nt, maxlen) in enumerate([(1, 10, 8), (3, 40, 30), (2, 90, 70), (4, 60, 20)]):
        tr = [[rng.randrange(1 << n_props) for _ in range(rng.randrange(0, maxlen + 1))] for _ in range(nt)]
        h = nt // 2
        out.append(("rand%d" % i, synth.TraceSet.from_list(tr[:h]), synth.TraceSet.from_list(tr[h:]), n_props, 6))
    s = synth.single_large(n_each=64)
    out.append(("large64", s.P, s.N, 3, 7))
    return out


PROBLEMS = _problems()
PID = [p[0] for p in PROBLEMS]
STOPS = {L.STOP_FIRST: 1, L.STOP_LEVEL: 2, L.STOP_NONE: 0}

VARIANTS = [
    dict(),
    dict(costs=[1, 2, 1, 1, 1, 1, 1, 3]),
    dict(nnf=True),
    dict(max_errors=2),
]


def _errors(formula, P, N, n_props):
    vp = O.evaluate_traces(formula, P, n_props)
    vn = O.evaluate_traces(formula, N, n_props)
    return sum(1 for v in vp if not (len(v) and v[0])) + sum(1 for v in vn if len(v) and v[0])


def _learn(ws, planning, stop, P, N, n_props, K, variant):
    ops = L.ALL | (L.NNF if variant.get("nnf") else 0)
    with L.Context(workspace=ws, stop=stop, planning=planning, costs=variant.get("costs"),
                   max_errors=variant.get("max_errors", 0)) as ctx:
        return ctx.learn(P, N, n_props, ops=ops, max_size=K)


def _same(a, b):
    assert a["status"] == b["status"], (a["status"], b["status"])
    assert a["size"] == b["size"]
    assert a["levels_done"] == b["levels_done"]
    d = a["levels_done"]
    assert a["unique"][1:d + 1] == b["unique"][1:d + 1]
    assert a["candidates"][1:d + 1] == b["candidates"][1:d + 1]


@pytest.mark.parametrize("pi", range(len(PROBLEMS)), ids=PID)
@pytest.mark.parametrize("stop", list(STOPS), ids=["first", "level", "none"])
def test_chain_equals_host_planning_and_oracle(ws, pi, stop):
    name, P, N, n_props, K = PROBLEMS[pi]
    auto = _learn(ws, L.PLAN_AUTO, stop, P, N, n_props, K, {})
    host = _learn(ws, L.PLAN_HOST, stop, P, N, n_props, K, {})
    _same(auto, host)
    o = O.learn(P, N, n_props, max_size=K, stop_mode=STOPS[stop])
    _same(auto, {"status": o["status"], "size": o["size"], "levels_done": o["levels_done"],
                 "unique": o["unique"], "candidates": o["candidates"]})
    for r in (auto, host):
        if r["status"] == "found":
            assert R.size(R.parse(r["formula"])) == r["size"], r["formula"]
            assert _errors(r["formula"], P, N, n_props) == 0, r["formula"]
    # the chain ran: level logs instead of per-level control blocks were read back
    assert auto["d2h_bytes"] != host["d2h_bytes"]


@pytest.mark.parametrize("vi", range(1, len(VARIANTS)))
def test_chain_variants(ws, vi):
    """Cost homomorphisms (levels without candidates inside a chain), negation
    normal form and noisy learning plan the same levels on the device."""
    variant = VARIANTS[vi]
    for name, P, N, n_props, K in PROBLEMS[:5]:
        K += 2 if variant.get("costs") else 0
        for stop in (L.STOP_LEVEL, L.STOP_NONE):
            auto = _learn(ws, L.PLAN_AUTO, stop, P, N, n_props, K, variant)
            host = _learn(ws, L.PLAN_HOST, stop, P, N, n_props, K, variant)
            _same(auto, host)
            o = O.learn(P, N, n_props, max_size=K, stop_mode=STOPS[stop], costs=variant.get("costs", [1] * 8),
                        nnf=variant.get("nnf", False), max_errors=variant.get("max_errors", 0))
            _same(auto, {"status": o["status"], "size": o["size"], "levels_done": o["levels_done"],
                         "unique": o["unique"], "candidates": o["candidates"]})
            if auto["status"] == "found":
                assert _errors(auto["formula"], P, N, n_props) <= variant.get("max_errors", 0)


def test_chain_hits_cache_cap(ws):
    """A cache that fills inside a chain stops it where host planning stops."""
    s = synth.single_large(n_each=64)
    res = []
    for planning in (L.PLAN_AUTO, L.PLAN_HOST):
        with L.Context(workspace=ws, stop=L.STOP_NONE, planning=planning, mem_budget=1 << 20) as ctx:
            res.append(ctx.learn(s.P, s.N, 3, max_size=9))
    _same(res[0], res[1])
    assert res[0]["status"] in ("cap", "found")
    assert res[0]["levels_done"] < 7, res[0]["levels_done"]


def test_context_reuse_mixes_modes(ws):
    """One context alternating problems keeps chain state per call."""
    with L.Context(workspace=ws, stop=L.STOP_LEVEL) as ctx:
        first = [ctx.learn(P, N, n_props, max_size=K) for _, P, N, n_props, K in PROBLEMS]
        again = [ctx.learn(P, N, n_props, max_size=K) for _, P, N, n_props, K in PROBLEMS]
    for a, b in zip(first, again):
        _same(a, b)


@pytest.mark.parametrize("stop", [L.STOP_NONE, L.STOP_FIRST], ids=["none", "first"])
def test_graph_replay_matches(ws, stop):
    """A chain shape enqueued often enough runs as a captured CUDA graph; every
    replay gives the result of host planning (the first calls are enqueued
    directly, later ones replay the graph)."""
    for name, P, N, n_props, K in (PROBLEMS[0], PROBLEMS[-1]):
        host = _learn(ws, L.PLAN_HOST, stop, P, N, n_props, K, {})
        assert host["device_planned_levels"] == 0 and host["graph_levels"] == 0
        with L.Context(workspace=ws, stop=stop, planning=L.PLAN_AUTO) as ctx:
            for i in range(12):
                r = ctx.learn(P, N, n_props, max_size=K)
                _same(r, host)
                if r["status"] == "found":
                    assert _errors(r["formula"], P, N, n_props) == 0, r["formula"]
                assert r["device_planned_levels"] >= 1
                # direct enqueues first; from the eighth call of the shape on, a graph
                assert (r["graph_levels"] == r["device_planned_levels"]) == (i >= 7), (i, r["graph_levels"])


def test_invalid_planning_rejected(ws):
    with pytest.raises(L.LtlError):
        L.Context(workspace=ws, planning=2)
