"""Batched and served learning (many problems resident in one workspace,
advanced in rounds, launches shared between problems) give every problem the
result it gets alone: the same status, minimal size, completed levels and
per-level unique and candidate counts; the returned formula separates under
the oracle's semantics.  Counts are integers, so the comparison is exact.

The problems of the batched workload itself (a fixed slice of
synth.batched_problem) and of the served workload (trace-scaling problems of
the served pool's seeds) are also compared with the oracle directly: status,
minimal size, completed levels and every completed level's counts."""
import concurrent.futures
import multiprocessing
import random
import time

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O
from paper_2402_12373_gb300 import _lib as L
from paper_2402_12373_gb300 import synth


@pytest.fixture(scope="module")
def ws():
    assert torch.cuda.is_available()
    return L.default_workspace(4 << 30)


def _mixed_problems(n, seed):
    """Uneven problems: 1..4 props, 2..600 traces, lengths 0..70 (narrow and
    wide layouts, several launch shapes), random connective masks."""
    rng = random.Random(seed)
    out = []
    for i in range(n):
        n_props = rng.choice([1, 2, 3, 4])
        nt = rng.choice([2, 7, 20, 64, 150, 600])
        maxlen = rng.choice([5, 12, 30, 45, 70])
        tr = [[rng.randrange(1 << n_props) for _ in range(rng.randrange(0, maxlen + 1))] for _ in range(nt)]
        h = rng.randrange(1, nt)
        ops = L.ALL if rng.random() < 0.7 else rng.randrange(1, 128)
        K = rng.choice([3, 4, 5])
        out.append((synth.TraceSet.from_list(tr[:h]), synth.TraceSet.from_list(tr[h:]), n_props, ops, K))
    return out


def _alone(ws, problems, stop):
    res = []
    with L.Context(workspace=ws, stop=stop) as ctx:
        for P, N, n_props, ops, K in problems:
            res.append(ctx.learn(P, N, n_props, ops=ops, max_size=K))
    return res


def _same(a, b, K):
    assert a["status"] == b["status"], (a, b)
    assert a["size"] == b["size"]
    assert a["levels_done"] == b["levels_done"]
    d = a["levels_done"]
    assert a["unique"][1:d + 1] == b["unique"][1:d + 1]
    assert a["candidates"][1:d + 1] == b["candidates"][1:d + 1]


@pytest.mark.parametrize("stop", [L.STOP_LEVEL, L.STOP_FIRST, L.STOP_NONE])
def test_batch_equals_alone(ws, stop):
    problems = _mixed_problems(40, 17)
    alone = _alone(ws, problems, stop)
    batch = L.learn_batch(problems, stop=stop, workspace=ws)
    for (P, N, n_props, ops, K), a, b in zip(problems, alone, batch):
        _same(a, b, K)
        if b["status"] == "found":
            assert O.separates(b["formula"], P, N, n_props), b["formula"]


def test_batch_matches_oracle_on_plain_and_large(ws):
    probs = [(synth.plain_single(seed=s).P, synth.plain_single(seed=s).N, 2, L.ALL, 7) for s in range(4)]
    s = synth.single_large(n_each=256)
    probs.append((s.P, s.N, 3, L.ALL, 6))
    batch = L.learn_batch(probs, stop=L.STOP_LEVEL, workspace=ws)
    for (P, N, n_props, ops, K), b in zip(probs, batch):
        want = O.learn(P, N, n_props, ops=ops, max_size=K, stop_mode=2)
        assert b["status"] == want["status"] and b["size"] == want["size"]
        d = b["levels_done"]
        assert d == want["levels_done"]
        assert b["unique"][1:d + 1] == want["unique"][1:d + 1]


def test_batch_admission_under_memory_pressure():
    """A workspace too small for all problems at once: problems wait for
    memory and still get their own results."""
    problems = _mixed_problems(24, 23)
    small = L.default_workspace(96 << 20)
    alone = _alone(small, problems, L.STOP_LEVEL)
    batch = L.learn_batch([p + (2 << 20,) for p in problems], stop=L.STOP_LEVEL, workspace=small)
    for (P, N, n_props, ops, K), a, b in zip(problems, alone, batch):
        if a["status"] == "cap" or b["status"] == "cap":
            continue   # a 2 MiB budget can cap a problem that a bigger one completes
        _same(a, b, K)


def test_server_alone_vs_mix(ws):
    """Requests that arrive while others run are admitted between rounds
    (continuous batching); each result equals the problem's result alone."""
    problems = _mixed_problems(30, 29)
    alone = _alone(ws, problems, L.STOP_LEVEL)
    with L.Server(workspace=ws, stop=L.STOP_LEVEL, max_resident=8) as srv:
        ids = {}
        results = {}
        for i, (P, N, n_props, ops, K) in enumerate(problems):
            ids[srv.submit(P, N, n_props, ops=ops, max_size=K)] = i
            if i % 5 == 4:      # stagger arrivals
                time.sleep(0.002)
                for r in srv.poll(64, 0):
                    results[ids[r["id"]]] = r
        t0 = time.time()
        while len(results) < len(problems) and time.time() - t0 < 120:
            for r in srv.poll(64, 100):
                results[ids[r["id"]]] = r
        assert srv.pending() == (0, 0)
    assert len(results) == len(problems)
    for i, (P, N, n_props, ops, K) in enumerate(problems):
        _same(alone[i], results[i], K)
        assert results[i]["latency_ms"] >= results[i]["queue_ms"] >= 0.0


# A fixed slice of the batched workload's own problems (synth.batched_problem,
# base seed 0) that the oracle solves in seconds: 34..6960 traces, 2..5
# propositions, minimal sizes 1..7, max size = planted size + 2.
BATCH_SLICE = [0, 1, 2, 3, 4, 5, 8, 10, 11, 15, 16, 22, 23, 30, 36, 37, 38, 40, 44, 45, 49, 50, 51, 56,
               59, 63]
# Seeds of the served workload's trace-scaling problems (65536 traces each):
# the benchmark's whole served pool.  Seven of them separate at size 3; the
# eighth (seed 1004) has no separator up to size 3 and fills its 2 GiB cache
# before the oracle's minimal size, which the oracle (O(n^2) U over 65,536
# traces) takes minutes to reach.  So the oracle enumerates the served
# problems up to SERVED_ORACLE_SIZE, and a problem it does not solve there is
# checked level by level up to that size.
SERVED_SEEDS = list(range(1000, 1008))
SERVED_ORACLE_SIZE = 3


def _spec(kind, i):
    return synth.batched_problem(i) if kind == "batched" else synth.trace_scaling(i)


def _max_size(kind, sp):
    return sp.planted_size + 2 if kind == "batched" else 11


def _oracle_job(kind, i):
    """Oracle result (stop at the first separator) of one problem; runs in a
    spawn-started worker process."""
    from oracle import oracle as Oc
    sp = _spec(kind, i)
    K = _max_size(kind, sp) if kind == "batched" else SERVED_ORACLE_SIZE
    return Oc.learn(sp.P, sp.N, sp.n_props, max_size=K, stop_mode=1)


@pytest.fixture(scope="module")
def oracle_results():
    jobs = [("batched", i) for i in BATCH_SLICE] + [("served", s) for s in SERVED_SEEDS]
    with concurrent.futures.ProcessPoolExecutor(max_workers=8,
                                                mp_context=multiprocessing.get_context("spawn")) as ex:
        futs = {j: ex.submit(_oracle_job, *j) for j in jobs}
        return {j: f.result() for j, f in futs.items()}


def _equals_oracle(got, want, sp):
    assert got["status"] == want["status"], (got["status"], want["status"])
    assert got["size"] == want["size"]
    d = want["levels_done"]
    assert got["levels_done"] == d
    assert got["unique"][1:d + 1] == want["unique"][1:d + 1]
    assert got["candidates"][1:d + 1] == want["candidates"][1:d + 1]
    if got["status"] == "found":
        assert O.separates(got["formula"], sp.P, sp.N, sp.n_props), got["formula"]
        assert O.size(got["formula"]) == got["size"]


def _equals_oracle_up_to(got, want, sp, K):
    """`want` is the oracle's result with sizes up to K.  Found there: the
    same result.  Not found: levels 1..K are complete on both sides with the
    same counts, and the GPU's separator, if any, is larger than K."""
    if want["status"] == "found":
        _equals_oracle(got, want, sp)
        return
    assert want["status"] == "not_found" and want["levels_done"] == K
    assert got["levels_done"] >= K
    assert got["unique"][1:K + 1] == want["unique"][1:K + 1]
    assert got["candidates"][1:K + 1] == want["candidates"][1:K + 1]
    assert got["status"] in ("found", "cap", "not_found"), got["status"]
    if got["status"] == "found":
        assert got["size"] > K
        assert O.separates(got["formula"], sp.P, sp.N, sp.n_props), got["formula"]


def _budgets(ws, specs):
    """Per-problem memory budgets proportional to the trace counts (as in the
    benchmark), at least 64 MiB so that no problem of the slice fills its cache
    before the oracle's minimal size."""
    T = [sp.n_traces for sp in specs]
    return [max(64 << 20, int(0.5 * ws.numel() * t / sum(T))) for t in T]


def test_batched_workload_slice_equals_oracle(ws, oracle_results):
    """The batched workload's problems through one ltl_learn_batch call, with
    budgets proportional to their trace counts as in the benchmark."""
    specs = [_spec("batched", i) for i in BATCH_SLICE]
    budgets = _budgets(ws, specs)
    items = [(sp.P, sp.N, sp.n_props, L.ALL, _max_size("batched", sp), b) for sp, b in zip(specs, budgets)]
    batch = L.learn_batch(items, stop=L.STOP_FIRST, workspace=ws)
    for i, sp, got in zip(BATCH_SLICE, specs, batch):
        _equals_oracle(got, oracle_results[("batched", i)], sp)


def _serve(ws, specs, kind, budgets, stagger):
    with L.Server(workspace=ws, stop=L.STOP_FIRST, max_resident=64) as srv:
        ids, results = {}, {}
        for n, sp in enumerate(specs):
            ids[srv.submit(sp.P, sp.N, sp.n_props, max_size=_max_size(kind, sp), budget=budgets[n])] = n
            if n % stagger == stagger - 1:   # requests arrive while others run
                time.sleep(0.002)
                for r in srv.poll(64, 0):
                    results[ids[r["id"]]] = r
        t0 = time.time()
        while len(results) < len(specs) and time.time() - t0 < 300:
            for r in srv.poll(64, 100):
                results[ids[r["id"]]] = r
        assert srv.pending() == (0, 0)
    assert len(results) == len(specs)
    return [results[n] for n in range(len(specs))]


def test_served_batched_slice_equals_oracle(ws, oracle_results):
    specs = [_spec("batched", i) for i in BATCH_SLICE]
    got = _serve(ws, specs, "batched", _budgets(ws, specs), 4)
    for i, sp, r in zip(BATCH_SLICE, specs, got):
        _equals_oracle(r, oracle_results[("batched", i)], sp)


def test_served_trace_scaling_requests_equal_oracle(oracle_results):
    """The served workload's requests (65536 two-word traces each, 2 GiB per
    problem as in the benchmark) through the continuous-batching server."""
    big = L.default_workspace(12 << 30)
    specs = [_spec("served", s) for s in SERVED_SEEDS]
    got = _serve(big, specs, "served", [2 << 30] * len(specs), 2)
    for s, sp, r in zip(SERVED_SEEDS, specs, got):
        _equals_oracle_up_to(r, oracle_results[("served", s)], sp, SERVED_ORACLE_SIZE)
    del big
