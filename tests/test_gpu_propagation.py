"""The two evaluations of F, G and U in the size-level kernels
(ltl_opts.propagation): the carry chain (the default, which every other GPU
test runs) and the paper's exponential propagation by log steps (Section 4).
Here the parity checks run again with the log steps forced, over narrow,
one-word, two-word and wider layouts, both kernels for matrices that fit a CTA
and the streaming and cluster kernels for larger ones; and both evaluations
store identical cache entries."""
import random

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import test_gpu_parity as P
import test_gpu_variants as V
from oracle import oracle as O
from paper_2402_12373_gb300 import _lib as L
from paper_2402_12373_gb300 import synth


@pytest.fixture(scope="module")
def ws():
    assert torch.cuda.is_available()
    return L.default_workspace(2 << 30)


@pytest.fixture
def logstep(monkeypatch):
    monkeypatch.setattr(L, "DEFAULT_PROPAGATION", L.PROP_LOGSTEP)


@pytest.fixture(params=[L.KERNEL_FUSED, L.KERNEL_WS], ids=["fused", "ws"])
def kernel(request, monkeypatch):
    monkeypatch.setattr(L, "DEFAULT_LEVEL_KERNEL", request.param)
    return request.param


@pytest.mark.parametrize("case", range(12))
def test_random_specs_logstep(ws, logstep, kernel, case):
    Pt, Nt, n_props, ops = list(P._random_specs(12, 4321))[case]
    K = 5 if n_props >= 3 else 6
    P._compare(P._ts(Pt), P._ts(Nt), n_props, ws, ops=ops, K=K, mode=L.STOP_LEVEL)


def test_plain_large_and_edges_logstep(ws, logstep, kernel):
    P.test_learn_plain_single_all_modes(ws)
    P.test_learn_single_large_levels_1_to_6(ws)
    P.test_learn_edge_cases(ws)


@pytest.mark.parametrize("L_len", [31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 257, 511, 512])
def test_word_boundaries_logstep(ws, logstep, kernel, L_len):
    P.test_learn_word_boundaries(ws, L_len)


def test_streaming_and_cluster_logstep(ws, logstep, kernel):
    """Matrices larger than a CTA: the streaming kernel (fused choice) and
    the cluster kernel (forced by the warp-specialised choice)."""
    P.test_learn_chunk_groups_streaming_path(ws)


def test_cache_entries_logstep(ws, logstep):
    P.test_cache_entries_are_their_formulas_and_distinct(ws)


@pytest.mark.parametrize("vi", range(len(V.VARIANTS)))
def test_variants_logstep(ws, logstep, vi):
    V.test_variant_matches_oracle(ws, vi, L.STOP_NONE)


def _entries(ws, spec, n_props, K, prop, kernel):
    """Every cache entry (formula, matrix words) of an enumeration to size K."""
    T = spec.n_traces
    with L.Context(workspace=ws, stop=L.STOP_NONE, propagation=prop, level_kernel=kernel) as ctx:
        got = ctx.learn(spec.P, spec.N, n_props, max_size=K)
        W = got["words_per_trace"]
        out = []
        for k in range(1, got["levels_done"] + 1):
            b, c = ctx.level_range(k)
            for idx in range(b, b + c):
                f, cs = ctx.entry(idx, T, W)
                out.append((k, cs.tobytes()))
    return got, out


@pytest.mark.parametrize("L_len", [24, 60, 100, 200])
def test_both_evaluations_store_the_same_matrices(ws, kernel, L_len):
    """Carry chain and log steps: the same counts and the same set of stored
    matrices per level (entry order within a level depends on timing)."""
    rng = random.Random(L_len)
    Pt = [[rng.randrange(8) for _ in range(rng.randrange(L_len // 2, L_len + 1))] for _ in range(12)]
    Nt = [[rng.randrange(8) for _ in range(rng.randrange(L_len // 2, L_len + 1))] for _ in range(12)]
    spec = synth.Spec(P=synth.TraceSet.from_list(Pt), N=synth.TraceSet.from_list(Nt), n_props=3)
    a, ea = _entries(ws, spec, 3, 4, L.PROP_CARRY, kernel)
    b, eb = _entries(ws, spec, 3, 4, L.PROP_LOGSTEP, kernel)
    assert a["unique"] == b["unique"] and a["candidates"] == b["candidates"]
    for k in range(1, a["levels_done"] + 1):
        assert sorted(x for lv, x in ea if lv == k) == sorted(x for lv, x in eb if lv == k), k
    want = O.learn(spec.P, spec.N, 3, max_size=4, stop_mode=0)
    assert a["unique"][1:5] == want["unique"][1:5]
