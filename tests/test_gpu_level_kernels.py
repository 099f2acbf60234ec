"""Both size-level kernels -- the fused one and the warp-specialised one
(compute warps hand each batch to hash warps through a shared-memory ring) --
give the oracle's results: the parity checks of the other GPU test files run
again with each kernel forced, over narrow, wide and multi-word layouts and
every launch shape."""
import random

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import test_gpu_parity as P
import test_gpu_ruc as RU
import test_gpu_variants as V
from oracle import oracle as O
from paper_2402_12373_gb300 import _lib as L
from paper_2402_12373_gb300 import synth


@pytest.fixture(scope="module")
def ws():
    assert torch.cuda.is_available()
    return L.default_workspace(2 << 30)


@pytest.fixture(params=[L.KERNEL_FUSED, L.KERNEL_WS], ids=["fused", "ws"])
def kernel(request, monkeypatch):
    monkeypatch.setattr(L, "DEFAULT_LEVEL_KERNEL", request.param)
    return request.param


def test_kernel_choice_is_reported(ws, kernel):
    s = synth.single_large(n_each=256)
    with L.Context(workspace=ws, stop=L.STOP_LEVEL) as ctx:
        r = ctx.learn(s.P, s.N, 3, max_size=4)
    nt = r["threads_per_cta"]
    if kernel == L.KERNEL_WS:
        assert nt % 32 == 0 and nt >= 96   # compute warps plus two hash warps
    want = O.learn(s.P, s.N, 3, max_size=4, stop_mode=2)
    assert r["unique"][1:5] == want["unique"][1:5]


@pytest.mark.parametrize("case", range(20))
def test_random_specs(ws, kernel, case):
    Pt, Nt, n_props, ops = list(P._random_specs(20, 1234))[case]
    K = 5 if n_props >= 3 else 6
    P._compare(P._ts(Pt), P._ts(Nt), n_props, ws, ops=ops, K=K, mode=L.STOP_LEVEL)


def test_plain_and_large(ws, kernel):
    P.test_learn_plain_single_all_modes(ws)
    P.test_learn_single_large_levels_1_to_6(ws)
    P.test_learn_edge_cases(ws)


@pytest.mark.parametrize("L_len", [31, 32, 33, 63, 64, 65, 127, 128, 129])
def test_word_boundaries(ws, kernel, L_len):
    P.test_learn_word_boundaries(ws, L_len)


@pytest.mark.parametrize("max_chunks", [1, 2, 4, 8])
def test_launch_shapes(ws, kernel, max_chunks):
    P.test_launch_shapes_narrow_and_wide(ws, max_chunks)


def test_cache_entries(ws, kernel):
    P.test_cache_entries_are_their_formulas_and_distinct(ws)
    P.test_cap_reached_with_small_budget(ws)
    P.test_context_reuse_across_shapes(ws)


@pytest.mark.parametrize("vi", range(len(V.VARIANTS)))
def test_variants(ws, kernel, vi):
    V.test_variant_matches_oracle(ws, vi, L.STOP_NONE)


def test_relaxed_admission(ws, kernel):
    RU.test_hash_without_mask_equals_exact(ws, L.STOP_NONE)
    RU.test_fkp_exact_when_key_holds_the_matrix(ws)
    RU.test_lossy_admission_properties(ws, L.RUC_HASH, 52)


def test_batch(ws, kernel):
    import test_gpu_batch_serve as B
    B.test_batch_equals_alone(ws, L.STOP_LEVEL)


def test_batch_same_shape_matches_oracle(ws, kernel):
    """Problems of one launch shape share every launch, so a CTA's consecutive
    batches can belong to different problems; each problem's counts still equal
    the oracle's (a deferred store must go to its own problem's cache)."""
    probs = []
    for s in range(12):
        sp = synth.plain_single(seed=s)
        probs.append((sp.P, sp.N, 2, L.ALL, 7))
    res = L.learn_batch(probs, stop=L.STOP_NONE, workspace=ws)
    for (P, N, n_props, ops, K), g in zip(probs, res):
        want = O.learn(P, N, n_props, max_size=K, stop_mode=0)
        assert g["levels_done"] == K
        assert g["unique"][1:K + 1] == want["unique"][1:K + 1]
        assert g["candidates"][1:K + 1] == want["candidates"][1:K + 1]
