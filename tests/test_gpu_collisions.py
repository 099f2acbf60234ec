"""The collision path of exact admission.

With 64-bit fingerprint keys two different characteristic matrices practically
never meet on one key, so the branch where the full compare finds a different
matrix and probing goes on would otherwise never run.  Masking the high bits
of the key in exact mode (`ruc_mask_bits` with LTL_RUC_EXACT) makes such
meetings common; the full compare still decides, so every count must stay
exactly the oracle's, on every kernel that admits candidates (fused,
warp-specialised, streaming and cluster), with host and device planning.
"""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O
from paper_2402_12373_gb300 import _lib as L
from paper_2402_12373_gb300 import synth


@pytest.fixture(scope="module")
def ws():
    assert torch.cuda.is_available()
    return L.default_workspace(2 << 30)


def _problems():
    out = []
    p = synth.plain_single(seed=0)
    out.append(("plain", p.P, p.N, 2, 6))
    s = synth.single_large(n_each=256)
    out.append(("large256", s.P, s.N, 3, 6))
    s = synth.single_large(n_each=3000)   # more traces than one CTA holds: chunk groups
    out.append(("groups", s.P, s.N, 3, 4))
    return out


PROBLEMS = _problems()
_WANT = {}


def _want(name):
    if name not in _WANT:
        _, P, N, n_props, K = next(p for p in PROBLEMS if p[0] == name)
        _WANT[name] = O.learn(P, N, n_props, max_size=K, stop_mode=0)
    return _WANT[name]


def _check(got, want):
    assert got["status"] == want["status"], (got["status"], want["status"])
    d = got["levels_done"]
    assert d == want["levels_done"]
    assert got["unique"][1:d + 1] == want["unique"][1:d + 1]
    assert got["candidates"][1:d + 1] == want["candidates"][1:d + 1]


@pytest.mark.parametrize("kernel", [L.KERNEL_FUSED, L.KERNEL_WS], ids=["fused", "ws"])
@pytest.mark.parametrize("planning", [L.PLAN_AUTO, L.PLAN_HOST], ids=["auto", "host"])
@pytest.mark.parametrize("pi", range(len(PROBLEMS)), ids=[p[0] for p in PROBLEMS])
def test_masked_keys_stay_exact(ws, kernel, planning, pi):
    name, P, N, n_props, K = PROBLEMS[pi]
    with L.Context(workspace=ws, stop=L.STOP_NONE, level_kernel=kernel, planning=planning,
                   ruc=L.RUC_EXACT, ruc_mask_bits=54) as ctx:
        got = ctx.learn(P, N, n_props, max_size=K)
    _check(got, _want(name))
    # 9 key bits for hundreds to thousands of matrices: different matrices met
    # on one key, and the full compare told them apart
    assert got["collisions"] > 0, got["collisions"]
    assert got["compares"] >= got["collisions"]


def test_unmasked_keys_meet_no_collision(ws):
    name, P, N, n_props, K = PROBLEMS[1]
    with L.Context(workspace=ws, stop=L.STOP_NONE) as ctx:
        got = ctx.learn(P, N, n_props, max_size=K)
    _check(got, _want(name))
    assert got["collisions"] == 0
    assert got["compares"] > 0   # duplicates are confirmed by the full compare


def test_masked_keys_batch_and_first_separator(ws):
    """Batched learning and stopping at the first separator on masked keys."""
    probs = [(P, N, n_props, L.ALL, K) for _, P, N, n_props, K in PROBLEMS[:2]]
    res = L.learn_batch(probs, stop=L.STOP_NONE, workspace=ws, ruc=L.RUC_EXACT, ruc_mask_bits=54)
    for (name, *_), g in zip(PROBLEMS[:2], res):
        _check(g, _want(name))
    name, P, N, n_props, K = PROBLEMS[0]
    with L.Context(workspace=ws, stop=L.STOP_FIRST, ruc_mask_bits=56) as ctx:
        got = ctx.learn(P, N, n_props, max_size=K)
    want = O.learn(P, N, n_props, max_size=K, stop_mode=1)
    assert got["status"] == want["status"] and got["size"] == want["size"]
    assert O.separates(got["formula"], P, N, n_props), got["formula"]
