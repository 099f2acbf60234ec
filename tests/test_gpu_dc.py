"""Divide and conquer (Section 6) through the C ABI: the returned formula
separates the whole specification under the oracle's semantics, its reported
size is its syntax-tree size, and the split statistics are consistent.  A
specification that fits the window is one enumeration, so its formula has
the oracle's minimal size."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O
from paper_2402_12373_gb300 import _lib as L
from paper_2402_12373_gb300 import synth

NNF_NO_U = (L.ALL & ~L.U) | L.NNF     # the setting of the Hamming experiments


@pytest.fixture(scope="module")
def ws():
    assert torch.cuda.is_available()
    return L.default_workspace(4 << 30)


def _check(r, spec, ops, trivial=False):
    assert r["status"] == "found", r
    f = r["formula"]
    assert O.separates(f, spec.P, spec.N, spec.n_props), f
    assert O.size(f) == r["formula_size"]
    assert r["formula_len"] == len(f)
    assert r["enum_failed"] <= r["enum_calls"]
    assert (r["enum_calls"] == 0) if trivial else (r["enum_calls"] >= 1)
    assert r["min_window"] >= 2
    if ops & L.NNF:
        g = f.replace(" ", "")
        assert all(g[i + 1] == "p" for i, c in enumerate(g) if c == "!"), f
    if not ops & L.U:
        assert "U" not in f


@pytest.mark.parametrize("mode", [L.DC_DETERMINISTIC, L.DC_RANDOM])
@pytest.mark.parametrize("l,delta,window", [(6, 1, 8), (9, 2, 16), (15, 1, 16), (24, 2, 32), (48, 1, 64)])
def test_hamming(ws, mode, l, delta, window):
    spec = synth.hamming(l, delta, seed=l + delta)
    for ops in (L.ALL, NNF_NO_U):
        r = L.learn_dc(spec.P, spec.N, 2, ops=ops, max_size=6, mode=mode, window=window, seed=5, workspace=ws)
        _check(r, spec, ops)


@pytest.mark.parametrize("mode", [L.DC_DETERMINISTIC, L.DC_RANDOM])
def test_hamming_48_2(ws, mode):
    """The largest Hamming case of Section 7: 1 + 4560 traces of length 48."""
    spec = synth.hamming(48, 2, seed=1)
    r = L.learn_dc(spec.P, spec.N, 2, ops=NNF_NO_U, max_size=6, mode=mode, window=64, seed=3, workspace=ws)
    _check(r, spec, NNF_NO_U)
    # deterministic splitting needs several levels of halves; random splitting
    # may close the whole specification at once with the overfitting formula
    if mode == L.DC_DETERMINISTIC:
        assert r["max_depth"] >= 1
    assert r["formula_size"] <= (7 if mode == L.DC_RANDOM else 14) * 48


def test_fits_window_is_one_minimal_enumeration(ws):
    for seed in range(3):
        spec = synth.plain_single(seed=seed)
        want = O.learn(spec.P, spec.N, 2, max_size=7, stop_mode=1)
        for mode in (L.DC_DETERMINISTIC, L.DC_RANDOM):
            r = L.learn_dc(spec.P, spec.N, 2, max_size=7, mode=mode, window=64, workspace=ws)
            _check(r, spec, L.ALL)
            assert r["enum_calls"] == 1 and r["max_depth"] == 0
            assert r["formula_size"] == want["size"]


@pytest.mark.parametrize("mode", [L.DC_DETERMINISTIC, L.DC_RANDOM])
def test_large_random_specification(ws, mode):
    spec = synth.single_large(n_each=512)
    r = L.learn_dc(spec.P, spec.N, 3, max_size=5, mode=mode, window=128, seed=9, workspace=ws)
    _check(r, spec, L.ALL)


def _distinct_random(seed, n, n_props=2, lo=3, hi=7):
    sp = synth.random_small(seed=seed, n_traces=n, n_props=n_props, lo=lo, hi=hi)
    pos = {tuple(t) for t in sp.P.to_list()}
    return synth.Spec(sp.P, synth.TraceSet.from_list([t for t in sp.N.to_list() if tuple(t) not in pos]), n_props)


@pytest.mark.parametrize("mode", [L.DC_DETERMINISTIC, L.DC_RANDOM])
def test_window_halving_and_fallback(ws, mode):
    """With max_size 2 most parts of a random specification find nothing:
    windows are halved, and small parts are closed by fallback formulas."""
    spec = _distinct_random(3, 60)
    r = L.learn_dc(spec.P, spec.N, 2, max_size=2, mode=mode, window=32, seed=1, workspace=ws)
    _check(r, spec, L.ALL)
    assert r["enum_failed"] > 0 and r["min_window"] < 32
    assert r["fallbacks"] > 0


@pytest.mark.parametrize("mode", [L.DC_DETERMINISTIC, L.DC_RANDOM])
@pytest.mark.parametrize("l", [12, 24, 48])
def test_single_positive_overfits(ws, mode, l):
    """Hamming specifications have one positive trace: a part the enumerator
    cannot solve takes that trace's overfitting formula, about 6 nodes per
    position with 2 propositions, instead of one formula per negative."""
    spec = synth.hamming(l, 2, seed=7)
    r = L.learn_dc(spec.P, spec.N, 2, ops=NNF_NO_U, max_size=6, mode=mode, window=16, seed=2, workspace=ws)
    _check(r, spec, NNF_NO_U)
    assert r["fallbacks"] >= 1
    assert r["formula_size"] <= (7 * l if mode == L.DC_RANDOM else 14 * l)


@pytest.mark.parametrize("ruc,mask", [(L.RUC_FKP, 0), (L.RUC_HASH, 40)])
def test_relaxed_admission_parts(ws, ruc, mask):
    spec = synth.hamming(30, 2, seed=2)
    r = L.learn_dc(spec.P, spec.N, 2, ops=NNF_NO_U, max_size=6, mode=L.DC_RANDOM, window=32, ruc=ruc,
                   ruc_mask_bits=mask, workspace=ws)
    _check(r, spec, NNF_NO_U)


def test_costs_apply_to_parts(ws):
    spec = synth.hamming(9, 1, seed=6)
    r = L.learn_dc(spec.P, spec.N, 2, max_size=8, mode=L.DC_RANDOM, window=16, costs=[1, 1, 1, 1, 2, 1, 1, 1],
                   workspace=ws)
    _check(r, spec, L.ALL)


def test_unsolvable_and_trivial(ws):
    both = synth.TraceSet.from_list([[1, 2, 3], [0, 1]])
    r = L.learn_dc(both, synth.TraceSet.from_list([[0, 1]]), 2, max_size=4, window=2, workspace=ws)
    assert r["status"] == "not_found" and r["formula"] is None
    prefix = L.learn_dc(synth.TraceSet.from_list([[1]]), synth.TraceSet.from_list([[1, 1]]), 1, ops=L.ALL | L.NNF,
                        max_size=3, window=2, workspace=ws)
    assert prefix["status"] == "not_found"
    # without NNF the end of the shorter trace tells them apart
    spec = synth.Spec(synth.TraceSet.from_list([[1]]), synth.TraceSet.from_list([[1, 1]]), 1)
    r = L.learn_dc(spec.P, spec.N, 1, max_size=3, window=2, workspace=ws)
    _check(r, spec, L.ALL)
    # no negatives: a formula true everywhere, without any enumeration
    spec = synth.Spec(synth.TraceSet.from_list([[1], [0, 1]]), synth.TraceSet.from_list([]), 1)
    r = L.learn_dc(spec.P, spec.N, 1, max_size=3, window=2, workspace=ws)
    _check(r, spec, L.ALL, trivial=True)


@pytest.mark.parametrize("mode", [L.DC_DETERMINISTIC, L.DC_RANDOM])
@pytest.mark.parametrize("window", [16, 64])
def test_planted_large_parts_are_enumerated(ws, mode, window):
    """2048 traces labelled by F(p0 & X p1) (size 5): every part of a split
    has a U-free NNF separator of size <= 6, so the enumerator closes parts
    (no part needs the overfitting fallback)."""
    spec = synth.planted_large()
    r = L.learn_dc(spec.P, spec.N, 2, ops=NNF_NO_U, max_size=6, mode=mode, window=window, seed=2, workspace=ws)
    _check(r, spec, NNF_NO_U)
    assert r["enum_failed"] < r["enum_calls"]
    assert r["fallbacks"] == 0


@pytest.mark.parametrize("mode", [L.DC_DETERMINISTIC, L.DC_RANDOM])
def test_single_large_parts_are_enumerated_and_combined(ws, mode):
    """The single-large specification (2048 traces, minimal separator of size
    8) with parts limited to size 6: no one enumeration separates it, so the
    result combines several parts learned by enumeration."""
    spec = synth.single_large(seed=1)
    r = L.learn_dc(spec.P, spec.N, 3, ops=NNF_NO_U, max_size=6, mode=mode, window=64, seed=4, workspace=ws)
    _check(r, spec, NNF_NO_U)
    assert r["enum_calls"] >= 2
    assert r["enum_failed"] < r["enum_calls"]
