"""ltl_eval_noalloc: formula evaluation for callers that cannot allocate device
memory (a framework that owns the whole device through its own pool, a
real-time loop that must not allocate after start-up, code that cannot afford
the synchronisation of cudaMalloc / cudaFree).  The call takes device-resident
traces, writes a device-resident result and keeps its scratch in one static
device array of LTL_NOALLOC_SCRATCH_BYTES.

Its result must equal that of ltl_eval (the allocating entry point) bit for
bit, on two calls in a row -- the second one smaller than the first, so stale
scratch contents from the first call would show up if a part that must start
at zero were not cleared.  This file is collected last on purpose.
"""
import ctypes
import random

import numpy as np
import pytest

from paper_2402_12373_gb300 import _lib as L
from paper_2402_12373_gb300 import synth


def _rand_traces(seed, n, n_props, lo, hi):
    rng = random.Random(seed)
    return synth.TraceSet.from_list(
        [[rng.randrange(1 << n_props) for _ in range(rng.randrange(lo, hi + 1))] for _ in range(n)])


@pytest.mark.gpu
def test_noalloc_matches_ltl_eval_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    cases = [
        # larger first: three words per trace, U / G / X nesting
        ("((p0 U (p1 & X p2)) | G !p3)", _rand_traces(1, 3000, 4, 100, 190), 4),
        # then smaller: the plain-single traces
        ("F (p0 & X p1)", synth.plain_single().P, 2),
    ]
    for formula, ts, n_props in cases:
        n = ts.n
        max_len = int(ts.lengths().max())
        W = (max_len + 63) // 64
        want = L.evaluate(formula, ts, n_props, words_per_trace=W)          # allocating entry point
        d_letters = torch.from_numpy(ts.letters.astype(np.int32)).cuda()
        d_offsets = torch.from_numpy(ts.offsets.astype(np.int64)).cuda()
        d_out = torch.full((n, W), -1, dtype=torch.int64, device="cuda")   # poisoned output
        L.evaluate_noalloc(formula, d_letters, d_offsets, n, max_len, n_props, d_out, W)
        torch.cuda.synchronize()
        got = d_out.cpu().numpy().view(np.uint64)
        assert got.shape == want.shape
        assert np.array_equal(got, want), formula


def test_noalloc_rejects_work_beyond_the_static_scratch():
    """A size beyond LTL_NOALLOC_SCRATCH_BYTES is refused before any device work."""
    lib = L.load()
    n = 1 << 20                                    # 1M traces x 16 words x (1 + 2 + 2) CMs > 64 MiB
    fake = ctypes.c_void_p(256)                     # never dereferenced: rejected on the host
    rc = lib.ltl_eval_noalloc(b"(p0 U p1)", fake, fake, n, 1024, 2, fake, 16, None)
    assert rc == L.LTL_ERR_OOM
    msg = L.last_error()
    assert "static scratch" in msg and "bytes" in msg


@pytest.mark.gpu
def test_noalloc_trace_longer_than_max_len_within_its_words():
    """max_len below the longest trace, but every trace within the
    ceil(max_len / 64) words the call sizes from it: the evaluation must still
    be exact (F, G and U reach across the whole trace), equal to ltl_eval's."""
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    ts = _rand_traces(7, 500, 3, 20, 60)          # up to 60 positions: one word
    for formula in ("F p0", "G (p1 | p2)", "(p0 U (p1 & p2))", "X X F (p2 & X G p0)"):
        want = L.evaluate(formula, ts, 3, words_per_trace=1)
        d_letters = torch.from_numpy(ts.letters.astype(np.int32)).cuda()
        d_offsets = torch.from_numpy(ts.offsets.astype(np.int64)).cuda()
        d_out = torch.full((ts.n, 1), -1, dtype=torch.int64, device="cuda")
        L.evaluate_noalloc(formula, d_letters, d_offsets, ts.n, 10, 3, d_out, 1)   # max_len 10 < 60
        torch.cuda.synchronize()
        got = d_out.cpu().numpy().view(np.uint64)
        assert np.array_equal(got, want), formula


@pytest.mark.gpu
def test_noalloc_rejects_decreasing_offsets_then_evaluates_exactly():
    """Offsets that decrease: the pack kernel packs that trace as empty (no
    letter of it is read) and flags the input, the call returns
    LTL_ERR_INVALID; the next call with valid offsets is exact."""
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    ts = _rand_traces(11, 300, 2, 1, 40)
    bad = ts.offsets.astype(np.int64).copy()
    bad[5] = bad[6] + 1                        # offsets[5] > offsets[6], still inside the letters
    assert bad.max() <= len(ts.letters)
    d_letters = torch.from_numpy(ts.letters.astype(np.int32)).cuda()
    d_out = torch.full((ts.n, 1), -1, dtype=torch.int64, device="cuda")
    with pytest.raises(L.LtlError) as e:
        L.evaluate_noalloc("F (p0 & X p1)", d_letters, torch.from_numpy(bad).cuda(), ts.n, 40, 2, d_out, 1)
    assert e.value.status == L.LTL_ERR_INVALID
    assert "offsets decrease" in str(e.value)
    want = L.evaluate("F (p0 & X p1)", ts, 2, words_per_trace=1)
    L.evaluate_noalloc("F (p0 & X p1)", d_letters, torch.from_numpy(ts.offsets.astype(np.int64)).cuda(), ts.n, 40,
                       2, d_out, 1)
    torch.cuda.synchronize()
    assert np.array_equal(d_out.cpu().numpy().view(np.uint64), want)
