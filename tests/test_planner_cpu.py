"""CPU pins of the level planner (host logic; no GPU).

The host planner and the device planner cut a size level into segments and
tiles with the same code (paper_2402_12373_gb300/csrc/ltl_plan.h).  Built
here with the host compiler through tests/planner_harness.cpp, it must give,
from the oracle's per-level unique counts, exactly the oracle's candidate
count of every level -- the candidate space of Section 3's handleOp, under
uniform and non-uniform connective costs, negation normal form and connective
subsets (readings r6, r15, r16) -- and its tiles must cover each segment's
candidates exactly once.
"""
import ctypes
import os
import random
import shutil
import subprocess

import pytest

from oracle import oracle as O
from paper_2402_12373_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ALL, NNF = 127, 256


@pytest.fixture(scope="module")
def planner(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    out = str(tmp_path_factory.mktemp("planner") / "libplanner.so")
    subprocess.run([cxx, "-std=c++17", "-O1", "-shared", "-fPIC", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2402_12373_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "planner_harness.cpp"), "-o", out], check=True)
    lib = ctypes.CDLL(out)
    lib.level_candidates.restype = ctypes.c_uint64
    lib.level_candidates.argtypes = [ctypes.c_uint32, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64), ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_int)]
    lib.tiles_cover.restype = ctypes.c_int
    lib.tiles_cover.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                ctypes.POINTER(ctypes.c_uint64)]
    return lib


def _planned(lib, ops, n_props, unique, k, costs):
    counts = (ctypes.c_uint64 * 64)(*([0] + [int(u) for u in unique[1:k]] + [0] * (63 - max(0, k - 1))))
    c = (ctypes.c_int * 8)(*costs)
    return int(lib.level_candidates(ops, n_props, counts, k, c))


CASES = [
    ("all", ALL, [1] * 8),
    ("nnf", ALL | NNF, [1] * 8),
    ("costs", ALL, [1, 2, 1, 1, 1, 1, 1, 3]),
    ("costs_nnf", ALL | NNF, [2, 1, 3, 1, 2, 1, 2, 3]),
    ("no_until", ALL & ~64, [1] * 8),
    ("and_or_x", 2 | 4 | 8, [1] * 8),
    ("banned", ALL, [1, 1, 1, 1, 1, 1, 1, 9]),
]


@pytest.mark.parametrize("name,ops,costs", CASES, ids=[c[0] for c in CASES])
def test_planned_candidates_equal_the_oracle(planner, name, ops, costs):
    specs = [synth.plain_single(seed=s) for s in range(2)]
    rng = random.Random(4)
    for n_props in (1, 3):
        tr = [[rng.randrange(1 << n_props) for _ in range(rng.randrange(1, 9))] for _ in range(12)]
        specs.append(synth.Spec(synth.TraceSet.from_list(tr[:6]), synth.TraceSet.from_list(tr[6:]), n_props,
                                "", 0, "rand"))
    for sp in specs:
        K = 6 if costs == [1] * 8 else 8
        o = O.learn(sp.P, sp.N, sp.n_props, ops=ops & ~NNF, max_size=K, stop_mode=0, costs=costs,
                    nnf=bool(ops & NNF))
        for k in range(1, o["levels_done"] + 1):
            got = _planned(planner, ops, sp.n_props, o["unique"], k, costs)
            assert got == o["candidates"][k], (name, k, got, o["candidates"][k])


@pytest.mark.parametrize("kind", [0, 1, 2], ids=["unary", "rect", "tri"])
def test_tiles_cover_every_candidate_once(planner, kind):
    rng = random.Random(kind)
    n = ctypes.c_uint64()
    for _ in range(300):
        a = rng.randrange(1 if kind != 2 else 2, 200)
        b = rng.randrange(1, 200) if kind == 1 else 0
        cpt = 1 << rng.randrange(0, 7)
        assert planner.tiles_cover(kind, a, b, cpt, ctypes.byref(n)) == 1, (kind, a, b, cpt)
        assert n.value >= 1
