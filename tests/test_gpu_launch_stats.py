"""The per-launch statistics the benchmark's roofline is computed from:
which level kernel ran each (size level, connective) launch, and how many
operand matrices it copied into shared memory.  A unary launch stages exactly
one matrix per candidate; a binary one stages every right operand once per
candidate plus the left operand once per reload (at least once per distinct
left operand, at most once per candidate).  Host- and device-planned levels
report the same kernel choices and, for the fused and warp-specialised
kernels, counts within those bounds."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2402_12373_gb300 import _lib as L
from paper_2402_12373_gb300 import synth

OP_UNARY = (1, 4, 5, 6)      # Not, X, F, G
OP_BINARY = (2, 3, 7)        # And, Or, U


def _left_operands(unique, k, op):
    """Distinct left operands of connective op at size k (sum over splits)."""
    n = 0
    for i in range(1, k - 1):
        j = k - 1 - i
        if op == 7:
            n += unique[i] if unique[j] else 0
        elif i < j:
            n += unique[i] if unique[j] else 0
        elif i == j:
            n += max(unique[i] - 1, 0)
    return n


@pytest.mark.parametrize("planning", [L.PLAN_AUTO, L.PLAN_HOST])
def test_staged_counts_and_kernels_single_large(planning):
    s = synth.single_large()
    ws = L.default_workspace(8 << 30)
    with L.Context(workspace=ws, stop=L.STOP_NONE, planning=planning) as ctx:
        r = ctx.learn(s.P, s.N, 3, max_size=8)
    assert r["levels_done"] == 8
    u, kern, staged = r["unique"], r["op_kernel"], r["op_staged"]
    # rounds of at least 2^15 candidates run the warp-specialised kernel
    for k in (7, 8):
        assert r["candidates"][k] >= 1 << 15
        for op in range(1, 8):
            assert kern[k][op] == "ws_level_kernel", (k, op, kern[k])
    for k in (7, 8):
        for op in OP_UNARY:
            assert staged[k][op] == u[k - 1], (k, op)
        for op in OP_BINARY:
            cand = _cands(u, k, op)
            assert cand + _left_operands(u, k, op) <= staged[k][op] <= 2 * cand, (k, op, staged[k][op], cand)


def _cands(u, k, op):
    tot = 0
    for i in range(1, k - 1):
        j = k - 1 - i
        if op == 7:
            tot += u[i] * u[j]
        elif i < j:
            tot += u[i] * u[j]
        elif i == j:
            tot += u[i] * (u[i] - 1) // 2
    return tot


def test_forced_fused_kernel_reports_it():
    s = synth.single_large(n_each=256)
    ws = L.default_workspace(4 << 30)
    with L.Context(workspace=ws, stop=L.STOP_NONE, level_kernel=L.KERNEL_FUSED, planning=L.PLAN_HOST) as ctx:
        r = ctx.learn(s.P, s.N, 3, max_size=7)
    for k in range(2, 8):
        for op in range(1, 8):
            if r["op_ms"][k][op] > 0:
                assert r["op_kernel"][k][op] == "fused_level_kernel", (k, op)


def test_which_launches_ran_alone():
    """op_alone marks the launches whose op_ms is their own duration: in a
    level of one problem with at least 2^18 candidates U runs alone first and
    the other connectives after it concurrently; smaller levels run their
    launches concurrently (or, planned on the device, in a chain)."""
    s = synth.single_large()
    ws = L.default_workspace(16 << 30)
    with L.Context(workspace=ws, stop=L.STOP_NONE, mem_budget=10 << 30) as ctx:
        r = ctx.learn(s.P, s.N, 3, max_size=9)
    assert r["levels_done"] == 9 and r["candidates"][9] >= 1 << 18 and r["candidates"][8] < 1 << 18
    alone = r["op_alone"]
    assert alone[9][7] and not any(alone[9][op] for op in range(1, 7))
    assert not any(alone[k][op] for k in range(1, 9) for op in range(8))
    assert r["op_ms"][9][7] > 0 and r["op_ms"][9][7] <= r["ms"][9]
