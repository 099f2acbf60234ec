"""The binding's conversion of the C structs it reads back (ltl_stats,
ltl_result) into Python dicts: every field, level and connective carried
over with its value and a plain Python type (no ctypes objects), on structs
filled with seeded random values.  CPU only: the structs are built here."""
import random

from paper_2402_12373_gb300 import _lib as L


def _filled_stats(rng):
    st = L.Stats()
    for name, _ in L.Stats._fields_:
        v = getattr(st, name)
        if isinstance(v, int):
            setattr(st, name, rng.randrange(1 << 31))
        elif isinstance(v, float):
            setattr(st, name, rng.random())
    for c in range(L.MAX_LEVELS):
        st.unique[c] = rng.randrange(1 << 60)
        st.candidates[c] = rng.randrange(1 << 60)
        st.ms[c] = rng.random()
        for o in range(8):
            st.op_ms[c][o] = rng.random()
            st.op_staged[c][o] = rng.randrange(1 << 40)
            st.op_kernel[c][o] = rng.randrange(len(L.LAUNCH_KINDS))
            st.op_alone[c][o] = rng.randrange(2)
    return st


def test_stats_dict_carries_every_field():
    rng = random.Random(5)
    for K in (1, 6, 9, L.MAX_LEVELS - 1):
        st = _filled_stats(rng)
        d = st.to_dict(K)
        for name, _ in L.Stats._fields_:
            v = getattr(st, name)
            if isinstance(v, (int, float)):
                assert d[name] == v and type(d[name]) is type(v), name
        assert d["unique"] == [st.unique[c] for c in range(K + 1)]
        assert d["candidates"] == [st.candidates[c] for c in range(K + 1)]
        assert d["ms"] == [st.ms[c] for c in range(K + 1)]
        for c in range(K + 1):
            assert d["op_ms"][c] == [st.op_ms[c][o] for o in range(8)]
            assert d["op_staged"][c] == [st.op_staged[c][o] for o in range(8)]
            assert d["op_kernel"][c] == [L.LAUNCH_KINDS[st.op_kernel[c][o]] for o in range(8)]
            assert d["op_alone"][c] == [bool(st.op_alone[c][o]) for o in range(8)]
            assert all(type(x) is bool for x in d["op_alone"][c])
            assert all(type(x) is float for x in d["op_ms"][c])
            assert all(type(x) is int for x in d["op_staged"][c])


def test_result_dict_carries_every_field():
    rng = random.Random(6)
    for status in (L.LTL_OK, L.LTL_NOT_FOUND, L.LTL_CAP_REACHED, L.LTL_ERR_INVALID):
        r = L.Result()
        r.id = rng.randrange(1 << 60)
        r.status = status
        r.found_size = rng.randrange(1, 12)
        r.formula = b"(G (F p1 | !p0) U p2)"
        r.levels_done = rng.randrange(12)
        for c in range(L.MAX_LEVELS):
            r.unique[c] = rng.randrange(1 << 60)
            r.candidates[c] = rng.randrange(1 << 60)
        r.n_traces = rng.randrange(1 << 30)
        r.rounds = rng.randrange(100)
        r.queue_ms = rng.random()
        r.latency_ms = rng.random()
        d = r.to_dict()
        assert d["id"] == r.id and d["status"] == L.STATUS[status]
        assert d["levels_done"] == r.levels_done and d["n_traces"] == r.n_traces and d["rounds"] == r.rounds
        assert d["queue_ms"] == r.queue_ms and d["latency_ms"] == r.latency_ms
        assert d["unique"] == [r.unique[c] for c in range(L.MAX_LEVELS)]
        assert d["candidates"] == [r.candidates[c] for c in range(L.MAX_LEVELS)]
        assert all(type(x) is int for x in d["unique"] + d["candidates"])
        if status == L.LTL_OK:
            assert d["size"] == r.found_size and d["formula"] == "(G (F p1 | !p0) U p2)"
        else:
            assert d["size"] is None and d["formula"] is None
