"""CPU-only checks of the C-ABI boundary: the library builds and loads, it
exports every entry point include/ltl.h declares, host-side argument checks
reject bad input before any device work, and the oracle and the CUDA path
share no code."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ltl.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:ltl_status|void|const char \*)\s*\*?\s*(ltl_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("ltl_learn", "ltl_eval", "ltl_ctx_create", "ltl_ctx_destroy", "ltl_ctx_learn",
              "ltl_ctx_learn_device", "ltl_ctx_level_range", "ltl_ctx_entry", "ltl_last_error", "ltl_version"):
        assert n in names, n


def test_library_builds_loads_and_exports_every_declared_symbol():
    from paper_2402_12373_gb300 import _lib, build
    path = build.build()
    lib = _lib.load()
    for n in _declared():
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    for n in _declared():
        assert re.search(r"\bT %s$" % n, out, flags=re.M), n
    assert _lib.version().startswith("ltl-gb300")
    assert sorted(_lib.EXPORTS) == _declared()


def test_sm_103a_only():
    from paper_2402_12373_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_host_side_validation_without_gpu():
    """Argument errors are reported before any CUDA call."""
    from paper_2402_12373_gb300 import _lib
    from paper_2402_12373_gb300.synth import TraceSet
    ts = TraceSet.from_list([[1, 2], [3]])
    with pytest.raises(_lib.LtlError) as e:
        _lib.evaluate("(p0 &", ts, 2)
    assert e.value.status == _lib.LTL_ERR_INVALID
    with pytest.raises(_lib.LtlError) as e:
        _lib.evaluate("p5", ts, 2)
    assert e.value.status == _lib.LTL_ERR_INVALID
    with pytest.raises(_lib.LtlError) as e:
        _lib.evaluate("p0", ts, 0)
    assert e.value.status == _lib.LTL_ERR_INVALID
    bad = TraceSet(np.array([1, 2, 3], np.uint32), np.array([0, 2, 1], np.uint64))
    with pytest.raises(_lib.LtlError) as e:
        _lib.evaluate("p0", bad, 2)
    assert e.value.status == _lib.LTL_ERR_INVALID
    assert "decrease" in _lib.last_error()
    # divide and conquer: window, split mode and connectives are checked first
    for kw in (dict(window=1), dict(mode=7), dict(ops=_lib.ALL & ~_lib.OR)):
        with pytest.raises(_lib.LtlError) as e:
            _lib.learn_dc(ts, ts, 2, **kw)
        assert e.value.status == _lib.LTL_ERR_INVALID
    # option values are checked before any CUDA call
    import ctypes
    lib = _lib.load()
    hp = _lib._HostTraces(ts)
    for field, bad in (("level_planning", 2), ("level_kernel", 3), ("ruc", 3), ("ruc_mask_bits", 63),
                       ("propagation", 2)):
        o = _lib._opts()
        setattr(o, field, bad)
        buf = ctypes.create_string_buffer(64)
        st = _lib.Stats()
        rc = lib.ltl_learn(ctypes.byref(hp.struct), ctypes.byref(hp.struct), 2, _lib.ALL, 3, ctypes.byref(o), buf,
                           len(buf), ctypes.byref(st))
        assert rc == _lib.LTL_ERR_INVALID, field
        assert field.split("_")[0] in _lib.last_error(), (field, _lib.last_error())
    # the integer-throughput probe checks its arguments before touching a device
    for kw in (dict(iters=3), dict(repeats=0)):
        with pytest.raises(_lib.LtlError) as e:
            _lib.int32_peak(**kw)
        assert e.value.status == _lib.LTL_ERR_INVALID


def _files(d, exts):
    for dp, _, fs in os.walk(os.path.join(ROOT, d)):
        for f in fs:
            if f.endswith(exts):
                yield os.path.join(dp, f)


def test_oracle_and_cuda_path_share_no_code():
    for f in _files("paper_2402_12373_gb300", (".py", ".cu", ".cuh", ".h", ".cpp")):
        text = open(f).read()
        assert not re.search(r"^\s*(from|import)\s+oracle\b", text, flags=re.M), f
        assert "ltl_oracle" not in text, f
    for f in _files("oracle", (".py", ".c", ".h")):
        text = open(f).read()
        assert "paper_2402_12373_gb300" not in text, f
        assert "ltl_device" not in text and "ltl_types" not in text, f
