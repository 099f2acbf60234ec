"""The integer-throughput probe (ltl_int32_peak) that the candidate launches'
integer roofline is measured against: its rate is positive, does not depend
on the number of steps (it is a rate, not a latency), and stays below the
issue limit of one warp instruction per scheduler and cycle."""
import subprocess

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2402_12373_gb300 import _lib as L


def _max_sm_mhz():
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits", "-i", "0"],
                             capture_output=True, text=True, timeout=30).stdout.strip().splitlines()
        return float(out[0])
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        return 2100.0


def test_int32_peak_is_a_plausible_rate():
    assert torch.cuda.is_available()
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    issue_limit = n_sm * 4 * 32 * _max_sm_mhz() * 1e6   # 4 schedulers x 32 lanes per SM and cycle
    a = L.int32_peak(iters=1 << 14, repeats=3)
    b = L.int32_peak(iters=1 << 16, repeats=3)
    for r in (a, b):
        assert 0.05 * issue_limit < r["ops_per_s"] < 1.02 * issue_limit, (r, issue_limit)
    assert b["ms"] > 2.0 * a["ms"]
    assert abs(a["ops_per_s"] - b["ops_per_s"]) < 0.25 * b["ops_per_s"], (a, b)
