"""The launch autotuner (ltl_opts.autotune_path): trying the six tile-size and
occupancy configurations on real launches changes no result -- every learn
call of the sequence gives the oracle's counts -- every configuration of a
tuned launch class gets tried, and the measurements persist through a file."""
import os

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O
from paper_2402_12373_gb300 import _lib as L
from paper_2402_12373_gb300 import synth


@pytest.fixture(scope="module")
def ws():
    assert torch.cuda.is_available()
    return L.default_workspace(4 << 30)


def _classes(dump):
    out = {}
    for line in dump.strip().splitlines():
        parts = line.split()
        out[parts[0]] = [tuple(map(float, p.split(":"))) for p in parts[1:]]
    return out


def test_tuning_changes_no_result(ws, tmp_path):
    """Size 9 is the first level with a launch that runs alone (its U launch:
    the level has at least 2^18 candidates), so that launch is tuned; every
    tuned call equals the untuned one, which equals the oracle up to size 6."""
    s = synth.single_large(n_each=512)
    K = 9
    want6 = O.learn(s.P, s.N, 3, max_size=6, stop_mode=0)
    with L.Context(workspace=ws, stop=L.STOP_NONE) as ctx:
        want = ctx.learn(s.P, s.N, 3, max_size=K)
    assert want["unique"][1:7] == want6["unique"][1:7]
    path = str(tmp_path / "tune.txt")
    with L.Context(workspace=ws, stop=L.STOP_NONE, autotune=path) as ctx:
        for _ in range(7):
            g = ctx.learn(s.P, s.N, 3, max_size=K)
            assert g["unique"][1:K + 1] == want["unique"][1:K + 1]
            assert g["candidates"][1:K + 1] == want["candidates"][1:K + 1]
        dump = ctx.autotune_dump()
    classes = _classes(dump)
    assert classes, "no launch was large enough to tune"
    for key, confs in classes.items():
        assert len(confs) == 6
        tried = [c for c in confs if c[1] > 0]
        assert len(tried) in (3, 6), (key, confs)    # 3 when one CTA per SM is the maximum
        assert all(t[0] > 0 for t in tried)
    # persisted on close, read back by the next context
    assert os.path.exists(path)
    with L.Context(workspace=ws, stop=L.STOP_NONE, autotune=path) as ctx:
        assert _classes(ctx.autotune_dump()) == classes
        g = ctx.learn(s.P, s.N, 3, max_size=K)
        assert g["unique"][1:K + 1] == want["unique"][1:K + 1]


def test_tuning_off_by_default(ws):
    s = synth.plain_single()
    with L.Context(workspace=ws, stop=L.STOP_NONE) as ctx:
        ctx.learn(s.P, s.N, 2, max_size=6)
        assert ctx.autotune_dump() == ""
