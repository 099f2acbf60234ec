"""Writes the oracle's per-level counts for the full-size workloads.

The characteristic-matrix enumeration of the paper (Section 3, `enum` and
`handleOp`, exact uniqueness check) is run by the plain CPU oracle alone, on
the seeded synthetic inputs, with every level enumerated completely (stop mode
0).  The JSON files it writes hold, per size level, the number of candidates
built and the number of characteristic matrices first reached at that size;
the GPU parity tests compare the library's counts with them level by level.

Nothing here touches the CUDA path: it imports the oracle and the input
generators only.  Usage (from the repository root):

    python tests/golden/make_fullsize_levels.py single_large 9
    python tests/golden/make_fullsize_levels.py trace_scaling 6

Memory: the oracle keeps one byte per trace position for every cached
matrix, about 49 KB per matrix for the 2048-trace workload and 3.8 MB for the
65,536-trace one.
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import oracle as O  # noqa: E402
from paper_2402_12373_gb300 import synth  # noqa: E402

WORKLOADS = {
    "single_large": (lambda: synth.single_large(), 3),
    "trace_scaling": (lambda: synth.trace_scaling(), 4),
}


def input_digest(spec) -> str:
    """SHA-256 over the letters and offsets of P then N (the exact inputs)."""
    h = hashlib.sha256()
    for ts in (spec.P, spec.N):
        h.update(np.ascontiguousarray(ts.letters, dtype=np.uint32).tobytes())
        h.update(np.ascontiguousarray(ts.offsets, dtype=np.uint64).tobytes())
    return h.hexdigest()


def main():
    name, K = sys.argv[1], int(sys.argv[2])
    make, n_props = WORKLOADS[name]
    spec = make()
    t0 = time.time()
    res = O.learn(spec.P, spec.N, n_props, ops=O.OPS_ALL, max_size=K, stop_mode=0)
    wall = time.time() - t0
    out = {
        "workload": name,
        "generator": "synth.%s() (default seed and sizes)" % name,
        "input_sha256": input_digest(spec),
        "n_traces": spec.n_traces,
        "n_props": n_props,
        "ops": O.OPS_ALL,
        "max_size": K,
        "stop_mode": 0,
        "status": res["status"],
        "size": res["size"],
        "levels_done": res["levels_done"],
        "unique": res["unique"],
        "candidates": res["candidates"],
        "oracle_seconds": [round(s, 3) for s in res["seconds"]],
        "oracle_wall_seconds": round(wall, 1),
        "written_by": "tests/golden/make_fullsize_levels.py (oracle only)",
    }
    path = os.path.join(HERE, "%s_levels.json" % name)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps({k: out[k] for k in ("workload", "status", "size", "levels_done",
                                          "unique", "candidates", "oracle_wall_seconds")}))


if __name__ == "__main__":
    main()
