"""Builds the in-tree CUDA library libltl_gb300.so for sm_103a with nvcc.

The translation units (two size-level kernels, the small kernels, the host
driver) are compiled in parallel and
linked into one shared library next to this file.  A rebuild happens only
when a source or header is newer than the library.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libltl_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["ltl_level_fused_w1.cu", "ltl_level_fused_w2.cu", "ltl_level_fused_w48.cu",
           "ltl_level_fused_narrow.cu", "ltl_level_stream.cu", "ltl_level_cluster.cu",
           "ltl_level_ws_w1.cu", "ltl_level_ws_wn.cu",
           "ltl_misc.cu", "ltl_host.cu", "ltl_engine.cu", "ltl_noalloc.cu", "ltl_dc.cu",
           "ltl_peak.cu", "ltl_plan.cu"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libltl_gb300.so")


def _deps():
    return (glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(INCLUDE, "*.h"))
            + [os.path.abspath(__file__)])


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    if not force and not ptxas_info and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                    "-I" + INCLUDE, "-I" + CSRC]
    if ptxas_info:
        flags += ["-Xptxas", "-v"]
    procs = []
    objs = []
    for s in SOURCES:
        obj = os.path.join(BUILD, s.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [cc] + flags + ["-c", os.path.join(CSRC, s), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    outs = []
    for cmd, p in procs:
        out, _ = p.communicate()
        outs.append(out.decode(errors="replace"))
        if p.returncode != 0:
            raise RuntimeError("nvcc failed:\n%s\n%s" % (" ".join(cmd), out.decode(errors="replace")[-6000:]))
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    if ptxas_info:
        return "\n".join(outs)
    return LIB


if __name__ == "__main__":
    info = "-v" in sys.argv
    r = build(force=True, verbose=True, ptxas_info=info)
    print(r)
