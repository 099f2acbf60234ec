#!/usr/bin/env python3
"""Benchmark of the GB300 enumerative LTL learner.

Workload (the single-large learning problem): 3 propositions, 1024 positive +
1024 negative seeded synthetic traces of length U{16..32}, Bernoulli(0.3)
proposition bits, labelled by the planted formula (G(!p0 | F p1) | p2); all
seven connectives; sizes 1..9, every level enumerated completely
(enumeration-only mode), the language cache and hash set resident in HBM
within a 32 GB memory budget.

One step = one whole learn call (trace packing, then every size level's
candidate kernel, reading back the control block after each level).  Before
the W warm-up steps the library's launch autotuner gets six untimed calls,
one per launch configuration it tries; the warm-up and timed steps run the
fastest configuration of every tuned launch class.

Metric: candidates x traces per second = sum over completed size levels of
(candidates built at that size) * |P u N|, divided by the step's device time.

  value    traces already resident in HBM (ltl_ctx_learn_device), CUDA events
           on the library's stream around each step; L2 flushed between steps.
           The timed region is the whole call: levels 1..6 run as one
           device-planned chain (a CUDA graph), and between the host-planned
           levels 7, 8 and 9 the library reads the control block back, so the
           host's round trips are inside it.  `kernel_ms_per_step` is the sum
           of the level launches' own device times, beside it.
  e2e      the same metric through ltl_ctx_learn with HOST trace buffers: the
           host->device copy of the traces and the device->host reads of the
           control block and formula are inside the wall-clock timed region.
  roofline the dominant kernel (the longest (size level, connective) launch):
           algorithmic bytes with the left operand staged in shared memory --
           the operand matrices the launch copied into shared memory (left
           operands once per reload, counted on the device) plus one matrix
           per candidate stored (new) or read for the full compare
           (duplicate) -- over its event-timed duration, against the
           measured HBM copy bandwidth; beside it the same launch's
           algorithmic 32-bit operations against the measured integer roof
           (alu), the count with both operands streamed, and the physical
           DRAM bytes of an ncu capture of the same kernel sources.  `bound`
           names the roof the launch uses the larger fraction of.
  cpu_baseline  the oracle on the host's cores: every core (the OpenMP
           variant, identical results) and one core (the plain C oracle), on
           a bounded sample.
  other_propagation  the same steps with the other evaluation of F, G and U
           (by default the kernels use the carry chain; this runs the paper's
           log-step exponential propagation), timed the same way, with its
           counts checked equal.

`--impl reference` times the oracle alone on every host core (the CPU
reference of this workload) with the same metric.  With torchrun (N > 1)
every rank learns its own independent problem (seed = rank); there is no
collective on the path.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "candidates×traces/s"
MAX_SIZE = 9
WORKLOAD = ("single_large: 3 props, 1024+1024 traces, length U{16..32}, Bernoulli(0.3) bits, "
            "planted (G(!p0 | F p1) | p2), all 7 connectives, sizes 1..9 enumerated completely")
N_UNARY = 4   # !, X, F, G


def units_of(stats, T):
    d = stats["levels_done"]
    return sum(stats["candidates"][k] for k in range(1, d + 1)) * T


def level_bytes(stats, k, T, n_props):
    """Algorithmic HBM bytes of level k's launches: every candidate reads its
    operand matrices and either writes its matrix (new) or reads one for the
    full compare (duplicate): (operands + 1) * (bytes per trace) per trace,
    8 * W bytes per trace (4 in the narrow layout, two traces per word)."""
    cand = stats["candidates"][k]
    if k == 1:
        unary, binary = cand, 0
    else:
        unary = min(cand, N_UNARY * stats["unique"][k - 1])
        binary = cand - unary
    per_trace = 4 if stats["traces_per_word"] == 2 else 8 * stats["words_per_trace"]
    return (unary * 2 + binary * 3) * T * per_trace


OP_NAMES = ["atoms", "not", "and", "or", "X", "F", "G", "U"]


def op_candidates(unique, k, op, n_props):
    """Candidates of connective `op` at size k, from the unique counts of the
    smaller sizes (the candidate space of the paper's handleOp, as read here:
    unary over size k-1; U over ordered splits and pairs; And/Or over splits
    i <= j, pairs a < b when i == j)."""
    if k == 1 or op == 0:
        return n_props if (k == 1 and op == 0) else 0
    if op in (1, 4, 5, 6):
        return unique[k - 1]
    tot = 0
    for i in range(1, k - 1):
        j = k - 1 - i
        if op == 7:
            tot += unique[i] * unique[j]
        elif i < j:
            tot += unique[i] * unique[j]
        elif i == j:
            tot += unique[i] * (unique[i] - 1) // 2
    return tot


def int_ops_per_candidate_trace(op, nsteps, carry=True):
    """Algorithmic 32-bit integer operations per candidate and trace in the
    narrow layout (one 32-bit word per trace).  Not, And, Or and X: one
    operation; atoms none.  By the carry chain (the kernels' default): F a
    bit reversal, a negation, an OR and the reversal back; G the same between
    two masked complements; U the reversal of both operands, an OR, an
    addition, a three-input update and the reversal back.  By the paper's
    exponential propagation (Section 4): F a shift and an OR per log step; G
    the same plus the masked complements; U per step a shift and a
    three-input update of the until-vector and, on every step but the last,
    a shift and an AND of the holds-so-far vector.  Plus 3 for the
    fingerprint (two additions and a widening multiply-add per 64-bit word of
    two traces) and the position-0 check."""
    if carry:
        core = {0: 0, 1: 1, 2: 1, 3: 1, 4: 1, 5: 4, 6: 6, 7: 6}[op]
    else:
        core = {0: 0, 1: 1, 2: 1, 3: 1, 4: 1, 5: 2 * nsteps, 6: 2 * nsteps + 2, 7: 4 * nsteps - 2}[op]
    return core + 3


def kernel_sources_sha():
    h = hashlib.sha256()
    for f in ("ltl_level_fused.cuh", "ltl_level_ws.cuh", "ltl_level_common.cuh", "ltl_device.cuh", "ltl_types.h"):
        with open(os.path.join(ROOT, "paper_2402_12373_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def stream_sources_sha():
    h = hashlib.sha256()
    for f in ("ltl_level_stream.cu", "ltl_level_common.cuh", "ltl_device.cuh", "ltl_types.h"):
        with open(os.path.join(ROOT, "paper_2402_12373_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def stream_traffic_per_candidate():
    """Physical DRAM bytes per candidate of the streaming kernel from a
    committed ncu summary of a small trace-scaling case whose cache fills
    during the captured level, if it was taken on the current sources."""
    p = os.path.join(ROOT, "profiles", "stream_kernel_trace_scaling.json")
    try:
        with open(p) as f:
            d = json.load(f)
        if d.get("stream_sources_sha") == stream_sources_sha():
            return d.get("dram_bytes_per_candidate")
    except Exception:
        pass
    return None


def profiled_traffic(sha):
    """DRAM bytes per launch of the dominant kernel from a committed ncu
    summary, if it was taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "level_kernel_single_large.json")
    try:
        with open(p) as f:
            d = json.load(f)
        if d.get("kernel_sources_sha") == sha:
            return d.get("dram_bytes_per_launch_full_size")
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms; only the
    samples whose timestamps fall inside the timed region (mark_start /
    mark_end) are summarised."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
            # wait for the first sample, so that sampling covers the timed region
            t_end = time.time() + 5.0
            while time.time() < t_end and os.path.getsize(self.f.name) == 0:
                time.sleep(0.02)
        except Exception:
            self.p = None
        return self

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()
        time.sleep(0.12)   # let the sample that covers the end arrive

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        import datetime
        self.f.flush()
        self.f.seek(0)
        rows = [l.strip().split(",") for l in self.f.read().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                ts = datetime.datetime.strptime(r[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                if self.t0 is not None and not (self.t0 - 0.05 <= ts <= self.t1 + 0.05):
                    continue
                sm.append(float(r[2]))
                mx.append(float(r[3]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[6:10]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "interval_ms": 50}


# Launch configurations the library's tuner tries per launch class (2, 4 or 8
# tiles per resident CTA, at the occupancy maximum or one CTA per SM fewer),
# one untried configuration per launch of the class.  A step launches each
# tuned class once, so this many calls end the exploration.
AUTOTUNE_CONFIGS = 6


def autotune_summary(ctx, off, calls):
    """The tuned launch classes: chosen configuration (tiles per resident CTA,
    CTAs per SM below the occupancy maximum) and its best time per candidate
    against the default configuration's (4 tiles per CTA, full occupancy)."""
    if off:
        return {"enabled": False}
    tpc = [2, 4, 8, 2, 4, 8]
    assert len(tpc) == AUTOTUNE_CONFIGS
    less = [0, 0, 0, 1, 1, 1]
    chosen = {}
    for line in ctx.autotune_dump().strip().splitlines():
        parts = line.split()
        conf = [tuple(map(float, p.split(":"))) for p in parts[1:]]
        assert len(conf) == AUTOTUNE_CONFIGS, line
        tried = [(v, c) for c, (v, n) in enumerate(conf) if n > 0]
        if not tried:
            continue
        v, c = min(tried)
        chosen[parts[0]] = {"tiles_per_cta": tpc[c], "ctas_per_sm_less": less[c], "ns_per_candidate": round(v, 3),
                            "default_ns_per_candidate": round(conf[1][0], 3) if conf[1][1] else None}
    return {"enabled": True, "tuning_calls": calls,
            "tuning": "the tuner tries its configurations in untimed calls before the warm-up steps; the warm-up and "
                      "timed steps run the fastest",
            "classes": chosen}


def _oracle_rate(learn, spec, max_size, target_s):
    """candidates x traces per second of one oracle entry point, sizes
    1..max_size of `spec` enumerated completely, repeated for ~target_s; and
    the oracle's own time per size level, averaged over the runs (ms)."""
    T = spec.n_traces
    units, secs, runs, used = 0, 0.0, 0, 1
    level_s = [0.0] * (max_size + 1)
    while secs < target_s or runs == 0:
        t0 = time.perf_counter()
        r = learn(spec.P, spec.N, spec.n_props, max_size=max_size, stop_mode=0)
        secs += time.perf_counter() - t0
        units += sum(r["candidates"][1:max_size + 1]) * T
        runs += 1
        used = r.get("threads", 1)
        for k in range(1, max_size + 1):
            level_s[k] += r["seconds"][k]
    level_ms = [round(1e3 * level_s[k] / runs, 3) for k in range(1, max_size + 1)]
    return units / secs, runs, secs, used, level_ms


def cpu_baseline(target_s: float = 10.0, max_size: int = 6):
    """The oracle on the same workload, sizes 1..max_size enumerated
    completely: on every host core (the OpenMP variant, whose results equal
    the serial oracle's) and single-threaded (the plain C oracle)."""
    from oracle import oracle as O
    from paper_2402_12373_gb300 import synth
    spec = synth.single_large()
    sample = "single_large traces (2048), sizes 1..%d enumerated completely, %d run(s), %.1f s"
    unit = METRIC.split("/")[0] + "/s"
    v1, runs1, secs1, _, lv1 = _oracle_rate(O.learn, spec, max_size, target_s)
    single = {"value": v1, "unit": unit, "cores": 1, "kind": "oracle", "sample": sample % (max_size, runs1, secs1),
              "level_ms": lv1, "total_ms": round(sum(lv1), 3)}
    try:
        vn, runsn, secsn, used, lvn = _oracle_rate(O.learn_par, spec, max_size, target_s)
    except Exception as e:   # no OpenMP toolchain: the single-core figure stands alone
        single["multi_core_unavailable"] = str(e)[:200]
        return single
    return {"value": vn, "unit": unit, "cores": used, "kind": "oracle",
            "sample": sample % (max_size, runsn, secsn) + " (OpenMP over each block of a level's candidates, "
                      "admitted in enumeration order)",
            "level_ms": lvn, "total_ms": round(sum(lvn), 3),
            "level_ms_note": "the oracle's time per size level 1..%d on the same traces (mean over its runs); the "
                             "GPU's per level are levels.ms" % max_size,
            "nproc": os.cpu_count(), "single_core": single}


def _units_all(r, T):
    """candidates x traces over every level a run touched (the partial last
    level included): the work both the batched and the one-at-a-time path do."""
    return sum(r["candidates"][1:]) * T


def _same_result(a, b):
    d = a["levels_done"]
    return (a["status"] == b["status"] and a["size"] == b["size"] and d == b["levels_done"]
            and a["unique"][1:d + 1] == b["unique"][1:d + 1])


def bench_batched(L, ws, problems):
    """Batched workload: one ltl_learn_batch call against the plain path
    (one ltl_ctx_learn per problem, same workspace, same memory budgets, host
    planning of every level)."""
    import torch
    nbytes = ws.numel()
    T = [p.n_traces for p in problems]
    budgets = [int(0.85 * nbytes * t / sum(T)) for t in T]
    items = [(p.P, p.N, p.n_props, L.ALL, p.planted_size + 2, b) for p, b in zip(problems, budgets)]
    # plain path: one problem at a time, every level planned on the host (for
    # this workload of many different small problems that stop at their first
    # separator, the faster setting of the plain path); one untimed pass first,
    # as for every other leg (the first launch of each kernel variant in a
    # process loads its module)
    with L.Context(workspace=ws, stop=L.STOP_FIRST, planning=L.PLAN_HOST) as ctx:
        for rep in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            alone = []
            for (P, N, n_props, ops, K, b) in items:
                ctx.set_mem_budget(b)
                alone.append(ctx.learn(P, N, n_props, ops=ops, max_size=K))
            t_alone = time.perf_counter() - t0
    # batched: every problem resident, one launch per connective and shape per
    # round; one untimed call, then the mean of three calls
    L.learn_batch(items, stop=L.STOP_FIRST, workspace=ws)
    t_calls = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        batch = L.learn_batch(items, stop=L.STOP_FIRST, workspace=ws)
        t_calls.append(time.perf_counter() - t0)
    t_batch = statistics.mean(t_calls)
    units = sum(_units_all(r, t) for r, t in zip(batch, T))
    units_alone = sum(_units_all(r, t) for r, t in zip(alone, T))
    same = all(_same_result(a, b) for a, b in zip(alone, batch))
    st = {}
    for r in batch:
        st[r["status"]] = st.get(r["status"], 0) + 1
    return {"workload": "batched: %d problems, props U{2..5}, |P|=|N| log-uniform 16..4096, length U{8..64}, "
                        "Bernoulli(0.3), planted size U{3..9}, max size planted+2, stop at first separator, "
                        "memory budget per problem proportional to |P|+|N|" % len(problems),
            "problems": len(problems), "n_traces_total": sum(T),
            "batched_s": t_batch, "batched_calls_s": t_calls, "one_at_a_time_s": t_alone,
            "timing": "host buffers, wall clock; both paths after one untimed pass; batched: mean of 3 calls",
            "problems_per_s": len(problems) / t_batch, "one_at_a_time_problems_per_s": len(problems) / t_alone,
            "speedup_vs_one_at_a_time": t_alone / t_batch,
            "candidates_x_traces_per_s": units / t_batch,
            "one_at_a_time_candidates_x_traces_per_s": units_alone / t_alone,
            "results_equal_alone_and_batched": same, "statuses": st,
            "rounds_max": max(r["rounds"] for r in batch)}


def bench_served(L, ws, pool, rates=(0.5, 0.9, 1.5), per_rate_s=1.5, seed=5):
    """Served workload: Poisson arrivals of trace-scaling-shaped problems
    (65536 traces, length U{33..128}) at fractions of the one-at-a-time rate."""
    import random as _random
    import threading
    import torch
    # one-at-a-time rate mu on the same problems (host buffers, learn mode)
    with L.Context(workspace=ws, stop=L.STOP_FIRST, mem_budget=2 << 30) as ctx:
        for sp in pool[:2]:
            ctx.learn(sp.P, sp.N, sp.n_props, max_size=11)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n_alone = 0
        alone = {}
        while time.perf_counter() - t0 < 1.0 or n_alone < len(pool):
            sp = pool[n_alone % len(pool)]
            r = ctx.learn(sp.P, sp.N, sp.n_props, max_size=11)
            alone[n_alone % len(pool)] = r
            n_alone += 1
        mu = n_alone / (time.perf_counter() - t0)
    out = {"workload": "served: Poisson arrivals of trace-scaling problems (65536 traces, length U{33..128}, "
                       "4 props, planted (((p0 U p1) & G !p3) & F p2), seeds 1000..%d cycled), max size 11, "
                       "stop at first separator, 2 GiB per problem; each server gets one untimed warm-up "
                       "request of every problem of the pool before the timed arrivals" % (1000 + len(pool) - 1),
           "one_at_a_time_problems_per_s": mu, "rates": []}
    rng = _random.Random(seed)
    for f in rates:
        lam = f * mu
        n_req = max(8, int(lam * per_rate_s))
        gaps = [rng.expovariate(lam) for _ in range(n_req)]
        arrivals = []
        acc = 0.0
        for g in gaps:
            acc += g
            arrivals.append(acc)
        results = {}
        with L.Server(workspace=ws, stop=L.STOP_FIRST, max_resident=64, mem_budget=2 << 30) as srv:
            # untimed requests first, one of every problem of the pool: a fresh
            # server's first admissions and the first rounds of each shape
            # pay one-time set-up (launch attributes, occupancy queries,
            # events, the first launch of each kernel)
            warm = {srv.submit(sp.P, sp.N, sp.n_props, max_size=11) for sp in pool}
            t_w = time.perf_counter()
            while warm and time.perf_counter() - t_w < 60:
                for r in srv.poll(64, 50):
                    warm.discard(r["id"])
            ids = {}
            t_start = time.perf_counter()

            def submitter():
                for i, t_a in enumerate(arrivals):
                    dt = t_start + t_a - time.perf_counter()
                    if dt > 0:
                        time.sleep(dt)
                    sp = pool[i % len(pool)]
                    ids[srv.submit(sp.P, sp.N, sp.n_props, max_size=11)] = i

            th = threading.Thread(target=submitter)
            th.start()
            while len(results) < n_req and time.perf_counter() - t_start < 120:
                for r in srv.poll(256, 50):
                    results[r["id"]] = r
            th.join()
            t_end = time.perf_counter()
        lat = sorted(r["latency_ms"] for r in results.values())
        same = all(_same_result(alone[ids[i] % len(pool)], r) for i, r in results.items() if i in ids)
        out["rates"].append({
            "rate_fraction_of_mu": f, "arrival_rate_per_s": lam, "requests": n_req, "completed": len(results),
            "throughput_problems_per_s": len(results) / (t_end - t_start),
            "latency_ms_p50": lat[len(lat) // 2] if lat else None,
            "latency_ms_p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))] if lat else None,
            "results_equal_alone": same})
    return out


def bench_trace_scaling(L, ws, spec, steps=2):
    """Trace-scaling workload: enumeration-only until the cache budget (120 GB)
    or size 11 is reached; two-word sequences with cross-word carries."""
    import torch
    T = spec.n_traces
    letters = np.concatenate([spec.P.letters, spec.N.letters]).astype(np.int32)
    offs = np.concatenate([spec.P.offsets, spec.N.offsets[1:] + spec.P.offsets[-1]]).astype(np.int64)
    dl = torch.from_numpy(letters).to(ws.device)
    do = torch.from_numpy(offs).to(ws.device)
    budget = min(120 * 10**9, int(0.9 * ws.numel()))
    runs = []
    with L.Context(workspace=ws, stop=L.STOP_NONE, mem_budget=budget) as ctx:
        ctx.learn_device(dl, do, spec.P.n, spec.N.n, spec.max_len(), spec.n_props, max_size=11)   # warm-up
        for _ in range(steps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            r = ctx.learn_device(dl, do, spec.P.n, spec.N.n, spec.max_len(), spec.n_props, max_size=11)
            e1.record()
            e1.synchronize()
            runs.append((e0.elapsed_time(e1), r))
    ms = statistics.mean(t for t, _ in runs)
    r = runs[-1][1]
    done = r["levels_done"]
    units_done = sum(r["candidates"][1:done + 1]) * T
    units_all = sum(r["candidates"][1:]) * T
    # size levels against the HBM roof, all of a level's launches together (a
    # level of fewer than 2^17 candidates runs its connectives concurrently,
    # so only the level has a time of its own).  Algorithmic bytes: every
    # candidate streams its operand matrices (the kernels for matrices larger
    # than a CTA stage no operand across candidates); a candidate that was
    # stored or compared adds one matrix.  In a completed level that is every
    # candidate; in the level the cache filled during, only the candidates
    # stored (its unique count) or compared before that (the call's compares
    # less the duplicates of the completed levels): after it, a candidate is
    # only tested for separation.
    cm_bytes = T * 8 * r["words_per_trace"]
    peaks, peak_src = measured_peaks()

    def level_roof(k, completed):
        k_ms = statistics.mean(x["ms"][k] for _, x in runs)
        operands = sum(op_candidates(r["unique"], k, o, spec.n_props) * (2 if o in (2, 3, 7) else 1)
                       for o in range(1, 8))
        if completed:
            touched = r["candidates"][k]
        else:
            dups_before = sum(r["candidates"][i] - r["unique"][i] for i in range(1, k))
            touched = r["unique"][k] + max(0, r["compares"] - dups_before)
        k_bytes = (operands + touched) * cm_bytes
        ach = k_bytes / (k_ms / 1e3) / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": None,
                "kernel": "%s, every connective of size level %d%s" % (
                    "/".join(sorted({x for x in r["op_kernel"][k] if x})), k,
                    "" if completed else " (the cache filled during it)"),
                "count": "both operand matrices of every candidate, plus one per candidate stored or compared; the "
                         "streaming kernel copies each candidate's operands from global memory and L2 serves the left "
                         "operand that consecutive candidates share, so this fraction can exceed 1",
                "candidates": r["candidates"][k], "stored_or_compared": touched, "level_ms": k_ms,
                "algorithmic_bytes": k_bytes, "peak_source": peak_src + " (hbm_gbs, copy bandwidth)"}

    roof_done = level_roof(done, True) if done >= 1 else None
    # enumerating every level (no stop at a separator), a level that has
    # candidates but is not complete is the one the cache filled during
    capped = done + 1 < len(r["candidates"]) and r["candidates"][done + 1] > 0
    roof_cap = level_roof(done + 1, False) if capped else None
    # the roofline of the leg is its longest level's
    if roof_cap is not None:
        # physical DRAM bytes: an ncu capture of a small case scaled by candidates
        per_cand = stream_traffic_per_candidate()
        if per_cand:
            traffic = per_cand * roof_cap["candidates"]
            roof_cap["traffic"] = traffic
            roof_cap["dram"] = {"bytes": traffic, "gbs": traffic / (roof_cap["level_ms"] / 1e3) / 1e9,
                                "frac": traffic / (roof_cap["level_ms"] / 1e3) / 1e9 / peaks["hbm_gbs"],
                                "source": "ncu DRAM bytes per candidate of a size-5 trace-scaling launch whose cache "
                                          "fills during it (profiles/stream_kernel_trace_scaling.json), times this "
                                          "level's candidates"}
    roof = roof_done
    if roof_cap is not None and (roof is None or roof_cap["level_ms"] > roof["level_ms"]):
        roof = dict(roof_cap, completed_level=roof_done)
    return {"workload": "trace_scaling: 4 props, 32768+32768 traces, length U{33..128} (2 words per trace), "
                        "Bernoulli(0.25), every level until size 11 or a 120 GB cache budget",
            "status": r["status"], "levels_done": done, "unique": r["unique"][1:], "candidates": r["candidates"][1:],
            "ms": ms, "level_ms": [round(x, 3) for x in r["ms"][1:]],
            "candidates_x_traces_per_s_completed_levels": units_done / (ms / 1e3),
            "candidates_x_traces_per_s_all": units_all / (ms / 1e3),
            "launch": {"threads_per_cta": r["threads_per_cta"], "chunk_groups": r["chunk_groups"],
                       "words_per_trace": r["words_per_trace"]},
            "entries": r["entries"], "max_entries": r["max_entries"], "roofline": roof}


def bench_dc(L, ws, specs, windows=(16, 64)):
    """Divide and conquer on Hamming(B, l, delta) (Section 7's high-cost
    workload): U-free NNF formulae, max size 6 per part; wall time per
    specification with host buffers, formula size and split statistics."""
    ops = (L.ALL & ~L.U) | L.NNF
    rows = []
    for spec in specs:
        for mode, mname in ((L.DC_RANDOM, "random"), (L.DC_DETERMINISTIC, "deterministic")):
            for win in windows:
                t0 = time.perf_counter()
                r = L.learn_dc(spec.P, spec.N, spec.n_props, ops=ops, max_size=6, mode=mode, window=win, seed=1,
                               workspace=ws)
                wall = 1e3 * (time.perf_counter() - t0)
                rows.append({"spec": spec.name, "traces": spec.n_traces, "split": mname, "window": win,
                             "status": r["status"], "wall_ms": wall, "formula_size": r["formula_size"],
                             "parts_enumerated": r["enum_calls"] - r["enum_failed"],
                             "enum_calls": r["enum_calls"], "enum_failed": r["enum_failed"],
                             "fallbacks": r["fallbacks"], "rounds": r["rounds"], "evals": r["evals"],
                             "max_depth": r["max_depth"]})
    return {"workload": "planted_large: 1024 + 1024 traces of length U{4..10} over 2 propositions labelled by "
                        "F(p0 & X p1) (parts the enumerator solves); single_large: the bench's 2048 traces, whose "
                        "minimal separator (size 8) exceeds the parts' limit, so parts are enumerated and "
                        "combined; Hamming(B, l, delta): P = one random trace "
                        "of length l over 2 propositions, N = all traces at bit distance delta (parts closed by "
                        "the overfitting fallback); U-free NNF, max size 6 per part; enum_calls - enum_failed "
                        "= parts learned by enumeration", "runs": rows}


def run_reference(args):
    from paper_2402_12373_gb300 import dist
    rank, _, world = dist.env_rank()
    if rank != 0:
        return 0
    from oracle import oracle as O
    from paper_2402_12373_gb300 import synth
    spec = synth.single_large()
    T = spec.n_traces
    K = 5
    try:
        learn, kind = O.learn_par, "OpenMP over each block of a level's candidates"
        learn(spec.P, spec.N, spec.n_props, max_size=2, stop_mode=0)
    except Exception:
        learn, kind = O.learn, "single-threaded"
    for _ in range(args.warmup):
        learn(spec.P, spec.N, spec.n_props, max_size=K, stop_mode=0)
    units, secs, used = 0, 0.0, 1
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = learn(spec.P, spec.N, spec.n_props, max_size=K, stop_mode=0)
        secs += time.perf_counter() - t0
        units += sum(r["candidates"][1:K + 1]) * T
        used = r.get("threads", 1)
    value = units / secs
    sample = ("single_large traces (2048), sizes 1..%d enumerated completely per step (CPU oracle, %s)"
              % (K, kind))
    out = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": WORKLOAD, "reference_sample": sample, "n_traces": T},
           "cpu_baseline": {"value": value, "unit": METRIC, "cores": used, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=8,
                    help="untimed steps (at least 3), after the autotuner's untimed tuning calls")
    ap.add_argument("--no-autotune", action="store_true", help="fixed launch heuristics instead of the autotuner")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--max-size", type=int, default=MAX_SIZE)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the batched, served and trace-scaling measurements")
    ap.add_argument("--max-chunks", type=int, default=0,
                    help="launch-shape cap (16-byte chunks per thread); 0 = automatic")
    ap.add_argument("--planning", default="auto", choices=["auto", "host"],
                    help="where small size levels are planned (ltl_opts.level_planning)")
    ap.add_argument("--propagation", default="carry", choices=["carry", "logstep"],
                    help="F, G and U by the carry chain or by the paper's log-step exponential propagation")
    ap.add_argument("--level-kernel", default="auto", choices=["auto", "fused", "ws"],
                    help="size-level kernel: automatic choice, fused, or warp-specialised")
    ap.add_argument("--budget-gb", type=float, default=32.0,
                    help="device memory budget of the single-large problem's cache and hash set, in GB "
                         "(capped by the workspace)")
    ap.add_argument("--ws-gb", type=float, default=0.0,
                    help="workspace size in GB (default: half of the free device memory)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    args.warmup = max(args.warmup, 3)

    import numpy as np
    import torch

    from paper_2402_12373_gb300 import _lib as L
    from paper_2402_12373_gb300 import dist, synth

    rank, local_rank, world = dist.env_rank()
    # inputs of the extra workloads, generated before any GPU work (spawn pool)
    extra = None
    if not args.no_extra and rank == 0:
        procs = min(16, os.cpu_count() or 1)
        batched_probs = synth.batched_workload(256, processes=procs)
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(min(8, procs)) as pool:
            served_pool = pool.map(synth.trace_scaling, [1000 + i for i in range(8)])
        extra = (batched_probs, served_pool)
    torch.cuda.set_device(local_rank)
    world = dist.init("nccl")
    dev = torch.device("cuda", local_rank)

    spec = synth.single_large(seed=rank)
    T = spec.n_traces
    letters = np.concatenate([spec.P.letters, spec.N.letters]).astype(np.int32)
    offs = np.concatenate([spec.P.offsets, spec.N.offsets[1:] + spec.P.offsets[-1]]).astype(np.int64)
    d_letters = torch.from_numpy(letters).to(dev)
    d_offsets = torch.from_numpy(offs).to(dev)
    max_len = spec.max_len()
    K = args.max_size

    free, _ = torch.cuda.mem_get_info(local_rank)
    ws_bytes = int(args.ws_gb * 1e9) if args.ws_gb > 0 else int(free * 0.5)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    L.DEFAULT_LEVEL_KERNEL = {"auto": L.KERNEL_AUTO, "fused": L.KERNEL_FUSED, "ws": L.KERNEL_WS}[args.level_kernel]
    L.DEFAULT_PLANNING = {"auto": L.PLAN_AUTO, "host": L.PLAN_HOST}[args.planning]
    L.DEFAULT_PROPAGATION = {"carry": L.PROP_CARRY, "logstep": L.PROP_LOGSTEP}[args.propagation]
    budget = min(int(args.budget_gb * 1e9), int(ws_bytes * 0.9))   # the workspace also holds the fixed parts
    ctx = L.Context(workspace=ws, stop=L.STOP_NONE, max_chunks=args.max_chunks, mem_budget=budget,
                    autotune=None if args.no_autotune else "")

    def step():
        return ctx.learn_device(d_letters, d_offsets, spec.P.n, spec.N.n, max_len, spec.n_props, max_size=K)

    int_peak = L.int32_peak()   # integer roof, measured before the warm-up
    tune_calls = 0 if args.no_autotune else AUTOTUNE_CONFIGS
    for _ in range(tune_calls + args.warmup):
        step()
        flush.zero_()
    torch.cuda.synchronize()

    gpu_idx = local_rank
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES")
    if cvd:
        try:
            gpu_idx = int(cvd.split(",")[local_rank])
        except ValueError:
            pass
    results = []
    times = []
    # no cyclic-GC pass inside the timed region (the host drives every round,
    # so a collection over the extras' inputs would stretch a step)
    gc.collect()
    gc.disable()
    with ClockSampler(gpu_idx) as clk:
        dist.barrier()
        torch.cuda.synchronize()
        clk.mark_start()
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = step()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            results.append(r)
        torch.cuda.synchronize()
        clk.mark_end()
        dist.barrier()
    gc.enable()
    clocks = clk.summary()

    total_ms = sum(times)
    local_units = sum(units_of(r, T) for r in results)
    max_ms = dist.reduce_max(total_ms, dev)
    all_units = dist.reduce_sum(local_units, dev)
    value = all_units / (max_ms / 1e3)
    r0 = results[-1]
    W = r0["words_per_trace"]

    # dominant kernel: the (size level, connective) launch with the longest
    # device time (CUDA events the library records on its stream)
    # (only launches that ran alone, whose event time is their own)
    pairs = [(k, o) for k in range(1, r0["levels_done"] + 1) for o in range(8) if r0["op_alone"][k][o]]
    kd, od = max(pairs, key=lambda ko: sum(r["op_ms"][ko[0]][ko[1]] for r in results))
    kd_ms = statistics.mean(r["op_ms"][kd][od] for r in results)
    per_trace = 4 if r0["traces_per_word"] == 2 else 8 * W
    cm_bytes = T * per_trace                       # algorithmic bytes of one characteristic matrix
    n_operands = 2 if od in (2, 3, 7) else 1
    kd_cands = op_candidates(r0["unique"], kd, od, spec.n_props)
    kd_staged = statistics.mean(r["op_staged"][kd][od] for r in results)
    streamed_bytes = kd_cands * (n_operands + 1) * cm_bytes
    if kd_staged > 0:
        # operands as the kernel stages them (left operand once per reload),
        # plus the matrix stored or read for the full compare per candidate
        kd_bytes = (kd_staged + kd_cands) * cm_bytes
        count = "left operand staged: operand matrices copied into shared memory (device count) + 1 per candidate"
    else:
        kd_bytes = streamed_bytes
        count = "both operands streamed (this kernel reports no staged-operand count)"
    peaks, peak_src = measured_peaks()
    hbm_achieved = kd_bytes / (kd_ms / 1e3) / 1e9
    hbm_frac = hbm_achieved / peaks["hbm_gbs"]
    sha = kernel_sources_sha()
    traffic = profiled_traffic(sha)
    kname = ("%s connective %s, size level %d (%s layout)"
             % (r0["op_kernel"][kd][od], OP_NAMES[od], kd, "narrow" if r0["traces_per_word"] == 2 else "wide"))
    hbm = {"achieved": hbm_achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": hbm_frac,
           "peak_source": peak_src + " (hbm_gbs, copy bandwidth)", "count": count,
           "algorithmic_bytes_per_launch": kd_bytes, "operand_matrices_staged": kd_staged,
           "matrix_bytes": cm_bytes,
           "frac_both_operands_streamed": streamed_bytes / (kd_ms / 1e3) / 1e9 / peaks["hbm_gbs"]}

    # the same launch against the integer roof: algorithmic shift and logic
    # operations over the measured throughput of such operations
    alu = None
    if r0["traces_per_word"] == 2:
        nsteps = max(1, (spec.max_len() - 1).bit_length())
        carry = L.DEFAULT_PROPAGATION == L.PROP_CARRY
        ops_ct = int_ops_per_candidate_trace(od, nsteps, carry)
        kd_ops = kd_cands * T * ops_ct
        alu_achieved = kd_ops / (kd_ms / 1e3) / 1e9
        alu = {"achieved": alu_achieved, "peak": int_peak["ops_per_s"] / 1e9, "unit": "Gop/s",
               "frac": alu_achieved / (int_peak["ops_per_s"] / 1e9), "ops_per_candidate_trace": ops_ct,
               "log_steps": nsteps, "propagation": "carry chain" if carry else "log steps",
               "algorithmic_ops_per_launch": kd_ops,
               "peak_source": "measured on this GPU (ltl_int32_peak: chains of 32-bit shifts and three-input "
                              "logic operations, %.2f ms)" % int_peak["ms"]}
    # the roof the launch uses more of, by these algorithmic counts
    main = alu if (alu is not None and alu["frac"] > hbm_frac) else hbm
    roofline = {"bound": "alu" if main is alu else "hbm", "achieved": main["achieved"], "peak": main["peak"],
                "unit": main["unit"], "frac": main["frac"], "traffic": traffic, "kernel": kname,
                "candidates_per_launch": kd_cands, "launch_ms": kd_ms,
                "level_ms": statistics.mean(r["ms"][kd] for r in results),
                "hbm": hbm, "alu": alu, "kernel_sources_sha": sha}
    if traffic:
        # physical DRAM bytes of the launch (ncu, same kernel sources) over its event time
        roofline["dram"] = {"bytes_per_launch": traffic, "gbs": traffic / (kd_ms / 1e3) / 1e9,
                            "frac": traffic / (kd_ms / 1e3) / 1e9 / peaks["hbm_gbs"]}
        if alu is not None and max(roofline["dram"]["frac"], alu["frac"]) < 0.5:
            # neither physical roof is near: say what the launch waits on
            roofline["limiter"] = ("latency: physical DRAM traffic at %.2f of the copy bandwidth and integer work at "
                                   "%.2f of the measured integer roof; the hash warps' global round trips (claim, "
                                   "allocation or compare, publication) and the compute warps' dependent chains "
                                   "(ncu: long-scoreboard and wait stalls lead, profiles/level_kernel_single_large.md)"
                                   % (roofline["dram"]["frac"], alu["frac"]))
    kernel_ms = [sum(r["ms"][k] for k in range(1, r["levels_done"] + 1)) for r in results]

    # end to end: host trace buffers through ltl_ctx_learn (one untimed call
    # first: the first copy from these pageable host buffers sets up the
    # driver's staging)
    ctx.learn(spec.P, spec.N, spec.n_props, max_size=K)
    e2e_times, e2e_units, h2d, d2h = [], 0, 0, 0
    gc.collect()
    gc.disable()
    for _ in range(max(2, min(args.steps, 10))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = ctx.learn(spec.P, spec.N, spec.n_props, max_size=K)
        e2e_times.append(time.perf_counter() - t0)
        e2e_units += units_of(r, T)
        h2d, d2h = r["h2d_bytes"], r["d2h_bytes"]
    gc.enable()
    e2e_value = dist.reduce_sum(e2e_units, dev) / dist.reduce_max(sum(e2e_times), dev)

    # time to learn (stop at the first separator), host buffers, wall clock
    ctx_first = L.Context(workspace=ws, stop=L.STOP_FIRST, mem_budget=budget)
    ttl = []
    found = None
    for _ in range(5):
        t0 = time.perf_counter()
        r = ctx_first.learn(spec.P, spec.N, spec.n_props, max_size=K)
        ttl.append(1e3 * (time.perf_counter() - t0))
        found = r
    ctx_first.close()

    # the paper's evaluation of F, G and U (log-step exponential propagation,
    # Section 4) on the same workload, timed the same way, for comparison
    other = None
    if rank == 0 and not args.no_extra:
        alt = L.PROP_LOGSTEP if L.DEFAULT_PROPAGATION == L.PROP_CARRY else L.PROP_CARRY
        ctx_alt = L.Context(workspace=ws, stop=L.STOP_NONE, max_chunks=args.max_chunks, mem_budget=budget,
                            autotune=None if args.no_autotune else "", propagation=alt)
        for _ in range(tune_calls + args.warmup):
            ctx_alt.learn_device(d_letters, d_offsets, spec.P.n, spec.N.n, max_len, spec.n_props, max_size=K)
            flush.zero_()
        alt_times, alt_res = [], []
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ra = ctx_alt.learn_device(d_letters, d_offsets, spec.P.n, spec.N.n, max_len, spec.n_props, max_size=K)
            e1.record(stream)
            e1.synchronize()
            alt_times.append(e0.elapsed_time(e1))
            alt_res.append(ra)
        ctx_alt.close()
        other = {"propagation": "log steps (the paper's exponential propagation)" if alt == L.PROP_LOGSTEP
                 else "carry chain",
                 "ms_per_step": sum(alt_times) / len(alt_times),
                 "value": sum(units_of(x, T) for x in alt_res) / (sum(alt_times) / 1e3),
                 "dominant_launch_ms": statistics.mean(x["op_ms"][kd][od] for x in alt_res),
                 "top_level_op_ms": {name: round(statistics.mean(x["op_ms"][K][op] for x in alt_res), 4)
                                     for op, name in enumerate(OP_NAMES) if op > 0 and alt_res[0]["op_alone"][K][op]},
                 "top_level_ms": round(statistics.mean(x["ms"][K] for x in alt_res), 4),
                 "same_counts": all(x["unique"] == r0["unique"] and x["candidates"] == r0["candidates"]
                                    for x in alt_res)}

    launches = sum(r["launches"] for r in results)
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
            "step_ms": {"median": statistics.median(times), "min": min(times), "max": max(times)},
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_traces": T, "words_per_trace": W, "max_size": K,
                       "mode": "enumeration-only (every level complete)",
                       "l2": "flushed between steps (512 MiB write); cache working set > L2",
                       "memory_budget_gb": budget / 1e9,
                       "propagation": "carry chain" if L.DEFAULT_PROPAGATION == L.PROP_CARRY else "log steps",
                       "parallelism": "independent problem per rank (seed = rank)" if world > 1 else "1 GPU",
                       "launch": {"threads_per_cta": r0["threads_per_cta"],
                                  "traces_per_thread": r0["traces_per_thread"],
                                  "traces_per_word": r0["traces_per_word"],
                                  "batch": r0["batch"], "ctas_per_sm": r0["ctas_per_sm"],
                                  "chunk_groups": r0["chunk_groups"]}},
            "levels": {"unique": r0["unique"][1:], "candidates": r0["candidates"][1:],
                       "device_planned": r0["device_planned_levels"], "from_cuda_graph": r0["graph_levels"],
                       "ms": [round(x, 4) for x in r0["ms"][1:]], "entries": r0["entries"],
                       # own launch times of the last level's connectives that ran alone; the
                       # others ran concurrently after them (the level's time covers both)
                       "top_level_op_ms": {name: round(statistics.mean(r["op_ms"][K][op] for r in results), 4)
                                           for op, name in enumerate(OP_NAMES)
                                           if r0["op_ms"][K][op] > 0 and r0["op_alone"][K][op]},
                       "top_level_concurrent": [name for op, name in enumerate(OP_NAMES)
                                                if r0["op_ms"][K][op] > 0 and not r0["op_alone"][K][op]],
                       "top_level_concurrent_ms": round(statistics.mean(
                           r["ms"][K] - sum(r["op_ms"][K][op] for op in range(8) if r["op_alone"][K][op])
                           for r in results), 4)},
            "roofline": roofline,
            "kernel_ms_per_step": statistics.mean(kernel_ms),
            "value_by_kernel_time": local_units / (sum(kernel_ms) / 1e3),
            "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "time_to_learn_ms": {"median": statistics.median(ttl), "size": found["size"],
                                 "formula": found["formula"], "mode": "stop at first separator, host buffers"},
            "gpu_launches": launches,
            "clocks": clocks,
            "autotune": autotune_summary(ctx, args.no_autotune, tune_calls),
        }
        if other is not None:
            out["other_propagation"] = other
        if extra is not None:
            out["batched"] = bench_batched(L, ws, extra[0])
            out["served"] = bench_served(L, ws, extra[1])
            out["trace_scaling"] = bench_trace_scaling(L, ws, extra[1][0])
            out["divide_and_conquer"] = bench_dc(L, ws, [synth.planted_large(seed=1), synth.single_large(seed=1),
                                                          synth.hamming(24, 2, seed=1), synth.hamming(48, 2, seed=1)])
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline()
        print(json.dumps(out))
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
