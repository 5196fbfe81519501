#!/usr/bin/env python3
"""Benchmark of the GKR/CMT prover on the F2 circuit, n = 2^20 (inputs uniform
in [0, 2^16]): one step = one proof (evaluation, all sum-check rounds, all line
reductions) plus its verification, on inputs already resident in HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `value` is whole-job non-input gates per
second (device time, CUDA events around each step, L2 flushed between steps);
`e2e` is the same metric through the C ABI starting from page-locked host
inputs (each step uploads them, and downloads the transcript and the accept
bit, inside the timed region); `roofline` covers the
first sum-check wave, the dominant kernel; `cpu_baseline` is the CPU oracle
timed on this host.  Under torchrun every rank proves its own independent
instances (the proofs share nothing): weak scaling, no collective on the data
path.  `--impl reference` times the CPU oracle instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GKR prover gates/s (F2, n=2^20); batched proofs/s and p50/p99 proof latency"
UNIT = "gates/s"
WORKLOAD = "f2_2^20"
SC_CHUNK_LOG = 11


def env_rank():
    from paper_1202_1350_gb300 import replicas
    return replicas.rank_env()


# ---- clocks during the timed region --------------------------------------------------

class ClockSampler:
    """nvidia-smi every 100 ms from start() to stop(); the SM clock is the
    median over the samples that saw the GPU busy (all samples if none did)."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.12)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
            os.unlink(self.path)
        except Exception:
            return None
        if not rows:
            return None
        busy = [r for r in rows if len(r) >= 10 and r[9].isdigit() and int(r[9]) >= 50]
        sm = [float(r[1]) for r in (busy or rows) if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "busy_samples": len(busy)}


# ---- work of the dominant launch ---------------------------------------------------------

def algorithmic_work(widths, kinds):
    """Field multiplications the folding prover needs for what the wave launch
    computes, per layer i with S_i = 2^{s_i} gates over S_{i+1} = 2^{s_{i+1}}:
      phase 1 (three values and two folds per pair, over halving rounds)  5 S_i
      phase-2/3 P and B tables (formed from eq(r_P, .) and the wiring)     2 S_i
      phases 2 and 3 (A V, B, M V at t = 0, 1, 2 and four folds per pair) 20 S_{i+1}
      line polynomial (coefficient-form folding)                           4 S_{i+1}
    i.e. 7 S_i + 24 S_{i+1}.  (The eq tables themselves are built by the coin
    launch and not counted here.)  Bytes: the value tables the launch reads,
    each once: V_i for phase 1, V_{i+1} for phases 2 and 3 and the line,
    8 (S_i + 3 S_{i+1}) per layer."""
    mul = 0
    byts = 0
    for i in range(len(kinds)):
        S, Sn = 1 << widths[i], 1 << widths[i + 1]
        mul += 7 * S + 24 * Sn
        byts += 8 * (S + 3 * Sn)
    return mul, byts


def executed_work(widths, kinds, first_wave_log=12):
    """Field multiplications the wave launch actually performs on circuits of
    SQUARE and TREE layers (products of W values, 64-bit or in 31-bit limbs):
      * product-weighted instance over n variables (phase 1 of every layer,
        phase 3 of SQUARE and TREE layers; P stays implicit): per pair of
        entries of every round h(0), h(1) and the fold of V: 3 (2^n - 1);
      * general instance (phase 2): per pair P V at t = 0, 1, 2 and the folds
        of P and V (and B for TREE): 5 (6) per pair; SQUARE forms P = eq V at
        2 per entry; TREE with a first wave in registers (n > 7) does its
        round 0 at 5 per pair (eq(r_P, g), w (v0 + v1), w (3 v1 - v0), the V
        fold and B = w v1), smaller TREE instances form P and B at 2 per gate;
      * line reduction over n = s_{i+1} coordinates: folding coordinate j turns
        pairs of degree-j polynomials into one of degree j + 1 at 2 (j + 1)
        multiplications: sum_j 2^(n-j-1) 2 (j + 1)."""
    mul = 0
    for i, k in enumerate(kinds):
        si, sn = widths[i], widths[i + 1]
        assert k in (0, 1), "counted for SQUARE and TREE layers"
        for ph, n in ((1, si), (2, sn), (3, sn)):
            if n == 0:
                continue
            if ph == 2 and k == 0:
                mul += 5 * ((1 << n) - 1) + 2 * (1 << n)
            elif ph == 2 and min(n, first_wave_log) > 7:
                mul += 5 * (1 << (n - 1)) + 6 * ((1 << (n - 1)) - 1)
            elif ph == 2:
                mul += 6 * ((1 << n) - 1) + (1 << n)
            else:
                mul += 3 * ((1 << n) - 1)
        mul += sum((1 << (sn - j - 1)) * 2 * (j + 1) for j in range(sn))
    return mul


# DRAM bytes (read + write) of one k_waves launch on this workload, from an ncu
# capture of the current kernel; the V tables are mostly served from L2, so
# this is below the algorithmic bytes
K_WAVES_DRAM_BYTES = 25_572_096
# The same launch's integer pipes (ncu, % of peak sustained while active):
# the multiply pipe (fmaheavy) cycles, ALU instructions, issue slots
K_WAVES_PIPES = {"fmaheavy_cycles_pct": 52.4, "alu_inst_pct": 49.9, "issue_active_pct": 48.7}
# ncu: the pair-step microbenchmark keeps the multiply pipe (fmaheavy) busy
# this fraction of its cycles (83-86 % over its configurations), so the pipe
# saturated would give its rate / this fraction
PAIR_STEP_FMAHEAVY_FRAC = 0.847


def run_ablation(h, xd, tr, flush, reps=5):
    """The same proof by the paper's per-gate method (one thread per gate per
    round, vc_prove_pergate) against the folding prover, device time of one
    proof each (L2 flushed before every call; transcripts compared)."""
    import torch
    from paper_1202_1350_gb300 import vc
    out = {}
    ref = torch.empty_like(tr)
    for name, fn, dst in (("folding", vc.vc_prove, ref), ("pergate", vc.vc_prove_pergate, tr)):
        ts = []
        for k in range(reps + 2):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn(h, xd, 4242, dst)
            e1.record()
            e1.synchronize()
            if k >= 2:
                ts.append(e0.elapsed_time(e1))
        out[name + "_prove_ms"] = statistics.median(ts)
    vc.vc_circuit_sync(h)
    assert bool((ref == tr).all().item()), "per-gate and folding transcripts differ"
    out["speedup_of_folding"] = out["pergate_prove_ms"] / out["folding_prove_ms"]
    out["note"] = "prove only (no verification), median of 5, same transcript"
    return out


def run_residency(widths, kinds, xd, flush, reps=5):
    """Proof time with the layer values in mapped host memory (read and
    written over the host link at every use), staged through host memory
    (copy-once-per-layer: the wide layers pass through device slots of the
    widest layer's size) and windowed (the same slots, each iteration run
    while its layers are there, nothing copied to the host), against
    device-resident values; transcripts compared.  link_bytes: what a mode
    moves over the host link per proof (staged: each wide layer written once,
    plus the layers copied back in), as the library reports it."""
    import torch
    from paper_1202_1350_gb300 import vc
    out = {}
    trs = {}
    for name, kw in (("device", {}), ("host_values", {"host_values": True}), ("staged", {"staged": True}),
                     ("windowed", {"windowed": True})):
        h = vc.vc_circuit_create(widths, kinds, **kw)
        tr = torch.empty(vc.vc_transcript_len(h), dtype=torch.int64, device="cuda")
        ts = []
        for k in range(reps + 2):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            vc.vc_prove(h, xd, 4343, tr)
            e1.record()
            e1.synchronize()
            if k >= 2:
                ts.append(e0.elapsed_time(e1))
        vc.vc_circuit_sync(h)
        out[name + "_prove_ms"] = statistics.median(ts)
        out[name + "_device_bytes"] = vc.vc_circuit_bytes(h)
        trs[name] = tr.clone()
        if name in ("staged", "windowed"):
            out[name + "_link_bytes"] = vc.vc_circuit_get_info(h)["link_bytes"]
        else:
            out[name + "_stage_ms"] = _stage_split(h, xd, tr, flush)
        vc.vc_circuit_destroy(h)
    for name in ("host_values", "staged", "windowed"):
        assert bool((trs["device"] == trs[name]).all().item()), f"residency {name} changed the transcript"
    out["slowdown"] = out["host_values_prove_ms"] / out["device_prove_ms"]
    out["staged_slowdown"] = out["staged_prove_ms"] / out["device_prove_ms"]
    out["windowed_slowdown"] = out["windowed_prove_ms"] / out["device_prove_ms"]
    out["note"] = ("F2's wide layers (2^20, 2^20 and 2^19 values) pass through two slots of 2^20 values, "
                   "so staging saves F2 half a slot and copies the input layer back in once; windowed values "
                   "use the same slots with no host copies (each iteration runs while its two layers are "
                   "there); the deep F0 circuit (62 layers of values, eight slots) shows the saving: see `deep`")
    return out


def _stage_split(h, xd, tr, flush, reps=3):
    """Device time of the evaluation, wave and final-reduction stages of a
    proof (CUDA events the library records around them), medians of `reps`
    proofs after one warm-up."""
    import torch
    from paper_1202_1350_gb300 import vc
    names = ("eval", "waves", "final")
    ev = [None] * (2 * vc.NUM_STAGES)
    for nm in names:
        i = vc.STAGES.index(nm)
        ev[2 * i] = torch.cuda.Event(enable_timing=True)
        ev[2 * i + 1] = torch.cuda.Event(enable_timing=True)
    vc.vc_circuit_set_stage_events(h, ev)
    got = {nm: [] for nm in names}
    for k in range(reps + 1):
        flush.zero_()
        vc.vc_prove(h, xd, 4545 + k, tr)
        torch.cuda.synchronize()
        if k:
            for nm in names:
                i = vc.STAGES.index(nm)
                got[nm].append(ev[2 * i].elapsed_time(ev[2 * i + 1]))
    vc.vc_circuit_sync(h)
    vc.vc_circuit_set_stage_events(h, None)
    return {nm: statistics.median(v) for nm, v in got.items()}


def run_residency_deep(flush, reps=3):
    """The same comparison on the F0 circuit with 2^16 inputs (61 power
    layers of 2^17 values each): staged and windowed values need eight slots
    of device memory instead of every layer."""
    import torch
    from paper_1202_1350_gb300 import circuits, vc
    from paper_1202_1350_gb300 import inputs as I
    widths, kinds = circuits.f0(16)
    x = torch.from_numpy(I.f0_inputs(16, 0xC0FFEE + 1).view(np.int64).copy()).cuda()
    out = {"workload": "F0, 2^16 inputs (Poisson(1) capped at 2^10)"}
    trs = {}
    for name, kw in (("device", {}), ("staged", {"staged": True}), ("windowed", {"windowed": True})):
        h = vc.vc_circuit_create(widths, kinds, **kw)
        tr = torch.empty(vc.vc_transcript_len(h), dtype=torch.int64, device="cuda")
        ts = []
        for k in range(reps + 1):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            vc.vc_prove(h, x, 4444, tr)
            e1.record()
            e1.synchronize()
            if k >= 1:
                ts.append(e0.elapsed_time(e1))
        vc.vc_circuit_sync(h)
        out[name + "_prove_ms"] = statistics.median(ts)
        out[name + "_device_bytes"] = vc.vc_circuit_bytes(h)
        if name == "staged":
            out["staged_link_bytes"] = vc.vc_circuit_get_info(h)["link_bytes"]
        trs[name] = tr
        vc.vc_circuit_destroy(h)
    for name in ("staged", "windowed"):
        assert bool((trs["device"] == trs[name]).all().item()), f"{name} values changed the F0 transcript"
    out["values_bytes"] = 8 * sum(1 << s for s in widths)
    return out


def run_special_purpose(flush, shapes=((1048, 1001), (4995, 5005)), reps=3):
    """The special-purpose non-interactive F2 protocol: prover and streaming
    verifier times for a v x h grid of frequencies uniform in [0, 2^16]
    (n ~ 2^20 with h = 1001 = 7 11 13, and the paper's n ~ 25 million with
    h = 5005 = 5 7 11 13, v = 4995: Sec. 6.3's table row of 39.1 KB of verifier
    space and 78.1 KB of proof); the answer is checked against sum a_i^2.
    verify_stream_ms: the verifier fed from page-locked host memory in 16
    asynchronous absorb calls of whole rows (as rows would arrive),
    double-buffered through the device, from begin to the end's answer;
    stream_gbs: the rows' bytes over that time."""
    import torch
    from paper_1202_1350_gb300 import vc
    from paper_1202_1350_gb300 import inputs as I
    P = (1 << 61) - 1
    out = []
    for v, h in shapes:
        a = I.uniform_ints(SEED_SP + v, v * h, 1 << 16)
        ad = torch.from_numpy(a.view(np.int64)).cuda()
        proof = torch.empty(2 * h, dtype=torch.int64, device="cuda")
        ah = torch.from_numpy(a.view(np.int64)).pin_memory()
        s = vc.vc_f2sp_create(v, h)
        pt, vt, st = [], [], []
        ok = True
        parts = np.linspace(0, v, 17).astype(int)
        for k in range(reps + 1):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            vc.vc_f2sp_prove(s, ad, proof)
            t1 = time.perf_counter()
            vc.vc_f2sp_verify_begin(s, 77 + k)
            vc.vc_f2sp_verify_absorb(s, ad, 0, v)
            acc, f2 = vc.vc_f2sp_verify_end(s, proof)
            t2 = time.perf_counter()
            ok &= acc
            flush.zero_()
            torch.cuda.synchronize()
            t3 = time.perf_counter()
            vc.vc_f2sp_verify_begin(s, 177 + k)
            for x0, x1 in zip(parts[:-1], parts[1:]):  # each part its own rows: no buffer is refilled
                vc.vc_f2sp_verify_absorb_async(s, ah[x0 * h:x1 * h], int(x0), int(x1 - x0))
            acc2, f2s = vc.vc_f2sp_verify_end(s, proof)
            t4 = time.perf_counter()
            ok &= acc2 and f2s == f2
            if k >= 1:
                pt.append(1000 * (t1 - t0))
                vt.append(1000 * (t2 - t1))
                st.append(1000 * (t4 - t3))
        vc.vc_f2sp_destroy(s)
        want = int((a.astype(object) ** 2).sum()) % P
        out.append({"n": v * h, "v": v, "h": h, "prove_ms": statistics.median(pt),
                    "verify_ms": statistics.median(vt), "verify_stream_ms": statistics.median(st),
                    "stream_gbs": 8 * v * h / (statistics.median(st) / 1000) / 1e9,
                    "accepted": bool(ok), "answer_ok": f2 == want,
                    "proof_words": 2 * h, "verifier_words": v,
                    "transform_products": 2 * v * h * sum(_f2sp_factors(h))})
        del ad, ah
    return out


def run_size_sweep(flush, reps=5):
    """Prover and verifier time against input size for each of the paper's
    benchmark problems (its scaling experiment, on synthetic inputs): F2, F0,
    MatMult (n^2 outputs), pattern matching (pattern of 2^4 symbols) and the
    single-output MatMult check.  Device inputs and transcripts, L2 flushed
    before each proof, median of `reps`; the proof's transcript is checked
    by the device verifier (one pass) each time."""
    import torch
    from paper_1202_1350_gb300 import circuits, vc
    from paper_1202_1350_gb300 import inputs as I
    cases = [("f2", n, circuits.f2(n), None, lambda n=n: I.f2_inputs(n, 1 << 16, 11 + n)) for n in (10, 14, 18, 22)]
    cases += [("f0", n, circuits.f0(n), None, lambda n=n: I.f0_inputs(n, 11 + n)) for n in (8, 12, 16)]
    cases += [("matmult", 1 << n, circuits.matmult(n), None, lambda n=n: I.matmult_inputs(n, 1 << 10, 11 + n))
              for n in (4, 6, 7)]
    cases += [("pattern_match", n, circuits.pattern_match(n, 4)[:2], circuits.pattern_match(n, 4)[2],
               lambda n=n: I.pm_inputs(n, 4, 11 + n)) for n in (10, 14, 18)]
    cases += [("matmult_check", 1 << m, circuits.matmult_check(m)[:2], circuits.matmult_check(m)[2],
               lambda m=m: I.mm1_inputs(m, 11 + m)) for m in (4, 6)]
    out = []
    for fam, size, (w, k), ex, gen in cases:
        h = vc.vc_circuit_create(w, k, ex)
        x = torch.from_numpy(np.ascontiguousarray(gen()).view(np.int64).copy()).cuda()
        tr = torch.empty(vc.vc_transcript_len(h), dtype=torch.int64, device="cuda")
        pt, vt, ok = [], [], True
        for r in range(reps + 2):
            flush.zero_()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record()
            vc.vc_prove(h, x, 300 + r, tr)
            e1.record()
            ok &= vc.vc_verify(h, x, 300 + r, tr)
            e2.record()
            e2.synchronize()
            if r >= 2:
                pt.append(e0.elapsed_time(e1))
                vt.append(e1.elapsed_time(e2))
        vc.vc_circuit_sync(h)
        gates = circuits.non_input_gates(w)
        out.append({"problem": fam, "size": size, "inputs": 1 << w[-1], "gates": gates,
                    "prove_ms": statistics.median(pt), "verify_ms": statistics.median(vt),
                    "prove_gates_per_s": gates / (statistics.median(pt) / 1000), "accepted": bool(ok)})
        vc.vc_circuit_destroy(h)
    return out


def _f2sp_factors(h):
    q = []
    for pr in (3, 5, 7, 11, 13, 31, 41, 61):
        pp = 1
        while h % pr == 0:
            h //= pr
            pp *= pr
        if pp > 1:
            q.append(pp)
    return q


SEED_SP = 0xC0FFEE + 7


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ---- the oracle on the host cores ---------------------------------------------------------

def _oracle_warm(_):
    """Pool warm-up: load the oracle library and run one tiny proof."""
    sys.path.insert(0, ROOT)
    import oracle
    c = oracle.Circuit(*oracle.f2_layers(4))
    c.prove(np.arange(16, dtype=np.uint64), 1)
    return os.getpid()


def _oracle_layers(fam, logn):
    import oracle
    return {"f2": oracle.f2_layers, "f0": oracle.f0_layers, "matmult": oracle.matmult_layers}[fam](logn)


def _oracle_run(args):
    """Prove (and optionally verify) a list of jobs with the C oracle; returns
    the seconds spent in the proofs."""
    jobs, verify = args
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1202_1350_gb300 import inputs as I
    t = 0.0
    for fam, logn, seed in jobs:
        c = oracle.Circuit(*_oracle_layers(fam, logn))
        x = I.job_inputs(fam, logn, seed)
        t0 = time.perf_counter()
        tr = c.prove(x, seed & 0xFFFFFFFF)
        if verify:
            ok, _ = c.verify(x, seed & 0xFFFFFFFF, tr)
            assert ok
        t += time.perf_counter() - t0
    return t


def _oracle_pool_run(job_lists, verify):
    """Run job_lists[k] in worker k (one process per host core, spawned and
    warmed up before the clock starts); returns (wall seconds, CPU seconds)."""
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    n = len(job_lists)
    with ctx.Pool(n) as pool:
        pool.map(_oracle_warm, range(n), chunksize=1)
        t0 = time.perf_counter()
        cpu = pool.map(_oracle_run, [(jl, verify) for jl in job_lists], chunksize=1)
        wall = time.perf_counter() - t0
    return wall, sum(cpu)


def _deal(jobs, n, weight):
    """Split jobs over n workers, heaviest first to the least loaded."""
    lists, load = [[] for _ in range(n)], [0.0] * n
    for j in sorted(jobs, key=weight, reverse=True):
        k = min(range(n), key=load.__getitem__)
        lists[k].append(j)
        load[k] += weight(j)
    return [jl for jl in lists if jl]


def host_cores() -> int:
    return max(1, os.cpu_count() or 1)


def cpu_baseline(logn: int = 20, per_core: int = 2):
    """The C oracle on every host core: each process proves and verifies
    `per_core` F2 n = 2^logn instances (after a warm-up proof); value = all
    gates / the wall time of the timed phase."""
    cores = host_cores()
    jobs = [[("f2", logn, 5000 + cores * r + j) for r in range(per_core)] for j in range(cores)]
    wall, cpu = _oracle_pool_run(jobs, True)
    gates = 2 * (1 << logn) - 1
    return {"value": cores * per_core * gates / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} processes (one per host core, os.cpu_count() = {cores}), each proving and verifying "
                      f"{per_core} F2 n=2^{logn} instances with the C oracle after a warm-up proof "
                      f"({wall:.1f} s wall, {cpu:.1f} s CPU)"}


def cpu_baseline_jobs(jobs, what: str):
    """Proofs per second of the C oracle over a job list, one process per host
    core (jobs dealt heaviest first); prove only, as the GPU legs time."""
    from paper_1202_1350_gb300 import circuits
    cores = host_cores()
    weight = lambda j: float(circuits.non_input_gates(circuits.by_name(j[0], j[1])[0]))  # noqa: E731
    wall, cpu = _oracle_pool_run(_deal(jobs, cores, weight), False)
    return {"proofs_per_s": len(jobs) / wall, "jobs": len(jobs), "cores": cores, "kind": "oracle",
            "wall_s": wall, "cpu_s": cpu,
            "sample": f"{what}: {len(jobs)} proofs by the C oracle on {cores} processes (one per host core)"}


REFERENCE_BUDGET_S = 100.0
REFERENCE_MIN_LOGN = 10


def reference_logn(steps: int, warmup: int, probe_s: float, probe_logn: int = 14,
                   budget_s: float = REFERENCE_BUDGET_S, max_logn: int = 20) -> int:
    """Size of the F2 instance the reference arm proves per step: the largest
    log2 n <= max_logn whose estimated (steps + warmup) proofs fit in budget_s,
    never below REFERENCE_MIN_LOGN.  The oracle's prove + verify time grows
    linearly in n (folding prover, one MLE pass), so a step at log2 n is
    estimated from one probe proof at probe_logn, with a 25 % margin."""
    n_runs = max(1, steps + warmup)
    logn = max_logn
    while logn > REFERENCE_MIN_LOGN and n_runs * 1.25 * probe_s * 2.0 ** (logn - probe_logn) > budget_s:
        logn -= 1
    return logn


def run_reference(args):
    rank, local, world = env_rank()
    if rank != 0:
        return
    import oracle
    from paper_1202_1350_gb300 import inputs as I
    oracle.build()
    # size each step so the whole run stays within about REFERENCE_BUDGET_S
    probe = oracle.Circuit(*oracle.f2_layers(14))
    xp = I.f2_inputs(14, 1 << 16, 6999)
    t0 = time.perf_counter()
    probe.verify(xp, 1, probe.prove(xp, 1))
    logn = reference_logn(args.steps, args.warmup, time.perf_counter() - t0)
    c = oracle.Circuit(*oracle.f2_layers(logn))
    gates = 2 * (1 << logn) - 1
    times = []
    for k in range(args.warmup + args.steps):
        x = I.f2_inputs(logn, 1 << 16, 7000 + k)
        t0 = time.perf_counter()
        tr = c.prove(x, k + 1)
        ok, _ = c.verify(x, k + 1, tr)
        dt = time.perf_counter() - t0
        assert ok
        if k >= args.warmup:
            times.append(dt)
    ms = 1000 * statistics.mean(times)
    value = gates / (ms / 1000)
    sample = f"F2 n=2^{logn} prove+verify per step, single thread of the C oracle"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"F2 n=2^{logn}, x uniform in [0, 2^16], prove + verify", "gates": gates},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- the CUDA path ------------------------------------------------------------------------------

def event_recorder():
    """Record a torch CUDA event through the driver (cuEventRecord on the
    event's and stream's handles): torch's Event.record adds about 5 us of
    host time, and the start event's record is inside the timed region.
    Falls back to Event.record."""
    import ctypes
    try:
        drv = ctypes.CDLL("libcuda.so.1")
        fn = drv.cuEventRecord
        fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        fn.restype = ctypes.c_int
    except (OSError, AttributeError):
        return lambda ev, st: ev.record(st)

    def rec(ev, st):
        if not ev.cuda_event:  # torch creates the event at its first record
            ev.record(st)
        elif fn(ev.cuda_event, st.cuda_stream) != 0:
            raise RuntimeError("cuEventRecord failed")
    return rec


def e2e_pipelined(h, step, xh, n_in, tr_len, side, main, ev_start, nsteps, dist):
    """A stream of proofs from page-locked host inputs: step k's upload runs
    on a copy stream into one of two device input buffers while step k - 1
    proves and verifies from the other, and each step's transcript and accept
    bit are read back into page-locked host memory on the step's stream.
    Every step's copies are inside the timed region (host wall clock from the
    first upload to the last read-back); the per-step figure is throughput,
    not the latency of one step."""
    import torch
    from paper_1202_1350_gb300 import replicas
    copy = torch.cuda.Stream()
    xe = [torch.empty(n_in, dtype=torch.int64, device="cuda") for _ in range(2)]
    # the accept word sits after the transcript: one read-back per step
    tr = [torch.empty(tr_len + 1, dtype=torch.int64, device="cuda") for _ in range(2)]
    acc = [t[tr_len:].view(torch.int32) for t in tr]
    trh = torch.empty((nsteps, tr_len + 1), dtype=torch.int64).pin_memory()
    up = [torch.cuda.Event() for _ in range(2)]
    free = [torch.cuda.Event() for _ in range(2)]

    def run(seed0):
        for k in range(nsteps):
            b = k & 1
            if k >= 2:
                copy.wait_event(free[b])  # step k - 2 is done with buffer b
            with torch.cuda.stream(copy):
                xe[b].copy_(xh, non_blocking=True)
            up[b].record(copy)
            main.wait_event(up[b])
            ev_start.record(main)
            step(seed0 + k, ev_start, xe[b], tr[b], acc[b])
            free[b].record(main)
            trh[k].copy_(tr[b], non_blocking=True)
        main.synchronize()
        return int(trh[:, tr_len:].contiguous().view(torch.int32)[:, 0].sum()) == nsteps

    assert run(7000)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ok = run(8000)
    ms = 1000 * (time.perf_counter() - t0) / nsteps
    assert ok, "a pipelined proof was rejected"
    ms = replicas.max_over_ranks(ms, dist, "cuda")
    return {"ms_per_step": ms, "steps": nsteps, "h2d_bytes_per_step": n_in * 8, "d2h_bytes_per_step": (tr_len + 1) * 8,
            "note": "throughput of a stream of proofs with each step's upload overlapping the previous step's "
                    "proof; not the latency of one step (the `modes` above)"}


def run_ours(args):
    import torch
    from paper_1202_1350_gb300 import build as vcbuild
    from paper_1202_1350_gb300 import circuits, vc
    from paper_1202_1350_gb300 import inputs as I

    rank, local, world = env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    vcbuild.build()
    fam, logn, gen, seed0 = I.WORKLOADS[WORKLOAD]
    widths, kinds = circuits.by_name(fam, logn)
    gates = circuits.non_input_gates(widths)
    h = vc.vc_circuit_create(widths, kinds, None, local)
    info = vc.vc_circuit_get_info(h)
    from paper_1202_1350_gb300 import replicas
    x = gen(replicas.replica_seed(seed0, rank))
    xd = torch.from_numpy(x.view(np.int64).copy()).cuda()
    tr = torch.empty(info["transcript_len"], dtype=torch.int64, device="cuda")
    acc = torch.zeros(1, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 8, dtype=torch.int64, device="cuda")
    # the timed region records only the dominant launch's two events (each
    # recorded event costs device time); the stage breakdown is a separate pass
    iw = vc.STAGES.index("waves")
    wave_ev = [None] * (2 * vc.NUM_STAGES)
    wave_ev[2 * iw] = torch.cuda.Event(enable_timing=True)
    wave_ev[2 * iw + 1] = torch.cuda.Event(enable_timing=True)
    vc.vc_circuit_set_stage_events(h, wave_ev)

    main = torch.cuda.current_stream()
    side = torch.cuda.Stream()
    ev_start, ev_input = torch.cuda.Event(), torch.cuda.Event()

    def step(seed, start, x=xd, t=tr, a=acc):
        # the proof on the main stream; the verifier's input pass (its coins and
        # the inputs' MLE at the final point, fixed by the seed alone) beside it
        # on a second stream, from the step's start event `start` on; then the
        # transcript pass
        vc.vc_prove(h, x, seed, t)
        side.wait_event(start)
        vc.vc_verify_input(h, x, seed, stream=side)
        ev_input.record(side)
        main.wait_event(ev_input)
        return vc.vc_verify_transcript(h, seed, t, accept=a)

    for w in range(args.warmup):
        flush.zero_()
        ev_start.record(main)
        step(100 + w, ev_start)
    torch.cuda.synchronize()
    vc.vc_circuit_sync(h)
    assert int(acc.item()) == 1, "warm-up proof rejected"

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    # the timed steps take a few ms, less than the sampler's period: the same
    # step runs untimed for 0.5 s first, so that the samples see the clocks
    # under this load right up to the timed region
    t_soak = time.perf_counter()
    k = 0
    while time.perf_counter() - t_soak < 0.5:
        flush.zero_()
        ev_start.record(main)
        step(5000 + k, ev_start)
        k += 1
        if k % 64 == 0:
            main.synchronize()
    torch.cuda.synchronize()
    vc.vc_circuit_sync(h)
    step_ms, wave_ms = [], []
    oks = 0
    rec = event_recorder()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for e0, e1 in evs:  # create the events outside the timed region
        e0.record(main)
        e1.record(main)
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()
        e0, e1 = evs[k]
        rec(e0, main)
        step(1 + k, e0)
        rec(e1, main)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        wave_ms.append(wave_ev[2 * iw].elapsed_time(wave_ev[2 * iw + 1]))
        oks += int(acc.item())
    torch.cuda.synchronize()
    clocks = sampler.stop()
    vc.vc_circuit_sync(h)
    assert oks == args.steps, "a timed proof was rejected"
    total_ms = replicas.max_over_ranks(sum(step_ms), dist, "cuda")
    ms_per_step = total_ms / args.steps
    value = replicas.whole_job_rate(gates * args.steps, world, total_ms / 1000)

    # end to end through the C ABI with pinned host buffers
    xh = torch.from_numpy(x.view(np.int64).copy()).pin_memory()
    # the e2e steps' transcript with the accept word after it: one read-back
    ntr = info["transcript_len"]
    trx = torch.empty(ntr + 1, dtype=torch.int64, device="cuda")
    accx = trx[ntr:].view(torch.int32)
    trh = torch.empty(ntr + 1, dtype=torch.int64).pin_memory()
    # stage breakdown (diagnostic, outside the timed region): every stage's events
    stage_ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * vc.NUM_STAGES)]
    vc.vc_circuit_set_stage_events(h, stage_ev)
    stage_ms = {}
    for k in range(5):
        flush.zero_()
        vc.vc_prove(h, xd, 900 + k, tr)
        torch.cuda.synchronize()
        if k >= 2:
            for i, name in enumerate(vc.STAGES):
                if name in ("wavesn", "build", "tabwaves"):  # no work in SQUARE/TREE circuits
                    continue
                try:
                    stage_ms.setdefault(name, []).append(stage_ev[2 * i].elapsed_time(stage_ev[2 * i + 1]))
                except RuntimeError:  # a stage with no work records nothing
                    pass
    vc.vc_circuit_set_stage_events(h, None)
    ablation = residency = special = size_sweep = None
    if not args.no_ablation:
        ablation = run_ablation(h, xd, tr, flush)
        residency = run_residency(widths, kinds, xd, flush)
        residency["deep"] = run_residency_deep(flush)
        special = run_special_purpose(flush)
        size_sweep = run_size_sweep(flush)
    # end to end from page-locked host memory, four ways; each step ends with
    # the transcript and the accept bit read back into page-locked host
    # memory.  "upload": the C ABI gets the host inputs and copies them itself
    # (a circuit created with VC_INPUTS_UPLOAD): the prover's upload comes
    # first, the verifier's input pass uploads its own copy on a second stream
    # from the end of the evaluation stage on, beside the sum-check waves.
    # "upload_one_call": the same circuit through vc_prove_verify: one upload
    # into the input layer, which the prover and the verifier both read, and
    # one graph launch.  "copy": the caller uploads the inputs once (torch)
    # and the prover and the verifier's input pass both read that device
    # copy.  "in_place" (vc_prove_verify): nothing is copied; the prover's
    # first evaluation launch reads the inputs across the host link where they
    # lie, and the verifier's input pass reads them again, so the inputs cross
    # the link twice.  The fastest is reported; all are measured.
    xe = torch.empty_like(xd)
    ev_eval = torch.cuda.Event()
    e2e_ev = [None] * (2 * vc.NUM_STAGES)
    e2e_ev[2 * vc.STAGES.index("eval") + 1] = ev_eval
    h_up = vc.vc_circuit_create(widths, kinds, upload=True)
    vc.vc_circuit_set_stage_events(h_up, e2e_ev)

    def e2e_upload(seed):
        vc.vc_prove(h_up, xh, seed, trx)  # asynchronous: uploads, then proves
        side.wait_event(ev_eval)
        vc.vc_verify_input(h_up, xh, seed, stream=side)
        ev_input.record(side)
        main.wait_event(ev_input)
        vc.vc_verify_transcript(h_up, seed, trx, accept=accx)

    def e2e_upload_one_call(seed):
        vc.vc_prove_verify(h_up, xh, seed, trx, accept=accx)  # asynchronous

    def e2e_copy(seed):
        xe.copy_(xh, non_blocking=True)
        ev_start.record(main)
        step(seed, ev_start, xe, trx, accx)

    def e2e_in_place(seed):
        vc.vc_prove_verify(h, xh, seed, trx, accept=accx)  # asynchronous: inputs read in place

    def e2e_time(run, hh=h):
        def one(seed):
            run(seed)
            trh.copy_(trx, non_blocking=True)
            main.synchronize()
            return int(trh[ntr:].view(torch.int32)[0]) == 1
        assert one(999) and one(998)
        ms = []
        for k in range(max(5, args.steps)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ok = one(500 + k)
            ms.append(1000 * (time.perf_counter() - t0))
            assert ok
        vc.vc_circuit_sync(hh)
        return replicas.max_over_ranks(statistics.mean(ms), dist, "cuda")

    n_in, tr_bytes = 1 << widths[-1], (ntr + 1) * 8
    modes = {"upload": {"ms_per_step": e2e_time(e2e_upload, h_up), "h2d_bytes_per_step": 2 * n_in * 8}}
    vc.vc_circuit_set_stage_events(h_up, None)
    modes["upload_one_call"] = {"ms_per_step": e2e_time(e2e_upload_one_call, h_up), "h2d_bytes_per_step": n_in * 8}
    modes["copy"] = {"ms_per_step": e2e_time(e2e_copy), "h2d_bytes_per_step": n_in * 8}
    vc.vc_circuit_destroy(h_up)
    modes["in_place"] = {"ms_per_step": e2e_time(e2e_in_place), "h2d_bytes_per_step": 2 * n_in * 8}
    best = min(modes, key=lambda m: modes[m]["ms_per_step"])
    e2e = {"value": world * gates / (modes[best]["ms_per_step"] / 1000), "unit": UNIT,
           "h2d_bytes_per_step": modes[best]["h2d_bytes_per_step"], "d2h_bytes_per_step": tr_bytes,
           "ms_per_step": modes[best]["ms_per_step"], "mode": best, "modes": modes,
           "pipelined": e2e_pipelined(h, step, xh, x.size, info["transcript_len"], side, main, ev_start,
                                      max(8, args.steps), dist)}

    if rank != 0:
        vc.vc_circuit_destroy(h)
        if dist:
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel: the first persistent wave launch,
    # which runs every sum-check round and line reduction of the F2 circuit
    wave_launch_ms = statistics.mean(wave_ms)
    mul, byts = algorithmic_work(widths, kinds)
    executed = executed_work(widths, kinds, vc.vc_circuit_get_tiles(h)["gn_chunk_log"])
    rate = vc.vc_field_mul_rate(local, 2, 1 << 12)
    achieved = mul / (wave_launch_ms / 1000)
    stages = {name: round(statistics.mean(v), 4) for name, v in stage_ms.items()}
    launches = (info["prove_launches"] + info["verify2_launches"]) * args.steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "F2 n=2^20, x uniform in [0, 2^16], prove + verify per step",
                   "gates": gates, "transcript_u64": info["transcript_len"], "rounds": info["n_rounds"],
                   "l2": "flushed between steps (256 MiB write outside the step events)",
                   "clock_sampling": "nvidia-smi every 100 ms over 0.5 s of the same step run untimed right before "
                                     "the timed steps, and over them; SM clock median over the busy samples",
                   "parallelism": f"replicas x{world}"},
        "e2e": e2e,
        "roofline": {"bound": "alu", "kernel": "k_waves (persistent launch: every sum-check round and line "
                                                "reduction of the F2 circuit)",
                     "achieved": achieved / 1e12, "peak": rate / 1e12, "unit": "Tmulmod/s",
                     "frac": achieved / rate, "traffic": K_WAVES_DRAM_BYTES,
                     "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                     "peak_source": "measured on this GPU: vc_field_mul_rate variant 2, the kernel's own "
                                    "pair step (2 exact multiply-adds + 1 lazy fold), best of 5 chain-count and "
                                    "register-budget configurations on a one-wave grid; ncu shows that step keeps "
                                    "the integer-multiply (fmaheavy) pipe 83-86 % of its cycles busy "
                                    "(profiles/int_rate_microbench.md)",
                     "peak_pipe_saturated": rate / PAIR_STEP_FMAHEAVY_FRAC / 1e12,
                     "frac_of_pipe_saturated": achieved / (rate / PAIR_STEP_FMAHEAVY_FRAC),
                     "kernel_pipes_ncu": K_WAVES_PIPES,
                     "algorithmic_mulmods": mul, "algorithmic_rule": "7 S_i + 24 S_{i+1} per layer (folding prover)",
                     "executed_mulmods": executed, "executed_frac": executed / (wave_launch_ms / 1000) / rate,
                     "algorithmic_bytes": byts, "kernel_ms": wave_launch_ms,
                     "bytes_frac_of_hbm": (byts / (wave_launch_ms / 1000)) / (measured_peaks().get("hbm_gbs", 6787.9) * 1e9)},
        "stage_ms": stages,
        "ablation": ablation,
        "residency": residency,
        "special_purpose_f2": special,
        "size_sweep": size_sweep,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    # serving first: the batch leg runs the autotuner, whose per-class tile
    # shapes every later circuit of those classes in this process would use
    if not args.no_serve:
        line["serving"] = run_serving(local)
    if not args.no_batch:
        line["batched"] = run_batch(local)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
        if "batched" in line:
            line["batched"]["cpu_baseline"] = cpu_baseline_jobs(I.batch_mix(), "the batched workload (every job)")
        if "serving" in line:
            line["serving"]["cpu_baseline"] = cpu_baseline_jobs(
                I.serving_mix(0xC0FFEE + 6, 64), "the first 64 jobs of the serving mix's closed-loop trace")
    print(json.dumps(line), flush=True)
    vc.vc_circuit_destroy(h)
    if dist:
        dist.destroy_process_group()


# ---- batched proving (576 independent circuits of uneven sizes) -----------------------------

def run_batch(local: int, reps: int = 5):
    """512 F2 circuits (log2 n uniform in [8, 18]) and 64 MatMult circuits
    (n in {16, 32, 64}) proved as one batch (merged launches, CUDA graph)
    against the same proofs one at a time (vc_prove per circuit, each its own
    graph) on one stream.  Inputs and transcripts resident in HBM.  The tile
    shapes are the autotuner's: vc_autotune_batch searches one configuration
    for the whole mix by timing the merged batch itself and records it for
    every member's size class, so the circuits built afterwards use it.  The
    same batch with each circuit's default shapes is timed first, for
    comparison."""
    import torch
    from paper_1202_1350_gb300 import circuits, vc
    from paper_1202_1350_gb300 import inputs as I

    jobs = I.batch_mix()
    xs = [torch.from_numpy(I.job_inputs(fam, logn, seed).view(np.int64).copy()).cuda() for fam, logn, seed in jobs]
    gates = sum(circuits.non_input_gates(circuits.by_name(fam, logn)[0]) for fam, logn, _ in jobs)
    n = len(jobs)
    seeds = list(range(1, n + 1))

    def build():
        hs = [vc.vc_circuit_create(*circuits.by_name(fam, logn), None, local) for fam, logn, _ in jobs]
        trs = [torch.empty(vc.vc_transcript_len(h), dtype=torch.int64, device="cuda") for h in hs]
        return hs, trs, vc.vc_batch_create(hs)

    def destroy(hs, b):
        vc.vc_batch_destroy(b)
        for h in hs:
            vc.vc_circuit_destroy(h)

    def time_batch(b, trs):
        for _ in range(3):
            vc.vc_batch_prove(b, xs, seeds, trs)
        vc.vc_batch_sync(b)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for r in range(reps):
            vc.vc_batch_prove(b, xs, [s + 1000 * r for s in seeds], trs)
        e1.record()
        e1.synchronize()
        vc.vc_batch_sync(b)
        return e0.elapsed_time(e1) / reps

    # each circuit's default tile shapes (no size class tuned yet in this process)
    hs, trs, b = build()
    default_tiles = vc.vc_circuit_get_tiles(hs[0])
    times = {"default": time_batch(b, trs)}
    destroy(hs, b)
    t0 = time.perf_counter()
    tuned, tuned_ms = vc.vc_autotune_batch([circuits.by_name(fam, logn) for fam, logn, _ in jobs], local, reps=3)
    tune_s = time.perf_counter() - t0
    hs, trs, b = build()  # the circuits take the recorded configuration
    assert vc.vc_circuit_get_tiles(hs[0]) == tuned
    times["autotuned"] = time_batch(b, trs)
    batch_ms = times["autotuned"]
    info = vc.vc_batch_get_info(b)
    try:
        # spot-check: the batched transcript of job 0 equals its standalone proof
        ref = torch.empty_like(trs[0])
        vc.vc_prove(hs[0], xs[0], seeds[0] + 1000 * (reps - 1), ref)
        vc.vc_circuit_sync(hs[0])
        same = bool(torch.equal(ref, trs[0]))
        # one at a time
        for j in range(n):
            vc.vc_prove(hs[j], xs[j], seeds[j], trs[j])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for r in range(max(1, reps // 2)):
            for j in range(n):
                vc.vc_prove(hs[j], xs[j], seeds[j] + r, trs[j])
        e1.record()
        e1.synchronize()
        single_ms = e0.elapsed_time(e1) / max(1, reps // 2)
        for h in hs:
            vc.vc_circuit_sync(h)
    finally:
        destroy(hs, b)
    return {"workload": "512 F2 (log2 n uniform in [8,18], x uniform in [0,2^16]) + 64 MatMult "
                        "(n in {16,32,64}, entries uniform in [0,2^10]), inputs resident in HBM",
            "proofs_per_s": n / (batch_ms / 1000), "gates_per_s": gates / (batch_ms / 1000),
            "ms_per_batch": batch_ms, "jobs": n, "gates_per_batch": gates,
            "launches_per_batch": info["prove_launches"],
            "one_at_a_time_proofs_per_s": n / (single_ms / 1000), "one_at_a_time_ms": single_ms,
            "speedup_vs_one_at_a_time": single_ms / batch_ms, "batched_equals_standalone": same,
            "reps": reps, "tiles": "autotuned (vc_autotune_batch on this batch)",
            "ms_per_batch_by_tiles": times, "default_tiles": default_tiles, "autotuned_tiles": tuned,
            "autotune_s": tune_s, "autotune_ms_per_batch": tuned_ms}


# ---- serving: Poisson arrivals into the proof server ---------------------------------------

def run_serving(local: int, seconds_per_rate: float = 1.5, repeats: int = 3):
    """70% F2 (log2 n uniform in [10, 22]) and 30% MatMult (n in {32, 64, 128})
    jobs submitted to vc_server (admission cap 150 GB, continuous batching);
    inputs resident in HBM, one input vector per shape.  Jobs are submitted
    from this thread and collected (vc_server_wait, in submission order) by a
    second one, so collection never delays a submission.  Saturation: a closed
    loop keeps max_inflight x max_batch x 16 jobs outstanding (a queue deep
    enough that every launch set is formed from a full choice of jobs, as
    under overload); its rate over windows of 1000 completions, after the
    first window, is the saturated throughput.  Then Poisson arrivals at 0.5x, 0.9x and 1.2x of it, each rate
    `repeats` times with other seeds: proofs/s and p50/p99 latency (submit to
    transcript written, on the server's own clock)."""
    import queue
    import threading

    import torch
    from paper_1202_1350_gb300 import Server, circuits
    from paper_1202_1350_gb300 import inputs as I

    shapes = {}
    for logn in range(10, 23):
        shapes[("f2", logn)] = circuits.f2(logn)
    for logn in (5, 6, 7):
        shapes[("matmult", logn)] = circuits.matmult(logn)
    xin = {k: torch.from_numpy(I.job_inputs(k[0], k[1], 11 + k[1]).view(np.int64).copy()).cuda() for k in shapes}
    trl = {k: circuits.transcript_len(w) for k, (w, _) in shapes.items()}
    gates = {k: circuits.non_input_gates(w) for k, (w, _) in shapes.items()}
    max_batch, max_inflight = 16, 4
    srv = Server(local, mem_cap_bytes=150 << 30, max_batch=max_batch, max_inflight=max_inflight)

    def run(jobs, arrivals=None, outstanding=None):
        trbuf = torch.empty(sum(trl[(f, n)] for f, n, _ in jobs), dtype=torch.int64, device="cuda")
        q = queue.Queue()
        infos = []
        slots = threading.Semaphore(outstanding) if outstanding else None

        def collect():
            while True:
                jid = q.get()
                if jid is None:
                    return
                infos.append(srv.wait(jid))
                if slots:
                    slots.release()

        th = threading.Thread(target=collect)
        th.start()
        off = 0
        t0 = time.perf_counter()
        for k, (fam, logn, seed) in enumerate(jobs):
            if arrivals is not None:
                wait = arrivals[k] - (time.perf_counter() - t0)
                if wait > 2e-4:
                    time.sleep(wait - 1e-4)
                while time.perf_counter() - t0 < arrivals[k]:
                    pass
            if slots:
                slots.acquire()
            w, kinds = shapes[(fam, logn)]
            n = trl[(fam, logn)]
            q.put(srv.submit(w, kinds, xin[(fam, logn)], seed, trbuf[off:off + n]))
            off += n
        q.put(None)
        th.join()
        assert all(i["status"] == 0 for i in infos)
        lat = np.array([(i["done_ns"] - i["submit_ns"]) / 1e6 for i in infos])
        span = (max(i["done_ns"] for i in infos) - min(i["submit_ns"] for i in infos)) / 1e9
        g = sum(gates[(f, n)] for f, n, _ in jobs)
        return {"proofs_per_s": len(jobs) / span, "gates_per_s": g / span, "jobs": len(jobs),
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean())}, infos

    def windows(infos, size=1000):
        done = np.sort(np.array([i["done_ns"] for i in infos], dtype=np.float64))
        rates = []
        for a in range(0, len(done) - size, size):
            rates.append(size / ((done[a + size] - done[a]) / 1e9))
        return rates

    try:
        warm = I.serving_mix(0xC0FFEE + 5, 1500)
        run(warm, outstanding=2 * max_batch * max_inflight)  # fills the circuit pool
        closed = I.serving_mix(0xC0FFEE + 6, 10000)
        sat, infos = run(closed, outstanding=16 * max_batch * max_inflight)
        win = windows(infos)
        sat["window_proofs_per_s"] = win
        sat["outstanding"] = 16 * max_batch * max_inflight
        sat_rate = float(np.median(win[1:])) if len(win) > 1 else sat["proofs_per_s"]
        sat["saturated_proofs_per_s"] = sat_rate
        if len(win) > 1:
            sat["saturated_proofs_per_s_range"] = [float(min(win[1:])), float(max(win[1:]))]
        rates = []
        for mult in (0.5, 0.9, 1.2):
            rate = mult * sat_rate
            n = int(min(30000, max(300, rate * seconds_per_rate)))
            reps = []
            for r in range(repeats):
                jobs = I.serving_mix(0xC0FFEE + 5 + int(mult * 10) + 100 * r, n)
                arr = I.poisson_arrivals(0xC0FFEE + int(mult * 10) + 100 * r, n, rate)
                res, _ = run(jobs, arrivals=arr)
                reps.append(res)
            summ = {"load": mult, "offered_per_s": rate, "jobs_per_repeat": n, "repeats": reps}
            for key in ("proofs_per_s", "p50_ms", "p99_ms"):
                vals = [x[key] for x in reps]
                summ[key] = float(np.median(vals))
                summ[key + "_range"] = [float(min(vals)), float(max(vals))]
            rates.append(summ)
        st = srv.stats()
    finally:
        srv.close()
    return {"workload": "Poisson arrivals; 70% F2 (log2 n uniform in [10,22], x uniform in [0,2^16]), "
                        "30% MatMult (n in {32,64,128}); admission cap 150 GB; inputs resident in HBM",
            "saturated": sat, "rates": rates,
            "server": {"max_batch": max_batch, "max_inflight": max_inflight, "launch_sets": st["launch_sets"],
                       "max_jobs_in_flight": st["max_jobs_in_flight"], "circuits": st["circuits_created"],
                       "peak_held_gb": st["peak_held_bytes"] / 1e9}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-ablation", action="store_true",
                    help="skip the per-gate prover, host-residency and special-purpose protocol measurements")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-workload measurement")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--residency-only", action="store_true",
                    help="print only the residency comparison on the F2 n=2^20 workload (for profiling it)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.residency_only:
        run_residency_only()
    else:
        run_ours(args)


def run_residency_only():
    import torch
    from paper_1202_1350_gb300 import build as vcbuild
    from paper_1202_1350_gb300 import circuits
    from paper_1202_1350_gb300 import inputs as I
    vcbuild.build()
    fam, logn, gen, seed0 = I.WORKLOADS[WORKLOAD]
    widths, kinds = circuits.by_name(fam, logn)
    xd = torch.from_numpy(gen(seed0).view(np.int64).copy()).cuda()
    flush = torch.empty(256 * 1024 * 1024 // 8, dtype=torch.int64, device="cuda")
    print(json.dumps(run_residency(widths, kinds, xd, flush)), flush=True)


if __name__ == "__main__":
    main()
