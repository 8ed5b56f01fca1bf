#!/usr/bin/env python3
"""Benchmark: two-vector Four-Russians Nussinov folding on one B300 per rank.

Prints ONE JSON line (rank 0).  The headline is DP cells/s of one fold of a
single n = 6000 uniform-ACGU sequence (q = 8, pair set AU UA CG GC GU UG),
device-resident inputs, L2 flushed between steps; beside it the plain
Nussinov kernel on the same input, the end-to-end host-buffer call, batched
and served throughput, the lookup roofline of the persistent kernel, SM
clocks sampled during the timed region, and the CPU oracle baseline.

A step is one complete fold (every cell of the table).  With --gpus N > 1
(torchrun, one rank per GPU) every rank folds its own replica of the
workload (a single fold does not shard); value = all ranks' cells / max time.

--impl reference times the CPU oracle (the plain cubic recurrence) on the
host cores instead: every timed step folds the whole input once.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DP cells/s at n=6000 vs plain GPU Nussinov; batched seq/s; serve p50/p99 ms"
UNIT = "cells/s"
L2_FLUSH_BYTES = 256 << 20


DRAM_PROFILE = os.path.join(ROOT, "profiles", "fold_kernel_n6000_dram.md")


# the sources that make a single two-vector q = 8 fold launch: the kernel and its q = 8
# instantiation, the task list and the work-split planner (serving, batch plans, the other methods
# and the benchmarks of the library do not change it)
KERNEL_SOURCES = ("api.cu", "api_internal.h", "fold_column.cuh", "fold_common.h", "fold_inst_tv8.cu", "fold_kernel.cu",
                  "fold_kernel.cuh", "kernels.h", "schedule.cpp", "schedule.h")


def kernel_source_hash() -> str:
    """sha256 over the sources of the two-vector fold launch, in name order."""
    h = hashlib.sha256()
    for name in sorted(KERNEL_SOURCES):
        path = os.path.join(ROOT, "paper_1307_7820_b300", "csrc", name)
        h.update(name.encode())
        with open(path, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(n: int, q: int):
    """DRAM bytes per launch of the two-vector fold kernel from the committed ncu summary, or None
    when that summary was taken on other sources (the kernel changed since) or another workload."""
    try:
        text = open(DRAM_PROFILE).read()
    except OSError:
        return None
    got = dict(re.findall(r"^- (\w+): (\S+)$", text, re.M))
    if got.get("source_sha256") != kernel_source_hash() or got.get("workload") != f"n{n}_q{q}":
        return None
    try:
        return float(got["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def hbm_peak_gbs() -> float:
    """Measured HBM copy bandwidth of the B300s (MEASURED_PEAKS.json), else the fallback."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6400.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=6000)
    ap.add_argument("--q", type=int, default=8)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-qsweep", action="store_true")
    ap.add_argument("--no-sliding", action="store_true", help="skip Section 4's per-column organisation")
    ap.add_argument("--trace", default="", help="write a per-task trace of one fold to this .npy file")
    ap.add_argument("--no-sizes", action="store_true", help="skip the single-fold size sweep")
    ap.add_argument("--serve-rates", default="50,100,200,500,1000,2000",
                    help="Poisson arrival rates (req/s) for the serving run")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="arrival window per rate (cut to --serve-requests requests at high rates)")
    ap.add_argument("--serve-requests", type=int, default=2000, help="requests per rate at most")
    return ap.parse_args()


def workload_config(a):
    return {
        "workload": f"single RNA sequence n={a.n}, i.i.d. uniform ACGU (seed 1308), pair set AU,UA,CG,GC,GU,UG, "
                    f"no minimum hairpin, two-vector q={a.q}, int16 D (row-major; a column-major copy where a "
                    f"kernel reads columns)",
        "n": a.n,
        "q": a.q,
        "pair_mask": "0x5A48",
        "seed": 1308,
        "l2": "flushed between timed steps by a 256 MiB device write outside the timed events",
        "launch": "a ~0.1 ms device spin precedes each timed step's first event, so that the step's launches "
                  "are queued when the device reaches it (the host's enqueue time is in e2e, not in value)",
        "replicas": "each rank folds its own copy (a single fold does not shard)",
    }


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
                power.append(float(p[3]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "power_w_max": max(power),
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ CPU side
# The paper's own figures (Section 6), with the hardware it states: context only.
PAPER_FIGURES = {
    "gpu_tesla_c2070_s_at_6000": 2.50,
    "gpu_geforce_gtx550ti_s_at_6000": 4.97,
    "serial_two_vector_desktop_s_at_6150": round(1027.8 / 18.1, 1),
    "serial_nussinov_desktop_s_at_6150": 1027.8,
    "serial_two_vector_server_s_at_6000": 15,
    "desktop": "Pentium II 3 GHz, 1 MB cache (as the paper states); the server is not described",
    "note": "the paper's times on its own hardware; not this metric on this workload",
}


def host_info():
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    try:
        usable = len(os.sched_getaffinity(0))
    except AttributeError:
        usable = os.cpu_count()
    return {"cpu_model": model, "cpu_count": os.cpu_count(), "cpus_usable": usable}


def cpu_oracle_fold(seq: str):
    """Seconds of one whole fold of seq by the CPU oracle (single-threaded C, Eq. 1), and its answer."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    mp = oracle.score(seq)
    return time.perf_counter() - t0, mp


def cpu_two_vector_fold(seq: str, q: int, threads: int):
    """Seconds of one whole fold by the multi-threaded CPU two-vector program, answer, threads used."""
    import baseline
    baseline.build()
    t0 = time.perf_counter()
    mp, _, _, used = baseline.fold(seq, q=q, threads=threads)
    return time.perf_counter() - t0, mp, used


def run_reference(a):
    """--impl reference: the CPU oracle as it stands, on the host cores; every timed step is one
    whole fold of the workload's input (warm-up steps fold a 1000-base prefix: there is nothing to
    warm in a CPU program beyond its code and pages)."""
    from paper_1307_7820_b300 import metrics, synth
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    seq = synth.uniform(a.n, 1308)
    for _ in range(a.warmup):
        cpu_oracle_fold(seq[:1000])
    times = []
    answers = set()
    for _ in range(a.steps):
        dt, mp = cpu_oracle_fold(seq)
        times.append(dt)
        answers.add(mp)
    assert len(answers) == 1
    ms = 1e3 * statistics.mean(times)
    value = metrics.cells(a.n) / (ms * 1e-3)
    sample = (f"every timed step folds the whole n={a.n} input once with the cubic oracle (single-threaded C, "
              f"Eq. 1); measured, not scaled; warm-up steps fold its first 1000 bases")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic", "config": workload_config(a),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         **host_info()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "max_pairs": answers.pop(), "paper": PAPER_FIGURES,
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ serving
def serve_bench(f, rates, seconds, max_requests, dev, stream, torch, fold, metrics, synth):
    """Continuous batching under Poisson arrivals vs folding the same requests one at a time."""
    import threading
    out = []
    budget = 60 << 30
    # warm-up: the task lists of every request length in the range are built before the arrivals
    tw = time.perf_counter()
    fold.fold_serve_warm(f.ctx, 8000)
    warm_s = time.perf_counter() - tw
    ws = torch.empty(f.workspace_bytes(8000), dtype=torch.uint8, device=dev)
    o = torch.zeros(1, dtype=torch.int32, device=dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for ri, rate in enumerate(rates):
        count = max(8, min(int(rate * seconds), max_requests))
        reqs = synth.serve_requests(rate, count, 50, 8000, synth.SEED_BASE + 4 + ri)
        fold.fold_serve_start(f.ctx, budget, 4096)
        submit_t = {}
        done_t = {}
        t2k = {}   # ticket -> request index, written by the submitter
        t0 = time.perf_counter()

        def submitter():
            for k, (at, s, _) in enumerate(reqs):
                while time.perf_counter() - t0 < at:
                    time.sleep(0.0002)
                submit_t[k] = time.perf_counter()
                while True:
                    try:
                        t2k[fold.fold_serve_submit(f.ctx, s)] = k
                        break
                    except fold.FoldError as e:
                        if e.code != fold.FOLD_EAGAIN:
                            raise
                        time.sleep(0.001)

        th = threading.Thread(target=submitter)
        th.start()
        results = {}
        seen = {}   # finished tickets -> time reported (kept until the submitter has recorded them)
        while len(results) < count:
            # blocks (GIL released) until the server reports a finished request
            t = fold.fold_serve_wait_any(f.ctx, 50)
            if t is not None:
                seen[t] = time.perf_counter()
            for t, tdone in list(seen.items()):
                k = t2k.get(t)
                if k is None:
                    continue
                results[k] = fold.fold_serve_poll(f.ctx, t)
                done_t[k] = tdone
                del seen[t]
        th.join()
        wall = max(done_t.values()) - t0
        st = fold.fold_serve_stats(f.ctx)
        fold.fold_serve_stop(f.ctx)
        lat = np.array([1e3 * (done_t[k] - submit_t[k]) for k in range(count)])
        # one at a time: the device time of every request folded alone (single-fold path, one
        # reused workspace); results must agree with the served ones
        alone_s = 0.0
        for k in range(count):
            s = reqs[k][1]
            codes = torch.from_numpy(fold.encode_codes(s)).to(dev)
            torch.cuda.synchronize()
            e0.record(stream)
            f.score_dev(codes, ws, o, None, stream=stream.cuda_stream)
            e1.record(stream)
            e1.synchronize()
            alone_s += e0.elapsed_time(e1) / 1e3
            assert (int(o.item()) if len(s) else 0) == results[k]
        cells = sum(metrics.cells(len(r[1])) for r in reqs)
        out.append({"rate_req_s": rate, "requests": count, "p50_ms": float(np.percentile(lat, 50)),
                    "p99_ms": float(np.percentile(lat, 99)), "throughput_req_s": count / wall,
                    "throughput_cells_s": cells / wall,
                    "one_at_a_time_req_s": count / alone_s,
                    "one_at_a_time_note": "device time of every request folded alone, back to back",
                    "slices": st["slices"], "solo": st["solo"], "tasks_per_slice": st["tasks"] / max(1, st["slices"]),
                    "gpu_busy": st["gpu_ms"] / (1e3 * wall), "host_prep_ms": st["prep_ms"],
                    "window_s": float(reqs[-1][0]),
                    "lengths": "log-uniform [50, 8000]; 80% uniform, 10% GC-rich, 10% structured",
                    "budget_bytes": budget, "warm_s": warm_s})
    return out


# ------------------------------------------------------------------ GPU side
def main():
    a = parse_args()
    if a.impl == "reference":
        return run_reference(a)

    import torch
    from paper_1307_7820_b300 import fold, metrics, ranks, synth

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rk = ranks.Ranks(backend="nccl", device=dev)
    world, rank = rk.world, rk.rank
    torch.cuda.set_device(dev)
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count

    def barrier_sync():
        torch.cuda.synchronize()
        rk.barrier()
        torch.cuda.synchronize()

    max_over_ranks = rk.max

    n, q = a.n, a.q
    seq = synth.uniform(n, 1308)
    cells = metrics.cells(n)
    lam = metrics.lookups(n, q)

    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def make(method):
        f = fold.Folder(q=q, method=method, device=local)
        f.option(fold.FOLD_OPT_TIMING, 1)
        return f

    def queue_ahead():
        # outside the timed events: the device spins ~0.1 ms while the host enqueues the step, so the
        # events bracket device work only (torch's spin kernel; the host path is timed by e2e)
        torch.cuda._sleep(200_000)

    def device_run(f, steps, warmup, sampler=None):
        codes = torch.from_numpy(fold.encode_codes(seq)).to(dev)
        ws = torch.empty(f.workspace_bytes(n), dtype=torch.uint8, device=dev)
        out = torch.zeros(1, dtype=torch.int32, device=dev)
        torch.cuda.synchronize()
        for _ in range(warmup):
            with torch.cuda.stream(stream):
                f.score_dev(codes, ws, out, None, stream=stream.cuda_stream)
        barrier_sync()
        if sampler:
            sampler.start()
        l0 = f.launches
        step_ms, kern_ms = [], []
        barrier_sync()
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                queue_ahead()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                f.score_dev(codes, ws, out, None, stream=stream.cuda_stream)
                e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            kern_ms.append(f.option(fold.FOLD_OPT_KERNEL_NS) / 1e6)
        barrier_sync()
        clocks = sampler.stop() if sampler else None
        launches = f.launches - l0
        return {"step_ms": step_ms, "kern_ms": kern_ms, "max_pairs": int(out.item()), "launches": launches,
                "clocks": clocks}

    # ---- headline: two-vector fold, device-resident
    tv = make("two_vector")
    sampler = ClockSampler(local)
    r_tv = device_run(tv, a.steps, a.warmup, sampler)
    total_ms = max_over_ranks(sum(r_tv["step_ms"]))
    ms_per_step = total_ms / a.steps
    value = world * cells / (ms_per_step * 1e-3)
    kern_ms = statistics.mean(r_tv["kern_ms"])

    # ---- plain comparison kernel, same input and procedure
    pl = make("plain")
    r_pl = device_run(pl, max(3, a.steps // 4), a.warmup)
    pl_ms = statistics.mean(r_pl["step_ms"])
    assert r_pl["max_pairs"] == r_tv["max_pairs"], "plain and two-vector disagree"

    # ---- single folds by size: two-vector vs plain, device time (best of a few, L2 flushed before
    # each), cells/s and the lookup-roofline fraction; uniform at every size, GC-rich at 6000
    sizes = None
    if not a.no_sizes and rank == 0:
        sizes = []
        for kind, nn in (("uniform", 2000), ("uniform", 4000), ("gc_rich", 6000), ("uniform", 8000),
                         ("uniform", 16384), ("uniform", 32768)):
            s_seq = synth.variant(kind, nn, 1308)
            reps = 5 if nn <= 8000 else (3 if nn <= 16384 else 2)
            row = {"n": nn, "kind": kind, "q": q}
            answers = {}
            for method in ("two_vector", "plain"):
                fm = make(method)
                codes = torch.from_numpy(fold.encode_codes(s_seq)).to(dev)
                wsm = torch.empty(fm.workspace_bytes(nn), dtype=torch.uint8, device=dev)
                outm = torch.zeros(1, dtype=torch.int32, device=dev)
                ts, ks = [], []
                for k in range(reps + 1):
                    with torch.cuda.stream(stream):
                        flush.zero_()
                        queue_ahead()
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        fm.score_dev(codes, wsm, outm, None, stream=stream.cuda_stream)
                        e1.record(stream)
                    e1.synchronize()
                    if k > 0:
                        ts.append(e0.elapsed_time(e1))
                        ks.append(fm.option(fold.FOLD_OPT_KERNEL_NS) / 1e6)
                answers[method] = int(outm.item())
                row[method] = {"ms": min(ts), "kernel_ms": min(ks), "cells_per_s": metrics.cells(nn) / (min(ts) * 1e-3)}
                fm.close()
                del wsm
            assert answers["two_vector"] == answers["plain"], f"n={nn}: kernels disagree"
            lam_n = metrics.lookups(nn, q)
            row["max_pairs"] = answers["two_vector"]
            row["two_vector_speedup"] = row["plain"]["ms"] / row["two_vector"]["ms"]
            row["lookups"] = lam_n
            row["lookup_frac"] = lam_n / (row["two_vector"]["kernel_ms"] * 1e-3) / metrics.lookup_peak(n_sm, 2032.0)
            row["plain_dpx_frac"] = (metrics.splits(nn) / (row["plain"]["kernel_ms"] * 1e-3)
                                     / (n_sm * 128 * 2032e6))
            sizes.append(row)
        torch.cuda.empty_cache()

    # ---- Section 3.2's partially memoised variant: R rows tabulated on first sight in each CTA
    memo = None
    if q <= 9:
        mf = make("two_vector")
        mf.option(fold.FOLD_OPT_R_MEMO, 1)
        r_m = device_run(mf, max(3, a.steps // 4), a.warmup)
        assert r_m["max_pairs"] == r_tv["max_pairs"], "memoised and precomputed R disagree"
        m_ms = statistics.mean(r_m["step_ms"])
        memo = {"ms_per_step": m_ms, "cells_per_s": cells / (m_ms * 1e-3),
                "kernel_ms": statistics.mean(r_m["kern_ms"]),
                "slowdown_vs_precomputed": m_ms / statistics.mean(r_tv["step_ms"]),
                "note": "Section 3.2 partially memoised: each CTA tabulates R[h][*] the first time it stages h"}
        mf.close()

    # ---- Section 3.2's FG algorithm (a table per row and group), per-column kernel, same input
    fgr = None
    if not a.no_sliding:
        fgr = {}
        for fq in (3, 8):
            ff = fold.Folder(q=fq, method="fg", device=local)
            ff.option(fold.FOLD_OPT_TIMING, 1)
            r_f = device_run(ff, 3, 1)
            assert r_f["max_pairs"] == r_tv["max_pairs"], "FG and two-vector disagree"
            f_ms = statistics.mean(r_f["step_ms"])
            fgr[f"q{fq}"] = {"ms_per_step": f_ms, "cells_per_s": cells / (f_ms * 1e-3),
                             "kernel_ms": statistics.mean(r_f["kern_ms"]),
                             "row_group_tables": metrics.fg_tables(n, fq),
                             "tiled_speedup": f_ms / statistics.mean(r_tv["step_ms"])}
            ff.close()
        fgr["note"] = ("Section 3.2 FG: Algorithm 1's groups, a table per row and group built when the group "
                       "completes; one warp per column like 'sliding'")

    # ---- Section 4's organisation as printed (one warp per column, per-cell vectors), same input
    sliding = None
    if not a.no_sliding:
        sl = make("sliding")
        r_sl = device_run(sl, 3, 1)
        assert r_sl["max_pairs"] == r_tv["max_pairs"], "sliding and two-vector disagree"
        sl_ms = statistics.mean(r_sl["step_ms"])
        sliding = {"ms_per_step": sl_ms, "cells_per_s": cells / (sl_ms * 1e-3),
                   "kernel_ms": statistics.mean(r_sl["kern_ms"]),
                   "lookups": metrics.lookups_relative(n, q),
                   "tiled_speedup": sl_ms / statistics.mean(r_tv["step_ms"]),
                   "note": "Section 4: one warp per column bottom to top, groups relative to i, "
                           "difference vectors at every cell"}
        sl.close()

    # ---- end to end through the public host API (pinned staging inside the library)
    e2e_times = []
    for k in range(a.warmup + a.steps):
        barrier_sync()
        t0 = time.perf_counter()
        mp = tv.score(seq)
        dt = time.perf_counter() - t0
        if k >= a.warmup:
            e2e_times.append(dt)
        assert mp == r_tv["max_pairs"]
    e2e_s = max_over_ranks(statistics.mean(e2e_times))
    e2e = {"value": world * cells / e2e_s, "unit": UNIT, "h2d_bytes_per_step": n, "d2h_bytes_per_step": 4,
           "ms_per_step": e2e_s * 1e3, "api": "fold_score (host string in, max pairs out)"}

    # ---- one optimal structure (fold + traceback kernel), device-resident, CUDA events
    structure = None
    if rank == 0:
        wsb = fold.fold_structure_workspace_bytes(tv.ctx, n)
        ws_s = torch.empty(wsb, dtype=torch.uint8, device=dev)
        codes_s = torch.from_numpy(fold.encode_codes(seq)).to(dev)
        out_s = torch.zeros(1, dtype=torch.int32, device=dev)
        part_s = torch.empty(n, dtype=torch.int32, device=dev)
        ts = []
        for k in range(4):
            with torch.cuda.stream(stream):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fold.fold_structure_dev(tv.ctx, codes_s.data_ptr(), n, ws_s.data_ptr(), wsb, out_s.data_ptr(),
                                        part_s.data_ptr(), stream.cuda_stream)
                e1.record(stream)
            e1.synchronize()
            if k > 0:
                ts.append(e0.elapsed_time(e1))
        assert int(out_s.item()) == r_tv["max_pairs"]
        pairs = int((part_s > torch.arange(n, device=dev)).sum().item())
        assert pairs == r_tv["max_pairs"]
        structure = {"ms_fold_and_traceback": min(ts), "ms_traceback": min(ts) - statistics.mean(r_tv["step_ms"]),
                     "pairs": pairs, "note": "fold_structure_dev: the fold, then the traceback (intervals traced in parallel by warps)"}
        del ws_s

    # ---- trace of one fold (optional)
    if a.trace and rank == 0:
        tv.option(fold.FOLD_OPT_TRACE, 1)
        tv.score(seq)
        np.save(a.trace, fold.fold_trace_copy(tv.ctx))
        tv.option(fold.FOLD_OPT_TRACE, 0)

    # ---- batched folding: 4096 sequences, log-uniform lengths in [64, 3000]; with several ranks
    # each folds its longest-processing-time share (independent sequences, no collective)
    batch = None
    if not a.no_batch:
        all_seqs = synth.batch(4096, 64, 3000, synth.SEED_BASE + 3)
        mine = ranks.partition_lpt([len(x) for x in all_seqs], world)[rank]
        seqs = [all_seqs[k] for k in mine]
        # one untimed call of the same batch sizes the context's buffers and device templates (a
        # serving process's steady state); then the median of three timed calls
        tv.batch(seqs)
        bts, bks = [], []
        for _ in range(3):
            barrier_sync()
            t0 = time.perf_counter()
            res = tv.batch(seqs)
            bts.append(time.perf_counter() - t0)
            bks.append(tv.option(fold.FOLD_OPT_KERNEL_NS) / 1e9)
        bt = max_over_ranks(statistics.median(bts))
        bk = max_over_ranks(statistics.median(bks))
        # one-at-a-time baseline on a 1-in-16 sample, device-timed, scaled to all sequences
        sample = seqs[::16]
        loop_s = 0.0
        for s in sample:
            codes = torch.from_numpy(fold.encode_codes(s)).to(dev)
            ws = torch.empty(max(256, tv.workspace_bytes(len(s))), dtype=torch.uint8, device=dev)
            out = torch.zeros(1, dtype=torch.int32, device=dev)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            tv.score_dev(codes, ws, out, None, stream=stream.cuda_stream)
            e1.record(stream)
            e1.synchronize()
            loop_s += e0.elapsed_time(e1) / 1e3
        loop_s *= len(seqs) / len(sample)
        # the same batch planned once and recorded into a CUDA graph (fold_batch_plan_create +
        # fold_batch_dev): device time of a replay, and end to end with the codes copied in from pinned
        # host memory and the answers copied out
        bp = fold.BatchPlan(tv.ctx, [len(s) for s in seqs])
        cat = torch.from_numpy(bp.encode(seqs)).pin_memory()
        d_codes = torch.empty(max(1, cat.numel()), dtype=torch.uint8, device=dev)
        d_codes[:cat.numel()].copy_(cat)
        wsb_ = torch.empty(bp.workspace_bytes, dtype=torch.uint8, device=dev)
        d_out = torch.zeros(len(seqs), dtype=torch.int32, device=dev)
        h_out = torch.zeros(len(seqs), dtype=torch.int32).pin_memory()
        bp.fold_dev(d_codes.data_ptr(), wsb_.data_ptr(), wsb_.numel(), d_out.data_ptr(), stream=stream.cuda_stream)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        tv.option(fold.FOLD_OPT_TIMING, 0)   # per-launch timing events cannot be recorded into a graph
        with torch.cuda.graph(graph, stream=stream):
            bp.fold_dev(d_codes.data_ptr(), wsb_.data_ptr(), wsb_.numel(), d_out.data_ptr(),
                        stream=stream.cuda_stream)
        tv.option(fold.FOLD_OPT_TIMING, 1)
        gts, gets = [], []
        for _ in range(3):
            barrier_sync()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):   # a graph replays on the current stream
                e0.record(stream)
                graph.replay()
                e1.record(stream)
            e1.synchronize()
            gts.append(e0.elapsed_time(e1) / 1e3)
        for _ in range(3):
            barrier_sync()
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                d_codes[:cat.numel()].copy_(cat, non_blocking=True)
                graph.replay()
                h_out.copy_(d_out, non_blocking=True)
            stream.synchronize()
            gets.append(time.perf_counter() - t0)
        assert h_out.numpy().tolist() == res.tolist(), "graph-replayed batch disagrees with fold_batch"
        g_dev = max_over_ranks(statistics.median(gts))
        g_e2e = max_over_ranks(statistics.median(gets))
        graph_batch = {"seq_per_s_replay": len(all_seqs) / g_dev, "seq_per_s_e2e": len(all_seqs) / g_e2e,
                       "replay_ms": g_dev * 1e3, "e2e_ms": g_e2e * 1e3, "h2d_bytes": int(cat.numel()),
                       "d2h_bytes": 4 * len(seqs),
                       "api": "fold_batch_plan_create once; fold_batch_dev recorded by stream capture, replayed",
                       "timing": "median of 3 replays (CUDA events) / 3 end-to-end replays with pinned copies"}
        del graph, wsb_
        bp.close()
        batch = {"sequences": len(all_seqs), "lengths": "log-uniform [64, 3000]", "graph": graph_batch,
                 "ranks": world, "split": "longest processing time first across ranks" if world > 1 else None,
                 "seq_per_s_e2e": len(all_seqs) / bt,
                 "seq_per_s_kernel": len(all_seqs) / bk if bk > 0 else None,
                 "seq_per_s_one_at_a_time": len(seqs) / loop_s,   # this rank's share on one GPU
                 "speedup_vs_one_at_a_time": (loop_s / bk) if bk > 0 else None,
                 "one_at_a_time_sample": "device time of every 16th sequence, scaled to 4096",
                 "timing": "median of 3 calls after one untimed call of the same batch",
                 "total_cells": int(sum(metrics.cells(len(s)) for s in seqs)), "checksum": int(res.sum())}

    # ---- serving: Poisson arrivals, lengths log-uniform in [50, 8000], 60 GB D budget
    serve = None
    if not a.no_serve:
        serve = serve_bench(tv, [float(x) for x in a.serve_rates.split(",") if x], a.serve_seconds,
                            a.serve_requests, dev, stream, torch, fold, metrics, synth)

    # ---- q sweep of the same fold (device time, best of 3 per q, automatic work split)
    qsweep = None
    if not a.no_qsweep:
        qsweep = {}
        for qq in range(4, 11):
            fq = fold.Folder(q=qq, device=local)
            codes = torch.from_numpy(fold.encode_codes(seq)).to(dev)
            wsq = torch.empty(fq.workspace_bytes(n), dtype=torch.uint8, device=dev)
            outq = torch.zeros(1, dtype=torch.int32, device=dev)
            ts = []
            for k in range(4):
                with torch.cuda.stream(stream):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    fq.score_dev(codes, wsq, outq, None, stream=stream.cuda_stream)
                    e1.record(stream)
                e1.synchronize()
                if k > 0:
                    ts.append(e0.elapsed_time(e1))
            assert int(outq.item()) == r_tv["max_pairs"], f"q={qq} disagrees"
            qsweep[str(qq)] = {"ms": min(ts), "cells_per_s": cells / (min(ts) * 1e-3),
                               "lookups": metrics.lookups(n, qq)}
            fq.close()
        best = min(qsweep, key=lambda k: qsweep[k]["ms"])
        qsweep["best_q"] = int(best)

    # ---- CPU baselines, whole folds of the same input, measured (rank 0, N = 1 only)
    cpu = None
    cpu_tv = None
    cpu_tv_mt = None
    if not a.no_cpu and rank == 0 and world == 1:
        hinfo = host_info()
        dt, mp = cpu_oracle_fold(seq)
        assert mp == r_tv["max_pairs"], "CPU oracle and GPU disagree"
        cpu = {"value": cells / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"one whole fold of the n={n} input by the cubic oracle (single-threaded C, Eq. 1): "
                         f"{dt:.1f} s, measured", **hinfo}
        dt1, mp1, _ = cpu_two_vector_fold(seq, q, 1)
        assert mp1 == r_tv["max_pairs"]
        cpu_tv = {"value": cells / dt1, "unit": UNIT, "cores": 1, "q": q,
                  "kind": "CPU two-vector (Algorithm 1, tiled wavefront; independent C program)",
                  "seconds": dt1, "sample": f"one whole fold of the n={n} input on 1 thread, measured"}
        per_q = {}
        used = 1
        for qq in range(4, 11):
            dq, mq, used = cpu_two_vector_fold(seq, qq, 0)
            assert mq == r_tv["max_pairs"]
            per_q[str(qq)] = {"seconds": dq, "cells_per_s": cells / dq}
        best_q = min(per_q, key=lambda k: per_q[k]["seconds"])
        cpu_tv_mt = {"value": per_q[str(q)]["cells_per_s"], "unit": UNIT, "cores": used, "q": q,
                     "seconds": per_q[str(q)]["seconds"], "best_q": int(best_q),
                     "best_q_value": per_q[best_q]["cells_per_s"], "best_q_seconds": per_q[best_q]["seconds"],
                     "per_q": per_q, "kind": "CPU two-vector (Algorithm 1, OpenMP over tile anti-diagonals)",
                     "sample": f"one whole fold of the n={n} input per q on all {used} host threads, measured",
                     **hinfo}

    # ---- attainable shared-memory lookup rate (microbenchmark; lookups per SM clock per SM)
    lookup_rates = None
    if rank == 0:
        lookup_rates = {}
        for mode, name in ((0, "uniform_row_registers"), (1, "uniform_row_kernel_step"), (2, "random_row")):
            r, kms = fold.fold_lookup_rate(local, 8, mode, 4096)
            lookup_rates[name] = r
        lookup_rates["analytic"] = 32.0
        lookup_rates["note"] = ("R-sized (q = 8, 16 KiB) byte table in shared memory, every SM full of resident "
                                "warps, cycles from clock64: uniform row = one row of R per warp-wide lookup "
                                "(the fold kernel's pattern); random row = independent (h, c) per lane")

    clocks = r_tv["clocks"] or {}
    sm_mhz = clocks.get("sm_mhz") or 2032.0
    peak = metrics.lookup_peak(n_sm, 2032.0)
    achieved = lam / (kern_ms * 1e-3)
    roofline = {
        "bound": "alu", "unit": "Glookups/s", "achieved": achieved / 1e9, "peak": peak / 1e9,
        "frac": achieved / peak, "traffic": measured_traffic(n, q),
        "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
        "kernel": "fold_kernel<8,two-vector> (persistent)", "kernel_ms": kern_ms,
        "algorithmic_lookups": lam,
        "peak_basis": f"{n_sm} SMs x 32 conflict-free shared-memory lookups/clk x 2032 MHz max SM clock",
        "frac_at_sampled_clock": achieved / metrics.lookup_peak(n_sm, sm_mhz),
        "hbm_floor_ms": metrics.hbm_bytes(n) / hbm_peak_gbs() / 1e6,
        "hbm_floor_basis": (f"8 B/cell (two int16 copies written and read once) at {hbm_peak_gbs():.1f} GB/s "
                            f"measured copy bandwidth; the two-vector kernel in column mode writes one row-major "
                            f"int16 copy plus packed (D << 16 | bits) row and column features instead of the "
                            f"column-major copy, so its compulsory bytes are 2 B/cell + 8 B per q cells"),
    }
    if lookup_rates:
        per_clk = achieved / (n_sm * 2032e6)
        roofline["lookups_per_clk_sm"] = per_clk
        roofline["measured_ceiling_lookups_per_clk_sm"] = lookup_rates["uniform_row_registers"]
        roofline["frac_of_measured_ceiling"] = per_clk / lookup_rates["uniform_row_registers"]
        roofline["frac_of_kernel_step_rate"] = per_clk / lookup_rates["uniform_row_kernel_step"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int16", "data": "synthetic", "config": workload_config(a),
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": r_tv["launches"], "clocks": clocks,
        "plain": {"ms_per_step": pl_ms, "cells_per_s": cells / (pl_ms * 1e-3),
                  "two_vector_speedup": pl_ms / statistics.mean(r_tv["step_ms"]),
                  "kernel_ms": statistics.mean(r_pl["kern_ms"])},
        "memoized": memo,
        "sliding": sliding,
        "fg": fgr,
        "sizes": sizes, "lookup_rates": lookup_rates,
        "batch": batch, "serve": serve, "q_sweep": qsweep, "cpu_two_vector": cpu_tv,
        "cpu_two_vector_mt": cpu_tv_mt, "paper": PAPER_FIGURES, "structure": structure,
        "max_pairs": r_tv["max_pairs"],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    tv.close()
    pl.close()
    rk.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
