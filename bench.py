"""Benchmark: SLPF parse throughput (text GB/s) of one text per GPU.

One step = one full parse of a device-resident text: forward / backward
speculative reach, join, checkpoint fix-up and build & merge with compose
(every kernel of the path), the clean SLPF written to HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload log|dna|ab] [--mode ...]

Default workload (the headline): web-server-like log records, 1 GiB of text
(seed 2 on rank 0) under the RE ((good|[^\n]*)\n)* with 124 numbered
positions and 162 segments, 2 % of the lines malformed; DICT columns.  The
DNA-like motif text (256 MiB, seed 1) is measured after it in the same run
and reported under the "dna" key.  Both texts are larger than L2, so every
step streams them from HBM.  N > 1 (torchrun): every rank parses its own
text of the same size (weak scaling, no collective on the data path); time
is the max over ranks.

Printed: one JSON line (rank 0) with the contract keys plus ``roofline``
(the dominant kernel timed live with the library's per-phase CUDA events),
``cpu_baseline`` (the CPU oracle on a bounded sample), ``e2e`` (host buffers
in, SLPF back to host, through the same C-ABI call) and ``clocks``.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SLPF parse GB/s of text on 1 GB300, % of HBM roofline; p50/p99 latency served"
# name -> (description, RE attribute of workloads, text maker, default bytes, seed, oracle sample bytes)
WORKLOADS = {
    "log": ("log-records: RE ((IPv4 - - [timestamp] \"METHOD /path HTTP/1.x\" status size|[^\\n]*)\\n)*, "
            "124 positions, 162 segments; 1 GiB of web-server-like lines (paths Zipf over 1e5 tokens, "
            "status 200 w.p. 0.9, 2% malformed), seed 2", "LOG_RE", "log_text", 1 << 30, 2, 16 << 20),
    "dna": ("dna-motif: RE ([ACGT]|ATG([ACGT][ACGT][ACGT])*(TAA|TAG|TGA))*, 256 MiB uniform ACGT, "
            "ORFs 30-900 codons at 1 per 10 kB, seed 1", "DNA_RE", "dna_text", 256 << 20, 1, 256 << 20),
    "ab": ("ab: RE (a|b|ab)*, i.i.d. uniform {a,b}, seed 0", "AB_RE", "ab_text", 1 << 20, 0, 64 << 20),
}
WORKLOAD = WORKLOADS["log"][0]
FALLBACK_HBM = 6800.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="log", choices=sorted(WORKLOADS),
                    help="single mode: log (1 GiB, the headline), dna (256 MiB) or ab")
    ap.add_argument("--bytes", type=int, default=0, help="text size (default: the workload's)")
    ap.add_argument("--no-extra", action="store_true", help="single mode: skip the DNA line after the log one")
    ap.add_argument("--chunk-len", type=int, default=0)
    ap.add_argument("--reach-shape", type=int, default=0,
                    help="with --chunk-len: reach shape 1-4 (RE_PARSE_REACH); 0 = the library's default")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", default="single",
                    choices=["single", "batch", "serve", "matches", "latency", "ablation", "join", "shard",
                             "archive"],
                    help="single: one 256 MiB text (default); batch: 4096 texts under 8 random REs; "
                         "serve: Poisson request stream")
    ap.add_argument("--texts", type=int, default=4096, help="batch mode: number of texts")
    ap.add_argument("--rates", default="1000,3000,10000,30000,100000", help="serve mode: request rates (req/s)")
    ap.add_argument("--duration", type=float, default=1.0, help="serve mode: seconds of arrivals per rate")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        loaded = [r for r in rows if (num(r[4]) or 0) >= 50] or rows
        sm = [num(r[1]) for r in loaded if num(r[1]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in loaded:
            for j, nm in enumerate(names):
                if r[6 + j].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": num(loaded[0][2]), "reasons": sorted(reasons),
                "samples": len(loaded), "power_w_max": max((num(r[3]) or 0) for r in loaded)}


def cpu_baseline(text_host, pattern, sample_bytes):
    """The CPU oracle as it stands (serial two-way NFA parser, one core) on a
    bounded prefix of the same text."""
    from oracle import serial
    from oracle.re_front import compile_re
    c = compile_re(pattern)
    sample = text_host[:sample_bytes].tobytes()
    t0 = time.perf_counter()
    serial.parse(c, sample)
    dt = time.perf_counter() - t0
    return {"value": len(sample) / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"first {len(sample) >> 20} MiB of the workload text, serial oracle (Eq. matrixmul), "
                      f"{dt:.1f} s, host {os.uname().machine} nproc={os.cpu_count()}"}


def lsu_roofline(phase_ms: dict, n: int, device: int, ncls: int, shape: int):
    """Reach against the shared-memory pipe, its real bound.  Shared-memory
    lookups per text byte: 2 with byte-indexed tables (reach shape 1: one
    transition per byte and direction); with class tables 3 for at most 16
    byte classes (per direction and byte pair: two class lookups and one
    two-byte table lookup), else 4 (per direction and byte: one class and one
    transition lookup).  Peak: one 32-lane wavefront per SM and cycle at the
    maximum SM clock (bank conflicts make a lookup cost more)."""
    import torch
    props = torch.cuda.get_device_properties(device)
    peak = props.multi_processor_count * 32 * 2.07e9 / 1e12
    per_byte = 2 if shape == 1 else 3 if ncls <= 16 else 4
    achieved = per_byte * n / (phase_ms["reach"] / 1e3) / 1e12
    return {"kernel": "reach", "bound": "lsu", "lookups_per_byte": per_byte, "achieved": round(achieved, 3),
            "peak": round(peak, 3),
            "unit": "T lookups/s", "frac": round(achieved / peak, 4),
            "peak_source": "SM count x 32 lanes x 2070 MHz (one conflict-free wavefront per SM and cycle)"}


# The sources of the kernels whose DRAM traffic profiles/traffic.json records
# (reach, fix-up, build & merge) and of the structures they share.
KERNEL_SOURCES = ("kernels.cuh", "re_internal.h", "reach_impl.cuh", "reach_byte8.cu", "reach_ascii.cu", "merge.cu")


def csrc_hash() -> str:
    """SHA-256 over the sources of the profiled kernels, in name order."""
    d = os.path.join(ROOT, "paper_2503_06763_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(KERNEL_SOURCES):
        h.update(f.encode())
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()


def traffic_for(workload: str, kernel: str, n: int):
    """ncu DRAM bytes of the dominant kernel, scaled per text byte, if the
    committed capture of this workload matches the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("csrc_sha256") != csrc_hash():
            return None
        per = d.get("dram_bytes_per_text_byte", {}).get(workload, {}).get(kernel)
        return None if per is None else per * n
    except Exception:
        return None


def aggregate(ms_local: float, units_local: int, dist=None, device=None):
    """Whole-job timing over ranks: the slowest rank's timed region (max) and
    the units every rank processed (sum).  Single process: unchanged."""
    if dist is None:
        return ms_local, units_local
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([units_local], dtype=torch.int64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(u.item())


def rank_seed(base: int, rank: int) -> int:
    """Seed of rank r's input: every rank parses its own text (weak scaling)."""
    return base + 1000 * rank


def measure_single(args, name, n, rank, world, local, dist, full=True):
    """One workload on one text per rank: the timed headline loop, per-phase
    times, and (full) the recognizer, end-to-end and CPU-oracle legs.
    Returns the fields of the JSON line."""
    import torch
    import workloads as W
    from paper_2503_06763_gb300 import Regex
    from paper_2503_06763_gb300.native import PHASES

    desc, re_attr, maker, _, seed, cpu_bytes = WORKLOADS[name]
    pattern = getattr(W, re_attr)
    host = getattr(W, maker)(n, seed=rank_seed(seed, rank))
    n = int(host.size)
    rx = Regex(pattern)
    dev = torch.device("cuda", local)
    text = torch.from_numpy(host).to(dev)
    tuned = None
    if args.chunk_len == 0:                 # re_autotune on this text; later parses use its choice
        tuned = rx.autotune(text)
        torch.cuda.empty_cache()
    kind, cb, out_bytes = rx.layout(n, "auto")
    dt = {1: torch.uint8, 2: torch.int16, 4: torch.int32, 8: torch.int64}[cb]
    out = torch.empty(n + 1, dtype=dt, device=dev)
    status = torch.empty(1, dtype=torch.int32, device=dev)
    ws = torch.empty(rx.workspace_size(n, args.chunk_len), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(PHASES) + 1)] for _ in range(args.steps)]

    def step(i=None):
        rx.parse(text, kind=kind, chunk_len=args.chunk_len, out=out, status=status, workspace=ws,
                 events=ev[i] if i is not None else None, reach_shape=args.reach_shape)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    st = int(status.item())
    if st != 0:
        raise SystemExit(f"{name}: parse status {st}")
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(args.steps):
            step()
        t_end.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    clocks = clk.summary()
    ms_total, units = aggregate(t_start.elapsed_time(t_end), n, dist, dev)
    ms = ms_total / args.steps
    value = units / (ms / 1e3) / 1e9

    # per-phase device times: a second timed loop of the same K steps with an
    # event on the launching stream between phases (kept out of the loop
    # above: an event between two dependent launches serialises them)
    for i in range(args.steps):
        step(i)
    torch.cuda.synchronize()
    phase_ms = {p: statistics.mean(ev[i][j].elapsed_time(ev[i][j + 1]) for i in range(args.steps))
                for j, p in enumerate(PHASES)}
    dominant = max(phase_ms, key=phase_ms.get)
    shape = args.reach_shape if args.chunk_len else rx.tuned(n)[1]
    if not shape:                       # the library's default: byte tables when they fit, else warp pairs
        shape = 1 if rx.info["n_classes"] > 16 and rx.info["fwd_states"] < 256 and rx.info["bwd_states"] < 256 else 2
    # algorithmic bytes per launch: text read once, plus the SLPF written by build & merge
    alg = {"reach": n, "join": 0, "fixup": 0, "build_merge": n + (n + 1) * cb}
    hbm, src = peaks()
    achieved = alg[dominant] / (phase_ms[dominant] / 1e3) / 1e9 if alg[dominant] else 0.0
    roofline = {"bound": "hbm", "kernel": dominant, "achieved": round(achieved, 1), "peak": hbm,
                "peak_source": src, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                "traffic": traffic_for(name, dominant, n),
                "phase_ms": {k: round(v, 4) for k, v in phase_ms.items()},
                "phase_timing": "second loop of the same K steps, CUDA events between phases",
                "algorithmic_bytes": {k: v for k, v in alg.items() if v},
                "whole_step_frac": round((n + (n + 1) * cb) / (ms / 1e3) / 1e9 / hbm, 4),
                "lsu": lsu_roofline(phase_ms, n, local, rx.info["n_classes"], shape)}
    res = {"value": round(value, 3), "ms_per_step": round(ms, 4), "roofline": roofline, "clocks": clocks,
           "config": {"workload": desc, "text_bytes_per_gpu": n, "encoding": f"{kind}-{8 * cb}bit",
                      "chunk_len": args.chunk_len or tuned,
                      "chunk_len_from": "fixed" if args.chunk_len else "re_autotune",
                      "reach_shape": shape,
                      "segments": rx.ell,
                      "byte_classes": rx.info["n_classes"],
                      "l2": f"text {n >> 20} MiB > 129 MB L2 (no flush needed)",
                      "parallelism": f"independent texts per GPU x{world}"}}
    if not full:
        del text, out, ws
        torch.cuda.empty_cache()
        return res

    # recognizer mode (forward reach + join only, Sect. 4.2), same text, with
    # its own autotuned chunk length (one forward warp per 32-chunk tile, so it
    # prefers more, shorter chunks than the parse)
    rec_k = args.chunk_len
    if args.chunk_len == 0:
        rec_k = rx.autotune(text, recognize_only=True)
        torch.cuda.empty_cache()
    rec_ws = torch.empty(rx.workspace_size(n, rec_k, 1), dtype=torch.uint8, device=dev)
    for _ in range(3):
        rx.parse(text, chunk_len=args.chunk_len, status=status, workspace=rec_ws, recognize_only=True)
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    for _ in range(args.steps):
        rx.parse(text, chunk_len=args.chunk_len, status=status, workspace=rec_ws, recognize_only=True)
    r1.record(stream)
    torch.cuda.synchronize()
    res["recognizer"] = {"value": round(n / (r0.elapsed_time(r1) / args.steps / 1e3) / 1e9, 3), "unit": "GB/s",
                         "status": int(status.item()), "chunk_len": rec_k}
    del rec_ws

    # end to end through re_parse_host: pinned host text in, columns and status
    # back to pinned host memory, every step.  Three streams with their own
    # device buffers take steps in turn, so one step's copy in, another's
    # kernels and a third's copy out run at once (the link carries about 200
    # GB/s each way, 171 GB/s each way when both directions are busy).
    E2E_STREAMS = 3
    pin_in = torch.from_numpy(host).pin_memory()
    sets = []
    for _ in range(E2E_STREAMS):
        sets.append({"s": torch.cuda.Stream(dev), "out": torch.empty(n + 1, dtype=dt).pin_memory(),
                     "st": torch.empty(1, dtype=torch.int32).pin_memory(),
                     "d_text": torch.empty(n, dtype=torch.uint8, device=dev),
                     "d_out": torch.empty(n + 1, dtype=dt, device=dev),
                     "d_st": torch.empty(1, dtype=torch.int32, device=dev),
                     "ws": torch.empty(ws.numel(), dtype=torch.uint8, device=dev)})

    def e2e_step(k):
        b = sets[k % E2E_STREAMS]
        rx.parse_host(pin_in, b["out"], b["st"], b["d_text"], b["d_out"], b["d_st"], b["ws"], stream=b["s"],
                      kind=kind, chunk_len=args.chunk_len)

    for k in range(2 * E2E_STREAMS):            # warm-up: first use of the pinned buffers and copy paths
        e2e_step(k)
    torch.cuda.synchronize()
    e_steps = max(2 * E2E_STREAMS, min(args.steps, 9))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for b in sets:
        b["s"].wait_event(e0)
    for k in range(e_steps):
        e2e_step(k)
    for b in sets:
        done = torch.cuda.Event()
        done.record(b["s"])
        stream.wait_event(done)
    e1.record(stream)
    torch.cuda.synchronize()
    e_ms = e0.elapsed_time(e1) / e_steps
    if not all(int(b["st"][0]) == st for b in sets) or not torch.equal(sets[0]["out"], out.cpu()):
        raise SystemExit("end-to-end columns differ from the device-resident parse")
    res["e2e"] = {"value": round(n * world / (e_ms / 1e3) / 1e9, 3), "unit": "GB/s",
                  "h2d_bytes_per_step": n, "d2h_bytes_per_step": (n + 1) * cb + 4,
                  "api": f"re_parse_host, {E2E_STREAMS} streams taking steps in turn"}
    del sets, pin_in, text, out, ws
    torch.cuda.empty_cache()
    res["cpu_baseline"] = None
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        res["cpu_baseline"] = cpu_baseline(host, pattern, cpu_bytes)
    return res


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return reference_arm(args, rank, world)
    if args.mode == "batch":
        return batch_mode(args, rank, world, local)
    if args.mode == "serve":
        return serve_mode(args, rank, world, local)
    if args.mode == "matches":
        return matches_mode(args, rank, world, local)
    if args.mode == "latency":
        return latency_mode(args, rank, world, local)
    if args.mode == "ablation":
        return ablation_mode(args, rank, world, local)
    if args.mode == "join":
        return join_mode(args, rank, world, local)
    if args.mode == "shard":
        return shard_mode(args, rank, world, local)
    if args.mode == "archive":
        return archive_mode(args, rank, world, local)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    name = args.workload
    n = args.bytes or WORKLOADS[name][3]
    r = measure_single(args, name, n, rank, world, local, dist, full=True)
    extra = None
    if name == "log" and not args.no_extra:     # the DNA motif text, same protocol, headline loop only
        d = measure_single(args, "dna", WORKLOADS["dna"][3], rank, world, local, dist, full=False)
        extra = {"workload": d["config"]["workload"], "value": d["value"], "unit": "GB/s",
                 "ms_per_step": d["ms_per_step"], "chunk_len": d["config"]["chunk_len"],
                 "phase_ms": d["roofline"]["phase_ms"], "whole_step_frac": d["roofline"]["whole_step_frac"],
                 "dominant": {k: d["roofline"][k] for k in ("kernel", "achieved", "frac")}}
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": r["value"], "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic", "config": r["config"],
        "roofline": r["roofline"], "cpu_baseline": r.get("cpu_baseline"), "e2e": r.get("e2e"),
        "recognizer": r.get("recognizer"), "gpu_launches": 7 * args.steps, "clocks": r["clocks"],
    }
    if extra:
        line["dna"] = extra
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


_ORACLE_RES = {}


def _oracle_parse_job(job):
    """One text through the serial oracle in a pool worker (REs compiled
    once per worker).  Returns (bytes, parse seconds)."""
    pattern, text = job
    from oracle import serial
    from oracle.re_front import compile_re
    c = _ORACLE_RES.get(pattern)
    if c is None:
        c = _ORACLE_RES[pattern] = compile_re(pattern)
    t0 = time.perf_counter()
    serial.parse(c, text)
    return len(text), time.perf_counter() - t0


def batch_cpu_baseline(patterns, hosts, budget: int = 256 << 20):
    """The oracle on all host cores: the batch's first texts (about `budget`
    bytes) parsed one per task by a process pool started with spawn (safe
    after CUDA is initialised)."""
    import multiprocessing as mp
    jobs, tot = [], 0
    for pat, h in zip(patterns, hosts):
        if tot >= budget:
            break
        jobs.append((pat, h.tobytes()))
        tot += len(h)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        done = pool.map(_oracle_parse_job, jobs, chunksize=1)
    wall = time.perf_counter() - t0
    nbytes, parse_s = sum(d[0] for d in done), sum(d[1] for d in done)
    return {"value": round(nbytes / wall / 1e9, 6), "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"first {len(jobs)} texts of the batch ({nbytes >> 20} MiB), one per task on a spawn pool of "
                      f"{cores} processes, {wall:.1f} s wall including each worker's RE compiles; "
                      f"parsing alone {nbytes / parse_s / 1e6:.1f} MB/s per core, host {os.uname().machine}"}


def batch_res(seed0: int = 3000, count: int = 8, lo: int = 10, hi: int = 200):
    """count random REs (lo..hi positions, alphabet 4..64 each); an RE whose
    tables exceed the library's caps is replaced by the next seed."""
    import workloads as W
    from paper_2503_06763_gb300 import Regex, ReError
    out, seed = [], seed0
    while len(out) < count:
        pat, tree, _ = W.random_re(seed, lo, hi)
        seed += 1
        try:
            rx = Regex(pat)
        except ReError:
            continue
        out.append((pat, tree, rx))
    return out


def batch_mode(args, rank, world, local):
    """4096 texts (lengths log-uniform 1 KiB - 4 MiB) under 8 random REs:
    re_parse_batch (one launch per phase and RE), its CUDA-graph replay, and
    one re_parse per text for comparison -- the same outputs each time."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2503_06763_gb300 import Batch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    res = batch_res()
    lens, which = W.batch_lengths(args.texts, seed=rank_seed(3, rank))
    pools = [W.PiecePool(tree, 100 + i) for i, (_, tree, _) in enumerate(res)]
    hosts = [pools[w].text(int(n), seed=10_000 + j) for j, (n, w) in enumerate(zip(lens, which))]
    total = int(sum(len(h) for h in hosts))
    texts = [torch.from_numpy(h).to(dev) for h in hosts]
    rxs = [res[w][2] for w in which]
    b = Batch(rxs, [len(h) for h in hosts])
    outs, status, kinds = b.parse(texts)
    torch.cuda.synchronize()
    bad = int((status != 0).sum().item())
    if bad:
        raise SystemExit(f"{bad} batch texts not accepted")
    out_bytes = sum(o.numel() * o.element_size() for o in outs)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, steps):
        for _ in range(max(args.warmup, 3)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    ms_batch = timed(b.run, args.steps)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.run()
    ms_graph = timed(g.replay, args.steps)
    ws = torch.empty(max(rx.workspace_size(len(h)) for rx, h in zip(rxs, hosts)), dtype=torch.uint8, device=dev)

    def per_text():
        for j, (rx, t) in enumerate(zip(rxs, texts)):
            rx.parse(t, out=outs[j], status=status[j:j + 1], workspace=ws)

    t0 = time.perf_counter()
    ms_single = timed(per_text, max(1, min(args.steps, 3)))
    host_single = (time.perf_counter() - t0) * 1e3
    hbm, src = peaks()
    gbs = lambda ms: round(total / (ms / 1e3) / 1e9, 3)
    line = {
        "metric": "batched SLPF parse GB/s of text (re_parse_batch, 1 launch per phase and RE)",
        "value": gbs(ms_batch), "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms_batch, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u8", "data": "synthetic",
        "config": {"workload": f"{args.texts} valid texts, lengths log-uniform 1 KiB-4 MiB, 8 random REs "
                               "(10-200 positions, alphabets 4-64), seed 3",
                   "text_bytes": total, "slpf_bytes": out_bytes,
                   "segments": [r[2].ell for r in res], "encodings": sorted(set(kinds))},
        "graph_replay": {"value": gbs(ms_graph), "ms_per_step": round(ms_graph, 3)},
        "per_text_launches": {"value": gbs(ms_single), "ms_per_step": round(ms_single, 3),
                              "launches_per_step": 7 * args.texts},
        "roofline": {"bound": "hbm", "achieved": round((total + out_bytes) / (ms_batch / 1e3) / 1e9, 1),
                     "peak": hbm, "peak_source": src, "unit": "GB/s",
                     "frac": round((total + out_bytes) / (ms_batch / 1e3) / 1e9 / hbm, 4)},
        "cpu_baseline": None,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = batch_cpu_baseline([res[w][0] for w in which], hosts)
    if rank == 0:
        print(json.dumps(line))


def serve_mode(args, rank, world, local):
    """Poisson request streams against 16 resident random REs (20-300
    positions); lengths lognormal (median 64 KiB, sigma 1.5, at most 64 MiB).
    Each rate is served three times: continuous batching in the Python loop
    (slots of re_parse_batch), one launch per request (the same loop with
    batches of one), and the library's request loop (re_server)."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2503_06763_gb300 import serve
    torch.cuda.set_device(local)
    res = batch_res(seed0=4000, count=16, lo=20, hi=300)
    pools = [W.PiecePool(tree, 200 + i) for i, (_, tree, _) in enumerate(res)]
    rng = np.random.Generator(np.random.PCG64(rank_seed(4, rank)))
    bank = []
    for j in range(2048):
        ln = np.exp(rng.normal(np.log(64 << 10), 1.5))
        while ln > (64 << 20):
            ln = np.exp(rng.normal(np.log(64 << 10), 1.5))
        ri = int(rng.integers(0, len(res)))
        bank.append((ri, pools[ri].text(int(ln), seed=50_000 + j)))
    rates = [float(r) for r in args.rates.split(",")]
    results = []
    for mb, label in ((4096, "continuous_batching"), (1, "per_request")):
        srv = serve.Server([r[2] for r in res], slots=4, arena_bytes=2 << 30, max_batch=mb)
        warm = [serve.Request(rid=j, re_index=bank[j][0], text=bank[j][1]) for j in range(64)]
        srv.run(warm, realtime=False)
        for rate in rates:
            n = int(min(max(rate * args.duration, 200), 20_000))
            gaps = rng.exponential(1.0 / rate, size=n)
            arr = np.cumsum(gaps)
            reqs = [serve.Request(rid=j, re_index=bank[j % len(bank)][0], text=bank[j % len(bank)][1],
                                  arrival=float(arr[j])) for j in range(n)]
            wall = srv.run(reqs, realtime=True)
            nbytes = sum(len(r.text) for r in reqs)
            span = max(r.done for r in reqs) - reqs[0].arrival
            bad = sum(1 for r in reqs if r.status != 0)
            results.append({"mode": label, "rate_rps": rate, "requests": n, "text_bytes": nbytes,
                            "offered_GBps": round(nbytes / arr[-1] / 1e9, 3),
                            "served_GBps": round(nbytes / span / 1e9, 3),
                            "achieved_rps": round(n / span, 1), **serve.latency_summary(reqs),
                            "batches": srv.stats["batches"], "not_ok": bad, "wall_s": round(wall, 3)})
            srv.stats.update(batches=0, requests=0, max_batch=0, max_inflight=0)
        srv.close()
    # the library's own request loop (re_server): submissions from this thread at
    # the arrival times, completion times taken on the server's clock
    from paper_2503_06763_gb300.native import NativeServer
    nsrv = NativeServer([r[2] for r in res], slots=4, arena_bytes=2 << 30)
    for j in range(64):
        nsrv.wait(nsrv.submit(bank[j][0], bank[j][1]))
    nsrv.poll(cap=1 << 16)
    for j in range(64):
        nsrv.result(j + 1)
    for rate in rates:
        n = int(min(max(rate * args.duration, 200), 20_000))
        arr = np.cumsum(rng.exponential(1.0 / rate, size=n))
        st0 = dict(nsrv.stats())
        start = time.perf_counter()
        sub = {}
        for j in range(n):
            while time.perf_counter() - start < arr[j]:
                pass
            sub[nsrv.submit(bank[j % len(bank)][0], bank[j % len(bank)][1])] = (nsrv.clock_ns(), j)
        lat, done_ns = [], []
        got = 0
        while got < n:
            for t, ns in nsrv.poll(cap=1 << 16):
                if t in sub:
                    lat.append((ns - sub[t][0]) / 1e6)
                    done_ns.append(ns)
                    got += 1
                    _, st = nsrv.result(t)
        nbytes = sum(len(bank[j % len(bank)][1]) for j in range(n))
        first = min(v[0] for v in sub.values())
        span = (max(done_ns) - first) / 1e9
        lat = np.array(lat)
        st1 = nsrv.stats()
        results.append({"mode": "native_loop", "rate_rps": rate, "requests": n, "text_bytes": nbytes,
                        "offered_GBps": round(nbytes / arr[-1] / 1e9, 3), "served_GBps": round(nbytes / span / 1e9, 3),
                        "achieved_rps": round(n / span, 1), "p50_ms": round(float(np.percentile(lat, 50)), 3),
                        "p99_ms": round(float(np.percentile(lat, 99)), 3), "mean_ms": round(float(lat.mean()), 3),
                        "max_ms": round(float(lat.max()), 3), "batches": st1["batches"] - st0["batches"]})
    nsrv.close()
    best = max((r for r in results if r["mode"] == "continuous_batching"), key=lambda r: r["served_GBps"])
    line = {
        "metric": "served SLPF parse: p50/p99 latency (ms) and GB/s under Poisson load",
        "value": best["served_GBps"], "unit": "GB/s", "n_gpus": world, "steps": len(rates), "warmup": 1,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": "Poisson arrivals, lognormal lengths (median 64 KiB, sigma 1.5, <= 64 MiB), "
                               "16 random REs (20-300 positions), valid texts, seed 4",
                   "slots": 4, "arena_bytes_per_slot": 2 << 30,
                   "segments": [r[2].ell for r in res]},
        "p50_ms": best["p50_ms"], "p99_ms": best["p99_ms"], "rates": results,
    }
    if rank == 0:
        print(json.dumps(line))


def matches_mode(args, rank, world, local):
    """Match extraction (re_matches) after a parse of the DNA workload: the
    stop codons that close an ORF (group 13), as text GB/s of columns
    visited; the oracle's forest visit on a 1 MiB prefix beside it."""
    import torch
    import workloads as W
    from paper_2503_06763_gb300 import Regex
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.bytes or (256 << 20)
    host = W.dna_text(n, seed=rank_seed(1, rank))
    rx = Regex(W.DNA_RE)
    text = torch.from_numpy(host).to(dev)
    cols, st, kind = rx.parse(text)
    torch.cuda.synchronize()
    group = 13
    pairs, total = rx.matches(cols, st, n, group, kind)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 3)):
        rx.matches(cols, st, n, group, kind, cap=total)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        rx.matches(cols, st, n, group, kind, cap=total)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import matches as M
        from oracle import serial
        from oracle.re_front import compile_re
        c = compile_re(W.DNA_RE)
        sample = host[:1 << 20].tobytes()
        colsets = [serial.from_bits(row) for row in serial.parse(c, sample)]
        t0 = time.perf_counter()
        M.matches_by_slpf(c, sample, group, colsets)
        dt = time.perf_counter() - t0
        cpu = {"value": round(len(sample) / dt / 1e9, 6), "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": "first 1 MiB: forest visit of the oracle's own SLPF (columns given)"}
    line = {"metric": "match extraction GB/s of text (re_matches: count, scan, write)", "value": round(n / (ms / 1e3) / 1e9, 3),
            "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": WORKLOAD, "group": "13 (stop codon closing an ORF)", "matches": total},
            "cpu_baseline": cpu}
    if rank == 0:
        print(json.dumps(line))


def latency_mode(args, rank, world, local):
    """One small text, (a|b|ab)* over 1 MiB of uniform a/b (seed 0): latency of
    one parse with its 7 launches issued directly, and as a CUDA-graph
    replay of the same re_parse call."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2503_06763_gb300 import Regex
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = 1 << 20
    rx = Regex(W.AB_RE)
    text = torch.from_numpy(W.ab_text(n, seed=0)).to(dev)
    cols, st, kind = rx.parse(text)
    ws = torch.empty(rx.workspace_size(n), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    reps = max(args.steps, 50)

    def lat(fn):
        for _ in range(max(args.warmup, 3)):
            fn()
        torch.cuda.synchronize()
        out = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            out.append(e0.elapsed_time(e1))
        a = np.array(out)
        return {"p50_ms": round(float(np.percentile(a, 50)), 4), "p99_ms": round(float(np.percentile(a, 99)), 4),
                "GBps_at_p50": round(n / (float(np.percentile(a, 50)) / 1e3) / 1e9, 2)}

    direct = lat(lambda: rx.parse(text, out=cols, status=st, workspace=ws))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        rx.parse(text, out=cols, status=st, workspace=ws)
    graph = lat(g.replay)
    line = {"metric": "single-parse latency, 1 MiB (a|b|ab)* text (p50 ms)", "value": graph["p50_ms"], "unit": "ms",
            "n_gpus": world, "steps": reps, "warmup": args.warmup, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": "(a|b|ab)*, 1 MiB uniform a/b, seed 0", "encoding": kind},
            "graph_replay": graph, "direct_launches": direct}
    if rank == 0:
        print(json.dumps(line))


def ablation_mode(args, rank, world, local):
    """Speculation ablation (the ME-DFA of Sect. 3.1 against the DFA, as in
    Sect. 5): the DNA workload, (a|b|ab)* over uniform a/b and
    (a|b)*a(a|b){3} over uniform a/b (accepted: the fourth byte from the end
    is a), each as large as --bytes, parsed with the ME-DFA starts and with
    starts from every DFA state forward (RE_COMPILE_DFA_STARTS), backward
    (RE_COMPILE_DFA_STARTS_BWD) and both.  Per variant: runs per class pair
    each way, the autotuned chunk length, the full parse (GB/s, reach time)
    and the recognizer (forward reach + join); a variant whose runs exceed
    the 32 a lane holds is refused at compile and listed as such.  value =
    DNA full-parse time with forward DFA starts / with ME-DFA starts."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2503_06763_gb300 import Regex, ReError
    from paper_2503_06763_gb300.native import PHASES
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.bytes or (256 << 20)
    stream = torch.cuda.current_stream(dev)
    steps = max(args.steps, 5)
    rows = []
    suffix = np.random.Generator(np.random.PCG64(4)).choice(np.frombuffer(b"ab", dtype=np.uint8), size=n)
    suffix[max(n - 4, 0)] = ord("a")
    for name, pattern, host in (("dna", W.DNA_RE, W.dna_text(n, seed=1)), ("ab", W.AB_RE, W.ab_text(n, seed=0)),
                                ("suffix", "(a|b)*a(a|b){3}", suffix)):
        text = torch.from_numpy(host).to(dev)
        for starts, which in (("me-dfa", False), ("dfa-fwd", "fwd"), ("dfa-bwd", "bwd"), ("dfa-both", "both")):
            try:
                rx = Regex(pattern, dfa_starts=which)
            except ReError as e:
                rows.append({"workload": name, "starts": starts, "refused": str(e)})
                continue
            k = rx.autotune(text)
            kind, cb, _ = rx.layout(n, "auto")
            dt = {1: torch.uint8, 2: torch.int16, 4: torch.int32, 8: torch.int64}[cb]
            out = torch.empty(n + 1, dtype=dt, device=dev)
            status = torch.empty(1, dtype=torch.int32, device=dev)
            ws = torch.empty(rx.workspace_size(n, chunk_len=256), dtype=torch.uint8, device=dev)

            def run(recognize, events=None):
                rx.parse(text, kind=kind, out=out, status=status, workspace=ws, recognize_only=recognize,
                         events=events)

            res = {"workload": name, "starts": starts, "fwd_runs_max": rx.info["fwd_slots_max"],
                   "bwd_runs_max": rx.info["bwd_slots_max"], "chunk_len": k}
            for recognize in (False, True):
                for _ in range(max(args.warmup, 3)):
                    run(recognize)
                torch.cuda.synchronize()
                if int(status.item()) != 0:
                    raise SystemExit(f"{name}/{starts}: parse status {int(status.item())}")
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(steps):
                    run(recognize)
                e1.record(stream)
                e1.synchronize()
                ms = e0.elapsed_time(e1) / steps
                res["recognizer_GBps" if recognize else "parse_GBps"] = round(n / (ms / 1e3) / 1e9, 1)
                if not recognize:
                    res["parse_ms"] = round(ms, 4)
                    ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(PHASES) + 1)]
                    run(False, ev)
                    torch.cuda.synchronize()
                    res["reach_ms"] = round(ev[0].elapsed_time(ev[1]), 4)
                else:
                    res["recognizer_ms"] = round(ms, 4)
            rows.append(res)
            del rx, out, ws
            torch.cuda.empty_cache()
    by = {(r["workload"], r["starts"]): r for r in rows}
    ratio = by[("dna", "dfa-fwd")]["parse_ms"] / by[("dna", "me-dfa")]["parse_ms"]
    line = {"metric": "speculation ablation: DNA full-parse time, forward all-DFA-state starts / ME-DFA starts",
            "value": round(ratio, 3), "unit": "x", "n_gpus": world, "steps": steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": f"dna-motif, (a|b|ab)* and (a|b)*a(a|b){{3}}, {n} bytes each, text resident",
                       "variants": "ME-DFA starts with the last-class filter / starts from every DFA state "
                                   "forward, backward, both"},
            "rows": rows}
    if rank == 0:
        print(json.dumps(line))


def archive_mode(args, rank, world, local):
    """SLPF archives (App. C): the log, DNA and ab texts (256 MiB, or --bytes)
    parsed, their columns archived by the host encoder (checkpoint every 4096
    columns) and rebuilt by the device decoder.  Per workload: archive bytes
    against the columns' bytes, the exception rate, host encode time, and the
    device rebuild in GB/s of columns written (value: the log's rebuild)."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2503_06763_gb300 import Regex
    from paper_2503_06763_gb300 import native
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n0 = args.bytes or (256 << 20)
    stream = torch.cuda.current_stream(dev)
    rows = []
    for name, pattern, host in (("log", W.LOG_RE, W.log_text(n0, seed=2)), ("dna", W.DNA_RE, W.dna_text(n0, seed=1)),
                                ("ab", W.AB_RE, W.ab_text(n0, seed=0))):
        n = host.size
        rx = Regex(pattern)
        text = torch.from_numpy(host).to(dev)
        cols, st, kind = rx.parse(text)
        torch.cuda.synchronize()
        cb = cols.element_size()
        hcols = cols.cpu().numpy().view({1: np.uint8, 2: np.uint16, 4: np.uint32}[cb])
        t0 = time.perf_counter()
        arch = native.slpf_dfa_encode(hcols, host, 4096)
        enc_s = time.perf_counter() - t0
        hdr = native.slpf_dfa_header(arch)
        for _ in range(3):
            got, gst = native.slpf_dfa_decode(arch, text, cb)
        torch.cuda.synchronize()
        if int(gst.item()) != 0 or not torch.equal(got.view(torch.uint8), cols.view(torch.uint8)):
            raise SystemExit(f"{name}: rebuilt columns differ")
        steps = max(args.steps, 5)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        d_arch = torch.from_numpy(arch).to(dev)
        hdr_c = native.DfaHeader(**hdr)
        out = torch.empty_like(cols)
        status = torch.empty(1, dtype=torch.int32, device=dev)
        lib = native.load()
        e0.record(stream)
        for _ in range(steps):
            native.check(lib.re_slpf_dfa_decode(native.ctypes.byref(hdr_c), d_arch.data_ptr(), d_arch.numel(),
                                                text.data_ptr(), out.data_ptr(), out.numel() * cb, cb,
                                                status.data_ptr(), native.ctypes.c_void_p(stream.cuda_stream)))
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        rows.append({"workload": name, "text_bytes": n, "encoding": f"{kind}-{8 * cb}bit",
                     "column_bytes": (n + 1) * cb, "archive_bytes": int(arch.size),
                     "ratio": round((n + 1) * cb / arch.size, 3),
                     "exceptions_per_column": round(hdr["n_exceptions"] / (n + 1), 4),
                     "table_rows": hdr["n_ids"], "encode_s": round(enc_s, 3),
                     "rebuild_ms": round(ms, 4), "rebuild_GBps": round((n + 1) * cb / ms / 1e6, 1)})
        del text, cols, got, out, d_arch
        torch.cuda.empty_cache()
    line = {"metric": "SLPF archive rebuild GB/s of columns (App. C, re_slpf_dfa_decode), log text",
            "value": rows[0]["rebuild_GBps"], "unit": "GB/s", "n_gpus": world, "steps": max(args.steps, 5),
            "warmup": 3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic", "config": {"workload": f"log, DNA and (a|b|ab)* texts of {n0} bytes, "
                                                        "checkpoint every 4096 columns"}, "rows": rows}
    if rank == 0:
        print(json.dumps(line))


def join_mode(args, rank, world, local):
    """The join phase (Eq. joiner) on 256 MiB texts: the DNA and log
    workloads, whose speculative runs meet inside nearly every chunk, and
    (aa)* on a^n, whose even and odd runs never meet, so every chunk's map
    depends on its input and the join resolves a chain through all of them.
    Per-phase times from CUDA events between phases, autotuned chunk length."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2503_06763_gb300 import Regex
    from paper_2503_06763_gb300.native import PHASES
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.bytes or (256 << 20)
    steps = max(args.steps, 5)
    rows = {}
    cases = (("dna", W.DNA_RE, W.dna_text(n, seed=1)), ("log", W.LOG_RE, W.log_text(n, seed=2)),
             ("aa_star_on_a^n", "(aa)*", np.full(n, ord("a"), dtype=np.uint8)))
    for name, pattern, host in cases:
        rx = Regex(pattern)
        text = torch.from_numpy(host).to(dev)
        k = rx.autotune(text)
        torch.cuda.empty_cache()
        kind, cb, _ = rx.layout(n, "auto")
        dt = {1: torch.uint8, 2: torch.int16, 4: torch.int32, 8: torch.int64}[cb]
        out = torch.empty(n + 1, dtype=dt, device=dev)
        st = torch.empty(1, dtype=torch.int32, device=dev)
        ws = torch.empty(rx.workspace_size(n), dtype=torch.uint8, device=dev)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(PHASES) + 1)] for _ in range(steps)]
        for _ in range(max(args.warmup, 3)):
            rx.parse(text, kind=kind, out=out, status=st, workspace=ws)
        for i in range(steps):
            rx.parse(text, kind=kind, out=out, status=st, workspace=ws, events=ev[i])
        torch.cuda.synchronize()
        ph = {p: round(statistics.median(ev[i][j].elapsed_time(ev[i][j + 1]) for i in range(steps)), 4)
              for j, p in enumerate(PHASES)}
        rows[name] = {"status": int(st.item()), "chunk_len": k, "chunks": (n + k - 1) // k, "phase_ms": ph,
                      "parse_GBps": round(n / (sum(ph.values()) / 1e3) / 1e9, 1)}
        del text, out, ws
        torch.cuda.empty_cache()
    if rank == 0:
        print(json.dumps({"metric": "join phase ms (Eq. joiner, scan over chunk maps)", "unit": "ms",
                          "text_bytes": n, "rows": rows,
                          "join_ratio_to_dna": {k: round(v["phase_ms"]["join"] / rows["dna"]["phase_ms"]["join"], 2)
                                                for k, v in rows.items()}}))


def shard_mode(args, rank, world, local):
    """One text split across the N ranks (Sect. 3.2): every rank holds the
    whole log text (seed 2, default 1 GiB), computes the maps of its slice,
    the maps are all-gathered (the one exchange step, a few hundred bytes per
    rank), every rank composes them into its entry states and parses its
    slice.  A step is all of that; time is the max over ranks and the value
    the text's bytes over it (strong scaling: the work is one text)."""
    import torch
    import workloads as W
    from paper_2503_06763_gb300 import Regex, shard
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    n = args.bytes or (1 << 30)
    host = W.log_text(n, seed=2)
    n = int(host.size)
    rx = Regex(W.LOG_RE)
    text = torch.from_numpy(host).to(dev)
    a, b = shard.slice_bounds(n, world)[rank]
    piece = text[a:b]

    def step():
        return shard.parse_sharded(rx, piece, a > 0, b < n)

    for _ in range(max(args.warmup, 3)):
        cols, st, acc = step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cols, st, acc = step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms_local = (time.perf_counter() - t0) * 1e3
    ms_total, _ = aggregate(ms_local, b - a, dist, dev)
    ms = ms_total / args.steps
    if rank == 0:
        print(json.dumps({"metric": "sharded SLPF parse GB/s of one text (slice maps, all-gather, slice parse)",
                          "value": round(n / (ms / 1e3) / 1e9, 3), "unit": "GB/s", "n_gpus": world,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
                          "higher_is_better": True, "scaling": "strong", "status": int(st.item()),
                          "accepted": bool(acc),
                          "config": {"workload": WORKLOADS["log"][0], "text_bytes": n,
                                     "slices": world, "timing": "host clock around the steps (maps leave the "
                                     "device for the exchange every step)"}}))
    if dist:
        dist.destroy_process_group()


def reference_arm(args, rank, world):
    """The oracle timed on the host cores on a bounded sample per step."""
    if rank != 0:
        return
    import numpy as np
    import workloads as W
    from oracle import serial
    from oracle.re_front import compile_re
    name = args.workload
    desc, re_attr, maker, _, seed, _ = WORKLOADS[name]
    host = getattr(W, maker)(4 << 20, seed=seed)
    c = compile_re(getattr(W, re_attr))
    sample = host[:1 << 20].tobytes()
    for _ in range(args.warmup):
        serial.parse(c, sample)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        serial.parse(c, sample)
    dt = (time.perf_counter() - t0) / args.steps
    v = len(sample) / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": desc, "text_bytes_per_step": len(sample)},
            "cpu_baseline": {"value": round(v, 6), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": "first 1 MiB of the workload text per step, serial oracle"},
            "e2e": {"value": round(v, 6), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
