"""Serving loop: continuous batching of parse requests on one GPU.

Compiled automata stay resident on the device (one ``Regex`` per RE).
Requests -- (RE index, text bytes) -- are admitted as they arrive into the
next free *slot*.  A slot owns a CUDA stream, a device arena and pinned host
staging buffers, all allocated once when the server starts.  A request joins
a slot's batch only if its device footprint fits in the slot's arena:

    text + SLPF columns + its share of the batch workspace.

So the device memory a request's SLPF output needs is what admits it.  Each
slot runs one ``re_parse_batch`` over its requests:

    one host->device copy of all their texts,
    the batch kernels (one launch per phase and RE),
    one device->host copy of all their columns and status words.

While a slot is on the GPU, requests that arrive meanwhile fill the other
slots.  Their work overlaps on the device, and a slot is reused as soon as
its event completes.

Every request gets back the same bytes as ``Regex.parse`` on its text alone:
the batch kernels compute each text independently.
"""
from __future__ import annotations

import time
from collections import deque
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

from .native import Batch, Regex


def _align(v: int, a: int = 256) -> int:
    return (v + a - 1) // a * a


@dataclass
class Request:
    rid: int
    re_index: int
    text: np.ndarray                 # host bytes (uint8)
    arrival: float = 0.0             # seconds on the server clock
    done: float = 0.0
    status: int = -100
    cols: np.ndarray | None = None   # host copy of the SLPF columns
    kind: str = ""


@dataclass
class _Slot:
    stream: object
    arena: object                    # device uint8
    pin_in: object                   # pinned host uint8 (texts)
    pin_out: object                  # pinned host uint8 (columns + status words)
    event: object = None
    reqs: list = field(default_factory=list)
    batch: Batch | None = None
    views: list = field(default_factory=list)


class Server:
    """Continuous-batching request loop over resident compiled REs."""

    def __init__(self, patterns, slots: int = 4, arena_bytes: int = 2 << 30, max_batch: int = 4096,
                 device=None, copy_threads: int = 8):
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.regexes = [p if isinstance(p, Regex) else Regex(p) for p in patterns]
        self.max_batch = max_batch
        self.arena_bytes = arena_bytes
        self.slots = []
        for _ in range(slots):
            self.slots.append(_Slot(
                stream=torch.cuda.Stream(self.dev),
                arena=torch.empty(arena_bytes, dtype=torch.uint8, device=self.dev),
                pin_in=torch.empty(arena_bytes // 4, dtype=torch.uint8).pin_memory(),
                pin_out=torch.empty(arena_bytes // 2, dtype=torch.uint8).pin_memory()))
        self.stats = {"batches": 0, "requests": 0, "max_batch": 0, "max_inflight": 0}
        # staging copies of a batch's texts run on several host threads (numpy
        # releases the interpreter lock while it copies)
        self._copy_pool = ThreadPoolExecutor(max_workers=copy_threads) if copy_threads > 1 else None
        self._prepare()

    # ------------------------------------------------------------------ sizing
    def _prepare(self):
        """Per RE: its column encoding (independent of the text length) and a
        bound on a text's workspace for any chunk length of at least 256 (the
        shortest the library picks): 8 bytes of checkpoints per 64 text bytes,
        the slot ends, run records and join-scan maps of every 256-byte chunk, and
        the alignment of the workspace arrays."""
        self._enc, self._ws_chunk = [], []
        for rx in self.regexes:
            kname, cb, _ = rx.layout(1, "auto")
            info = rx.info
            self._enc.append((kname, cb))
            scan = 2 * (info["fwd_dfa_states"] + 1) + 2 * (info["bwd_dfa_states"] + 1) + 16   # join scan maps
            self._ws_chunk.append(4 * (info["fwd_slots_max"] + info["bwd_slots_max"]) + 64 + 2 * (32 * 4 + 96 * 8)
                                  + scan)

    def ws_bound(self, re_index: int, n: int) -> int:
        # + per-position forward and backward states (one byte each, when the
        # library stores them)
        return 12288 + (n // 256 + 1) * self._ws_chunk[re_index] + (n // 64 + 1) * 8 + 2 * (n + 1 + 128) + 512

    def footprint(self, req: Request) -> tuple[int, int, int]:
        """(device bytes, pinned-in bytes, pinned-out bytes) a request needs:
        its text, its columns, a bound on its workspace and its share of the
        batch descriptors (under 1 KiB a text)."""
        n = len(req.text)
        _, cb = self._enc[req.re_index]
        cols = _align((n + 1) * cb)
        return _align(n) + cols + _align(self.ws_bound(req.re_index, n)) + 1024, _align(n), cols

    def fits_alone(self, req: Request) -> bool:
        d, i, o = self.footprint(req)
        s = self.slots[0]
        return d + (1 << 20) <= self.arena_bytes and i <= s.pin_in.numel() and o + 4096 <= s.pin_out.numel()

    # ------------------------------------------------------------------ one slot
    def _launch(self, slot: _Slot, reqs: list):
        torch = self.torch
        lens = [len(r.text) for r in reqs]
        enc = [self._enc[r.re_index] for r in reqs]
        # arena: [texts][columns][status words][workspace]
        offs_t, o = [], 0
        for n in lens:
            offs_t.append(o)
            o += _align(n)
        text_end = o
        offs_c = []
        for n, (_, cb) in zip(lens, enc):
            offs_c.append(o)
            o += _align((n + 1) * cb)
        st_off = o
        o += _align(4 * len(reqs))
        out_end = o
        ws_off = o
        single = len(reqs) == 1
        if single:                                            # one text: plain re_parse, no batch plan
            b = None
            ws_bytes = self.regexes[reqs[0].re_index].workspace_size(lens[0])
        else:
            b = Batch([self.regexes[r.re_index] for r in reqs], lens)
            ws_bytes = b.workspace_size
        if ws_off + ws_bytes > self.arena_bytes or text_end > slot.pin_in.numel() \
                or out_end - text_end > slot.pin_out.numel():
            if b is not None:
                b.close()
            raise RuntimeError("slot arena too small for the admitted batch")
        pin_in = slot.pin_in.numpy()                         # texts into pinned staging

        def stage(lo, hi):
            for r, ot in zip(reqs[lo:hi], offs_t[lo:hi]):
                pin_in[ot:ot + len(r.text)] = r.text

        if self._copy_pool is not None and text_end > (4 << 20):
            parts = self._copy_pool._max_workers
            cut = [0]                                         # equal bytes per thread
            for j, ot in enumerate(offs_t):
                if ot >= text_end * len(cut) / parts and len(cut) < parts:
                    cut.append(j)
            cut.append(len(reqs))
            list(self._copy_pool.map(lambda ab: stage(*ab), zip(cut[:-1], cut[1:])))
        else:
            stage(0, len(reqs))
        A = slot.arena
        base = A.data_ptr()
        with torch.cuda.stream(slot.stream):
            if text_end:
                A[:text_end].copy_(slot.pin_in[:text_end], non_blocking=True)
            sp = slot.stream.cuda_stream
            if single:
                kname, cb = enc[0]
                self.regexes[reqs[0].re_index].parse_raw(base + offs_t[0], lens[0], base + offs_c[0],
                                                         (lens[0] + 1) * cb, kname, cb, base + st_off,
                                                         base + ws_off, max(ws_bytes, 256), sp)
            else:
                b.parse_raw([base + ot for ot in offs_t], [base + oc for oc in offs_c],
                            [(n + 1) * cb for n, (_, cb) in zip(lens, enc)], [k for k, _ in enc],
                            [cb for _, cb in enc], base + st_off, base + ws_off, max(ws_bytes, 256), sp)
            slot.pin_out[:out_end - text_end].copy_(A[text_end:out_end], non_blocking=True)
            slot.event = torch.cuda.Event()
            slot.event.record(slot.stream)
        slot.reqs = reqs
        slot.batch = b
        slot.views = [(oc - text_end, n, cb, k) for oc, n, (k, cb) in zip(offs_c, lens, enc)] + [st_off - text_end]

    def _retire(self, slot: _Slot, now: float, keep_cols: bool):
        out = slot.pin_out.numpy()
        st_rel = slot.views[-1]
        status = out[st_rel:st_rel + 4 * len(slot.reqs)].view(np.int32).tolist()
        dt = {1: np.uint8, 2: np.uint16, 4: np.uint32, 8: np.uint64}
        for j, (r, (oc, n, cb, k)) in enumerate(zip(slot.reqs, slot.views[:-1])):
            r.status = status[j]
            r.kind = k
            r.done = now
            if keep_cols:
                r.cols = out[oc:oc + (n + 1) * cb].view(dt[cb]).copy()
        if slot.batch is not None:
            slot.batch.close()
        slot.batch, slot.reqs, slot.event, slot.views = None, [], None, []

    # ------------------------------------------------------------------ loop
    def run(self, requests: list, realtime: bool = True, keep_cols: bool = False, poll_sleep: float = 20e-6):
        """Serve ``requests`` (sorted by arrival, seconds from start).  With
        realtime=False every request is available at once (offline).  Fills
        each request's status / done (and cols with keep_cols); returns the
        wall time the loop took."""
        for r in requests:
            if not self.fits_alone(r):
                raise ValueError(f"request {r.rid} ({len(r.text)} bytes) exceeds a slot's arena")
        fp = {id(r): self.footprint(r) for r in requests}
        waiting = deque()
        nxt = 0
        t0 = time.perf_counter()
        pending = len(requests)
        while pending:
            now = time.perf_counter() - t0
            while nxt < len(requests) and (not realtime or requests[nxt].arrival <= now):
                waiting.append(requests[nxt])
                nxt += 1
            progressed = False
            for s in self.slots:                                   # retire finished slots
                if s.event is not None and s.event.query():
                    pending -= len(s.reqs)
                    self._retire(s, time.perf_counter() - t0, keep_cols)
                    progressed = True
            free = sum(1 for s in self.slots if s.event is None)
            for s in self.slots:                                   # admit into free slots
                if not waiting:
                    break
                if s.event is not None:
                    continue
                # light load (no more waiting requests than free slots): every request
                # gets a slot of its own at once; otherwise one slot takes all it can
                share = 1 if len(waiting) <= free else self.max_batch
                free -= 1
                take, dev_used, in_used, out_used = [], 1 << 20, 0, 4096
                while waiting and len(take) < min(self.max_batch, share):
                    d, i, o = fp[id(waiting[0])]
                    if take and (dev_used + d > self.arena_bytes or in_used + i > s.pin_in.numel()
                                 or out_used + o > s.pin_out.numel()):
                        break
                    take.append(waiting.popleft())
                    dev_used, in_used, out_used = dev_used + d, in_used + i, out_used + o
                self._launch(s, take)
                self.stats["batches"] += 1
                self.stats["requests"] += len(take)
                self.stats["max_batch"] = max(self.stats["max_batch"], len(take))
                self.stats["max_inflight"] = max(self.stats["max_inflight"],
                                                 sum(1 for q in self.slots if q.event is not None))
                progressed = True
            if not progressed:
                if nxt < len(requests) and realtime and not waiting:
                    gap = requests[nxt].arrival - (time.perf_counter() - t0)
                    if gap > 0:
                        time.sleep(min(gap, 1e-3))
                else:
                    time.sleep(poll_sleep)
        return time.perf_counter() - t0

    def close(self):
        self.torch.cuda.synchronize(self.dev)
        if self._copy_pool is not None:
            self._copy_pool.shutdown()
        for s in self.slots:
            if s.batch is not None:
                s.batch.close()
        self.slots = []


def latency_summary(requests: list) -> dict:
    lat = np.array([r.done - r.arrival for r in requests]) * 1e3
    return {"p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "mean_ms": round(float(lat.mean()), 3), "max_ms": round(float(lat.max()), 3)}
