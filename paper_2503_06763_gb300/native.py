"""ctypes binding of libslpf.so (include/slpf_parser.h), argument marshalling only.

Every step of the parse runs in the library's CUDA kernels; this module only
allocates device buffers with PyTorch and passes their pointers and the
current CUDA stream.  There is no CPU fallback: importing it without the built
library raises ImportError.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libslpf.so")

RE_OK, RE_REJECTED = 0, 1
STATUS_NAMES = {0: "RE_OK", 1: "RE_REJECTED", -1: "RE_E_INVALID_ARG", -2: "RE_E_SYNTAX",
                -3: "RE_E_INFINITE_AMBIGUITY", -4: "RE_E_TOO_MANY_STATES", -5: "RE_E_NOMEM",
                -6: "RE_E_CUDA", -7: "RE_E_TIMEOUT", -8: "RE_E_CAPACITY", -9: "RE_E_INTERNAL"}
KINDS = {"auto": 0, "dense": 1, "dict": 2, "pairs": 3}
KIND_NAMES = {0: "auto", 1: "dense", 2: "dict", 3: "pairs"}
RE_COMPILE_HOST_ONLY = 1
RE_COMPILE_DFA_STARTS = 2
RE_COMPILE_DFA_STARTS_BWD = 4
RE_PARSE_RECOGNIZE_ONLY = 1
RE_PARSE_TEST_STALL_JOIN = 0x80000000     # tests of the join's bounded waits only
REACH_SHAPES = {1: "byte tables, one direction per block, 2 stages", 2: "warp pairs, class tables, 3 stages",
                3: "warp pairs, class tables, 2 stages", 4: "one lane per chunk, both directions, 3 stages"}


def reach_flag(shape: int) -> int:
    """RE_PARSE_REACH(shape): force a reach kernel shape (0: automatic)."""
    return (shape & 7) << 8

EXPORTS = ["re_compile", "re_free", "re_get_info", "re_segment_name", "re_dict_copy",
           "re_slpf_layout", "re_workspace_size", "re_parse", "re_batch_plan", "re_batch_workspace_size",
           "re_batch_chunk_len", "re_parse_batch", "re_batch_run", "re_batch_free", "re_match_workspace_size",
           "re_matches", "re_autotune", "re_tuned", "re_parse_host",
           "re_shard_map_size", "re_shard_map", "re_shard_entry", "re_parse_slice", "re_state_bits",
           "re_parse_static", "re_slpf_dfa_encode", "re_slpf_dfa_decode",
           "re_server_create", "re_server_submit", "re_server_wait", "re_server_poll", "re_server_stats",
           "re_server_clock_ns", "re_server_destroy",
           "re_last_error"]
RE_STATIC_SCRATCH_BYTES = 64 << 20


class ReError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class CompileOpts(ctypes.Structure):
    _fields_ = [("max_states", ctypes.c_uint32), ("max_dict", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("sample_limit", ctypes.c_uint32)]


class ParseOpts(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("chunk_len", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("n_events", ctypes.c_uint32), ("events", ctypes.POINTER(ctypes.c_void_p))]


RE_PHASE_EVENTS = 5
PHASES = ["reach", "join", "fixup", "build_merge"]


class Slpf(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("col_bytes", ctypes.c_uint32), ("n_cols", ctypes.c_uint64),
                ("d_cols", ctypes.c_void_p), ("cols_cap_bytes", ctypes.c_uint64),
                ("d_status", ctypes.c_void_p)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_uint32), ("arena_bytes", ctypes.c_uint64), ("staging_bytes", ctypes.c_uint64),
                ("max_batch", ctypes.c_uint32)]


class DfaHeader(ctypes.Structure):
    _fields_ = [("magic", ctypes.c_uint32), ("version", ctypes.c_uint32), ("n", ctypes.c_uint64),
                ("n_ids", ctypes.c_uint32), ("interval", ctypes.c_uint32), ("n_exceptions", ctypes.c_uint64),
                ("n_checkpoints", ctypes.c_uint64)]


class Info(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in (
        "n_segments", "n_positions", "n_classes", "words_per_col", "fwd_states", "fwd_dfa_states",
        "bwd_states", "bwd_dfa_states", "fwd_slots_max", "bwd_slots_max")] + [("dict_size", ctypes.c_uint64)] + [
        ("inf_ambiguous", ctypes.c_uint32), ("sample_limit", ctypes.c_uint32), ("ascii_rows", ctypes.c_uint32),
        ("reach_shapes", ctypes.c_uint32)]


_lib = None


def load():
    """Load libslpf.so; raise ImportError when it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    lib.re_compile.argtypes = [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(CompileOpts), ctypes.POINTER(vp)]
    lib.re_compile.restype = i32
    lib.re_free.argtypes = [vp]
    lib.re_free.restype = None
    lib.re_get_info.argtypes = [vp, ctypes.POINTER(Info)]
    lib.re_get_info.restype = i32
    lib.re_segment_name.argtypes = [vp, u32, ctypes.c_char_p, ctypes.c_size_t]
    lib.re_segment_name.restype = i32
    lib.re_dict_copy.argtypes = [vp, vp, u64]
    lib.re_dict_copy.restype = i32
    lib.re_slpf_layout.argtypes = [vp, u64, i32, ctypes.POINTER(i32), ctypes.POINTER(u32), ctypes.POINTER(u64)]
    lib.re_slpf_layout.restype = i32
    lib.re_workspace_size.argtypes = [vp, u64, ctypes.POINTER(ParseOpts), ctypes.POINTER(u64)]
    lib.re_workspace_size.restype = i32
    lib.re_parse.argtypes = [vp, vp, u64, vp, ctypes.POINTER(Slpf), vp, u64, ctypes.POINTER(ParseOpts)]
    lib.re_parse.restype = i32
    lib.re_batch_plan.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(u64), u32, ctypes.POINTER(ParseOpts),
                                  ctypes.POINTER(vp)]
    lib.re_batch_plan.restype = i32
    lib.re_batch_workspace_size.argtypes = [vp, ctypes.POINTER(u64)]
    lib.re_batch_workspace_size.restype = i32
    lib.re_batch_chunk_len.argtypes = [vp, u32, ctypes.POINTER(u32)]
    lib.re_batch_chunk_len.restype = i32
    lib.re_parse_batch.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(Slpf), vp, u64, vp]
    lib.re_parse_batch.restype = i32
    lib.re_batch_run.argtypes = [vp, vp]
    lib.re_batch_run.restype = i32
    lib.re_batch_free.argtypes = [vp]
    lib.re_batch_free.restype = None
    lib.re_match_workspace_size.argtypes = [vp, u64, ctypes.POINTER(u64)]
    lib.re_match_workspace_size.restype = i32
    lib.re_matches.argtypes = [vp, ctypes.POINTER(Slpf), u64, u32, vp, u64, vp, vp, u64, vp]
    lib.re_matches.restype = i32
    lib.re_autotune.argtypes = [vp, vp, u64, ctypes.POINTER(Slpf), vp, u64, vp, ctypes.POINTER(ParseOpts),
                                ctypes.POINTER(u32)]
    lib.re_autotune.restype = i32
    lib.re_shard_map_size.argtypes = [vp, ctypes.POINTER(u32), ctypes.POINTER(u32)]
    lib.re_shard_map_size.restype = i32
    lib.re_shard_map.argtypes = [vp, vp, u64, u32, vp, vp, u64, vp, vp]
    lib.re_shard_map.restype = i32
    lib.re_shard_entry.argtypes = [vp, vp, u32, vp, vp, ctypes.POINTER(ctypes.c_int32)]
    lib.re_shard_entry.restype = i32
    lib.re_parse_slice.argtypes = [vp, vp, u64, u32, u32, vp, ctypes.POINTER(Slpf), vp, u64, ctypes.POINTER(ParseOpts)]
    lib.re_parse_slice.restype = i32
    lib.re_state_bits.argtypes = [vp, ctypes.c_int32, u32, vp, u32]
    lib.re_server_create.argtypes = [vp, u32, ctypes.POINTER(ServerOpts), ctypes.POINTER(vp)]
    lib.re_server_create.restype = i32
    lib.re_server_submit.argtypes = [vp, u32, vp, u64, vp, u64, vp, ctypes.POINTER(u64)]
    lib.re_server_submit.restype = i32
    lib.re_server_wait.argtypes = [vp, u64, ctypes.c_int32]
    lib.re_server_wait.restype = i32
    lib.re_server_poll.argtypes = [vp, vp, vp, u32, ctypes.POINTER(u32)]
    lib.re_server_poll.restype = i32
    lib.re_server_stats.argtypes = [vp, vp]
    lib.re_server_stats.restype = i32
    lib.re_server_clock_ns.argtypes = [vp]
    lib.re_server_clock_ns.restype = u64
    lib.re_server_destroy.argtypes = [vp]
    lib.re_server_destroy.restype = None
    lib.re_slpf_dfa_encode.argtypes = [vp, u32, vp, u64, u32, vp, u64, ctypes.POINTER(u64)]
    lib.re_slpf_dfa_encode.restype = i32
    lib.re_slpf_dfa_decode.argtypes = [ctypes.POINTER(DfaHeader), vp, u64, vp, vp, u64, u32, vp, vp]
    lib.re_slpf_dfa_decode.restype = i32
    lib.re_state_bits.restype = i32
    lib.re_tuned.argtypes = [vp, u64, u32, ctypes.POINTER(u32), ctypes.POINTER(u32)]
    lib.re_tuned.restype = i32
    lib.re_parse_host.argtypes = [vp, vp, u64, vp, vp, vp, ctypes.POINTER(Slpf), vp, u64, vp, ctypes.POINTER(ParseOpts)]
    lib.re_parse_host.restype = i32
    lib.re_parse_static.argtypes = [vp, vp, u64, vp, ctypes.POINTER(Slpf), ctypes.POINTER(ParseOpts)]
    lib.re_parse_static.restype = i32
    lib.re_last_error.argtypes = []
    lib.re_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def check(status: int):
    if status != RE_OK:
        raise ReError(status, load().re_last_error().decode(errors="replace"))


class Regex:
    """A compiled RE (owns the library handle and its device tables)."""

    def __init__(self, pattern, max_states: int = 0, max_dict: int = 0, host_only: bool = False,
                 dfa_starts=False, sample_limit: int = 0):
        """dfa_starts: speculation from every DFA state instead of the ME-DFA
        starts, an ablation: True or "fwd" forward (RE_COMPILE_DFA_STARTS),
        "bwd" backward (RE_COMPILE_DFA_STARTS_BWD), "both".  sample_limit: 0
        rejects an infinitely ambiguous RE; L >= 1 samples its LSTs, each
        numbered symbol at most L times per segment (App. A)."""
        lib = load()
        pat = pattern.encode("latin-1") if isinstance(pattern, str) else bytes(pattern)
        self.pattern = pat
        if dfa_starts not in (False, True, "fwd", "bwd", "both"):
            raise ValueError(f"dfa_starts: {dfa_starts!r}")
        flags = (RE_COMPILE_HOST_ONLY if host_only else 0)
        flags |= RE_COMPILE_DFA_STARTS if dfa_starts in (True, "fwd", "both") else 0
        flags |= RE_COMPILE_DFA_STARTS_BWD if dfa_starts in ("bwd", "both") else 0
        opts = CompileOpts(max_states, max_dict, flags, sample_limit)
        h = ctypes.c_void_p()
        check(lib.re_compile(pat, len(pat), ctypes.byref(opts), ctypes.byref(h)))
        self._h = h
        info = Info()
        check(lib.re_get_info(h, ctypes.byref(info)))
        self.info = {n: getattr(info, n) for n, _ in Info._fields_}

    def close(self):
        if getattr(self, "_h", None):
            load().re_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def ell(self) -> int:
        return self.info["n_segments"]

    @property
    def words(self) -> int:
        return self.info["words_per_col"]

    def segment_names(self):
        lib = load()
        buf = ctypes.create_string_buffer(1 << 16)
        out = []
        for i in range(self.ell):
            check(lib.re_segment_name(self._h, i, buf, len(buf)))
            out.append(buf.value.decode())
        return out

    def dictionary(self):
        import numpy as np
        d = self.info["dict_size"]
        arr = np.zeros((d, self.words), dtype=np.uint64)
        if d:
            check(load().re_dict_copy(self._h, arr.ctypes.data, arr.size))
        return arr

    def layout(self, n: int, kind: str = "auto"):
        k, cb, nb = ctypes.c_int(), ctypes.c_uint32(), ctypes.c_uint64()
        check(load().re_slpf_layout(self._h, n, KINDS[kind], ctypes.byref(k), ctypes.byref(cb), ctypes.byref(nb)))
        return KIND_NAMES[k.value], cb.value, nb.value

    def workspace_size(self, n: int, chunk_len: int = 0, flags: int = 0) -> int:
        b = ctypes.c_uint64()
        opts = ParseOpts(0, chunk_len, flags, 0, None)
        check(load().re_workspace_size(self._h, n, ctypes.byref(opts), ctypes.byref(b)))
        return b.value

    def parse(self, text, kind: str = "auto", chunk_len: int = 0, stream=None, out=None, status=None,
              workspace=None, recognize_only: bool = False, events=None, extra_flags: int = 0,
              reach_shape: int = 0):
        """Enqueue the parse of a CUDA uint8 tensor; returns (cols, status, kind).

        ``cols`` is a CUDA tensor of n+1 columns (uint8/int16/int32/int64 view of
        the DENSE bitsets or DICT indices), ``status`` a one-element int32 CUDA
        tensor holding the re_status word.  Nothing is synchronised here.
        Buffers allocated here are allocated on the parse's stream, so torch's
        caching allocator does not give them to other streams' work while the
        parse still uses them."""
        import torch
        if not (isinstance(text, torch.Tensor) and text.is_cuda and text.dtype == torch.uint8):
            raise TypeError("text must be a CUDA uint8 tensor")
        text = text.contiguous()
        n = text.numel()
        kname, cb, nbytes = self.layout(n, kind)
        dt = {1: torch.uint8, 2: torch.int16, 4: torch.int32, 8: torch.int64}[cb]
        flags = (RE_PARSE_RECOGNIZE_ONLY if recognize_only else 0) | extra_flags | reach_flag(reach_shape)
        wsz = self.workspace_size(n, chunk_len, flags & RE_PARSE_RECOGNIZE_ONLY)
        s = stream if stream is not None else torch.cuda.current_stream(text.device)
        with torch.cuda.stream(s):
            if out is None and not recognize_only:  # the recognizer writes no columns
                out = torch.empty(n + 1, dtype=dt, device=text.device)
            if status is None:
                status = torch.empty(1, dtype=torch.int32, device=text.device)
            if workspace is None or workspace.numel() < wsz:
                workspace = torch.empty(max(wsz, 256), dtype=torch.uint8, device=text.device)
            slpf = Slpf(KINDS[kname], cb, 0, out.data_ptr() if out is not None else None,
                        out.numel() * out.element_size() if out is not None else 0, status.data_ptr())
            opts = ParseOpts(KINDS[kname], chunk_len, flags, 0, None)
            if events is not None:          # RE_PHASE_EVENTS torch.cuda.Event objects
                for e in events:
                    if not e.cuda_event:        # torch creates the CUDA event on first record
                        e.record(s)
                arr = (ctypes.c_void_p * RE_PHASE_EVENTS)(*[ctypes.c_void_p(e.cuda_event) for e in events])
                opts.n_events, opts.events = RE_PHASE_EVENTS, ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p))
            check(load().re_parse(self._h, text.data_ptr() if n else None, n, ctypes.c_void_p(s.cuda_stream),
                                  ctypes.byref(slpf), workspace.data_ptr(), workspace.numel(), ctypes.byref(opts)))
        return out, status, kname

    def parse_raw(self, text_ptr: int, n: int, out_ptr: int, out_cap: int, kind: str, cb: int, status_ptr: int,
                  ws_ptr: int, ws_bytes: int, stream_ptr: int):
        """re_parse on raw device pointers (no tensor views): for callers that
        lay out their own buffers, such as the serving loop."""
        slpf = Slpf(KINDS[kind], cb, 0, out_ptr, out_cap, status_ptr)
        opts = ParseOpts(KINDS[kind], 0, 0, 0, None)
        check(load().re_parse(self._h, text_ptr if n else None, n, ctypes.c_void_p(stream_ptr), ctypes.byref(slpf),
                              ws_ptr, ws_bytes, ctypes.byref(opts)))

    def parse_static(self, text, kind: str = "auto", chunk_len: int = 0, stream=None, out=None, status=None,
                     recognize_only: bool = False):
        """Like ``parse`` but through re_parse_static: the library's fixed device
        scratch serves as workspace, so only the output tensors are allocated
        here (pass ``out`` and ``status`` to allocate nothing)."""
        import torch
        if not (isinstance(text, torch.Tensor) and text.is_cuda and text.dtype == torch.uint8):
            raise TypeError("text must be a CUDA uint8 tensor")
        text = text.contiguous()
        n = text.numel()
        kname, cb, _ = self.layout(n, kind)
        dt = {1: torch.uint8, 2: torch.int16, 4: torch.int32, 8: torch.int64}[cb]
        s = stream if stream is not None else torch.cuda.current_stream(text.device)
        with torch.cuda.stream(s):                  # outputs allocated on the parse's stream
            if out is None and not recognize_only:  # the recognizer writes no columns
                out = torch.empty(n + 1, dtype=dt, device=text.device)
            if status is None:
                status = torch.empty(1, dtype=torch.int32, device=text.device)
        slpf = Slpf(KINDS[kname], cb, 0, out.data_ptr() if out is not None else None,
                    out.numel() * out.element_size() if out is not None else 0, status.data_ptr())
        opts = ParseOpts(KINDS[kname], chunk_len, RE_PARSE_RECOGNIZE_ONLY if recognize_only else 0, 0, None)
        check(load().re_parse_static(self._h, text.data_ptr() if n else None, n, ctypes.c_void_p(s.cuda_stream),
                                     ctypes.byref(slpf), ctypes.byref(opts)))
        return out, status, kname

    def matches(self, cols, status, n: int, group: int, kind: str, cap=None, stream=None):
        """re_matches over the columns of a parse of an n-byte text: returns
        an int64 [m, 2] CUDA tensor of (i, j) spans of group ``group`` in
        (i, j) order.  With cap=None a first call counts the matches.  The
        counts are read on the call's stream, after its kernels."""
        import torch
        dev = cols.device
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        cb = cols.element_size()
        slpf = Slpf(KINDS[kind], cb, n + 1, cols.data_ptr(), cols.numel() * cb, status.data_ptr())
        w = ctypes.c_uint64()
        check(load().re_match_workspace_size(self._h, n, ctypes.byref(w)))
        with torch.cuda.stream(s):
            ws = torch.empty(max(w.value, 256), dtype=torch.uint8, device=dev)
            count = torch.zeros(1, dtype=torch.int64, device=dev)
            if cap is None:
                check(load().re_matches(self._h, ctypes.byref(slpf), n, group, None, 0, count.data_ptr(),
                                        ws.data_ptr(), ws.numel(), ctypes.c_void_p(s.cuda_stream)))
                cap = int(count.item())
            pairs = torch.empty((max(cap, 1), 2), dtype=torch.int64, device=dev)
            check(load().re_matches(self._h, ctypes.byref(slpf), n, group, pairs.data_ptr(), cap, count.data_ptr(),
                                    ws.data_ptr(), ws.numel(), ctypes.c_void_p(s.cuda_stream)))
            total = int(count.item())
        return pairs[:min(total, cap)], total

    def autotune(self, text, kind: str = "auto", workspace=None, stream=None, recognize_only: bool = False) -> int:
        """re_autotune on a CUDA uint8 tensor: returns the chunk length chosen
        (and kept for texts of this length bucket, parse or recognizer mode)."""
        import torch
        n = text.numel()
        kname, cb, _ = self.layout(n, kind)
        dt = {1: torch.uint8, 2: torch.int16, 4: torch.int32, 8: torch.int64}[cb]
        s = stream if stream is not None else torch.cuda.current_stream(text.device)
        with torch.cuda.stream(s):                  # scratch allocated on the stream the trials run on
            out = torch.empty(n + 1, dtype=dt, device=text.device)
            status = torch.empty(1, dtype=torch.int32, device=text.device)
            if workspace is None:               # room for every candidate (the shortest chunks need the most)
                workspace = torch.empty(self.workspace_size(n, chunk_len=256), dtype=torch.uint8,
                                        device=text.device)
        slpf = Slpf(KINDS[kname], cb, 0, out.data_ptr(), out.numel() * out.element_size(), status.data_ptr())
        opts = ParseOpts(KINDS[kname], 0, RE_PARSE_RECOGNIZE_ONLY if recognize_only else 0, 0, None)
        k = ctypes.c_uint32()
        check(load().re_autotune(self._h, text.data_ptr(), n, ctypes.byref(slpf), workspace.data_ptr(),
                                 workspace.numel(), ctypes.c_void_p(s.cuda_stream), ctypes.byref(opts),
                                 ctypes.byref(k)))
        return k.value

    def tuned(self, n: int, recognize_only: bool = False):
        """(chunk length, reach shape) re_autotune kept for n-byte texts, or (0, 0)."""
        k, v = ctypes.c_uint32(), ctypes.c_uint32()
        check(load().re_tuned(self._h, n, RE_PARSE_RECOGNIZE_ONLY if recognize_only else 0, ctypes.byref(k),
                              ctypes.byref(v)))
        return k.value, v.value

    def parse_host(self, text, cols, status, d_text, d_cols, d_status, workspace, stream=None, kind: str = "auto",
                   chunk_len: int = 0):
        """re_parse_host: ``text`` / ``cols`` / ``status`` are host tensors
        (pinned for overlap), ``d_*`` and ``workspace`` device tensors.
        Enqueues copy-in, parse and copy-back on the stream; nothing waits."""
        import torch
        n = text.numel()
        kname, cb, _ = self.layout(n, kind)
        s = stream if stream is not None else torch.cuda.current_stream()
        slpf = Slpf(KINDS[kname], cb, 0, d_cols.data_ptr(), d_cols.numel() * d_cols.element_size(),
                    d_status.data_ptr())
        opts = ParseOpts(KINDS[kname], chunk_len, 0, 0, None)
        check(load().re_parse_host(self._h, text.data_ptr() if n else None, n, cols.data_ptr(), status.data_ptr(),
                                   d_text.data_ptr() if n else None, ctypes.byref(slpf), workspace.data_ptr(),
                                   workspace.numel(), ctypes.c_void_p(s.cuda_stream), ctypes.byref(opts)))
        return kname

    # ------------------------------------------------------------------ sharded parse
    def shard_map_size(self):
        """(forward entries, backward entries) of a slice's maps."""
        f, b = ctypes.c_uint32(), ctypes.c_uint32()
        check(load().re_shard_map_size(self._h, ctypes.byref(f), ctypes.byref(b)))
        return f.value, b.value

    def shard_map(self, text, prev: bool, nxt: bool, stream=None):
        """re_shard_map on a CUDA uint8 slice (a view whose neighbouring bytes
        are readable where prev / nxt is set): a host uint8 array of the
        forward then backward map."""
        import numpy as np
        import torch
        n = text.numel()
        nf, nb = self.shard_map_size()
        s = stream if stream is not None else torch.cuda.current_stream(text.device)
        with torch.cuda.stream(s):
            maps = torch.empty(nf + nb, dtype=torch.uint8, device=text.device)
            st = torch.empty(1, dtype=torch.int32, device=text.device)
            ws = torch.empty(max(self.workspace_size(n), 256), dtype=torch.uint8, device=text.device)
        flags = (1 if prev else 0) | (2 if nxt else 0)
        check(load().re_shard_map(self._h, text.data_ptr(), n, flags, ctypes.c_void_p(s.cuda_stream),
                                  ws.data_ptr(), ws.numel(), maps.data_ptr(), st.data_ptr()))
        s.synchronize()
        status = int(st.item())
        if status != RE_OK:
            raise ReError(status, "slice map")
        return maps.cpu().numpy().astype(np.uint8)

    def shard_entry(self, maps):
        """Host composition of the slices' maps (a [N, nf + nb] uint8 array):
        (forward entry states, backward entry states, accepted)."""
        import numpy as np
        m = np.ascontiguousarray(maps, dtype=np.uint8)
        cnt = m.shape[0]
        e = np.zeros(cnt, dtype=np.uint32)
        eb = np.zeros(cnt, dtype=np.uint32)
        acc = ctypes.c_int32()
        check(load().re_shard_entry(self._h, m.ctypes.data, cnt, e.ctypes.data, eb.ctypes.data, ctypes.byref(acc)))
        return e, eb, bool(acc.value)

    def parse_slice(self, text, entry: int, entry_bwd: int, kind: str = "auto", stream=None):
        """re_parse_slice: the slice's len + 1 columns of the whole text's SLPF."""
        import torch
        n = text.numel()
        kname, cb, _ = self.layout(n, kind)
        dt = {1: torch.uint8, 2: torch.int16, 4: torch.int32, 8: torch.int64}[cb]
        s = stream if stream is not None else torch.cuda.current_stream(text.device)
        with torch.cuda.stream(s):
            out = torch.empty(n + 1, dtype=dt, device=text.device)
            status = torch.empty(1, dtype=torch.int32, device=text.device)
            ws = torch.empty(max(self.workspace_size(n), 256), dtype=torch.uint8, device=text.device)
        slpf = Slpf(KINDS[kname], cb, 0, out.data_ptr(), out.numel() * out.element_size(), status.data_ptr())
        opts = ParseOpts(KINDS[kname], 0, 0, 0, None)
        check(load().re_parse_slice(self._h, text.data_ptr(), n, int(entry), int(entry_bwd),
                                    ctypes.c_void_p(s.cuda_stream), ctypes.byref(slpf), ws.data_ptr(), ws.numel(),
                                    ctypes.byref(opts)))
        return out, status, kname

    def state_bits(self, forward: bool, state: int):
        """Segment set of a state as a [W] uint64 array (host)."""
        import numpy as np
        v = np.zeros(self.words, dtype=np.uint64)
        check(load().re_state_bits(self._h, 1 if forward else 0, state, v.ctypes.data, self.words))
        return v

    # ------------------------------------------------------------------ decoding
    def decode(self, cols, kind: str):
        """Columns (host numpy array from ``parse``) -> [(n+1), W] uint64 bitsets."""
        import numpy as np
        cols = np.asarray(cols)
        if kind == "dense":
            v = cols.view({1: np.uint8, 2: np.uint16, 4: np.uint32, 8: np.uint64}[cols.dtype.itemsize])
            return v.astype(np.uint64).reshape(-1, 1)
        if kind == "pairs":                         # (forward state, backward state): C_r = B_r ∩ B̂_r
            if cols.dtype.itemsize == 4:
                v = cols.view(np.uint32).astype(np.uint64)
                f, b = v & 0xFFFF, v >> 16
            else:
                v = cols.view(np.uint64)
                f, b = v & 0xFFFFFFFF, v >> 32
            uf, fi = np.unique(f, return_inverse=True)
            ub, bi = np.unique(b, return_inverse=True)
            fb = np.stack([self.state_bits(True, int(s)) for s in uf]) if uf.size else np.zeros((0, self.words), np.uint64)
            bb = np.stack([self.state_bits(False, int(s)) for s in ub]) if ub.size else np.zeros((0, self.words), np.uint64)
            return fb[fi.reshape(-1)] & bb[bi.reshape(-1)]
        idx = cols.view({1: np.uint8, 2: np.uint16, 4: np.uint32}[cols.dtype.itemsize]).astype(np.int64)
        d = self.dictionary()
        table = np.concatenate([np.zeros((1, self.words), dtype=np.uint64), d], axis=0)
        return table[idx]


class Batch:
    """A planned batch (re_batch_plan): texts j of lens[j] bytes, each under
    regexes[j].  ``parse`` binds CUDA tensors and enqueues every phase as one
    launch per RE; ``run`` re-enqueues the kernels over the same buffers."""

    def __init__(self, regexes, lens, kind: str = "auto", chunk_len: int = 0, recognize_only: bool = False):
        self.regexes = list(regexes)
        self.lens = [int(n) for n in lens]
        if len(self.regexes) != len(self.lens):
            raise ValueError("one length per regex")
        self.count = len(self.lens)
        self.recognize_only = recognize_only
        self.kind = kind
        hs = (ctypes.c_void_p * max(self.count, 1))(*[r._h for r in self.regexes])
        ls = (ctypes.c_uint64 * max(self.count, 1))(*self.lens)
        flags = RE_PARSE_RECOGNIZE_ONLY if recognize_only else 0
        opts = ParseOpts(KINDS[kind], chunk_len, flags, 0, None)
        b = ctypes.c_void_p()
        check(load().re_batch_plan(hs, ls, self.count, ctypes.byref(opts), ctypes.byref(b)))
        self._b = b
        w = ctypes.c_uint64()
        check(load().re_batch_workspace_size(self._b, ctypes.byref(w)))
        self.workspace_size = w.value
        self._keep = None

    def chunk_len(self, j: int) -> int:
        k = ctypes.c_uint32()
        check(load().re_batch_chunk_len(self._b, j, ctypes.byref(k)))
        return k.value

    def parse(self, texts, outs=None, status=None, workspace=None, stream=None):
        """texts: CUDA uint8 tensors (16-byte aligned).  Returns (outs, status,
        kinds): per text a column tensor (None in recognizer mode), one int32
        status word per text, and the encoding name per text."""
        import torch
        if len(texts) != self.count:
            raise ValueError("one text per planned length")
        dev = texts[0].device if self.count else torch.device("cuda", torch.cuda.current_device())
        kinds, specs = [], []
        for rx, n, t in zip(self.regexes, self.lens, texts):
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.uint8 and t.numel() == n):
                raise TypeError("each text must be a CUDA uint8 tensor of its planned length")
            if self.recognize_only:
                kinds.append(None)
                specs.append((0, 1))
            else:
                kname, cb, _ = rx.layout(n, self.kind)
                kinds.append(kname)
                specs.append((KINDS[kname], cb))
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        with torch.cuda.stream(s):                  # buffers allocated on the batch's stream
            if outs is None:
                dts = {1: torch.uint8, 2: torch.int16, 4: torch.int32, 8: torch.int64}
                outs = [None if self.recognize_only else torch.empty(n + 1, dtype=dts[cb], device=dev)
                        for n, (_, cb) in zip(self.lens, specs)]
            if status is None:
                status = torch.empty(max(self.count, 1), dtype=torch.int32, device=dev)
            if workspace is None or workspace.numel() < self.workspace_size:
                workspace = torch.empty(max(self.workspace_size, 256), dtype=torch.uint8, device=dev)
        arr = (Slpf * max(self.count, 1))()
        ptrs = (ctypes.c_void_p * max(self.count, 1))()
        for j in range(self.count):
            o = outs[j]
            k, cb = specs[j]
            arr[j] = Slpf(k, cb, 0, o.data_ptr() if o is not None else None,
                          o.numel() * o.element_size() if o is not None else 0, status.data_ptr() + 4 * j)
            ptrs[j] = texts[j].data_ptr() if self.lens[j] else None
        check(load().re_parse_batch(self._b, ptrs, arr, workspace.data_ptr(), workspace.numel(),
                                    ctypes.c_void_p(s.cuda_stream)))
        self._keep = (list(texts), outs, status, workspace)     # bound buffers stay alive with the batch
        return outs, status, kinds

    def parse_raw(self, text_ptrs, out_ptrs, out_caps, kinds, cbs, status_ptr: int, ws_ptr: int, ws_bytes: int,
                  stream_ptr: int):
        """re_parse_batch on raw device pointers: text j at text_ptrs[j], its
        columns at out_ptrs[j] (out_caps[j] bytes, encoding kinds[j] / cbs[j]),
        status words at status_ptr + 4 j.  The caller keeps the buffers alive."""
        m = max(self.count, 1)
        arr = (Slpf * m)()
        ptrs = (ctypes.c_void_p * m)()
        for j in range(self.count):
            arr[j] = Slpf(KINDS[kinds[j]], cbs[j], 0, out_ptrs[j], out_caps[j], status_ptr + 4 * j)
            ptrs[j] = text_ptrs[j] if self.lens[j] else None
        check(load().re_parse_batch(self._b, ptrs, arr, ws_ptr, ws_bytes, ctypes.c_void_p(stream_ptr)))

    def run(self, stream=None):
        """Enqueue the kernels again over the buffers bound by ``parse``."""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        check(load().re_batch_run(self._b, ctypes.c_void_p(s.cuda_stream)))

    def close(self):
        if getattr(self, "_b", None):
            load().re_batch_free(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------- SLPF archives (App. C)
def slpf_dfa_encode(cols, text, interval: int = 4096):
    """re_slpf_dfa_encode on host arrays: ``cols`` the n + 1 column ids (a numpy
    array of 1, 2 or 4 bytes per id: DICT indices or DENSE values), ``text``
    the n bytes.  Returns the archive as a numpy uint8 array."""
    import numpy as np
    cols = np.ascontiguousarray(cols)
    x = np.ascontiguousarray(np.frombuffer(bytes(text), dtype=np.uint8) if isinstance(text, (bytes, bytearray))
                             else np.asarray(text, dtype=np.uint8))
    if cols.size != x.size + 1:
        raise ValueError("one column per position 0..n")
    lib = load()
    size = ctypes.c_uint64()
    st = lib.re_slpf_dfa_encode(cols.ctypes.data, cols.dtype.itemsize, x.ctypes.data if x.size else None, x.size,
                                interval, None, 0, ctypes.byref(size))
    if st not in (RE_OK, -8):
        check(st)
    out = np.zeros(size.value, dtype=np.uint8)
    check(lib.re_slpf_dfa_encode(cols.ctypes.data, cols.dtype.itemsize, x.ctypes.data if x.size else None, x.size,
                                 interval, out.ctypes.data, out.size, ctypes.byref(size)))
    return out


def slpf_dfa_header(archive) -> dict:
    """The header of an archive (host numpy array) as a dict."""
    import numpy as np
    h = DfaHeader.from_buffer_copy(np.asarray(archive, dtype=np.uint8)[:ctypes.sizeof(DfaHeader)].tobytes())
    return {n: getattr(h, n) for n, _ in DfaHeader._fields_}


def slpf_dfa_decode(archive, text, col_bytes: int, stream=None):
    """re_slpf_dfa_decode: ``archive`` a host numpy array (copied to the
    device) and ``text`` a CUDA uint8 tensor.  Returns (columns, status) as
    CUDA tensors; enqueued on ``stream``."""
    import numpy as np
    import torch
    arch = np.ascontiguousarray(archive, dtype=np.uint8)
    hdr = DfaHeader.from_buffer_copy(arch[:ctypes.sizeof(DfaHeader)].tobytes())
    dev = text.device
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    dt = {1: torch.uint8, 2: torch.int16, 4: torch.int32}[col_bytes]
    with torch.cuda.stream(s):
        d_arch = torch.from_numpy(arch).to(dev, non_blocking=False)
        cols = torch.empty(hdr.n + 1, dtype=dt, device=dev)
        status = torch.empty(1, dtype=torch.int32, device=dev)
    check(load().re_slpf_dfa_decode(ctypes.byref(hdr), d_arch.data_ptr(), d_arch.numel(),
                                    text.data_ptr() if hdr.n else None, cols.data_ptr(), cols.numel() * col_bytes,
                                    col_bytes, status.data_ptr(), ctypes.c_void_p(s.cuda_stream)))
    cols._archive = d_arch                       # keep the device archive alive until the columns are used
    return cols, status


# ---------------------------------------------------------------------- request loop in the library
class NativeServer:
    """re_server: the library's request loop over resident compiled REs.
    ``submit`` queues a host text and returns a ticket; the columns and status
    land in host numpy arrays the server allocates and keeps until the ticket
    is collected with ``result``."""

    def __init__(self, regexes, slots: int = 4, arena_bytes: int = 1 << 30, staging_bytes: int = 0,
                 max_batch: int = 0):
        import numpy as np
        self._np = np
        self.regexes = list(regexes)
        hs = (ctypes.c_void_p * len(self.regexes))(*[r._h for r in self.regexes])
        opts = ServerOpts(slots, arena_bytes, staging_bytes, max_batch)
        h = ctypes.c_void_p()
        check(load().re_server_create(hs, len(self.regexes), ctypes.byref(opts), ctypes.byref(h)))
        self._h = h
        self._live = {}                      # ticket -> (text, cols, status) kept alive until collected

    def clock_ns(self) -> int:
        return load().re_server_clock_ns(self._h)

    def submit(self, re_index: int, text) -> int:
        np = self._np
        x = np.ascontiguousarray(text, dtype=np.uint8)
        _, cb, nbytes = self.regexes[re_index].layout(x.size, "auto")
        cols = np.empty(nbytes // cb, dtype={1: np.uint8, 2: np.uint16, 4: np.uint32, 8: np.uint64}[cb])
        status = np.full(1, -100, dtype=np.int32)
        t = ctypes.c_uint64()
        check(load().re_server_submit(self._h, re_index, x.ctypes.data if x.size else None, x.size,
                                      cols.ctypes.data, cols.nbytes, status.ctypes.data, ctypes.byref(t)))
        self._live[t.value] = (x, cols, status)
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1):
        check(load().re_server_wait(self._h, ticket, timeout_ms))

    def result(self, ticket: int):
        """(columns, status) of a completed request (call after wait/poll)."""
        x, cols, status = self._live.pop(ticket)
        return cols, int(status[0])

    def poll(self, cap: int = 4096):
        """[(ticket, completion time in ns on the server clock)] since the last poll."""
        np = self._np
        t = np.zeros(cap, dtype=np.uint64)
        ns = np.zeros(cap, dtype=np.uint64)
        n = ctypes.c_uint32()
        check(load().re_server_poll(self._h, t.ctypes.data, ns.ctypes.data, cap, ctypes.byref(n)))
        return list(zip(t[:n.value].tolist(), ns[:n.value].tolist()))

    def stats(self) -> dict:
        np = self._np
        v = np.zeros(4, dtype=np.uint64)
        check(load().re_server_stats(self._h, v.ctypes.data))
        return dict(zip(("batches", "requests", "max_batch", "max_inflight"), v.tolist()))

    def close(self):
        if getattr(self, "_h", None):
            load().re_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
