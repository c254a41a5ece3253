"""GPU parity: the CUDA path through the C ABI vs the CPU oracle, bit-exact.

The SLPF is integer data: every column (a set of segments) must be identical.
Segment ids agree because both sides use the canonical segment order, which
``test_native_abi`` checks by name.  Sizes span many chunks and sub-chunks and
end in ragged tails; chunk lengths are swept so speculation, join chains and
checkpoint fixups all run.
"""
import numpy as np
import pytest

import workloads as W
from oracle import serial
from oracle.re_front import compile_re

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2503_06763_gb300 import Regex
    return Regex


_oracle_cache = {}


def oracle_cols(pattern, text: bytes):
    c = _oracle_cache.get(pattern)
    if c is None:
        c = _oracle_cache[pattern] = compile_re(pattern)
    return serial.parse(c, text)


def gpu_cols(rx, host: np.ndarray, kind="auto", chunk_len=0):
    t = torch.from_numpy(np.array(host, dtype=np.uint8, copy=True)).cuda()
    cols, status, k = rx.parse(t, kind=kind, chunk_len=chunk_len)
    torch.cuda.synchronize()
    return rx.decode(cols.cpu().numpy(), k), int(status.item())


def check(rx, pattern, host, kind="auto", chunk_len=0):
    got, st = gpu_cols(rx, host, kind, chunk_len)
    want = oracle_cols(pattern, host.tobytes())
    accepted = serial.accepted(want)
    assert st == (0 if accepted else 1), f"status {st}, oracle accepted={accepted}"
    assert got.shape == want.shape
    bad = np.nonzero(np.any(got != want, axis=1))[0]
    assert bad.size == 0, f"{bad.size} columns differ, first at r={bad[:5].tolist()}"
    return st


SIZES = [0, 1, 2, 63, 64, 65, 127, 1000, 4097, 20000]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("chunk_len", [64, 192, 0])
def test_ab_star(lib, n, chunk_len):
    rx = lib(W.AB_RE)
    check(rx, W.AB_RE, W.ab_text(n, seed=n), chunk_len=chunk_len)
    check(rx, W.AB_RE, W.ab_text(n, seed=n), kind="dict", chunk_len=chunk_len)


@pytest.mark.parametrize("n", [5, 64, 1000, 30000, 100_003])
@pytest.mark.parametrize("chunk_len", [64, 128, 1024, 0])
def test_dna(lib, n, chunk_len):
    rx = lib(W.DNA_RE)
    x = W.dna_text(n, seed=1, mean_gap=500)
    check(rx, W.DNA_RE, x, chunk_len=chunk_len)
    if n <= 30000:
        check(rx, W.DNA_RE, x, kind="dense", chunk_len=chunk_len)


def _ab(rng, lo, hi):
    return "".join(rng.choice(["a", "b"]) for _ in range(int(rng.integers(lo, hi + 1))))


# Texts in each RE's language, built from its own structure: a prefix, then
# pieces of the top-level iteration until about n bytes, then a suffix.
FIXED_RES = {
    "(ab|a)*": (lambda r: "", lambda r: str(r.choice(["ab", "a"])), lambda r: ""),
    "(a|ab|aba)+": (lambda r: "aba", lambda r: str(r.choice(["a", "ab", "aba"])), lambda r: ""),
    "(a|b)*a(a|b){3}": (lambda r: "", lambda r: str(r.choice(["a", "b"])), lambda r: "a" + _ab(r, 3, 3)),
    "((ab)*c|a(bc)*)*": (lambda r: "", lambda r: ("ab" * int(r.integers(0, 4)) + "c") if r.random() < 0.5
                         else ("a" + "bc" * int(r.integers(0, 4))), lambda r: ""),
    "[ab]([^b]|bb)*": (lambda r: str(r.choice(["a", "b"])), lambda r: str(r.choice(["a", "c", "bb"])),
                       lambda r: ""),
    "(aa)*": (lambda r: "", lambda r: "aa", lambda r: ""),
    "(a|b)*(aaa|bbb)(a|b)*": (lambda r: "", lambda r: str(r.choice(["a", "b"])),
                              lambda r: str(r.choice(["aaa", "bbb"])) + _ab(r, 0, 5)),
    "((a|b){1,3}|c{1,2})*": (lambda r: "", lambda r: _ab(r, 1, 3) if r.random() < 0.7
                             else "c" * int(r.integers(1, 3)), lambda r: ""),
    "(a{0,2}b|a|c)*": (lambda r: "", lambda r: str(r.choice(["a" * int(r.integers(0, 3)) + "b", "a", "c"])),
                       lambda r: ""),
    "((a|b){2,}|a|b|c)*": (lambda r: "", lambda r: _ab(r, 2, 6) if r.random() < 0.5
                           else str(r.choice(["a", "b", "c"])), lambda r: ""),
}


def _valid_text(pattern, n, rng):
    pre, piece, post = FIXED_RES[pattern]
    parts, total = [pre(rng)], 0
    total = len(parts[0])
    while total < n:
        p = piece(rng)
        parts.append(p)
        total += len(p)
    parts.append(post(rng))
    return np.frombuffer("".join(parts).encode(), dtype=np.uint8).copy()


@pytest.mark.parametrize("pattern", list(FIXED_RES))
def test_fixed_res_valid_and_corrupted_texts(lib, pattern):
    """Each RE on texts drawn from its own structure (accepted: the columns
    carry the parse), and on corrupted copies of them (one byte replaced by a
    byte the RE has no position for: rejected, every column empty)."""
    import re
    rx = lib(pattern)
    rng = np.random.Generator(np.random.PCG64(len(pattern)))
    accepted = rejected = 0
    for n in (0, 1, 100, 777, 5000):
        x = _valid_text(pattern, n, rng)
        if n <= 100:                              # independent language check (backtracking: short texts)
            assert re.fullmatch(pattern.encode(), x.tobytes()), (pattern, n)
        bad = None
        for _ in range(20):                       # a one-byte change that leaves the language
            if not len(x):
                break
            y = x.copy()
            at = int(rng.integers(0, len(y)))
            y[at] = ord("c") if at == 0 else ord("d")
            if not serial.accepted(oracle_cols(pattern, y.tobytes())):
                bad = y
                break
        for chunk_len in (64, 128, 0):
            assert check(rx, pattern, x, chunk_len=chunk_len) == 0
            accepted += 1
            if bad is not None:
                assert check(rx, pattern, bad, chunk_len=chunk_len) == 1
                rejected += 1
    assert accepted == 15 and rejected >= 9


def test_unconverged_parity_chunks(lib):
    """(aa)* on a^n: speculative runs never meet, every chunk is chained."""
    rx = lib("(aa)*")
    for n in (64 * 5, 64 * 5 + 1, 64 * 40, 64 * 40 + 2):
        x = np.full(n, ord("a"), dtype=np.uint8)
        check(rx, "(aa)*", x, chunk_len=64)
        check(rx, "(aa)*", x, chunk_len=128)


@pytest.mark.parametrize("seed", range(6))
def test_random_res_valid_texts(lib, seed):
    pattern, tree, _ = W.random_re(100 + seed, max_pos=80)
    rx = lib(pattern)
    for n, cl in ((300, 64), (5000, 128), (20000, 0)):
        x = W.sample_text(tree, n, seed)
        check(rx, pattern, x, chunk_len=cl)


def test_rejected_texts(lib):
    rx = lib("(ab|a)*")
    x = np.frombuffer(b"ab" * 500 + b"b" + b"a" * 300, dtype=np.uint8)
    got, st = gpu_cols(rx, x, chunk_len=64)
    assert st == 1 and not got.any()
    x2 = np.frombuffer(b"ab" * 2000 + b"bb", dtype=np.uint8)      # dies in the last chunk
    got, st = gpu_cols(rx, x2, chunk_len=64)
    assert st == 1 and not got.any()


def test_log_records(lib):
    x = W.log_text(60_000, seed=2)
    rx = lib(W.LOG_RE)
    check(rx, W.LOG_RE, x, chunk_len=256)
    check(rx, W.LOG_RE, x, chunk_len=0)


def test_epsilon_and_single_terminal(lib):
    for pattern, text in (("(a|)b", b"b"), ("(a|)b", b"ab"), ("a", b"a"), ("a", b""), ("()", b""),
                          ("()", b"x"), ("(a|b)?", b"")):
        rx = lib(pattern)
        check(rx, pattern, np.frombuffer(text, dtype=np.uint8).copy())


@pytest.mark.parametrize("chunk_len", [64, 128, 0])
def test_recognizer_matches_oracle_acceptance(lib, chunk_len):
    """Recognizer mode (Sect. 4.2): forward reach + join only; the status word
    must be the oracle's accept / reject, for valid and corrupted texts."""
    rng = np.random.Generator(np.random.PCG64(17))
    cases = [(W.DNA_RE, W.dna_text(50_000, seed=3)), (W.AB_RE, W.ab_text(20_001, seed=4))]
    for s in range(4):
        pat, tree, _ = W.random_re(800 + s, 10, 80)
        cases.append((pat, W.sample_text(tree, 6000, seed=s)))
    for pat, host in cases:
        rx = lib(pat)
        for corrupt in (False, True):
            h = np.array(host, dtype=np.uint8, copy=True)
            if corrupt and len(h):
                j = int(rng.integers(0, len(h)))
                h[j] = (int(h[j]) + 1 + int(rng.integers(0, 254))) % 256
            t = torch.from_numpy(h).cuda()
            _, st, _ = rx.parse(t, chunk_len=chunk_len, recognize_only=True)
            torch.cuda.synchronize()
            want = serial.accepted(oracle_cols(pat, h.tobytes()))
            assert int(st.item()) == (0 if want else 1), (pat[:30], corrupt, len(h))


def test_parse_captured_in_cuda_graph(lib):
    """re_parse enqueues kernels only (after a first call has set up the
    launch attributes), so it can be captured in a CUDA graph and replayed on
    new text bytes; each replay gives the parse of the bytes present."""
    rx = lib(W.DNA_RE)
    n = 1 << 20
    text = torch.from_numpy(W.dna_text(n, seed=51)).cuda()
    cols, status, kind = rx.parse(text)
    ws = torch.empty(rx.workspace_size(n), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        rx.parse(text, out=cols, status=status, workspace=ws, stream=side)      # warm-up on the side stream
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        rx.parse(text, out=cols, status=status, workspace=ws)
    for seed in (52, 53):
        host = W.dna_text(n, seed=seed)
        if seed == 53:
            host[n // 2] = ord("N")                                             # rejected text
        text.copy_(torch.from_numpy(host))
        g.replay()
        torch.cuda.synchronize()
        want = oracle_cols(W.DNA_RE, host.tobytes())
        assert int(status.item()) == (0 if serial.accepted(want) else 1)
        assert np.array_equal(rx.decode(cols.cpu().numpy(), kind), want)


def test_parse_host_and_host_columns(lib):
    """re_parse_host with pinned and with pageable host buffers equals the
    device parse; re_parse also writes its columns straight into pinned host
    memory when given it (plain stores: no tensor stores into host memory)."""
    rx = lib(W.DNA_RE)
    n = 3_000_017
    host = W.dna_text(n, seed=61)
    want_cols, want_st, kind = rx.parse(torch.from_numpy(host).cuda())
    torch.cuda.synchronize()
    _, cb, _ = rx.layout(n, kind)
    dt = {1: torch.uint8, 2: torch.int16, 4: torch.int32, 8: torch.int64}[cb]
    pin_in = torch.from_numpy(host).pin_memory()
    d_text = torch.empty(n, dtype=torch.uint8, device="cuda")
    d_cols = torch.zeros(n + 1, dtype=dt, device="cuda")
    d_st = torch.empty(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(rx.workspace_size(n), dtype=torch.uint8, device="cuda")
    for pinned in (True, False):
        cols = torch.zeros(n + 1, dtype=dt)
        st = torch.zeros(1, dtype=torch.int32)
        if pinned:
            cols, st = cols.pin_memory(), st.pin_memory()
        rx.parse_host(pin_in, cols, st, d_text, d_cols, d_st, ws, kind=kind)
        torch.cuda.synchronize()
        assert int(st[0]) == int(want_st.item()) == 0
        assert torch.equal(cols, want_cols.cpu()), pinned
    direct = torch.zeros(n + 1, dtype=dt).pin_memory()
    st2 = torch.zeros(1, dtype=torch.int32, device="cuda")
    rx.parse(torch.from_numpy(host).cuda(), out=direct, status=st2, workspace=ws)
    torch.cuda.synchronize()
    assert int(st2.item()) == 0 and torch.equal(direct, want_cols.cpu())


@pytest.mark.parametrize("pattern,cb", [("(ab)*|b", 1), ("(a|b)*a(a|b){3}", 2), ("(a|b)*a(a|b){5}", 4),
                                        ("(a|b)*a(a|b){13}", 8)])
@pytest.mark.parametrize("kind", ["dense", "dict"])
def test_every_column_width(lib, pattern, cb, kind):
    """DENSE at 1, 2, 4 and 8 bytes per column and DICT (1 byte below 255
    dictionary entries), on texts that reach the tensor-store path (full
    32-group tiles) and end in a ragged tail, against the oracle."""
    rx = lib(pattern)
    got_kind, got_cb, _ = rx.layout(100, kind)
    dict_cb = 1 if rx.info["dict_size"] < 255 else 2
    assert got_kind == kind and (got_cb == cb if kind == "dense" else got_cb == dict_cb)
    rng = np.random.Generator(np.random.PCG64(cb))
    for n in (2048 + 37, 9000):
        if pattern.startswith("(ab)*"):
            host = np.frombuffer((b"ab" * (n // 2)), dtype=np.uint8).copy()
        else:
            host = rng.choice(np.frombuffer(b"ab", dtype=np.uint8), size=n)
        check(rx, pattern, host, kind=kind, chunk_len=0)
        check(rx, pattern, host, kind=kind, chunk_len=256)


@pytest.mark.parametrize("pattern", ["(a|b)*a(a|b){9}", "(a|b)*a(a|b){14}"])
def test_large_automata(lib, pattern):
    """REs with 2^10 .. 2^15 DFA states: one-byte tables in shared memory,
    and (k = 14, about 200 KB of tables) tables read from global memory."""
    rx = lib(pattern)
    rng = np.random.Generator(np.random.PCG64(77))
    for n in (3000, 20_001):
        host = rng.choice(np.frombuffer(b"ab", dtype=np.uint8), size=n)
        check(rx, pattern, host, kind="dict", chunk_len=0)
        check(rx, pattern, host, kind="dense", chunk_len=256)


DFA_START_RES = [W.DNA_RE, W.AB_RE, "(a|b)*a(a|b){3}", "((ab)*c|a(bc)*)*", "(a{0,2}b|a|c)*", "(a|ab|aba)+"]


@pytest.mark.parametrize("pattern", DFA_START_RES)
@pytest.mark.parametrize("which", ["fwd", "bwd", "both"])
def test_dfa_starts_give_the_same_slpf(lib, pattern, which):
    """Speculation from every DFA state (RE_COMPILE_DFA_STARTS forward,
    RE_COMPILE_DFA_STARTS_BWD backward: the ablation of the ME-DFA of
    Sect. 3.1) changes only the speculation: the columns and the recognizer's
    verdict equal the oracle's."""
    import paper_2503_06763_gb300 as pkg
    if pattern == W.DNA_RE and which != "fwd":
        pytest.skip("36 backward runs from every reverse DFA state: refused at compile")
    rx = pkg.Regex(pattern, dfa_starts=which)
    rng = np.random.Generator(np.random.PCG64(31))
    if pattern == W.DNA_RE:
        texts = [W.dna_text(n, seed=5) for n in (1, 5000, 70_001)]
    elif pattern == W.AB_RE:
        texts = [W.ab_text(n, seed=6) for n in (1, 5000, 70_001)]
    else:
        texts = [rng.choice(np.frombuffer(b"aabbc", dtype=np.uint8), size=n) for n in (1, 777, 20_000)]
    for host in texts:
        for chunk_len in (64, 192, 0):
            check(rx, pattern, host, chunk_len=chunk_len)
            t = torch.from_numpy(np.array(host, dtype=np.uint8, copy=True)).cuda()
            _, st, _ = rx.parse(t, chunk_len=chunk_len, recognize_only=True)
            torch.cuda.synchronize()
            assert int(st.item()) == (0 if serial.accepted(oracle_cols(pattern, host.tobytes())) else 1)


# ---------------------------------------------------------------- reach shapes
def _log_high_bytes(n, seed):
    """Log records with 2 % of the bytes other than newlines replaced by bytes
    >= 128 (the lines hit become malformed; [^\\n]* still takes them)."""
    rng = np.random.default_rng(seed)
    host = W.log_text(n, seed=seed).copy()
    hit = (rng.random(host.size) < 0.02) & (host != ord("\n"))
    host[hit] = rng.integers(128, 256, size=int(hit.sum()))
    return host


def _tokens(n, seed, toks):
    rng = np.random.default_rng(seed)
    parts = [toks[j] for j in rng.integers(0, len(toks), size=n)]
    return np.frombuffer(b"".join(parts), dtype=np.uint8).copy()


SHAPE_CASES = [("dna", W.DNA_RE, lambda: W.dna_text(200_003, seed=5, mean_gap=700)),
               ("ab", W.AB_RE, lambda: W.ab_text(100_001, seed=6)),
               ("log", W.LOG_RE, lambda: W.log_text(150_000, seed=7)),
               ("aa", "(aa)*", lambda: np.full(70_000, ord("a"), dtype=np.uint8)),
               # bytes >= 128 folded onto their class's ASCII byte before the byte-table lookups
               ("log-high-bytes", W.LOG_RE, lambda: _log_high_bytes(150_000, seed=8)),
               ("fold-many", r"([\x7f-\xff]a|b)*",
                lambda: _tokens(40_000, 9, [bytes([v, 97]) for v in range(127, 256)] + [b"b"] * 40)),
               # a class of high bytes alone: full 256-byte rows
               ("high-class", r"([ab]|[\x80-\xff]c)*",
                lambda: _tokens(40_000, 10, [b"a", b"b"] + [bytes([v, 99]) for v in range(128, 256, 7)]))]


@pytest.mark.parametrize("shape", [1, 2, 3, 4])
@pytest.mark.parametrize("case", range(len(SHAPE_CASES)))
def test_every_reach_shape(lib, shape, case):
    """Every reach kernel shape (RE_PARSE_REACH: byte tables with a block per
    direction, warp pairs with 3 or 2 ring stages, one lane per chunk) gives
    the oracle's columns, with automatic and short chunks, and the oracle's
    verdict in recognizer mode."""
    name, pattern, make = SHAPE_CASES[case]
    rx = lib(pattern)
    host = make()
    want = oracle_cols(pattern, host.tobytes())
    for chunk_len in (0, 128):
        t = torch.from_numpy(host).cuda()
        cols, st, kind = rx.parse(t, chunk_len=chunk_len, reach_shape=shape)
        _, rst, _ = rx.parse(t, chunk_len=chunk_len, reach_shape=shape, recognize_only=True)
        torch.cuda.synchronize()
        acc = serial.accepted(want)
        assert int(st.item()) == int(rst.item()) == (0 if acc else 1), (name, shape, chunk_len)
        got = rx.decode(cols.cpu().numpy(), kind)
        bad = np.nonzero(np.any(got != want, axis=1))[0]
        assert bad.size == 0, (name, shape, chunk_len, bad[:5].tolist())


# ---------------------------------------------------------------- sampled infinite ambiguity (App. A)
SAMPLED_RES = {
    "(a*|ab)+": (lambda r: str(r.choice(["a", "ab", "aa"])), ""),
    "(a?b?)*": (lambda r: str(r.choice(["a", "b", "ab"])), ""),
    "((a*)*b)*": (lambda r: "a" * int(r.integers(0, 4)) + "b", ""),
    "((ab)?|c*)+a": (lambda r: str(r.choice(["ab", "c", "cc"])), "a"),
    "(a|()|b)*c?": (lambda r: str(r.choice(["a", "b"])), "c"),
}


@pytest.mark.parametrize("pattern", list(SAMPLED_RES))
@pytest.mark.parametrize("limit", [1, 2, 3])
def test_sampled_infinite_ambiguity(lib, pattern, limit):
    """An infinitely ambiguous RE compiled with a sample limit (each numbered
    symbol at most L times per segment) parses on the GPU to the oracle's
    sampled SLPF, on valid texts across chunks and on corrupted ones."""
    rx = lib(pattern, sample_limit=limit)
    c = compile_re(pattern, sample_limit=limit)
    assert rx.segment_names() == c.names() and rx.info["inf_ambiguous"] == 1
    piece, suffix = SAMPLED_RES[pattern]
    rng = np.random.Generator(np.random.PCG64(limit))
    for n in (1, 70, 1000, 20_003):
        parts, size = [], 0
        while size < n:
            parts.append(piece(rng)); size += len(parts[-1])
        text = ("".join(parts) + suffix).encode()
        variants = [text]
        if len(text) > 8:
            bad = bytearray(text); bad[len(text) // 3] = ord("x")
            variants.append(bytes(bad))
        for t in variants:
            host = np.frombuffer(t, dtype=np.uint8)
            want = serial.parse(c, t)
            for chunk_len in (64, 0):
                got, st = gpu_cols(rx, host, chunk_len=chunk_len)
                assert st == (0 if serial.accepted(want) else 1), (pattern, limit, n)
                bad_cols = np.nonzero(np.any(got != want, axis=1))[0]
                assert bad_cols.size == 0, (pattern, limit, n, chunk_len, bad_cols[:5].tolist())


# ---------------------------------------------------------------- PAIRS columns (no dictionary needed)
@pytest.mark.parametrize("case", ["log", "dna", "log-nodict"])
def test_pair_columns(lib, case):
    """RE_SLPF_PAIRS: every column is the pair of the forward and backward DFA
    states there, and their segment sets meet in the oracle's column (Eq.
    merger).  Log and DNA force the encoding (per-position-state and
    checkpoint merges); the log RE (162 segments) compiled with no room for a
    dictionary gets it from AUTO."""
    if case == "log":
        pattern, rx, kind = W.LOG_RE, lib(W.LOG_RE), "pairs"
        texts = [W.log_text(n, seed=9) for n in (1, 900, 70_000)]
    elif case == "dna":
        pattern, rx, kind = W.DNA_RE, lib(W.DNA_RE), "pairs"
        texts = [W.dna_text(n, seed=9) for n in (1, 900, 70_001)]
    else:
        pattern = W.LOG_RE
        rx, kind = lib(pattern, max_dict=1), "auto"
        assert rx.info["dict_size"] == 0 and rx.ell > 64 and rx.layout(100, "auto")[0] == "pairs"
        texts = [W.log_text(n, seed=10) for n in (1, 900, 70_000)]
        bad = W.log_text(5000, seed=11).copy()
        bad[-1] = ord("x")                                   # no final newline: rejected
        texts.append(bad)
    for host in texts:
        host = np.ascontiguousarray(host)
        want = oracle_cols(pattern, host.tobytes())
        for chunk_len in (64, 0):
            t = torch.from_numpy(host.copy()).cuda()
            cols, st, kname = rx.parse(t, chunk_len=chunk_len, kind=kind)
            torch.cuda.synchronize()
            assert kname == "pairs"
            assert int(st.item()) == (0 if serial.accepted(want) else 1)
            got = rx.decode(cols.cpu().numpy(), kname)
            bad = np.nonzero(np.any(got != want, axis=1))[0]
            assert bad.size == 0, (case, len(host), chunk_len, bad[:5].tolist())
