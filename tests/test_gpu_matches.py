"""Match extraction on the device (re_matches) against the oracle.

Expected spans come from the oracle's own SLPF and its forest visit, which
brute force pins to the spans of every syntax tree; the device reads the
columns its parse wrote.  Also: the closed form of (a|b|ab)* at 1 MiB (group
5 spans exactly the occurrences of "ab"), rejected texts, the capacity
contract, and the ORF group of the DNA RE on 16 MiB (every span starts with
ATG, ends with a stop codon, and is a whole number of codons).
"""
import numpy as np
import pytest

import workloads as W
from oracle import matches as M
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


def groups(c):
    return sorted({s[1] for seg in c.segments for s in seg if s[0] == "("})


def device_matches(rx, host, group, chunk_len=0, kind="auto"):
    t = torch.from_numpy(np.ascontiguousarray(host)).cuda()
    cols, st, kind = rx.parse(t, chunk_len=chunk_len, kind=kind)
    pairs, total = rx.matches(cols, st, len(host), group, kind)
    torch.cuda.synchronize()
    return [tuple(p) for p in pairs.cpu().numpy().tolist()], total, int(st.item())


@pytest.mark.parametrize("pattern,make", [
    (W.AB_RE, lambda n, s: W.ab_text(n, seed=s)),
    (W.DNA_RE, lambda n, s: W.dna_text(n, seed=s, mean_gap=300, p_geom=0.2, max_codons=40)),
    ("(a|ab|aba)+", lambda n, s: W.ab_text(n, seed=s)),
    ("((ab)*c|a(bc)*)*", None),
])
def test_every_group_matches_oracle(lib, pattern, make):
    c = compile_re(pattern)
    rx = lib(pattern)
    for s, n in enumerate([0, 1, 7, 64, 200, 2001]):
        if make is not None:
            host = make(n, s)
        else:
            host = np.frombuffer((b"abc" * (n // 3 + 1))[:n], dtype=np.uint8).copy()
        cols = [serial.from_bits(row) for row in serial.parse(c, host.tobytes())]
        for k in groups(c):
            want = M.matches_by_slpf(c, host.tobytes(), k, cols)
            got, total, st = device_matches(rx, host, k, chunk_len=64 if n > 128 else 0)
            assert total == len(want) and got == want, (pattern, n, k)


def test_ab_group5_is_every_ab_at_1mib(lib):
    rx = lib(W.AB_RE)
    host = W.ab_text(1 << 20, seed=0)
    got, total, st = device_matches(rx, host, 5)
    idx = np.nonzero((host[:-1] == ord("a")) & (host[1:] == ord("b")))[0]
    assert st == 0 and total == len(idx)
    assert got == [(int(i), int(i) + 2) for i in idx]
    whole, total1, _ = device_matches(rx, host, 1)
    assert whole == [(0, len(host))] and total1 == 1


def test_rejected_text_and_capacity(lib):
    rx = lib(W.AB_RE)
    host = W.ab_text(5000, seed=4)
    bad = host.copy()
    bad[100] = ord("z")
    got, total, st = device_matches(rx, bad, 5)
    assert st == 1 and total == 0 and got == []
    t = torch.from_numpy(host).cuda()
    cols, st, kind = rx.parse(t)
    full, total = rx.matches(cols, st, len(host), 5, kind)
    part, total2 = rx.matches(cols, st, len(host), 5, kind, cap=10)
    torch.cuda.synchronize()
    assert total2 == total > 10 and torch.equal(part, full[:10])
    with pytest.raises(Exception):
        rx.matches(cols, st, len(host), 3, kind)              # 3 is a terminal, not a group


def test_dna_stop_codon_group_on_16mib(lib):
    """Group 13 of the DNA RE is the stop codon closing an ORF.  A stop codon
    at i is a match (i, i+3) exactly when an ATG starts in the same frame at
    some i' <= i - 3 (the codon star matches any codon, stops included, and
    every other byte parses as a single base): a closed form per frame."""
    rx = lib(W.DNA_RE)
    c = compile_re(W.DNA_RE)
    assert "8( )8 13( 14( t15" in c.names()                  # 8: codon star, 13: stop union
    host = W.dna_text(16 << 20, seed=7)
    got, total, st = device_matches(rx, host, 13)
    assert st == 0 and total == len(got)
    n = len(host)
    tri = host[:-2].astype(np.int64) << 16 | host[1:-1].astype(np.int64) << 8 | host[2:].astype(np.int64)
    code = lambda s: s[0] << 16 | s[1] << 8 | s[2]
    is_atg = tri == code(b"ATG")
    is_stop = (tri == code(b"TAA")) | (tri == code(b"TAG")) | (tri == code(b"TGA"))
    want = []
    for f in range(3):
        atg = np.nonzero(is_atg[f::3])[0]
        if len(atg) == 0:
            continue
        first = f + 3 * int(atg[0])
        stops = np.nonzero(is_stop[f::3])[0] * 3 + f
        want.extend(int(i) for i in stops if i >= first + 3)
    want = sorted((i, i + 3) for i in want)
    assert got == want and total > 100_000


def test_wide_columns_log_re(lib):
    """162 segments: three words per column (the kernels round up to four)."""
    rx = lib(W.LOG_RE)
    c = compile_re(W.LOG_RE)
    assert rx.words == 3
    host = W.log_text(20_000, seed=5)
    cols = [serial.from_bits(row) for row in serial.parse(c, host.tobytes())]
    ks = groups(c)
    pick = [ks[0], ks[1], ks[len(ks) // 3], ks[len(ks) // 2], ks[-1]]
    for k in pick:
        want = M.matches_by_slpf(c, host.tobytes(), k, cols)
        got, total, st = device_matches(rx, host, k)
        assert st == 0 and total == len(want) and got == want, k


def test_pair_columns_log_re(lib):
    """Columns written as (forward state, backward state) pairs (RE_SLPF_PAIRS)
    give the same spans: the device intersects the two states' segment sets."""
    rx = lib(W.LOG_RE)
    c = compile_re(W.LOG_RE)
    host = W.log_text(20_000, seed=6)
    cols = [serial.from_bits(row) for row in serial.parse(c, host.tobytes())]
    ks = groups(c)
    for k in (ks[0], ks[len(ks) // 2], ks[-1]):
        want = M.matches_by_slpf(c, host.tobytes(), k, cols)
        got, total, st = device_matches(rx, host, k, kind="pairs")
        assert st == 0 and total == len(want) and got == want, k
