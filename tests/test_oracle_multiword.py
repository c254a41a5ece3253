"""Pins of the oracle's multi-word bitset path (more than 64 segments).

``serial.parse`` runs Fig. (serialparser) in C over bitset columns of
W = ceil(ell / 64) words; every word index there matters only once ell > 64.
``serial.parse_small`` runs the same equations (Eq. matrixmul and the reverse
NFA of Eq. reverseNFAdef) over Python sets, which have no word layout at all,
so the two agreeing column by column on REs with ell > 64 pins the C loops'
word indexing.  A word-index slip planted in a copy of the C source (on the
CPU, compiled with gcc into a scratch directory) must make them disagree.

Also here: the optional operator against bounded repetition, App. A's
identity e? = e{0,1}, on the oracle and on the library's host compiler.
"""
import ctypes
import itertools
import os
import subprocess

import numpy as np
import pytest

import workloads as W
from oracle import serial
from oracle.re_front import compile_re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _log_lines(n_good: int, seed: int) -> bytes:
    """Whole lines of the log workload (about 90 bytes each)."""
    x = W.log_text(n_good * 120, seed=seed).tobytes()
    lines = x.split(b"\n")[:n_good]
    return b"\n".join(lines) + b"\n"


def _cases():
    """(pattern, text) pairs with ell > 64: accepted and rejected texts."""
    out = []
    log = W.LOG_RE
    good = _log_lines(24, seed=5)
    out.append((log, good))                                  # accepted, mostly well-formed lines
    bad = bytearray(good)
    for pos in (7, 300, 911, 1500):                          # malformed lines: the catch-all line parses them
        bad[pos] = ord("#")
    out.append((log, bytes(bad)))
    out.append((log, good[:-1]))                             # no final newline: rejected
    rng = np.random.Generator(np.random.PCG64(3))
    ab = "(a|b)*a(a|b){30}"
    for n in (31, 40, 200):
        out.append((ab, bytes(rng.choice(np.frombuffer(b"ab", dtype=np.uint8), size=n))))
    for seed in (11, 19):                                    # random REs of 140 and 103 segments
        pattern, tree, _ = W.random_re(seed, 10, 60)
        out.append((pattern, W.sample_text(tree, 600, seed=seed).tobytes()))
    return out


CASES = _cases()


def test_cases_need_several_words():
    for pattern, text in CASES:
        assert compile_re(pattern).ell > 64, pattern
    accepted = [serial.accepted(serial.parse(compile_re(p), t)) for p, t in CASES]
    assert any(accepted) and not all(accepted)


def _as_sets(cols):
    return [serial.from_bits(row) for row in cols]


@pytest.mark.parametrize("k", range(len(CASES)))
def test_multiword_c_loops_match_python_sets(k):
    """Eq. (matrixmul) over W-word bitsets (C) equals the same products over
    Python sets, at every column, for ell > 64."""
    pattern, text = CASES[k]
    c = compile_re(pattern)
    got = _as_sets(serial.parse(c, text))
    want = serial.parse_small(c, text)
    assert len(got) == len(want) == len(text) + 1
    for r, (g, w) in enumerate(zip(got, want)):
        assert g == w, (pattern[:40], r)


def _planted_library(tmp_path, old: str, new: str, name: str = "planted"):
    src = open(os.path.join(ROOT, "oracle", "serial_parser.c")).read()
    if old:                                                  # every occurrence: the plain and interned loops
        assert src.count(old) >= 1, old
        src = src.replace(old, new)
    path = tmp_path / f"{name}.c"
    path.write_text(src)
    lib = tmp_path / f"lib{name}.so"
    subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", str(lib), str(path)])
    so = ctypes.CDLL(str(lib))
    so.oracle_serial_parse.restype = ctypes.c_int
    so.oracle_serial_parse.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                       ctypes.c_void_p]
    return so


def _run(so, c, text):
    x = np.frombuffer(text, dtype=np.uint8).copy()
    Wd = serial.words(c.ell)
    ncol = serial.nfa_columns(c)
    I, F = serial.to_bits(c, c.initial), serial.to_bits(c, c.final)
    out = np.zeros((len(x) + 1, Wd), dtype=np.uint64)
    tmp = np.zeros(2 * Wd, dtype=np.uint64)
    assert so.oracle_serial_parse(c.ell, Wd, ncol.ctypes.data, I.ctypes.data, F.ctypes.data, x.ctypes.data,
                                  len(x), out.ctypes.data, tmp.ctypes.data) == 0
    return out


@pytest.mark.parametrize("old,new", [
    ("if (prev[j >> 6] >> (j & 63) & 1)", "if (prev[0] >> (j & 63) & 1)"),      # forward: bit j read in word 0
    ("chat[j >> 6] |= 1ull << (j & 63)", "chat[0] |= 1ull << (j & 63)"),        # backward: bit j set in word 0
])
def test_planted_word_index_mistake_is_caught(tmp_path, old, new):
    """A word-index slip for segments j >= 64 passes every single-word pin but
    must fail the multi-word pin above."""
    so = _planted_library(tmp_path, old, new)
    caught = False
    for pattern, text in CASES[:2]:
        c = compile_re(pattern)
        if _as_sets(_run(so, c, text)) != serial.parse_small(c, text):
            caught = True
    assert caught
    # the unplanted source built and run the same way agrees: the harness is sound
    so_ok = _planted_library(tmp_path, "", "", name="unplanted")
    for pattern, text in CASES[:2]:
        c = compile_re(pattern)
        assert _as_sets(_run(so_ok, c, text)) == serial.parse_small(c, text)


# --------------------------------------------------------------------------- e? = e{0,1} (App. A)
OPTIONAL_PAIRS = [("a?b", "a{0,1}b"), ("(ab|c)?a", "(ab|c){0,1}a"), ("(a(b|c)?)*", "(a(b|c){0,1})*"),
                  ("a*b", "a{0,}b"), ("(ab|c)*", "(ab|c){0,}")]


@pytest.mark.parametrize("p1,p2", OPTIONAL_PAIRS)
def test_optional_is_bounded_repetition_zero_one(p1, p2):
    """App. A states e? = e{0,1}; with h = 0 the repetition node is the
    optional itself (and e{0,} the star), so both spellings give the same
    numbered RE: the same segment names, FolSeg, and SLPF on every text over
    {a, b, c} up to length 5."""
    c1, c2 = compile_re(p1), compile_re(p2)
    assert c1.names() == c2.names()
    assert c1.folseg == c2.folseg and c1.initial == c2.initial and c1.final == c2.final
    for n in range(6):
        for tup in itertools.product(b"abc", repeat=n):
            t = bytes(tup)
            assert serial.parse_small(c1, t) == serial.parse_small(c2, t), (p1, t)


@pytest.mark.parametrize("p1,p2", OPTIONAL_PAIRS)
def test_native_compiler_keeps_the_identity(p1, p2):
    """The library's host compiler reads e{0,1} and e{0,} the same way."""
    try:
        from paper_2503_06763_gb300.native import Regex
        Regex("a", host_only=True)
    except ImportError:
        import __graft_entry__
        __graft_entry__.build()
        from paper_2503_06763_gb300.native import Regex
    r1, r2 = Regex(p1, host_only=True), Regex(p2, host_only=True)
    assert r1.segment_names() == r2.segment_names() == compile_re(p1).names()


# --------------------------------------------------------------------------- interned columns
def _interned_cases():
    rng = np.random.Generator(np.random.PCG64(9))
    out = list(CASES)
    out.append((W.DNA_RE, W.dna_text(50_000, seed=4).tobytes()))
    out.append((W.AB_RE, W.ab_text(20_000, seed=4).tobytes()))
    out.append(("(aa)*", b"a" * 999))                         # rejected: odd length
    out.append(("(aa)*", b"a" * 1000))
    out.append((W.AB_RE, b""))                                # empty text: one column I ∩ F
    out.append(("(a|b)*a(a|b){30}", bytes(rng.choice(np.frombuffer(b"ab", dtype=np.uint8), size=3000))))
    return out


@pytest.mark.parametrize("k", range(len(_interned_cases())))
def test_interned_columns_equal_the_plain_parser(k):
    """serial.parse_ids (each distinct column stored once, each product of a
    column with a byte computed once) gives the columns of serial.parse at
    every position; serial.parse is pinned above and in test_oracle_pins."""
    pattern, text = _interned_cases()[k]
    c = compile_re(pattern)
    want = serial.parse(c, text)
    ids, cols = serial.parse_ids(c, text)
    assert ids.shape == (len(text) + 1,)
    assert np.array_equal(cols[ids], want)
    assert len({tuple(r) for r in cols.tolist()}) == len(cols)     # each distinct column once
