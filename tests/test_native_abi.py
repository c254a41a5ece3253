"""CPU checks of the native library: exports, host-only compile vs the oracle.

No CUDA call is made here (handles are compiled with RE_COMPILE_HOST_ONLY).
"""
import os
import re

import numpy as np
import pytest

from oracle import parallel_equations as pe
from oracle.re_front import compile_re
from oracle import serial

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PATTERNS = ["(a|b|ab)*", "(ab|a)*", "(a|ab|aba)+", "(a|)b", "(a|b)*a(a|b){3}", "a", "()",
            "([ACGT]|ATG([ACGT][ACGT][ACGT])*(TAA|TAG|TGA))*", "((ab)*c|a(bc)*)*", "[ab]([^b]|bb)*",
            "(x(y|z)?w|[^a-c]+)*q", "a(b(c(d)))", "(a|(b|c)|d)*", "(\\.|[0-9]+\\.?)+", "((a|b)(a|b))*",
            "(a|bc){1,3}", "(ab|a){2,}", "a{0,2}b", "(a|b){2,3}c?", "(a?){2,3}", "(ab){0,}c", "((a|b){2}c){1,2}"]


@pytest.fixture(scope="module")
def native():
    try:
        from paper_2503_06763_gb300 import native
        native.load()
    except ImportError:
        import __graft_entry__
        __graft_entry__.build()
        from paper_2503_06763_gb300 import native
        native.load()
    return native


def header_functions():
    text = open(os.path.join(ROOT, "include", "slpf_parser.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(re_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(native):
    lib = native.load()
    names = header_functions()
    assert "re_parse" in names and "re_compile" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(native.EXPORTS) <= set(names)


@pytest.mark.parametrize("pattern", PATTERNS)
def test_host_compile_matches_oracle_segments_and_dfa(native, pattern):
    r = native.Regex(pattern, host_only=True)
    c = compile_re(pattern)
    assert r.segment_names() == c.names()
    assert r.info["fwd_dfa_states"] == len(pe.dfa_states(c))
    assert r.info["bwd_dfa_states"] == len(pe.dfa_states(c, reverse=True))
    # dictionary: distinct, non-empty, canonical order, every column a B ∩ B̂
    if r.info["dict_size"]:
        d = r.dictionary()
        sets = [tuple(sorted(serial.from_bits(row))) for row in d]
        assert all(sets) and len(set(sets)) == len(sets)
        assert sets == sorted(sets)
        fw, bw = pe.dfa_states(c), pe.dfa_states(c, reverse=True)
        inter = {tuple(sorted(a & b)) for a in fw for b in bw if a & b}
        assert set(sets) == inter


def test_ascii_rows_when_high_bytes_share_a_class_with_ascii(native):
    """The byte-table reach stages rows of the bytes below 128 only when
    every class holding a byte >= 128 holds one below it too: true for the
    benchmark REs (high bytes fall in the classes of [^\\n] or of no symbol),
    false once a class is made of high bytes alone."""
    import workloads as W
    for pattern in (W.LOG_RE, W.DNA_RE, W.AB_RE, "[^a]*", r"([\x7f-\xff]a|b)*"):
        assert native.Regex(pattern, host_only=True).info["ascii_rows"] == 1, pattern
    for pattern in (r"([ab]|[\x80-\xff]c)*", r"[\x80-\xff]*", r"(\xffa|b)*"):
        assert native.Regex(pattern, host_only=True).info["ascii_rows"] == 0, pattern


def test_ascii_rows_follow_the_byte_classes(native):
    """The library's choice of ASCII rows, checked against the byte classes
    as the oracle's segments define them (two bytes are alike when every
    segment reads both or neither): true exactly when each byte >= 128 has an
    alike byte below 128."""
    import workloads as W
    pats = [W.LOG_RE, W.DNA_RE, W.AB_RE, "[^a]*", r"(\xffa|b)*", r"([ab]|[\x80-\xff]c)*",
            r"([\x7f-\xff]a|b)*", r"([^\x00-\x7f]|x)*y", r"(a|[\x80-\x9f]|[\xa0-\xff])*"]
    pats += [W.random_re(seed, 8, 30)[0] for seed in (3, 4, 5)]
    for pattern in pats:
        c = compile_re(pattern)
        sig = [tuple(c.matches(q, b) for q in range(c.ell)) for b in range(256)]
        low = set(sig[:128])
        want = all(sig[h] in low for h in range(128, 256))
        assert native.Regex(pattern, host_only=True).info["ascii_rows"] == int(want), pattern


def test_reach_shapes_available(native):
    """Shapes 2-4 run for every automaton; shape 1 needs byte tables, that is
    at most 256 states per direction."""
    import workloads as W
    shapes = lambda p: native.Regex(p, host_only=True).info["reach_shapes"]
    for pattern in (W.DNA_RE, W.AB_RE, W.LOG_RE):
        assert shapes(pattern) == 0b11110, pattern
    assert shapes("(a|b)*a(a|b){10}") == 0b11100                 # 2^11 DFA states


def test_pair_layout_without_a_dictionary(native):
    """No dictionary and more than 64 segments: AUTO picks PAIRS (4 bytes per
    column while both automata have at most 65536 states); DICT is refused,
    DENSE too."""
    import workloads as W
    r = native.Regex(W.LOG_RE, host_only=True, max_dict=1)     # 162 segments, no room for a dictionary
    assert r.info["dict_size"] == 0 and r.ell > 64
    assert r.layout(100, "auto") == ("pairs", 4, 404)
    assert r.layout(100, "pairs") == ("pairs", 4, 404)
    for kind in ("dict", "dense"):
        with pytest.raises(native.ReError) as e:
            r.layout(100, kind)
        assert e.value.status == -8
    small = native.Regex("(a|b|ab)*", host_only=True)
    assert small.layout(10, "pairs") == ("pairs", 4, 44)


def test_layout_and_errors(native):
    r = native.Regex("(a|b|ab)*", host_only=True)
    assert r.layout(100, "auto") == ("dense", 2, 202)
    assert r.layout(100, "dict")[0] == "dict"
    big = native.Regex("([ACGT]|ATG([ACGT][ACGT][ACGT])*(TAA|TAG|TGA))*", host_only=True)
    assert big.layout(10, "auto") == ("dict", 2, 22)          # 351 dictionary entries: two bytes
    small = native.Regex("(a|b)*a(a|b){3}", host_only=True)     # fewer than 255 entries: one byte
    assert small.info["dict_size"] < 255 and small.layout(10, "dict") == ("dict", 1, 11)
    assert big.layout(10, "dense") == ("dense", 8, 88)
    for bad, code in (("(a", -2), ("a)", -2), ("(a|)*", -3), ("(a*)*", -3), ("a{0}", -2), ("a{3,2}", -2),
                      ("a{2,2}", -2), ("a{,2}", -2), ("a{}", -2), ("a{1,x}", -2), ("a{4097}", -2),
                      ("(a?){2,}", -3)):
        with pytest.raises(native.ReError) as e:
            native.Regex(bad, host_only=True)
        assert e.value.status == code
    with pytest.raises(native.ReError) as e:
        native.Regex("(a|b)*a(a|b){12}", max_states=200, host_only=True)
    assert e.value.status == -4


def oracle_dfa_start_count(pattern, reverse=False):
    """Most runs for one first byte when every classic DFA state is a start:
    distinct non-empty successors of the states reachable from I, computed
    with the oracle's NFA image (Sect. 3.1), one byte at a time; reverse: the
    same over the reverse DFA from F (Eq. reverseNFAdef), under the chunk's
    last byte."""
    from oracle.serial import nfa_image, nfa_preimage
    step = nfa_preimage if reverse else nfa_image
    c = compile_re(pattern)
    alphabet = sorted(set().union(*c.classes.values()))
    start = frozenset(c.final if reverse else c.initial)
    seen, todo = {start}, [start]
    while todo:
        s = todo.pop()
        for b in alphabet:
            t = step(c, s, b)
            if t and t not in seen:
                seen.add(t)
                todo.append(t)
    return max(len({step(c, s, b) for s in seen} - {frozenset()}) for b in alphabet)


@pytest.mark.parametrize("pattern", ["([ACGT]|ATG([ACGT][ACGT][ACGT])*(TAA|TAG|TGA))*", "(a|b|ab)*",
                                     "(a|b)*a(a|b){3}", "((ab)*c|a(bc)*)*", "(a{0,2}b|a|c)*", "(a|ab|aba)+"])
def test_dfa_starts_slot_counts(native, pattern):
    """RE_COMPILE_DFA_STARTS: the forward slots per class pair are the
    distinct successors of all DFA states, as the oracle counts them."""
    r = native.Regex(pattern, host_only=True, dfa_starts=True)
    assert r.info["fwd_slots_max"] == oracle_dfa_start_count(pattern)
    assert r.info["bwd_slots_max"] == native.Regex(pattern, host_only=True).info["bwd_slots_max"]
    if pattern.startswith("([ACGT]"):               # 36 backward runs: past the 32 a lane holds
        with pytest.raises(native.ReError) as e:
            native.Regex(pattern, host_only=True, dfa_starts="bwd")
        assert e.value.status == -4
        return
    rb = native.Regex(pattern, host_only=True, dfa_starts="bwd")
    assert rb.info["bwd_slots_max"] == oracle_dfa_start_count(pattern, reverse=True)
    assert rb.info["fwd_slots_max"] == native.Regex(pattern, host_only=True).info["fwd_slots_max"]
    both = native.Regex(pattern, host_only=True, dfa_starts="both")
    assert (both.info["fwd_slots_max"], both.info["bwd_slots_max"]) == (r.info["fwd_slots_max"],
                                                                      rb.info["bwd_slots_max"])


def test_dfa_starts_refused_past_32_runs(native):
    """The log RE needs more than 32 forward runs from all DFA states: the
    compile is refused with RE_E_TOO_MANY_STATES (its ME-DFA starts fit)."""
    import workloads as W
    assert oracle_dfa_start_count(W.LOG_RE) > 32
    assert native.Regex(W.LOG_RE, host_only=True).info["fwd_slots_max"] <= 32
    with pytest.raises(native.ReError) as e:
        native.Regex(W.LOG_RE, host_only=True, dfa_starts=True)
    assert e.value.status == -4


def test_ek_family_state_counts(native):
    for k in range(1, 8):
        r = native.Regex("(a|b)*a(a|b){%d}" % k, host_only=True)
        assert r.info["fwd_dfa_states"] == 2 ** (k + 1) + 1


def test_serving_workspace_bound_covers_the_library(native):
    """The serving loop admits requests with a workspace bound computed in
    Python; it must cover the library's workspace for every chunk length the
    library may pick (>= 256), for short and long texts."""
    from paper_2503_06763_gb300 import serve
    import workloads as W
    pats = [W.DNA_RE, W.AB_RE, W.LOG_RE] + [W.random_re(4000 + i, 20, 300)[0] for i in range(4)]
    srv = serve.Server.__new__(serve.Server)
    srv.regexes = [native.Regex(p, host_only=True) for p in pats]
    srv._prepare()
    for ri, rx in enumerate(srv.regexes):
        for n in (0, 1, 63, 64, 255, 256, 257, 4095, 65536, 1_000_003, 64 << 20):
            for k in (256, 320, 4608):
                assert rx.workspace_size(n, chunk_len=k) <= srv.ws_bound(ri, n), (pats[ri][:20], n, k)


def test_server_refuses_host_only_handles(native):
    """re_server_create checks its handles before touching the device."""
    r = native.Regex("(a|b|ab)*", host_only=True)
    with pytest.raises(native.ReError) as e:
        native.NativeServer([r])
    assert e.value.status == -1
