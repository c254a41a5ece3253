"""Pins of the speculation model (``oracle/speculation.py``).

The model counts a chunk's speculative runs under the start rules of
Sect. 3.1 and the reductions of Sect. 4.3.  Its start sets are pinned to the
library's own slot tables (the most runs any byte pair needs, ME-DFA and
all-DFA-state starts, both directions); the forward-restricted backward
starts are shown to leave the clean SLPF unchanged on every chunking; the
work count is pinned on runs that do not speculate at all.
"""
import itertools
import random

import pytest

import workloads as W
from oracle import parallel_equations as pe
from oracle import serial
from oracle import speculation as sp
from oracle.re_front import compile_re

RES = [W.DNA_RE, W.AB_RE, "(a|b)*a(a|b){3}", "((ab)*c|a(bc)*)*", "(a{0,2}b|a|c)*", "(a|ab|aba)+"]


def _alphabet(c):
    return sorted(set().union(*c.classes.values()))


def _native():
    try:
        from paper_2503_06763_gb300.native import Regex
        Regex("a", host_only=True)
    except ImportError:
        import __graft_entry__
        __graft_entry__.build()
        from paper_2503_06763_gb300.native import Regex
    return Regex


@pytest.mark.parametrize("pattern", RES)
def test_start_counts_equal_the_slot_tables(pattern):
    """Most ME-DFA runs (and most all-DFA-state runs) over every byte pair
    equal the compiled slot counts, forward and backward."""
    Regex = _native()
    c = compile_re(pattern)
    m = sp.Machine(c)
    dfa, rdfa = pe.dfa_states(c), pe.dfa_states(c, reverse=True)
    alpha = _alphabet(c)
    pairs = list(itertools.product(alpha, alpha))
    me = Regex(pattern, host_only=True).info
    assert max(len(sp.forward_starts(m, a, b, "me")) for a, b in pairs) == me["fwd_slots_max"]
    assert max(len(sp.backward_starts(m, a, b, "me")) for a, b in pairs) == me["bwd_slots_max"]
    f_dfa = max(len(sp.forward_starts(m, a, b, "dfa", dfa)) for a, b in pairs)
    b_dfa = max(len(sp.backward_starts(m, a, b, "dfa", rdfa=rdfa)) for a, b in pairs)
    assert Regex(pattern, host_only=True, dfa_starts=True).info["fwd_slots_max"] == f_dfa
    if b_dfa <= 32:
        assert Regex(pattern, host_only=True, dfa_starts="bwd").info["bwd_slots_max"] == b_dfa
    else:
        assert pattern == W.DNA_RE and b_dfa == 36


def _restricted_columns(c, text, edges):
    """Forward columns exact; at every chunk edge b (right to left) the
    backward set is cut to the segments of the exact forward column there
    before it is carried into the chunk (forward-restricted backward starts);
    returns B_r ∩ B̂_r."""
    n = len(text)
    fwd = [frozenset(c.initial)]
    for a in text:
        fwd.append(serial.nfa_image(c, fwd[-1], a))
    bwd = [None] * (n + 1)
    bwd[n] = frozenset(c.final)
    for r in range(n - 1, -1, -1):
        nxt = bwd[r + 1]
        if r + 1 in edges and r + 1 < n:
            nxt = nxt & fwd[r + 1]
        bwd[r] = serial.nfa_preimage(c, nxt, text[r])
    return [fwd[r] & bwd[r] for r in range(n + 1)]


@pytest.mark.parametrize("pattern", RES)
def test_forward_restricted_backward_keeps_the_slpf(pattern):
    """Cutting the backward set at chunk edges to the forward column leaves
    every clean column unchanged, for every chunk length."""
    c = compile_re(pattern)
    rng = random.Random(3)
    alpha = _alphabet(c)
    for _ in range(10):
        text = bytes(rng.choice(alpha) for _ in range(rng.randint(0, 24)))
        want = serial.parse_small(c, text)
        for k in range(1, len(text) + 2):
            edges = set(range(0, len(text) + 1, k))
            assert _restricted_columns(c, text, edges) == want, (pattern, text, k)


def test_restricted_starts_are_a_subset():
    c = compile_re(W.LOG_RE)
    m = sp.Machine(c)
    text = W.log_text(20_000, seed=4).tobytes()
    fwd = frozenset(c.initial)
    for e in range(1, len(text)):
        fwd = m.image(fwd, text[e - 1])
        if e % 997:
            continue
        full = sp.backward_starts(m, text[e - 1], text[e], "me")
        cut = sp.backward_starts(m, text[e - 1], text[e], "restricted", column=fwd & m.reads[text[e]])
        assert cut <= full and cut


def test_work_of_a_single_run_is_the_chunk():
    c = compile_re(W.DNA_RE)
    m = sp.Machine(c)
    text = W.dna_text(5000, seed=2).tobytes()
    S = frozenset(c.initial)
    assert sp.chunk_work(m, {S}, text, False) == (len(text), 0)
    assert sp.chunk_work(m, set(), text, False) == (0, 0)


def test_shifted_edges_stay_in_their_windows():
    c = compile_re(W.LOG_RE)
    m = sp.Machine(c)
    text = W.log_text(50_000, seed=4).tobytes()
    for k, s in ((1024, 8), (4096, 64)):
        e = sp.shifted_edges(m, text, k, s)
        assert e[0] == 0 and e[-1] == len(text)
        assert all(a < b for a, b in zip(e, e[1:]))
        assert all(abs(p - i * k) <= s for i, p in enumerate(e[1:-1], start=1))
