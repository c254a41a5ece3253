"""Pins of the CPU oracle to values the paper prints, closed forms and brute force.

Each test names the passage whose values it checks.  A plausible mistake in the
oracle (a dropped follower, a wrong index direction in N_a or N_a^T, a missing
intersection, a swapped I / F) fails at least one of them; see
``test_planted_mistakes_are_caught``.
"""
import itertools
import random

import numpy as np
import pytest

from oracle import parallel_equations as pe
from oracle import serial, trees
from oracle.re_front import (InfiniteAmbiguity, OracleSyntaxError, compile_re, seg_name,
                             sym_name)


def paper_ids(c, table):
    """Map the paper's segment numbers to oracle indices by name."""
    by_name = {n: i for i, n in enumerate(c.names())}
    return {int(k): by_name[v] for k, v in table.items()}


# --------------------------------------------------------------------------- e_1
def test_e1_numbering_and_trees(golden):
    g = golden["e1"]
    c = compile_re(g["pattern"])
    assert [sym_name(s) for s in c.symbols] == g["numbered_symbols"]
    got = sorted(" ".join(sym_name(s) for s in t) for t in trees.lsts(c, g["text"].encode()))
    assert got == sorted(g["lsts"])


# --------------------------------------------------------------------------- e_2
def test_e2_classic_followers(golden):
    g = golden["e2"]
    c = compile_re(g["pattern"])
    fol = {sym_name(s): sorted(sym_name(t) for t in v) for s, v in c.fol.items()}
    for s, printed in g["fol_printed"].items():
        want = set(printed)
        if s == "1(":
            want.add(")1")          # required by segment '1( )1 $' (see fol_note)
        if s == ")1":
            want.add("$")           # the end-mark is omitted in the printed table
        assert set(fol[s]) == want, s


def test_e2_segments_initial_final_folseg(golden):
    g = golden["e2"]
    c = compile_re(g["pattern"])
    assert sorted(c.names()) == sorted(g["segments"].values())
    pid = paper_ids(c, g["segments"])
    inv = {v: k for k, v in pid.items()}
    assert {inv[i] for i in c.initial} == set(g["initial"])
    assert {inv[i] for i in c.final} == set(g["final"])
    for p, fol in g["folseg"].items():
        assert {inv[j] for j in c.folseg[pid[int(p)]]} == set(fol)


def test_e2_connection_matrices(golden):
    g = golden["e2"]
    c = compile_re(g["pattern"])
    pid = paper_ids(c, g["segments"])
    ncol = serial.nfa_columns(c)
    for letter, key in (("a", "N_a_ones"), ("b", "N_b_ones")):
        ones = {(r, col) for r, col in g[key]}
        for r in range(1, 11):
            for col in range(1, 11):
                bit = (int(ncol[ord(letter), pid[col], 0]) >> pid[r]) & 1
                assert bit == ((r, col) in ones), (letter, r, col)


def test_e2_example4_serial_run(golden):
    g = golden["e2"]
    c = compile_re(g["pattern"])
    pid = paper_ids(c, g["segments"])
    inv = {v: k for k, v in pid.items()}
    text = g["ex4_text"].encode()
    fwd = [frozenset(c.initial)]
    for r in range(1, len(text) + 1):
        fwd.append(serial.nfa_image(c, fwd[-1], text[r - 1]))
    bwd = [frozenset(c.final)]
    for r in range(len(text) - 1, -1, -1):
        bwd.insert(0, serial.nfa_preimage(c, bwd[0], text[r]))
    assert [sorted(inv[q] for q in s) for s in fwd] == g["ex4_forward"]
    assert [sorted(inv[q] for q in s) for s in bwd] == g["ex4_backward"]
    clean = serial.parse_small(c, text)
    assert [sorted(inv[q] for q in s) for s in clean] == g["ex4_clean"]
    big = serial.parse(c, text)
    assert [sorted(inv[q] for q in serial.from_bits(r)) for r in big] == g["ex4_clean"]


def _state_names(c, g):
    pid = paper_ids(c, g["segments"])
    names = {}
    for k, v in g["dfa_states"].items():
        names[frozenset(pid[j] for j in v)] = k
    return pid, names


def test_e2_dfa_and_medfa(golden):
    g = golden["e2"]
    c = compile_re(g["pattern"])
    pid = paper_ids(c, g["segments"])
    T = {k: frozenset(pid[j] for j in v) for k, v in g["dfa_states"].items()}
    assert pe.dfa_states(c) == set(T.values())
    for s, row in g["dfa_delta"].items():
        for letter, tgt in row.items():
            got = serial.nfa_image(c, T[s], ord(letter))
            assert got == (T[tgt] if tgt else frozenset())
    S = {f"S{j}": frozenset([pid[j]]) for j in range(1, 11)}
    S.update({k: frozenset(pid[j] for j in v) for k, v in g["medfa_extra_states"].items()})
    assert pe.medfa_states(c) == set(S.values())
    assert len(S) == 13
    for s, row in g["medfa_delta"].items():
        for letter, tgt in row.items():
            got = serial.nfa_image(c, S[s], ord(letter))
            assert got == (S[tgt] if tgt else frozenset()), (s, letter)


def test_e2_example6_parallel_equations(golden):
    g = golden["e2"]
    c = compile_re(g["pattern"])
    pid = paper_ids(c, g["segments"])
    inv = {v: k for k, v in pid.items()}
    named = {k: frozenset(pid[j] for j in v) for k, v in g["dfa_states"].items()}
    named.update({k: frozenset(pid[j] for j in v) for k, v in g["medfa_extra_states"].items()})
    text = g["ex6_text"].encode()
    cols, tr = pe.parse_parallel(c, text, g["ex6_k"])
    for i in (1, 2, 3):
        want = {int(j): named[s] for j, s in g["ex6_R_nonempty"][str(i)].items()}
        for j in range(1, 11):
            assert tr["R"][i][pid[j]] == want.get(j, frozenset()), (i, j)
    assert tr["J"] == [named[s] for s in g["ex6_J"]]
    B = [b for i in (1, 2, 3) for b in tr["B"][i][1:]]
    assert B == [named[s] for s in g["ex6_B"]]
    Bh = [b for i in (1, 2, 3) for b in tr["Bh"][i][1:]]
    assert [sorted(inv[q] for q in s) for s in Bh] == g["ex6_Bhat"]
    assert sorted(inv[q] for q in tr["Jh"][1]) == g["ex6_Jhat1"]
    assert [sorted(inv[q] for q in s) for s in cols] == g["ex6_C"]
    assert cols == serial.parse_small(c, text)


# --------------------------------------------------------------------------- e_3
def test_e3_nfa_and_ambiguous_slpf(golden):
    g = golden["e3"]
    c = compile_re(g["pattern"])
    assert sorted(c.names()) == sorted(g["segments"])
    text = g["text"].encode()
    cols = serial.parse_small(c, text)
    names = c.names()
    assert [sorted(names[q] for q in s) for s in cols] == [sorted(x) for x in g["slpf"]]
    got = sorted(" ".join(sym_name(s) for s in t) for t in trees.lsts(c, text))
    assert got == sorted(g["lsts"])
    assert trees.count_paths(c, text, cols) == 4


# --------------------------------------------------------------------------- e_4
def test_e4_epsilon_segment(golden):
    g = golden["e4"]
    c = compile_re(g["pattern"])
    assert g["segment"] in c.names()
    cols = serial.parse_small(c, g["text"].encode())
    assert [sorted(c.names()[q] for q in s) for s in cols] == g["slpf"]


def test_bounded_repetition_printed_example(golden):
    """App. A's a^3: one numbered pair around three distinct terminal copies."""
    from oracle.re_front import sym_name
    g = golden["rep3"]
    c = compile_re(g["pattern"])
    assert sorted(n for n in c.names() if n.split()[-1].startswith("t")) == g["terminal_segments"]
    lsts = list(trees.lsts(c, g["text"].encode()))
    assert len(lsts) == 1 and [sym_name(s) for s in lsts[0]] == g["lst"]


# --------------------------------------------------------------------------- e(k)
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_ek_dfa_state_count(golden, k):
    g = golden["ek"]
    c = compile_re(g["pattern_template"] % k)
    assert len(pe.dfa_states(c)) == g["dfa_states"][str(k)] == 2 ** (k + 1) + 1


# --------------------------------------------------------------------------- brute force
BRUTE_RES = ["(a|b|ab)*", "(ab|a)*", "(a|ab|aba)+", "(a|)b", "a(b|c)*d", "(a*b|ac)+", "((ab)*c|a(bc)*)*",
             "(a|b)*a(a|b){2}", "a", "(ab){2}(a|b)?", "(a|b)(a|b)*", "[ab]([^b]|bb)*",
             "(a|bc){1,3}", "(ab|a){2,}", "a{0,2}b", "(a?){2,3}"]


@pytest.mark.parametrize("pattern", BRUTE_RES)
def test_brute_force_all_short_texts(pattern):
    """Union over all syntax trees == serial two-way parser; #trees == #paths."""
    c = compile_re(pattern)
    alphabet = b"abcd"
    for n in range(0, 7):
        for tup in itertools.product(alphabet, repeat=n):
            text = bytes(tup)
            want, ntrees = trees.slpf_by_trees(c, text)
            got = serial.parse_small(c, text)
            assert got == want, (pattern, text)
            assert trees.count_paths(c, text, got) == ntrees
            assert serial.accepted(serial.parse(c, text)) == (ntrees > 0)


def test_brute_force_ab_star_exhaustive_to_12():
    c = compile_re("(a|b|ab)*")
    for n in range(0, 13):
        for tup in itertools.product(b"ab", repeat=n):
            text = bytes(tup)
            got = [serial.from_bits(r) for r in serial.parse(c, text)]
            if n <= 9:
                want, _ = trees.slpf_by_trees(c, text)
                assert got == want


def ab_tree_count(text: bytes) -> int:
    """Closed form: tokenisations of x into a, b and ab."""
    f = [1, 1] + [0] * len(text)
    for r in range(2, len(text) + 1):
        f[r] = f[r - 1] + (1 if text[r - 2:r] == b"ab" else 0) * f[r - 2]
    return f[len(text)]


def test_closed_form_tree_count_on_prefixes():
    rng = np.random.Generator(np.random.PCG64(0))
    x = rng.choice(np.frombuffer(b"ab", dtype=np.uint8), size=4096).tobytes()
    c = compile_re("(a|b|ab)*")
    for n in (16, 64, 256, 4096):
        text = x[:n]
        cols = [serial.from_bits(r) for r in serial.parse(c, text)]
        assert trees.count_paths(c, text, cols) == ab_tree_count(text)


def test_16_byte_prefixes_against_trees():
    """Config 1 prefixes (seed 0): SLPF of each 16-byte prefix as a text."""
    rng = np.random.Generator(np.random.PCG64(0))
    x = rng.choice(np.frombuffer(b"ab", dtype=np.uint8), size=1 << 12).tobytes()
    c = compile_re("(a|b|ab)*")
    for start in range(0, 256, 16):
        text = x[start:start + 16]
        want, nt = trees.slpf_by_trees(c, text)
        got = [serial.from_bits(r) for r in serial.parse(c, text)]
        assert got == want and nt == ab_tree_count(text)


@pytest.mark.parametrize("pattern", ["(a|b|ab)*", "(ab|a)*", "a(b|c)*d", "((ab)*c|a(bc)*)*", "(a|b)*a(a|b){3}"])
def test_chunk_invariance_of_parallel_equations(pattern):
    """Sect. 3.2: every chunking reproduces the serial clean SLPF."""
    c = compile_re(pattern)
    rnd = random.Random(7)
    for _ in range(30):
        n = rnd.randint(0, 40)
        text = bytes(rnd.choice(b"abcd") for _ in range(n))
        serial_cols = serial.parse_small(c, text)
        for k in range(1, max(2, n + 2)):
            cols, _ = pe.parse_parallel(c, text, k)
            assert cols == serial_cols, (text, k)


@pytest.mark.parametrize("pattern", ["(a|b|ab)*", "(ab|a)*", "a(b|c)*d", "((ab)*c|a(bc)*)*", "(a{0,2}b|a|c)*"])
def test_dfa_start_equations_give_the_serial_slpf(pattern):
    """Reach from every DFA state with an exact-state join (the ablation of
    the ME-DFA, Sect. 3.1 / Sect. 5), forward, backward or both: for every
    chunk length the columns equal the serial parser's, and every J_i and
    Ĵ_i equals the ME-DFA join's."""
    c = compile_re(pattern)
    rng = random.Random(11)
    for trial in range(12):
        text = bytes(rng.choice(b"abcd") for _ in range(rng.randint(0, 18)))
        want = [serial.from_bits(row) for row in serial.parse(c, text)]
        for k in range(1, max(len(text), 1) + 2):
            _, me = pe.parse_parallel(c, text, k)
            for fwd, bwd in ((True, False), (False, True), (True, True)):
                cols, tr = pe.parse_parallel_dfa_starts(c, text, k, forward=fwd, backward=bwd)
                assert cols == want, (pattern, text, k, fwd, bwd)
                assert tr["J"] == me["J"] and tr["Jh"] == me["Jh"]


def test_invariants_on_random_texts():
    c = compile_re("( [ACGT] | ATG([ACGT][ACGT][ACGT])*(TAA|TAG|TGA) )*".replace(" ", ""))
    rng = np.random.Generator(np.random.PCG64(5))
    x = rng.choice(np.frombuffer(b"ACGT", dtype=np.uint8), size=3000).tobytes()
    cols = [serial.from_bits(r) for r in serial.parse(c, x)]
    assert all(cols)
    assert cols[0] <= c.initial and cols[-1] <= c.final
    for r in range(len(x) + 1):
        for q in cols[r]:
            if r < len(x):
                assert c.matches(q, x[r])
                assert c.folseg[q] & cols[r + 1]          # has a successor
            else:
                assert c.end_letter(q)[0] == "$"
            if r > 0:                                     # has a predecessor
                assert any(q in c.folseg[p] and c.matches(p, x[r - 1]) for p in cols[r - 1])


def test_unambiguous_re_has_singleton_columns():
    c = compile_re("(ab|a)*")
    rnd = random.Random(3)
    for _ in range(50):
        text = b"".join(rnd.choice([b"ab", b"a"]) for _ in range(rnd.randint(0, 30)))
        cols = serial.parse_small(c, text)
        assert all(len(s) == 1 for s in cols)


def test_rejected_texts_give_empty_columns():
    c = compile_re("(ab|a)*")
    for text in (b"b", b"abb", b"ba", b"aab b"):
        cols = serial.parse(c, text)
        assert not cols.any()
        assert not serial.accepted(cols)


def test_syntax_errors_and_infinite_ambiguity():
    for bad in ["(a", "a)", "*a", "[ab", "a{0}", "\\", "a{3,2}", "a{2,2}", "a{,2}", "a{}", "a{1,x}"]:
        with pytest.raises(OracleSyntaxError):
            compile_re(bad)
    for amb in ["(a|)*", "(a*)*", "(a?b?)+", "()*", "(a?){2,}"]:
        with pytest.raises(InfiniteAmbiguity):
            compile_re(amb)


# --------------------------------------------------------------------------- bounded repetition
BOUNDED = ["(a|bc){1,3}", "(ab|a){2,}", "a{0,2}b", "(a|b){2,3}c?", "(a|aa){2,3}", "(a?){2,3}", "(ab){0,}c"]


@pytest.mark.parametrize("pattern", BOUNDED)
def test_bounded_repetition_language(pattern):
    """App. A, bounded repetition: e{h}, e{h,k}, e{h,} accept the same texts
    as Python's re module (an independent definition), on every text over
    {a, b, c} up to length 7."""
    import re
    c = compile_re(pattern)
    rx = re.compile(pattern.encode())
    for n in range(0, 8):
        for tup in itertools.product(b"abc", repeat=n):
            text = bytes(tup)
            assert serial.accepted(serial.parse(c, text)) == (rx.fullmatch(text) is not None), (pattern, text)


def test_bounded_repetition_tree_counts():
    """(a|aa){h,k} on a^n: a tree is a sequence of j iterations, h <= j <= k,
    each 'a' or 'aa', so there are sum_j C(j, n - j) trees (compositions of n
    into j parts of size 1 or 2); e{h,} sums over every j >= h."""
    from math import comb
    for (h, k) in [(1, 1), (2, 3), (0, 2), (1, 4), (3, -1), (0, -1)]:
        pat = "(a|aa){%d}" % h if k == h else ("(a|aa){%d,}" % h if k < 0 else "(a|aa){%d,%d}" % (h, k))
        c = compile_re(pat)
        for n in range(0, 8):
            top = n if k < 0 else k
            want = sum(comb(j, n - j) for j in range(h, top + 1) if 0 <= n - j <= j)
            assert sum(1 for _ in trees.lsts(c, b"a" * n)) == want, (pat, n)


def test_bounded_repetition_iteration_numbering():
    """App. A: every iteration of a bounded repetition has its own numbered
    symbols, and a tree with j iterations uses copies 1 .. j in order, so
    the terminal numbers along a^2, a^3, a^4 under a{2,4} extend each other."""
    c = compile_re("a{2,4}")
    seen = []
    for n in (2, 3, 4):
        lsts = list(trees.lsts(c, b"a" * n))
        assert len(lsts) == 1
        nums = [s[1] for s in lsts[0] if s[0] == "t"]
        assert len(nums) == n and nums == sorted(nums) and len(set(nums)) == n
        seen.append(nums)
    assert seen[1][:2] == seen[0] and seen[2][:3] == seen[1]
    assert sum(1 for _ in trees.lsts(c, b"a" * 5)) == 0


# --------------------------------------------------------------------------- mutation check
def test_planted_mistakes_are_caught(golden, monkeypatch):
    """Plant plausible mistakes in the oracle and check a pin fails for each."""
    g = golden["e2"]

    def e2_clean():
        c = compile_re(g["pattern"])
        pid = paper_ids(c, g["segments"])
        inv = {v: k for k, v in pid.items()}
        cols, _ = pe.parse_parallel(c, g["ex6_text"].encode(), 2)
        return [sorted(inv[q] for q in s) for s in cols]

    assert e2_clean() == g["ex6_C"]
    # 1) transposed NFA in the backward step
    orig_pre = serial.nfa_preimage
    monkeypatch.setattr(pe, "nfa_preimage",
                        lambda c, S, b: frozenset(q for s in S for q in c.folseg[s] if c.matches(q, b)))
    with pytest.raises(Exception):
        assert e2_clean() == g["ex6_C"]
    monkeypatch.setattr(pe, "nfa_preimage", orig_pre)
    # 2) forgetting the label test in the forward image
    monkeypatch.setattr(pe, "nfa_image", lambda c, S, b: frozenset(q for s in S for q in c.folseg[s]))
    with pytest.raises(Exception):
        assert e2_clean() == g["ex6_C"]


def test_more_planted_mistakes_are_caught(golden, monkeypatch):
    """Further plausible mistakes, each planted in the oracle on the CPU,
    must make one of the pins fail: a dropped FolSeg arc, a wrong initial
    set, an end-letter test that looks at the wrong byte, a wrong numbering
    order, and a match rule that closes a group on its last parenthesis."""
    import itertools
    from oracle import matches as M
    from oracle import re_front

    def disagrees_with_trees(c, pattern_texts):
        for text in pattern_texts:
            want, _ = trees.slpf_by_trees(c, text)
            if serial.parse_small(c, text) != want:
                return True
        return False

    texts = [bytes(t) for n in range(0, 6) for t in itertools.product(b"ab", repeat=n)]
    # 1) a FolSeg arc dropped
    c = compile_re("(a|b|ab)*")
    q = next(i for i, f in enumerate(c.folseg) if len(f) > 1)
    c.folseg[q] = frozenset(sorted(c.folseg[q])[1:])
    assert disagrees_with_trees(c, texts)
    # 2) a segment wrongly taken as initial
    c = compile_re("(a|b|ab)*")
    extra = next(i for i in range(c.ell) if i not in c.initial and c.segments[i][-1][0] == "t")
    c.initial = frozenset(c.initial | {extra})
    assert disagrees_with_trees(c, texts)
    # 3) the arc label tested against the wrong byte
    c = compile_re("(a|b|ab)*")
    orig = re_front.Compiled.matches
    monkeypatch.setattr(re_front.Compiled, "matches", lambda self, q, b: orig(self, q, b ^ 3))
    assert disagrees_with_trees(c, texts)
    monkeypatch.setattr(re_front.Compiled, "matches", orig)
    # 4) numbering in postorder instead of preorder: the e_1 numbering pin fails
    g = golden["e1"]
    orig_number = re_front.number

    def postorder(root):
        counter = [0]

        def visit(nd):
            for ch in nd.children:
                visit(ch)
            counter[0] += 1
            nd.num = counter[0]
        visit(root)
        return counter[0]

    monkeypatch.setattr(re_front, "number", postorder)
    c = compile_re(g["pattern"])
    assert [sym_name(s) for s in c.symbols] != g["numbered_symbols"]     # the e_1 pin fails
    monkeypatch.setattr(re_front, "number", orig_number)
    assert [sym_name(s) for s in compile_re(g["pattern"]).symbols] == g["numbered_symbols"]
    # 5) a group closed on its last parenthesis instead of its first
    c = compile_re("((ab)*c|a(bc)*)*")
    orig_classes = M.segment_classes

    def wrong_classes(cc, k):
        opn, close_first, whole, none = orig_classes(cc, k)
        close_last = frozenset(q for q in range(cc.ell)
                               if M.k_parens(cc, q, k) and M.k_parens(cc, q, k)[-1] == ")")
        return opn, close_last, whole, none

    monkeypatch.setattr(M, "segment_classes", wrong_classes)
    found = False
    for n in range(1, 7):
        for t in itertools.product(b"abc", repeat=n):
            text = bytes(t)
            for k in (1, 2, 3):
                if M.matches_by_slpf(c, text, k) != M.matches_by_trees(c, text, k):
                    found = True
                    break
            if found:
                break
        if found:
            break
    assert found
