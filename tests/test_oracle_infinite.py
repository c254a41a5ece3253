"""Pins of the oracle's sampling of infinitely ambiguous REs (App. A).

App. A ("Infinite ambiguity") keeps such an RE and returns a finite sample of
the LSTs of a text: the segment computation counts the numbered symbols of a
meta-prefix and lets each occur up to a fixed limit.  The oracle's MetaPrefix
does that with ``sample_limit`` = L; ``trees.lsts_sampled`` builds the same
sample from the structure tree alone (no Fol, no segments), so the two
agreeing column by column, on every short text, pins the counters.  The
values the paper prints are the four LSTs of Fig. (infamb) for e_5.
"""
import itertools

import pytest

from oracle import serial, trees
from oracle.re_front import InfiniteAmbiguity, compile_re, sym_name

INFINITE = ["(a*|ab)+", "(a?b?)*", "((a*)*b)*", "(a*)+", "((ab)?|c*)+a", "(a|()|b)*c?", "(a{0,2}b?){2,}"]
FINITE = ["(a|ab|aba)+", "(ab|a)*", "(a|b)*a(a|b){2}", "a?b?c?", "(a|bc){1,3}"]


def _names(lst):
    return " ".join(sym_name(s) for s in lst)


def _node_kinds(root):
    out = {}

    def walk(n):
        out[n.num] = n.kind
        for ch in n.children:
            walk(ch)

    walk(root)
    return out


# --------------------------------------------------------------------------- e_5, Fig. (infamb)
def test_e5_numbering(golden):
    g = golden["e5"]
    c = compile_re(g["pattern"], sample_limit=2)
    assert [sym_name(s) for s in c.symbols] == g["numbered_symbols"]
    kinds = _node_kinds(c.root)
    assert {str(k): kinds[k] for k in (1, 2, 3, 5)} == g["operators"]
    assert c.infinitely_ambiguous


def test_e5_is_rejected_without_a_limit(golden):
    with pytest.raises(InfiniteAmbiguity):
        compile_re(golden["e5"]["pattern"])


@pytest.mark.parametrize("L,shown", [(2, 3), (3, 4), (4, 4)])
def test_e5_sample_holds_the_figure(golden, L, shown):
    """The figure's LSTs repeat the empty sub-LST 2( 3( )3 )2 zero, once or
    twice before or after the one that holds a4: with L = 2 the first three
    are in the sample, with L = 3 all four; each one is a path of the SLPF
    the parser computes (its r-th segment lies in column C_r)."""
    g = golden["e5"]
    c = compile_re(g["pattern"], sample_limit=L)
    text = g["text"].encode()
    sample = {_names(t) for t in trees.lsts_sampled(c, text, L)}
    cols = serial.parse_small(c, text)
    for k, lst in enumerate(g["lsts"]):
        assert (lst in sample) == (k < shown), (L, lst)
        segs = trees.factor(tuple(_symbol(c, tok) for tok in lst.split()))
        in_slpf = all(sg in c.index and c.index[sg] in cols[r] for r, sg in enumerate(segs))
        assert in_slpf == (k < shown), (L, lst)


def _symbol(c, tok):
    return next(s for s in c.symbols if sym_name(s) == tok)


@pytest.mark.parametrize("text", [b"a", b"ab"])
def test_e5_sample_size_closed_form(golden, text):
    """For 'a' (and 'ab') every tree of e_5 is 1( E^k X E^m )1 with E the empty
    sub-LST 2( 3( )3 )2 and X the sub-LST that reads the text.  Its first
    segment holds 2( k + 1 times and its last segment )2 m + 1 times, so the
    limit L admits k, m in [0, L - 1]: L^2 trees, and as many SLPF paths."""
    for L in range(1, 5):
        c = compile_re(golden["e5"]["pattern"], sample_limit=L)
        assert len(trees.lsts_sampled(c, text, L)) == L * L
        assert trees.count_paths(c, text, serial.parse_small(c, text)) == L * L


# --------------------------------------------------------------------------- brute force
def _texts(max_len):
    for n in range(max_len + 1):
        for tup in itertools.product(b"abc", repeat=n):
            yield bytes(tup)


@pytest.mark.parametrize("pattern", INFINITE)
@pytest.mark.parametrize("L", [1, 2, 3])
def test_sampled_slpf_equals_the_sampled_trees(pattern, L):
    """Column r of the parser's SLPF is the set of r-th segments over the
    sampled trees, and its paths count those trees, on every text over
    {a, b, c} up to length 3; the C bitset parser gives the same columns."""
    c = compile_re(pattern, sample_limit=L)
    assert c.infinitely_ambiguous
    accepted = 0
    for text in _texts(3):
        want, ntrees = trees.slpf_by_trees(c, text, L)
        got = serial.parse_small(c, text)
        assert [frozenset(x) for x in got] == want, (pattern, L, text)
        assert trees.count_paths(c, text, got) == ntrees
        assert _as_sets(serial.parse(c, text)) == [set(x) for x in got]
        accepted += ntrees > 0
    assert accepted > 3


def _as_sets(cols):
    return [serial.from_bits(row) for row in cols]


@pytest.mark.parametrize("pattern", INFINITE)
def test_the_sample_grows_with_the_limit(pattern):
    """A larger limit keeps every segment of a smaller one (the limit only
    prunes), and the SLPF of each text grows with it."""
    prev = None
    for L in (1, 2, 3):
        c = compile_re(pattern, sample_limit=L)
        if prev is not None:
            assert set(prev.segments) < set(c.segments)
            for text in (b"a", b"ab", b"ca"):
                small = [{prev.segments[q] for q in col} for col in serial.parse_small(prev, text)]
                big = [{c.segments[q] for q in col} for col in serial.parse_small(c, text)]
                assert all(s <= b for s, b in zip(small, big))
        prev = c


@pytest.mark.parametrize("pattern", FINITE)
def test_finitely_ambiguous_res_ignore_the_limit(pattern):
    """No meta-prefix of a finitely ambiguous RE repeats a symbol (Sect. 2.3.3),
    so every limit gives the exact segment set, and the sampled trees are all
    the trees (``trees.lsts``, whose iterations each read a byte)."""
    exact = compile_re(pattern)
    assert not exact.infinitely_ambiguous
    for L in (1, 2, 3):
        c = compile_re(pattern, sample_limit=L)
        assert c.segments == exact.segments and c.folseg == exact.folseg
        assert not c.infinitely_ambiguous
    for text in _texts(3):
        assert sorted(trees.lsts_sampled(exact, text, 1)) == sorted(trees.lsts(exact, text))


# --------------------------------------------------------------------------- the library's host compiler
def _regex():
    try:
        from paper_2503_06763_gb300.native import Regex
        Regex("a", host_only=True)
    except ImportError:
        import __graft_entry__
        __graft_entry__.build()
        from paper_2503_06763_gb300.native import Regex
    return Regex


@pytest.mark.parametrize("pattern", INFINITE + FINITE[:2])
def test_native_compiler_samples_the_same_segments(pattern):
    Regex = _regex()
    for L in (1, 2, 3):
        r = Regex(pattern, host_only=True, sample_limit=L)
        c = compile_re(pattern, sample_limit=L)
        assert r.segment_names() == c.names()
        assert r.info["inf_ambiguous"] == int(c.infinitely_ambiguous)
        assert r.info["sample_limit"] == L


def test_native_compiler_rejects_without_a_limit():
    from paper_2503_06763_gb300.native import ReError
    Regex = _regex()
    for pattern in INFINITE:
        with pytest.raises(ReError):
            Regex(pattern, host_only=True)
    with pytest.raises(ReError):
        Regex("(a*)+", host_only=True, sample_limit=17)
