"""Pins of the match-extraction oracle (Sect. 4.2, getMatches).

* The forest visit over the clean SLPF equals the spans read off every
  enumerated syntax tree, for every group of several REs and every text up
  to length 6 (brute force).
* Closed forms for (a|b|ab)* (1( 2( a3 | b4 | 5( a6 b7 )5 )2 )1): group 5
  matches exactly the occurrences of "ab"; group 2 every single byte and every
  "ab"; group 1 the whole text.
* A field query in the manner of Example 7: quoted values inside a header.
"""
import itertools
import re

import numpy as np
import pytest

from oracle import matches as M
from oracle import serial
from oracle.re_front import compile_re

BRUTE = ["(a|b|ab)*", "(ab|a)*", "(a|ab|aba)+", "(a|)b", "a(b|c)*d", "((ab)*c|a(bc)*)*", "(a*b|ac)+",
         "(a|b)*a(a|b){2}"]


def groups(c):
    return sorted({s[1] for seg in c.segments for s in seg if s[0] == "("})


@pytest.mark.parametrize("pattern", BRUTE)
def test_forest_visit_equals_tree_spans(pattern):
    c = compile_re(pattern)
    ks = groups(c)
    assert ks
    for n in range(0, 7):
        for tup in itertools.product(b"abcd", repeat=n):
            text = bytes(tup)
            cols = [serial.from_bits(row) for row in serial.parse(c, text)]
            for k in ks:
                assert M.matches_by_slpf(c, text, k, cols) == M.matches_by_trees(c, text, k), (pattern, text, k)


def test_ab_star_closed_forms():
    c = compile_re("(a|b|ab)*")
    names = c.names()
    assert "1( 2( 5( t6" in names and "t7" in names                    # a6 b7 inside group 5, as assumed below
    rng = np.random.Generator(np.random.PCG64(3))
    for n in (0, 1, 2, 17, 300):
        text = bytes(rng.choice(np.frombuffer(b"ab", dtype=np.uint8), size=n))
        ab = [(i, i + 2) for i in range(n - 1) if text[i:i + 2] == b"ab"]
        assert M.matches_by_slpf(c, text, 5) == ab
        assert M.matches_by_slpf(c, text, 2) == sorted([(i, i + 1) for i in range(n)] + ab)
        assert M.matches_by_slpf(c, text, 1) == [(0, n)]


def test_header_field_query():
    """Example 7's style: extra groups around the quoted values of a header."""
    pat = '<h3 id=("[^"]+") nam=("[^"]+")>'
    c = compile_re(pat)
    text = b'<h3 id="x1" nam="longer value">'
    ks = groups(c)
    spans = {k: M.matches_by_slpf(c, text, k) for k in ks}
    want_id = [(m.start(), m.end()) for m in re.finditer(rb'"x1"', text)]
    want_nam = [(m.start(), m.end()) for m in re.finditer(rb'"longer value"', text)]
    assert want_id in spans.values() and want_nam in spans.values()
    assert [(0, len(text))] in spans.values()                          # the outer concatenation
