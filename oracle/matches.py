"""Match extraction: the spans of a group (Sect. 4.2, "Match extraction").

Test infrastructure only (see ``oracle/__init__.py``).

A group is a numbered operator node k of e_# (a parenthesised
sub-expression, with its pair k( )k).  The paper's getMatches extracts the
offset pairs of the substrings that match a group.  Here a match of group k
in text x is a pair (i, j), 0 <= i <= j <= n, such that some syntax tree of
x has a node k whose yield is x[i:j].

Two definitions, pinned to each other by brute force in the tests:

* ``matches_by_trees`` -- from the enumerated LSTs (``trees.lsts``): along
  an LST, the text position advances at every terminal; k( at position i and
  the next )k at position j give (i, j).  A group never nests inside itself,
  so the next )k closes the k( just seen.

* ``matches_by_slpf`` -- from the clean SLPF alone (the visit of the forest
  the paper describes).  A segment is its parentheses and leaves before an
  end letter.  Within one segment, "k( ... )k" is a match (i, i) at that
  column.  A segment whose last k-parenthesis is k( leaves group k open.  From
  every column i, follow FolSeg arcs (Eq. folsegdef) through the next
  columns: segments without a k-parenthesis keep it open, and a segment whose
  first k-parenthesis is )k at column j closes it: (i, j).  The SLPF is
  clean, so every such partial path extends to a whole tree (every segment
  of a clean column has a predecessor and a successor), and every span in a
  tree is such a path.
"""
from __future__ import annotations

from . import serial, trees
from .re_front import Compiled


def matches_by_trees(c: Compiled, text: bytes, k: int) -> list:
    out = set()
    for lst in trees.lsts(c, text):
        pos, opened = 0, None
        for s in lst:
            if s == ("(", k):
                opened = pos
            elif s == (")", k):
                out.add((opened, pos))
                opened = None
            elif s[0] == "t":
                pos += 1
    return sorted(out)


def k_parens(c: Compiled, q: int, k: int) -> list:
    """The k-parentheses of segment q, in order: '(' or ')'."""
    return [s[0] for s in c.segments[q] if s[0] in "()" and s[1] == k]


def segment_classes(c: Compiled, k: int):
    """(OPEN, CLOSE_FIRST, EMPTY, NONE): segments leaving k open at their end,
    closing an open k first, holding a whole k( ... )k, and without any
    k-parenthesis."""
    opn, close_first, empty, none = set(), set(), set(), set()
    for q in range(c.ell):
        kp = k_parens(c, q, k)
        if not kp:
            none.add(q)
            continue
        if kp[-1] == "(":
            opn.add(q)
        if kp[0] == ")":
            close_first.add(q)
        if any(kp[a] == "(" and ")" in kp[a + 1:] for a in range(len(kp))):
            empty.add(q)
    return frozenset(opn), frozenset(close_first), frozenset(empty), frozenset(none)


def matches_by_slpf(c: Compiled, text: bytes, k: int, columns=None) -> list:
    if columns is None:
        columns = [serial.from_bits(row) for row in serial.parse(c, text)]
    n = len(text)
    opn, close_first, empty, none = segment_classes(c, k)
    out = set()
    for i in range(n + 1):
        if columns[i] & empty:
            out.add((i, i))
        S = columns[i] & opn
        r = i
        while S and r < n:
            nxt = set()
            for q in S:
                if c.matches(q, text[r]):
                    nxt |= c.folseg[q]
            r += 1
            N = frozenset(nxt) & columns[r]
            if N & close_first:
                out.add((i, r))
            S = N & none
    return sorted(out)
