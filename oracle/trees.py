"""Brute-force syntax-tree enumeration (independent definition of the SLPF).

Test infrastructure only (see ``oracle/__init__.py``).

Sect. 2.1 (Example 1) defines a syntax tree from the structure tree: a
concatenation node takes all its children in order, a union node takes exactly
one child, an iterator takes zero (star only) or more instances of its child.
Its LST is the parenthesised string whose pairs are the numbered inner nodes
(Sect. 2.2, Prop. 1).  An LST followed by ⊣ factors uniquely into segments
mu_1 a_1 ... mu_n a_n mu_{n+1} ⊣ (Sect. 2.3.2), and the r-th segment lies in
column C_r of the SLPF (Sect. 2.3.5).  So the clean SLPF of a text is, column
by column, the set of r-th segments over all its syntax trees, and the number
of SLPF paths equals the number of trees.

Nothing here uses Fol, FolSeg or any automaton.
"""
from __future__ import annotations

from functools import lru_cache

from .re_front import END, Compiled, Node


def lsts(c: Compiled, text: bytes, limit: int = 1_000_000):
    """All LSTs (tuples of numbered symbols, without ⊣) of ``text``."""
    n = len(text)

    @lru_cache(maxsize=None)
    def gen(node_id: int, i: int):
        node = nodes[node_id]
        k = node.num
        if node.kind == "term":
            if i < n and text[i] in node.chars:
                return ((i + 1, (("t", k),)),)
            return ()
        if node.kind == "eps":
            return ((i, (("e", k),)),)
        if node.kind in ("cat", "rep"):
            partial = [(i, ())]
            for ch in node.children:
                nxt = []
                for j, toks in partial:
                    for j2, t2 in gen(id(ch), j):
                        nxt.append((j2, toks + t2))
                partial = nxt
                if len(partial) > limit:
                    raise OverflowError("too many partial trees")
            return tuple((j, (("(", k),) + toks + ((")", k),)) for j, toks in partial)
        if node.kind == "alt":
            out = []
            for ch in node.children:
                out.extend(gen(id(ch), i))
            return tuple((j, (("(", k),) + toks + ((")", k),)) for j, toks in out)
        if node.kind in ("star", "plus"):
            body = node.children[0]
            # iterations: every body instance consumes >= 1 byte (finite ambiguity)
            results = []
            frontier = [(i, (), 0)]
            while frontier:
                nxt = []
                for j, toks, cnt in frontier:
                    if cnt >= 1 or node.kind == "star":
                        results.append((j, toks))
                    for j2, t2 in gen(id(body), j):
                        if j2 > j:
                            nxt.append((j2, toks + t2, cnt + 1))
                if len(nxt) > limit:
                    raise OverflowError("too many partial trees")
                frontier = nxt
            return tuple((j, (("(", k),) + toks + ((")", k),)) for j, toks in results)
        raise AssertionError(node.kind)

    nodes = {}

    def index(nd: Node):
        nodes[id(nd)] = nd
        for ch in nd.children:
            index(ch)

    index(c.root)
    return [toks for j, toks in gen(id(c.root), 0) if j == n]


def factor(lst) -> list:
    """Factor LST ⊣ into segments mu a (Sect. 2.3.2)."""
    segs, cur = [], []
    for s in tuple(lst) + (END,):
        cur.append(s)
        if s[0] in ("t", "$"):
            segs.append(tuple(cur))
            cur = []
    assert not cur
    return segs


def slpf_by_trees(c: Compiled, text: bytes):
    """(columns as sets of segment indices, number of trees) by enumeration."""
    trees = lsts(c, text)
    cols = [set() for _ in range(len(text) + 1)]
    for t in trees:
        segs = factor(t)
        assert len(segs) == len(text) + 1
        for r, sg in enumerate(segs):
            cols[r].add(c.index[sg])   # KeyError would mean a segment Q lacks
    return [frozenset(x) for x in cols], len(trees)


def count_paths(c: Compiled, text: bytes, columns) -> int:
    """Number of paths through the SLPF columns along parser-NFA arcs
    (exact integer), i.e. the number of LSTs it encodes (Sect. 2.3.5)."""
    n = len(columns) - 1
    ways = {q: 1 for q in columns[0] if q in c.initial}
    for r in range(1, n + 1):
        nxt = {}
        for q, w in ways.items():
            if not c.matches(q, text[r - 1]):
                continue
            for q2 in c.folseg[q]:
                if q2 in columns[r]:
                    nxt[q2] = nxt.get(q2, 0) + w
        ways = nxt
    return sum(w for q, w in ways.items() if q in c.final)
