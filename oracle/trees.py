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


def lsts_sampled(c: Compiled, text: bytes, sample_limit: int, cap: int = 200_000):
    """The LSTs of ``text`` (tuples without ⊣) in which every segment holds
    each numbered symbol at most ``sample_limit`` times (App. A, "Infinite
    ambiguity").

    Unlike ``lsts`` an iteration may derive the empty text, so an infinitely
    ambiguous RE has infinitely many trees; the limit keeps finitely many.
    The trees are built from the structure tree alone (Sect. 2.1, Example 1),
    their LST written left to right; a branch ends as soon as the current
    segment (the symbols since the last terminal) holds a symbol more than
    ``sample_limit`` times, a terminal misses its byte, or the text runs out.
    Every body instance of an iterator adds at least one symbol, so the search
    is finite.  Raises OverflowError past ``cap`` trees.
    """
    n = len(text)
    out = []
    # work items: ("sym", s) emits s; ("node", nd) expands nd;
    # ("iter", nd, k) decides on a further instance after k of them
    stack0 = (("node", c.root),)

    def run(work, pos, counts, lst):
        while work:
            item, work = work[0], work[1:]
            if item[0] == "sym":
                s = item[1]
                if s[0] == "t":
                    if pos >= n or text[pos] not in c.classes[s[1]]:
                        return
                    pos, counts = pos + 1, {}
                else:
                    k = counts.get(s, 0) + 1
                    if k > sample_limit:
                        return
                    counts = dict(counts); counts[s] = k
                lst = lst + (s,)
                continue
            nd = item[1]
            if item[0] == "node":
                num = nd.num
                if nd.kind == "term":
                    work = (("sym", ("t", num)),) + work
                elif nd.kind == "eps":
                    work = (("sym", ("e", num)),) + work
                elif nd.kind in ("cat", "rep"):
                    work = ((("sym", ("(", num)),) + tuple(("node", ch) for ch in nd.children)
                            + (("sym", (")", num)),) + work)
                elif nd.kind == "alt":
                    for ch in nd.children:
                        run((("sym", ("(", num)), ("node", ch), ("sym", (")", num))) + work, pos, counts, lst)
                    return
                elif nd.kind in ("star", "plus"):
                    work = (("sym", ("(", num)), ("iter", nd, 0), ("sym", (")", num))) + work
                else:
                    raise AssertionError(nd.kind)
                continue
            k = item[2]                                     # "iter"
            if k >= 1 or nd.kind == "star":                 # stop here
                run(work, pos, counts, lst)
            run((("node", nd.children[0]), ("iter", nd, k + 1)) + work, pos, counts, lst)
            return
        if pos == n and counts.get(END, 0) < 1:            # the last segment ends with ⊣
            out.append(lst)
            if len(out) > cap:
                raise OverflowError("too many trees")

    run(stack0, 0, {}, ())
    return out


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


def slpf_by_trees(c: Compiled, text: bytes, sample_limit: int = 0):
    """(columns as sets of segment indices, number of trees) by enumeration;
    with sample_limit >= 1 over ``lsts_sampled``."""
    trees = lsts_sampled(c, text, sample_limit) if sample_limit else lsts(c, text)
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
