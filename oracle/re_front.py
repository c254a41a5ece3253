"""Oracle front end: RE -> numbered RE -> Fol -> segments -> FolSeg.

Test infrastructure only (see ``oracle/__init__.py``).

Paper passages followed (arXiv 2503.06763):
  * RE operators and precedence: Sect. 2.1 ("What is RE parsing").
  * Numbered RE e_#: Sect. 2.2, Eq. (numberedRE).  Terminals, ε and operator
    parenthesis pairs are numbered with one counter in left-to-right preorder of
    the structure tree.  Concatenation and union are n-ary.  The scope of an
    iterator sits inside its pair, k( [body]* )k, so the inner pairs repeat per
    iteration and the outer pair appears once.
  * Classic followers Fol(e_# ⊣, s): Eq. (classicfollowers), over the language
    of LSTs, which is local (Sect. 2.3.4, "Local properties of LSTs").
  * Segments Q, initial I, final F: Fig. (segmentalgo), recursive MetaPrefix.
  * FolSeg: Eq. (folsegdef).
  * Character sets, wildcard, escapes, ε symbols, extra parentheses, bounded
    repetition e{h}, e{h,k}, e{h,}: App. A.

Readings where the paper is silent or ambiguous:
  * A parenthesised group creates a numbered node only through the operator it
    encloses; ``(a)`` is just ``a`` and ``((ab))`` is one node; a group nested
    in an operand list of the same operator stays a separate node (extra
    parenthesis, App. A).
  * ``e?`` is ``(e|ε)``; an empty alternative or an empty group is ε.
  * ``e{k}`` is one numbered node whose k children are fresh copies of e
    numbered progressively (App. A, "Bounded repetition"; Ex. 5).  ``e{h,k}``
    and ``e{h,}`` add the optional (resp. starred) further iterations, each
    with its own copy; see ``expand_repetitions``.  With h = 0 there is no
    mandatory copy and the optional (resp. starred) iterations are the node
    itself, so ``e{0,1}`` is ``e?`` and ``e{0,}`` is ``e*``: App. A states the
    identity e? = e{0,1}.
  * ``.`` matches every byte but newline (App. A, "wildcard").
  * The initial symbol test of MetaPrefix (``s = 1(``) is read as "s is the
    first symbol of every LST", which is ``1(`` whenever the root is an
    operator and the root leaf itself otherwise.
  * A star / cross whose body derives the empty text is infinitely ambiguous
    (Sect. 2.1, App. A "Infinite ambiguity").  With no sample limit such an RE
    is rejected.  With a limit L >= 1 it is sampled as App. A describes: the
    segment computation counts the numbered symbols of the meta-prefix being
    extended and keeps only meta-prefixes where each symbol (parenthesis or ε)
    occurs at most L times.  The count covers the whole segment, its first
    symbol included; end-letters cannot repeat inside one segment anyway.  The
    SLPF then holds exactly the LSTs whose every segment obeys the limit
    (``trees.lsts_sampled`` enumerates them from the trees alone).  On a
    finitely ambiguous RE no meta-prefix repeats a symbol (Sect. 2.3.3,
    termination of the segment algorithm), so any L gives the full segment set.
"""
from __future__ import annotations

from dataclasses import dataclass, field

ALL_BYTES = frozenset(range(256))
META = set("|*+?()[].\\{")


class OracleSyntaxError(ValueError):
    pass


class InfiniteAmbiguity(ValueError):
    pass


# ----------------------------------------------------------------------------
# Structure tree (Sect. 2.1)
# ----------------------------------------------------------------------------
@dataclass
class Node:
    kind: str                      # 'term' | 'eps' | 'cat' | 'alt' | 'star' | 'plus' | 'rep'
    children: list = field(default_factory=list)
    chars: frozenset = frozenset()  # for 'term'
    count: int = 0                  # for 'rep': the lower bound h of e{h}, e{h,k}, e{h,}
    num: int = 0                    # number assigned by numbering (Eq. numberedRE)
    hi: int = 0                     # for 'rep': the upper bound (= count for e{h}; -1: none)


def _escape_byte(s: bytes, i: int):
    """Read an escape after a backslash at s[i-1]; return (byte, next index)."""
    if i >= len(s):
        raise OracleSyntaxError("dangling backslash")
    c = s[i]
    if c == ord("n"):
        return 10, i + 1
    if c == ord("t"):
        return 9, i + 1
    if c == ord("r"):
        return 13, i + 1
    if c == ord("x"):
        h = s[i + 1:i + 3]
        if len(h) != 2:
            raise OracleSyntaxError("bad \\x escape")
        try:
            return int(h.decode(), 16), i + 3
        except ValueError as e:
            raise OracleSyntaxError("bad \\x escape") from e
    return c, i + 1


def _parse_set(s: bytes, i: int):
    """Character set [...] starting after '['.  Returns (frozenset, next)."""
    neg = False
    if i < len(s) and s[i] == ord("^"):
        neg = True
        i += 1
    items = set()
    first = True
    while True:
        if i >= len(s):
            raise OracleSyntaxError("unterminated [")
        c = s[i]
        if c == ord("]") and not first:
            i += 1
            break
        first = False
        if c == ord("\\"):
            lo, i = _escape_byte(s, i + 1)
        else:
            lo, i = c, i + 1
        if i + 1 < len(s) and s[i] == ord("-") and s[i + 1] != ord("]"):
            if s[i + 1] == ord("\\"):
                hi, i = _escape_byte(s, i + 2)
            else:
                hi, i = s[i + 1], i + 2
            if hi < lo:
                raise OracleSyntaxError("reversed range")
            items.update(range(lo, hi + 1))
        else:
            items.add(lo)
    cs = frozenset(ALL_BYTES - items) if neg else frozenset(items)
    if not cs:
        raise OracleSyntaxError("empty character set")
    return cs, i


def parse(pattern) -> Node:
    """Parse an RE into its structure tree (before numbering)."""
    s = pattern.encode("latin-1") if isinstance(pattern, str) else bytes(pattern)
    pos = 0

    def parse_alt():
        nonlocal pos
        branches = [parse_seq()]
        while pos < len(s) and s[pos] == ord("|"):
            pos += 1
            branches.append(parse_seq())
        if len(branches) == 1:
            return branches[0]
        return Node("alt", branches)

    def parse_seq():
        nonlocal pos
        items = []
        while pos < len(s) and s[pos] not in (ord("|"), ord(")")):
            items.append(parse_postfix())
        if not items:
            return Node("eps")
        if len(items) == 1:
            return items[0]
        return Node("cat", items)

    def parse_postfix():
        nonlocal pos
        node = parse_atom()
        while pos < len(s):
            c = s[pos]
            if c == ord("*"):
                node = Node("star", [node]); pos += 1
            elif c == ord("+"):
                node = Node("plus", [node]); pos += 1
            elif c == ord("?"):
                node = Node("alt", [node, Node("eps")]); pos += 1
            elif c == ord("{"):
                j = s.find(b"}", pos)
                if j < 0:
                    raise OracleSyntaxError("unterminated {")
                txt = s[pos + 1:j].decode("latin-1")
                lo_txt, comma, hi_txt = txt.partition(",")
                if not lo_txt.isdigit() or (hi_txt and not hi_txt.isdigit()):
                    raise OracleSyntaxError("bounded repetition is e{h}, e{h,k} or e{h,}")
                lo = int(lo_txt)
                hi = lo if not comma else (int(hi_txt) if hi_txt else -1)
                if (not comma and lo < 1) or (comma and hi_txt and not lo < hi):
                    raise OracleSyntaxError("bounded repetition needs 1 <= h in e{h} and h < k in e{h,k}")
                node = Node("rep", [node], count=lo, hi=hi); pos = j + 1
            else:
                break
        return node

    def parse_atom():
        nonlocal pos
        c = s[pos]
        if c == ord("("):
            pos += 1
            inner = parse_alt()
            if pos >= len(s) or s[pos] != ord(")"):
                raise OracleSyntaxError("missing )")
            pos += 1
            return inner
        if c == ord("["):
            cs, pos = _parse_set(s, pos + 1)
            return Node("term", chars=cs)
        if c == ord("."):
            pos += 1
            return Node("term", chars=frozenset(ALL_BYTES - {10}))
        if c == ord("\\"):
            b, pos = _escape_byte(s, pos + 1)
            return Node("term", chars=frozenset([b]))
        if c in b"*+?{":
            raise OracleSyntaxError("operator without operand")
        if c == ord("]"):
            raise OracleSyntaxError("unbalanced ]")
        pos += 1
        return Node("term", chars=frozenset([c]))

    root = parse_alt()
    if pos != len(s):
        raise OracleSyntaxError("unbalanced )")
    return root


def _copy(node: Node) -> Node:
    return Node(node.kind, [_copy(ch) for ch in node.children], node.chars, node.count, hi=node.hi)


def expand_repetitions(node: Node) -> Node:
    """Bounded repetition (App. A): one node whose children are fresh copies
    of e, so every iteration has its own numbered symbols.

    * e{h}: the h copies.
    * e{h,k}: the h copies, then copies h+1 .. k, each optional and present
      only after the one before it: (e (e (... e?)?)?)?.  A tree with j
      iterations therefore uses copies 1 .. j, in order.
    * e{h,}: the h copies, then copy h+1 under a star.
    * h = 0: the node is the outermost optional (resp. the star) itself,
      which makes e{0,1} the optional e? = (e|ε) and e{0,} the star e*
      (App. A: e? = e{0,1}).
    """
    kids = [expand_repetitions(ch) for ch in node.children]
    if node.kind == "rep":
        body, h, hi = kids[0], node.count, node.hi
        reps = [_copy(body) for _ in range(h)]
        if hi == -1:
            reps.append(Node("star", [_copy(body)]))
        elif hi > h:
            tail = Node("alt", [_copy(body), Node("eps")])            # copy k
            for _ in range(hi - h - 1):                               # copies k-1 .. h+1 around it
                tail = Node("alt", [Node("cat", [_copy(body), tail]), Node("eps")])
            reps.append(tail)
        if h == 0:
            return reps[0]
        return Node("rep", reps, count=h, hi=hi)
    return Node(node.kind, kids, node.chars, node.count, hi=node.hi)


def derives_empty_text(node: Node) -> bool:
    """Whether the sub-RE generates the empty text (used for infinite ambiguity)."""
    k = node.kind
    if k == "term":
        return False
    if k == "eps":
        return True
    if k in ("cat", "rep"):
        return all(derives_empty_text(ch) for ch in node.children)
    if k == "alt":
        return any(derives_empty_text(ch) for ch in node.children)
    if k == "star":
        return True
    if k == "plus":
        return derives_empty_text(node.children[0])
    raise AssertionError(k)


def check_finite_ambiguity(node: Node):
    if node.kind in ("star", "plus") and derives_empty_text(node.children[0]):
        raise InfiniteAmbiguity("iterated sub-expression derives the empty text")
    for ch in node.children:
        check_finite_ambiguity(ch)


def number(root: Node) -> int:
    """Left-to-right preorder numbering with one shared counter (Sect. 2.2)."""
    counter = [0]

    def visit(n: Node):
        counter[0] += 1
        n.num = counter[0]
        for ch in n.children:
            visit(ch)

    visit(root)
    return counter[0]


# ----------------------------------------------------------------------------
# Numbered symbols.  ('(',k) open paren, (')',k) close paren, ('t',k) terminal,
# ('e',k) epsilon, ('$',0) the end-mark ⊣.
# ----------------------------------------------------------------------------
END = ("$", 0)


def sym_name(s) -> str:
    kind, k = s
    if kind == "(":
        return f"{k}("
    if kind == ")":
        return f"){k}"
    if kind == "t":
        return f"t{k}"
    if kind == "e":
        return f"e{k}"
    return "$"


def seg_name(seg) -> str:
    return " ".join(sym_name(s) for s in seg)


def is_end_letter(s) -> bool:
    """End-letters are the numbered terminals and ⊣ (Sect. 2.3.2)."""
    return s[0] in ("t", "$")


# ----------------------------------------------------------------------------
# Classic followers Fol(e_# ⊣, s) (Eq. classicfollowers).  The LST language is
# described by a regular expression over numbered symbols in which every
# symbol occurs once (Prop. 1); for such a linear expression the followers are
# the textbook first / last / follow sets.
# ----------------------------------------------------------------------------
def _lst_expr(n: Node):
    """The LST expression of a numbered node as nested ('sym'|'seq'|'alt'|'star'|'plus')."""
    k = n.num
    if n.kind == "term":
        return ("sym", ("t", k))
    if n.kind == "eps":
        return ("sym", ("e", k))
    o, c = ("sym", ("(", k)), ("sym", (")", k))
    kids = [_lst_expr(ch) for ch in n.children]
    if n.kind in ("cat", "rep"):
        return ("seq", [o] + kids + [c])
    if n.kind == "alt":
        return ("seq", [o, ("alt", kids), c])
    if n.kind == "star":
        return ("seq", [o, ("star", kids[0]), c])
    if n.kind == "plus":
        return ("seq", [o, ("plus", kids[0]), c])
    raise AssertionError(n.kind)


def _glushkov(e, fol):
    """Return (nullable, first, last) of e; add follow pairs into fol."""
    tag = e[0]
    if tag == "sym":
        return False, {e[1]}, {e[1]}
    if tag == "seq":
        nullable, first, last = True, set(), set()
        for part in e[1]:
            pn, pf, pl = _glushkov(part, fol)
            for s in last:
                fol.setdefault(s, set()).update(pf)
            if nullable:
                first |= pf
            last = (last | pl) if pn else set(pl)
            nullable = nullable and pn
        return nullable, first, last
    if tag == "alt":
        nullable, first, last = False, set(), set()
        for part in e[1]:
            pn, pf, pl = _glushkov(part, fol)
            nullable |= pn
            first |= pf
            last |= pl
        return nullable, first, last
    if tag in ("star", "plus"):
        pn, pf, pl = _glushkov(e[1], fol)
        for s in pl:
            fol.setdefault(s, set()).update(pf)
        return (True if tag == "star" else pn), pf, pl
    raise AssertionError(tag)


@dataclass
class Compiled:
    """Everything the oracle derives from an RE (Sects. 2.2-2.3)."""
    pattern: bytes
    root: Node
    symbols: list            # all numbered symbols of e_# ⊣
    fol: dict                # symbol -> set of follower symbols
    first_symbol: tuple      # first symbol of every LST
    classes: dict            # terminal number -> frozenset of bytes
    segments: list           # canonical order (see segment_key)
    index: dict              # segment tuple -> index in ``segments``
    initial: frozenset       # indices of I
    final: frozenset         # indices of F
    folseg: list             # index -> frozenset of follower indices (Eq. folsegdef)
    sample_limit: int = 0    # 0: exact; L >= 1: each symbol at most L times per segment
    infinitely_ambiguous: bool = False

    @property
    def ell(self) -> int:
        return len(self.segments)

    def names(self):
        return [seg_name(q) for q in self.segments]

    def end_letter(self, q: int):
        return self.segments[q][-1]

    def matches(self, q: int, byte: int) -> bool:
        """NFA arc label test: byte in the class of the end-letter of q."""
        e = self.end_letter(q)
        return e[0] == "t" and byte in self.classes[e[1]]


def symbol_key(s):
    """Order of numbered symbols used for the canonical segment order."""
    kind, k = s
    if kind == "$":
        return (1 << 30, 3)
    return (k, {"(": 0, ")": 1, "t": 2, "e": 2}[kind])


def segment_key(seg):
    return tuple(symbol_key(s) for s in seg)


def compile_re(pattern, sample_limit: int = 0) -> Compiled:
    """RE text -> segments, I, F and FolSeg (Sects. 2.2-2.3).

    sample_limit = 0 rejects an infinitely ambiguous RE (InfiniteAmbiguity);
    L >= 1 accepts it and samples its LSTs (App. A, "Infinite ambiguity")."""
    c = compile_tree(parse(pattern), sample_limit)
    c.pattern = pattern if isinstance(pattern, bytes) else pattern.encode("latin-1")
    return c


def compile_tree(root: Node, sample_limit: int = 0) -> Compiled:
    """Compile an already built structure tree (used for Ex. 5's e(k) family)."""
    import copy
    root = expand_repetitions(copy.deepcopy(root))
    try:
        check_finite_ambiguity(root)
        infinite = False
    except InfiniteAmbiguity:
        if sample_limit < 1:
            raise
        infinite = True
    number(root)
    fol: dict = {}
    _, first, _ = _glushkov(("seq", [_lst_expr(root), ("sym", END)]), fol)
    c = _finish(root, fol, next(iter(first)), sample_limit)
    c.infinitely_ambiguous = infinite
    return c


def _finish(root, fol, first_symbol, sample_limit: int = 0) -> Compiled:
    """Symbols, Fig. segmentalgo (MetaPrefix), I, F and Eq. folsegdef."""
    symbols, classes = [], {}

    def collect(n: Node):
        if n.kind == "term":
            symbols.append(("t", n.num)); classes[n.num] = n.chars
        elif n.kind == "eps":
            symbols.append(("e", n.num))
        else:
            symbols.append(("(", n.num))
            for ch in n.children:
                collect(ch)
            symbols.append((")", n.num))

    collect(root)
    symbols.append(END)
    fol = {s: frozenset(fol.get(s, ())) for s in symbols}
    preds = {s: [r for r in symbols if s in fol[r]] for s in symbols}
    Q = set()

    def meta_prefix(s, sigma):
        if s == first_symbol:
            Q.add(sigma)
            return
        for r in preds[s]:
            if is_end_letter(r):
                Q.add(sigma)
            else:
                seen = sigma.count(r)
                if seen and sample_limit < 1:
                    raise InfiniteAmbiguity("repeated symbol in a meta-prefix")
                if seen >= max(sample_limit, 1):
                    continue                 # App. A: the counter of r is at its limit
                meta_prefix(r, (r,) + sigma)

    for a in symbols:
        if is_end_letter(a):
            meta_prefix(a, (a,))
    segments = sorted(Q, key=segment_key)
    index = {q: i for i, q in enumerate(segments)}
    initial = frozenset(i for i, q in enumerate(segments) if q[0] == first_symbol)
    final = frozenset(i for i, q in enumerate(segments) if q[-1] == END)
    folseg = [frozenset(j for j, sg in enumerate(segments) if sg[0] in fol[rho[-1]])
              for rho in segments]
    return Compiled(pattern=b"", root=root, symbols=symbols, fol=fol, first_symbol=first_symbol,
                    classes=classes, segments=segments, index=index, initial=initial,
                    final=final, folseg=folseg, sample_limit=sample_limit)
