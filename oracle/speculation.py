"""Speculative work of the chunked parse under different start rules.

Test infrastructure only (see ``oracle/__init__.py``).  A model of how many
speculative runs a chunk's reach carries, written with the oracle's segment
sets, to compare the start rules of Sect. 3.1 and the two speculation
reductions of Sect. 4.3 on the same text:

* ``me``   -- ME-DFA starts (Sect. 3.1) with the last-character filter: the
  forward runs of a chunk start from {q} for every segment q that reads the
  chunk's first byte and can follow a segment that reads the byte before;
  after that byte the run from {q} is in FolSeg(q), so runs with the same
  successor set are one run.  Backward runs start from {q} for every q that
  reads the byte after the chunk; after the chunk's last byte they are in the
  reverse image of {q}, one run per distinct image.
* ``dfa``  -- every classic DFA state (reachable from I), or reverse DFA
  state (reachable from F), as a start: the alternative Sect. 5 measures the
  ME-DFA against.
* ``restricted`` (backward only) -- the ME-DFA backward starts limited to
  the segments of the exact forward column at the chunk's right edge.  Only
  those can be in the clean column there (C = B ∩ B̂), and every LST through
  a column to the left passes through one of them, so the clean columns are
  unchanged; the price is that the backward reach must wait for the forward
  join.
* edge shifting (technique (ii) of Sect. 4.3, for which the paper gives no
  algorithm): each chunk edge moves within ±s bytes to the position whose
  byte pair gives the fewest ME-DFA starts (forward + backward), ties to the
  nearest.

The work of a chunk is the number of transitions its runs take: at every
byte after the first one each distinct live state steps once (runs that reach
the same state are one run from then on, runs that die stop).  The exact
parse takes one transition per byte.
"""
from __future__ import annotations

from .parallel_equations import dfa_states
from .re_front import Compiled
from .serial import nfa_image, nfa_preimage


class Machine:
    """Memoised forward and reverse images of segment sets under a byte."""

    def __init__(self, c: Compiled):
        self.c = c
        self._f, self._b = {}, {}
        self.reads = [frozenset(q for q in range(c.ell) if c.matches(q, a)) for a in range(256)]
        self.enter = {}                 # byte -> segments that can follow a segment reading it

    def image(self, S, a):
        key = (S, a)
        T = self._f.get(key)
        if T is None:
            T = self._f[key] = nfa_image(self.c, S, a)
        return T

    def preimage(self, S, a):
        key = (S, a)
        T = self._b.get(key)
        if T is None:
            T = self._b[key] = nfa_preimage(self.c, S, a)
        return T

    def followers_of_byte(self, a):
        T = self.enter.get(a)
        if T is None:
            T = self.enter[a] = self.image(self.reads[a], a)
        return T


def forward_starts(m: Machine, prev: int, first: int, rule: str, dfa=None):
    """Start sets after the chunk's first byte (the empty set dropped)."""
    if rule == "me":
        cand = m.followers_of_byte(prev) & m.reads[first]
        out = {m.image(frozenset([q]), first) for q in cand}
    elif rule == "dfa":
        out = {m.image(S, first) for S in dfa}
    else:
        raise ValueError(rule)
    out.discard(frozenset())
    return out


def backward_starts(m: Machine, last: int, nxt: int, rule: str, rdfa=None, column=None):
    """Backward start sets after the chunk's last byte (the empty set dropped).
    ``column``: the exact forward column at the edge, for ``restricted``."""
    if rule == "me":
        out = {m.preimage(frozenset([q]), last) for q in m.reads[nxt]}
    elif rule == "restricted":
        out = {m.preimage(frozenset([q]), last) for q in m.reads[nxt] & column}
    elif rule == "dfa":
        out = {m.preimage(S, last) for S in rdfa}
    else:
        raise ValueError(rule)
    out.discard(frozenset())
    return out


def chunk_work(m: Machine, starts, rest: bytes, reverse: bool):
    """Transitions the runs take over ``rest`` (the chunk without the byte
    the starts already read, in reading order), and the bytes read until at
    most one run is left."""
    live = set(starts)
    work, settle = 0, 0
    for t, a in enumerate(rest):
        if len(live) <= 1:
            return work + len(live) * (len(rest) - t), settle
        work += len(live)
        live = {m.preimage(S, a) if reverse else m.image(S, a) for S in live}
        live.discard(frozenset())
        settle = t + 1
    return work, settle


def shifted_edges(m: Machine, text: bytes, k: int, s: int):
    """Chunk edges moved within ±s bytes to the fewest ME-DFA starts."""
    n = len(text)
    cost = {}

    def starts_at(e):
        key = (text[e - 1], text[e])
        v = cost.get(key)
        if v is None:
            v = cost[key] = (len(forward_starts(m, text[e - 1], text[e], "me"))
                             + len(backward_starts(m, text[e - 1], text[e], "me")))
        return v

    edges, last = [0], 0
    for e in range(k, n, k):
        lo, hi = max(last + 1, e - s), min(n - 1, e + s)
        best = min(range(lo, hi + 1), key=lambda p: (starts_at(p), abs(p - e)))
        edges.append(best)
        last = best
    edges.append(n)
    return edges


def report(c: Compiled, text: bytes, k: int, shifts=(8, 64)):
    """Speculative work over every chunk but the first (forward) or the last
    (backward), which start from I (resp. F) exactly.  Returns a dict of
    variant -> (mean starts per chunk, transitions / exact transitions,
    mean bytes until one run is left)."""
    m = Machine(c)
    n = len(text)
    dfa, rdfa = dfa_states(c), dfa_states(c, reverse=True)
    fwd_cols = [frozenset(c.initial)]
    for a in text:                                     # exact forward columns at every position
        fwd_cols.append(m.image(fwd_cols[-1], a))

    def measure(edges, fwd_rule=None, bwd_rule=None):
        starts = work = exact = settle = chunks = 0
        for i in range(len(edges) - 1):
            a, b = edges[i], edges[i + 1]
            if fwd_rule and a > 0:
                st = forward_starts(m, text[a - 1], text[a], fwd_rule, dfa)
                w, sl = chunk_work(m, st, text[a + 1:b], False)
            elif bwd_rule and b < n:
                col = fwd_cols[b] & m.reads[text[b]]
                st = backward_starts(m, text[b - 1], text[b], bwd_rule, rdfa, col)
                w, sl = chunk_work(m, st, text[a:b - 1][::-1], True)
            else:
                continue
            starts += len(st); work += w; exact += b - a - 1; settle += sl; chunks += 1
        return (starts / max(chunks, 1), work / max(exact, 1), settle / max(chunks, 1))

    plain = list(range(0, n, k)) + [n]
    out = {
        "fwd me": measure(plain, fwd_rule="me"),
        "fwd dfa": measure(plain, fwd_rule="dfa"),
        "bwd me": measure(plain, bwd_rule="me"),
        "bwd dfa": measure(plain, bwd_rule="dfa"),
        "bwd restricted": measure(plain, bwd_rule="restricted"),
    }
    for s in shifts:
        e = shifted_edges(m, text, k, s)
        out[f"fwd me, edges ±{s}"] = measure(e, fwd_rule="me")
        out[f"bwd me, edges ±{s}"] = measure(e, bwd_rule="me")
    return out


if __name__ == "__main__":
    # python -m oracle.speculation: the table of speculative work on 1 MiB of
    # the DNA and log workloads at their tuned chunk lengths and at 1 KiB.
    import workloads as W
    from .re_front import compile_re
    for name, pattern, text, ks in (("dna", W.DNA_RE, W.dna_text(1 << 20, seed=1).tobytes(), (6912, 1024)),
                                    ("log", W.LOG_RE, W.log_text(1 << 20, seed=2).tobytes(), (13824, 1024))):
        c = compile_re(pattern)
        for k in ks:
            print(f"{name} k={k}")
            for key, (starts, work, settle) in report(c, text, k).items():
                print(f"  {key:22s} starts/chunk {starts:6.2f}  transitions/exact {work:.4f}  "
                      f"bytes to one run {settle:7.1f}")
