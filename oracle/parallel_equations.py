"""The parallel parser's equations, written with segment sets.

Test infrastructure only (see ``oracle/__init__.py``).

Sect. 3.1: DFA and ME-DFA states are segment sets; the transition function of
both is the NFA image of the set (powerset construction), the DFA starts from
T_1 = I and the ME-DFA from every singleton {q}.  The reverse machines use the
reverse NFA (Eq. reverseNFAdef).
Sect. 3.2: split, Eq. reacher, Eq. joiner, Eq. builder, Eq. merger, compose.
The chunks have length k except a shorter last one (the paper's equal-length
assumption relaxed).  The paper's splitter / composer index formulas are
garbled; the reading used is r = (i-1) k + t (Sect. 3.2, "split", Ex. 6).
The backward builder starts from Ĵ_{i+1} (the printed Eq. builder drops the
hat; Fig. builders&merger and the flow chart have it).
"""
from __future__ import annotations

from .re_front import Compiled
from .serial import nfa_image, nfa_preimage


def split(text: bytes, k: int):
    if k < 1:
        raise ValueError("chunk length must be >= 1")
    return [text[s:s + k] for s in range(0, len(text), k)]


def run(c: Compiled, S, chunk: bytes, reverse: bool = False):
    """delta*(S, chunk) of the (ME-)DFA, or of the reverse machine on chunk^R."""
    if reverse:
        for a in reversed(chunk):
            S = nfa_preimage(c, S, a)
    else:
        for a in chunk:
            S = nfa_image(c, S, a)
    return S


def backward_join(c: Compiled, y):
    """Eq. reacher (backward) from every reverse ME-DFA singleton and
    Eq. joiner: returns (R̂, Ĵ) with Ĵ_{c+1} = F."""
    cnum, ell = len(y), c.ell
    Rh = [None] + [[run(c, frozenset([j]), y[i - 1], reverse=True) for j in range(ell)]
                   for i in range(1, cnum + 1)]
    Jh = [None] * (cnum + 2)
    Jh[cnum + 1] = frozenset(c.final)
    for i in range(cnum, 0, -1):
        acc = set()
        for j in Jh[i + 1]:
            acc |= Rh[i][j]
        Jh[i] = frozenset(acc)
    return Rh, Jh


def build_merge_compose(c: Compiled, y, J, Jh):
    """Eq. builder (forward from J_{i-1}, backward from Ĵ_{i+1}), Eq. merger
    and compose: the clean columns C_0 .. C_n, and B, B̂."""
    cnum = len(y)
    B, Bh, M = [None], [None], [None]
    for i in range(1, cnum + 1):
        yi = y[i - 1]
        kk = len(yi)
        b = [None] * (kk + 1)
        b[1] = nfa_image(c, J[i - 1], yi[0])
        for t in range(2, kk + 1):
            b[t] = nfa_image(c, b[t - 1], yi[t - 1])
        bh = [None] * (kk + 1)
        bh[kk] = Jh[i + 1]
        for t in range(kk - 1, 0, -1):
            bh[t] = nfa_preimage(c, bh[t + 1], yi[t])      # y_{i,t+1}
        B.append(b)
        Bh.append(bh)
        M.append([None] + [b[t] & bh[t] for t in range(1, kk + 1)])
    cols = [J[0] & Jh[1]] if cnum else [frozenset(c.initial) & frozenset(c.final)]
    for i in range(1, cnum + 1):
        cols.extend(M[i][1:])
    return cols, B, Bh


def parse_parallel(c: Compiled, text: bytes, k: int):
    """Clean SLPF by Eqs. reacher, joiner, builder, merger.  Returns
    (columns, trace) where trace holds R, R̂, J, Ĵ, B, B̂ for inspection."""
    y = split(text, k)
    cnum = len(y)
    ell = c.ell
    # reach (FW) from every ME-DFA initial state S_j = {j}, and join
    R = [None] + [[run(c, frozenset([j]), y[i - 1]) for j in range(ell)] for i in range(1, cnum + 1)]
    J = [frozenset(c.initial)]
    for i in range(1, cnum + 1):
        acc = set()
        for j in J[i - 1]:
            acc |= R[i][j]
        J.append(frozenset(acc))
    Rh, Jh = backward_join(c, y)
    cols, B, Bh = build_merge_compose(c, y, J, Jh)
    return cols, dict(R=R, Rh=Rh, J=J, Jh=Jh, B=B, Bh=Bh)


def parse_parallel_dfa_starts(c: Compiled, text: bytes, k: int, forward: bool = True,
                              backward: bool = False):
    """The same equations with the reach started from every DFA state instead
    of every ME-DFA singleton: the alternative the ME-DFA of Sect. 3.1
    improves on (Sect. 5 measures both).  Forward: R_{i,T} = delta*(T, y_i)
    for every DFA state T; the join takes the run of the input state itself,
    J_i = R_{i,J_{i-1}} (J_{i-1} is a DFA state, or the empty set when the
    text cannot continue).  Backward likewise from every reverse DFA state,
    Ĵ_i = R̂_{i,Ĵ_{i+1}}.  A direction not selected keeps the ME-DFA starts."""
    y = split(text, k)
    cnum = len(y)
    if forward:
        starts = dfa_states(c)
        R = [None] + [{T: run(c, T, y[i - 1]) for T in starts} for i in range(1, cnum + 1)]
        J = [frozenset(c.initial)]
        for i in range(1, cnum + 1):
            J.append(R[i].get(J[i - 1], frozenset()))
    else:
        R = [None] + [[run(c, frozenset([j]), y[i - 1]) for j in range(c.ell)] for i in range(1, cnum + 1)]
        J = [frozenset(c.initial)]
        for i in range(1, cnum + 1):
            J.append(frozenset().union(*[R[i][j] for j in J[i - 1]]))
    if backward:
        starts = dfa_states(c, reverse=True)
        Rh = [None] + [{T: run(c, T, y[i - 1], reverse=True) for T in starts} for i in range(1, cnum + 1)]
        Jh = [None] * (cnum + 2)
        Jh[cnum + 1] = frozenset(c.final)
        for i in range(cnum, 0, -1):
            Jh[i] = Rh[i].get(Jh[i + 1], frozenset())
    else:
        Rh, Jh = backward_join(c, y)
    cols, B, Bh = build_merge_compose(c, y, J, Jh)
    return cols, dict(R=R, Rh=Rh, J=J, Jh=Jh, B=B, Bh=Bh)


def powerset_states(c: Compiled, starts, reverse: bool = False):
    """All segment sets reachable from ``starts`` under the (reverse) NFA image,
    over every byte.  The empty set is not included."""
    seen = set()
    stack = [frozenset(s) for s in starts if s]
    while stack:
        S = stack.pop()
        if S in seen:
            continue
        seen.add(S)
        for a in range(256):
            T = nfa_preimage(c, S, a) if reverse else nfa_image(c, S, a)
            if T and T not in seen:
                stack.append(T)
    return seen


def dfa_states(c: Compiled, reverse: bool = False):
    return powerset_states(c, [c.final if reverse else c.initial], reverse)


def medfa_states(c: Compiled, reverse: bool = False):
    return powerset_states(c, [[q] for q in range(c.ell)], reverse)
