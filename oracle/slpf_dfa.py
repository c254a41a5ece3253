"""SLPF compression by a text-specific transition table (App. C, "SLPF compression").

Test infrastructure only (see ``oracle/__init__.py``).

App. C stores the SLPF as the initial column and a table delta(C_{r-1}, x_r) =
C_r over the columns that occur, and rebuilds C_1 .. C_n by running the table
over the text.  On a clean SLPF the next column is not always a function of
the previous column and the byte: the columns carry the future too (C_r holds
only segments on a complete LST, and which of them survive can depend on
bytes after r).  The reading used here keeps the paper's table and makes the
archive exact with an exception list:

* the table maps each key (column id of C_{r-1}, byte x_r) to the column
  that follows the key's first occurrence (r smallest);
* every K-th column (r = 0, K, 2K, ...) is stored as a checkpoint, so the
  columns can be rebuilt in independent pieces ("a selection of evenly spaced
  columns stored together with the SLPF-DFA", the improvement App. C names);
* every other position r whose column differs from the table's value is an
  exception (r, id of C_r).

Columns are given as ids (any integer labelling of the distinct columns, e.g.
the DICT encoding or ``serial.parse_ids``).
"""
from __future__ import annotations

import numpy as np


def encode(ids, text: bytes, K: int):
    """Returns (table dict (id, byte) -> id, exceptions [(r, id)] ascending,
    checkpoints [ids of C_0, C_K, C_2K, ...])."""
    ids = [int(v) for v in ids]
    n = len(text)
    if len(ids) != n + 1:
        raise ValueError("one column per position 0..n")
    table, exceptions = {}, []
    for r in range(1, n + 1):
        key = (ids[r - 1], text[r - 1])
        if key not in table:
            table[key] = ids[r]
        elif table[key] != ids[r] and r % K:
            exceptions.append((r, ids[r]))
    checkpoints = [ids[r] for r in range(0, n + 1, K)]
    return table, exceptions, checkpoints


def decode(table, exceptions, checkpoints, text: bytes, K: int):
    """Columns C_0 .. C_n rebuilt piece by piece from the checkpoints."""
    n = len(text)
    exc = dict(exceptions)
    out = []
    for s, start in enumerate(checkpoints):
        cur = start
        out.append(cur)
        for r in range(s * K + 1, min((s + 1) * K, n + 1)):
            cur = exc[r] if r in exc else table[(cur, text[r - 1])]
            out.append(cur)
    return np.array(out, dtype=np.int64)
