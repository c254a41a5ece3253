"""Oracle serial parser (Eq. matrixmul, Eq. reverseNFAdef, Fig. serialparser).

Test infrastructure only (see ``oracle/__init__.py``).

The parser NFA (Sect. 2.3.4): states are the segments; there is an arc from
q_col to q_row labelled a iff q_row ∈ FolSeg(q_col) and a belongs to the class
of the end-letter of q_col.  N_a[row, col] is that arc (Sect. 2.4).  The
reverse NFA has N̂_a = N_a^T and I, F switched (Eq. reverseNFAdef).

``parse_small`` runs Fig. serialparser with Python sets, one column at a time.
``parse`` runs the same products in ``serial_parser.c`` over bitsets.  Both
return the clean SLPF columns C_r ∩ Ĉ_r, r = 0..n.  ``parse_ids`` returns
the same columns interned (an id per position and a table of distinct
columns), for texts too long to hold W words per position.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from .re_front import Compiled

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "serial_parser.c")
_LIB = os.path.join(_HERE, "liboracle_serial.so")
_lock = threading.Lock()
_lib = None


def build_library(force: bool = False) -> str:
    """Compile serial_parser.c with gcc (plain C, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build_library()
            lib = ctypes.CDLL(_LIB)
            lib.oracle_serial_parse.restype = ctypes.c_int
            lib.oracle_serial_parse.argtypes = [
                ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
            lib.oracle_serial_parse_ids.restype = ctypes.c_int
            lib.oracle_serial_parse_ids.argtypes = [
                ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                ctypes.c_void_p]
            _lib = lib
    return _lib


# ---------------------------------------------------------------------------
def nfa_image(c: Compiled, states, byte):
    """Column N_byte x V as a set: all targets of arcs labelled ``byte``."""
    out = set()
    for q in states:
        if c.matches(q, byte):
            out |= c.folseg[q]
    return frozenset(out)


def nfa_preimage(c: Compiled, states, byte):
    """N_byte^T x V as a set: sources of arcs labelled ``byte`` into V."""
    return frozenset(q for q in range(c.ell) if c.matches(q, byte) and c.folseg[q] & states)


def parse_small(c: Compiled, text: bytes):
    """Fig. serialparser with Python sets.  Returns list of n+1 frozensets."""
    n = len(text)
    fwd = [frozenset(c.initial)]
    for r in range(1, n + 1):
        fwd.append(nfa_image(c, fwd[r - 1], text[r - 1]))
    bwd = [None] * (n + 1)
    bwd[n] = frozenset(c.final)
    for r in range(n - 1, -1, -1):
        bwd[r] = nfa_preimage(c, bwd[r + 1], text[r])
    return [fwd[r] & bwd[r] for r in range(n + 1)]


# ---------------------------------------------------------------------------
def words(ell: int) -> int:
    return (ell + 63) // 64


def to_bits(c: Compiled, states) -> np.ndarray:
    W = words(c.ell)
    v = np.zeros(W, dtype=np.uint64)
    for q in states:
        v[q >> 6] |= np.uint64(1) << np.uint64(q & 63)
    return v


def from_bits(row) -> frozenset:
    out = []
    for w, word in enumerate(np.asarray(row, dtype=np.uint64).tolist()):
        while word:
            low = word & -word
            out.append(w * 64 + low.bit_length() - 1)
            word ^= low
    return frozenset(out)


def nfa_columns(c: Compiled) -> np.ndarray:
    """ncol[a, j] = column j of N_a as a bitset of rows (targets)."""
    W = words(c.ell)
    ncol = np.zeros((256, c.ell, W), dtype=np.uint64)
    for j in range(c.ell):
        tgt = to_bits(c, c.folseg[j])
        e = c.end_letter(j)
        if e[0] != "t":
            continue
        for a in c.classes[e[1]]:
            ncol[a, j] = tgt
    return ncol


def parse(c: Compiled, text) -> np.ndarray:
    """Clean SLPF as a [(n+1), W] uint64 bitset array, via serial_parser.c."""
    lib = _load()
    x = np.frombuffer(bytes(text), dtype=np.uint8) if not isinstance(text, np.ndarray) else text
    x = np.ascontiguousarray(x, dtype=np.uint8)
    n = int(x.shape[0])
    W = words(c.ell)
    ncol = nfa_columns(c)
    I = to_bits(c, c.initial)
    F = to_bits(c, c.final)
    out = np.zeros((n + 1, W), dtype=np.uint64)
    tmp = np.zeros(2 * W, dtype=np.uint64)
    rc = lib.oracle_serial_parse(c.ell, W, ncol.ctypes.data, I.ctypes.data, F.ctypes.data,
                                 x.ctypes.data, n, out.ctypes.data, tmp.ctypes.data)
    if rc != 0:
        raise RuntimeError("oracle_serial_parse failed")
    return out


def parse_ids(c: Compiled, text, cap: int = 1 << 20):
    """The clean SLPF of ``parse`` with every column interned, for long texts:
    returns (ids, cols) with ids a uint32 array of n+1 indices into cols, a
    [D, W] uint64 array of the distinct clean columns.  Column r of the SLPF
    is cols[ids[r]].  The forward and backward columns are interned as well,
    and each product of a stored column with a byte is computed once (the same
    loops as ``parse``), so a GiB of text needs 4 bytes per position."""
    lib = _load()
    x = np.frombuffer(bytes(text), dtype=np.uint8) if not isinstance(text, np.ndarray) else text
    x = np.ascontiguousarray(x, dtype=np.uint8)
    n = int(x.shape[0])
    W = words(c.ell)
    ncol = nfa_columns(c)
    I = to_bits(c, c.initial)
    F = to_bits(c, c.final)
    ids = np.empty(n + 1, dtype=np.uint32)
    cols = np.zeros((cap, W), dtype=np.uint64)
    nc = ctypes.c_int64(0)
    rc = lib.oracle_serial_parse_ids(c.ell, W, ncol.ctypes.data, I.ctypes.data, F.ctypes.data, x.ctypes.data,
                                     n, ids.ctypes.data, cols.ctypes.data, cap, ctypes.byref(nc))
    if rc != 0:
        raise RuntimeError(f"oracle_serial_parse_ids failed ({rc})")
    return ids, cols[:nc.value].copy()


def accepted(columns: np.ndarray) -> bool:
    """A text is in L(e) iff its clean C_0 is non-empty (Sect. 2.3.5)."""
    return bool(np.any(columns[0] != 0))
