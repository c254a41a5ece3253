"""SLPF compression (App. C): the oracle's archive and the library's encoder.

The oracle's archive (``oracle/slpf_dfa.py``) is pinned by its round trip
against the serial parser's columns: decoding must give back every column of
the SLPF, for several REs, texts and checkpoint intervals.  The measured fact
behind its exception list is pinned too: on (a|b|ab)* the column after an
``a`` depends on the next byte, so the paper's table alone cannot be a
function there, while on a text where every (column, byte) pair occurs once
there is no exception at all.  The library's host encoder must produce the
same table, checkpoints and exceptions as the oracle, byte for byte.
"""
import ctypes

import numpy as np
import pytest

import workloads as W
from oracle import serial
from oracle import slpf_dfa as SD
from oracle.re_front import compile_re

CASES = [(W.AB_RE, W.ab_text(3000, seed=1).tobytes()),
         (W.DNA_RE, W.dna_text(20_000, seed=2, mean_gap=500).tobytes()),
         (W.LOG_RE, W.log_text(8000, seed=3).tobytes()),
         ("(ab|a)*", b"ab" * 50 + b"a" * 7),
         ("(a|ab|aba)+", b"ababa"),
         (W.AB_RE, b""),
         (W.AB_RE, b"abc")]                      # rejected: every column empty


def _ids(pattern, text):
    ids, _ = serial.parse_ids(compile_re(pattern), text)
    return ids


@pytest.mark.parametrize("k", range(len(CASES)))
@pytest.mark.parametrize("K", [1, 7, 64, 4096])
def test_round_trip_gives_back_every_column(k, K):
    pattern, text = CASES[k]
    ids = _ids(pattern, text)
    table, exc, cps = SD.encode(ids, text, K)
    assert len(cps) == len(text) // K + 1
    assert np.array_equal(SD.decode(table, exc, cps, text, K), ids.astype(np.int64))


def test_the_next_column_depends_on_the_future():
    """(a|b|ab)*: after an 'a' the column holds the segments that read the
    next byte, so (C, 'a') is followed by different columns: exceptions."""
    text = b"aab" * 20
    ids = _ids(W.AB_RE, text)
    _, exc, _ = SD.encode(ids, text, 1 << 20)
    assert exc
    c = compile_re(W.AB_RE)
    cols = serial.parse_small(c, text)
    for r, v in exc:                           # an exception is a column the table's key cannot tell
        assert cols[r] != cols[[q for q in range(1, r) if ids[q - 1] == ids[r - 1] and text[q - 1] == text[r - 1]][0]]


def test_no_exception_when_every_key_is_new():
    text = b"ab"
    ids = _ids(W.AB_RE, text)
    table, exc, _ = SD.encode(ids, text, 1)
    assert exc == [] and len(table) == 2


def _native():
    try:
        from paper_2503_06763_gb300 import native
        native.load()
    except ImportError:
        import __graft_entry__
        __graft_entry__.build()
        from paper_2503_06763_gb300 import native
    return native


def _parse_archive(native, arch, cb):
    """Sections of an archive as the header of slpf_parser.h lays them out;
    exceptions come back as absolute positions and ids."""
    h = native.slpf_dfa_header(arch)
    hdr = ctypes.sizeof(native.DfaHeader)
    al = lambda v: (v + 15) & ~15
    off_t = al(hdr)
    off_c = off_t + al(h["n_ids"] * 256 * 2)
    off_s = off_c + al(h["n_checkpoints"] * 2)
    off_e = off_s + al((h["n_checkpoints"] + 1) * 8)
    table = arch[off_t:off_t + h["n_ids"] * 512].view(np.uint16).reshape(h["n_ids"], 256)
    cps = arch[off_c:off_c + h["n_checkpoints"] * 2].view(np.uint16)
    starts = arch[off_s:off_s + (h["n_checkpoints"] + 1) * 8].view(np.uint64)
    exc = arch[off_e:off_e + h["n_exceptions"] * 4].view(np.uint32)
    assert starts[0] == 0 and starts[-1] == h["n_exceptions"] and np.all(np.diff(starts.astype(np.int64)) >= 0)
    piece = np.repeat(np.arange(h["n_checkpoints"], dtype=np.uint64), np.diff(starts.astype(np.int64)))
    pos = piece * np.uint64(h["interval"]) + (exc >> 16).astype(np.uint64)
    ids = exc & 0xFFFF
    return h, table, cps, pos, ids


@pytest.mark.parametrize("k", range(len(CASES)))
@pytest.mark.parametrize("K", [7, 4096])
def test_native_encoder_equals_the_oracle(k, K):
    native = _native()
    pattern, text = CASES[k]
    ids = _ids(pattern, text)
    cb = 1 if ids.max() < 256 else 2
    cols = ids.astype({1: np.uint8, 2: np.uint16}[cb])
    arch = native.slpf_dfa_encode(cols, text, K)
    h, table, cps, pos, xids = _parse_archive(native, arch, cb)
    otable, oexc, ocps = SD.encode(ids, text, K)
    assert h["magic"] == 0x46504C53 and h["n"] == len(text) and h["interval"] == K
    assert h["n_ids"] == int(ids.max()) + 1
    want = np.full((h["n_ids"], 256), 0xFFFF, dtype=np.uint16)
    for (v, a), w in otable.items():
        want[v, a] = w
    assert np.array_equal(table, want)
    assert cps.tolist() == ocps
    assert list(zip(pos.tolist(), xids.tolist())) == oexc


def test_native_encoder_errors():
    native = _native()
    with pytest.raises(native.ReError):
        native.slpf_dfa_encode(np.zeros(3, dtype=np.uint8), b"ab", 0)       # interval 0
    with pytest.raises(ValueError):
        native.slpf_dfa_encode(np.zeros(2, dtype=np.uint8), b"ab", 4)       # one column short
    with pytest.raises(native.ReError):
        native.slpf_dfa_encode(np.full(3, 70000, dtype=np.uint32), b"ab", 4)  # ids past 65534
    with pytest.raises(native.ReError):
        native.slpf_dfa_encode(np.zeros(3, dtype=np.uint8), b"ab", 70000)    # interval past 65536
