"""The join as a pointer-jumping scan over chunk maps (Eq. joiner).

Chunks whose speculative runs never meet inside them have a map that depends
on their input; long runs of such chunks used to be evaluated one after the
other.  Here they are resolved by pointer jumping in a few rounds.  Cases:
(aa)* on a^n, where the even and odd runs never meet, so every chunk's map
depends on its input, at several MiB and tens of thousands of chunks; the
log RE with 64-byte chunks (a mix of both kinds); and the bounded wait of
the scan's grid barrier, made to run out by the test hook
RE_PARSE_TEST_STALL_JOIN (one block leaves before the barrier), which must
give the status RE_E_TIMEOUT and leave the device usable.
"""
import numpy as np
import pytest

import workloads as W
from oracle import serial
from oracle.re_front import compile_re

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2503_06763_gb300 import Regex, native
    return Regex, native


def parse(rx, host, chunk_len=0, flags=0):
    t = torch.from_numpy(np.ascontiguousarray(host)).cuda()
    cols, st, kind = rx.parse(t, chunk_len=chunk_len, extra_flags=flags)
    torch.cuda.synchronize()
    return cols.cpu().numpy(), int(st.item()), kind


def assert_equal_to_oracle(rx, pattern, host, cols, st):
    ids, table = serial.parse_ids(compile_re(pattern), host)
    want = table[ids]
    assert st == (0 if serial.accepted(want) else 1)
    got = rx.decode(cols, "dense" if rx.layout(1)[0] == "dense" else "dict")
    bad = np.nonzero(np.any(got != want, axis=1))[0]
    assert bad.size == 0, f"{bad.size} columns differ, first at r={bad[:5].tolist()}"


@pytest.mark.parametrize("n,chunk_len", [((4 << 20) + 2, 64), ((4 << 20) + 1, 64), ((8 << 20) + 2, 128),
                                         ((3 << 20) + 2, 0)])
def test_unconverged_chunks_at_several_mib(lib, n, chunk_len):
    Regex, _ = lib
    rx = Regex("(aa)*")
    host = np.full(n, ord("a"), dtype=np.uint8)
    cols, st, _ = parse(rx, host, chunk_len)
    assert st == (0 if n % 2 == 0 else 1)
    assert_equal_to_oracle(rx, "(aa)*", host, cols, st)


def test_ambiguous_mix_short_chunks(lib):
    Regex, _ = lib
    rx = Regex("(a|b|ab)*")
    host = W.ab_text((1 << 20) + 17, seed=41)
    cols, st, _ = parse(rx, host, 64)
    assert_equal_to_oracle(rx, "(a|b|ab)*", host, cols, st)


def test_log_records_short_chunks(lib):
    Regex, _ = lib
    rx = Regex(W.LOG_RE)
    host = W.log_text(2 << 20, seed=42)
    cols, st, _ = parse(rx, host, 64)
    assert st == 0
    assert_equal_to_oracle(rx, W.LOG_RE, host, cols, st)


def test_bounded_wait_runs_out(lib):
    Regex, native = lib
    rx = Regex("(aa)*")
    host = np.full((1 << 20) + 2, ord("a"), dtype=np.uint8)
    _, st, _ = parse(rx, host, 64, flags=native.RE_PARSE_TEST_STALL_JOIN)
    assert st == -7                                      # RE_E_TIMEOUT, read back from the device
    cols, st, _ = parse(rx, host, 64)                    # the device and the library still work
    assert st == 0
    assert_equal_to_oracle(rx, "(aa)*", host, cols, st)
