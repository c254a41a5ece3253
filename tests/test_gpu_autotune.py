"""re_autotune: the chosen chunk length is kept per handle and length bucket,
used by later parses and workspace queries, and never changes the result."""
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
    from paper_2503_06763_gb300 import Regex
    return Regex


def test_autotune_keeps_choice_and_result(lib):
    Regex = lib
    n = 3 << 20
    host = W.dna_text(n, seed=41)
    t = torch.from_numpy(host).cuda()
    fresh = Regex(W.DNA_RE)
    rx = Regex(W.DNA_RE)
    rule_ws = fresh.workspace_size(n)
    k = rx.autotune(t)
    assert k >= 256 and k % 64 == 0
    assert rx.workspace_size(n) == rx.workspace_size(n, chunk_len=k)
    assert rx.workspace_size(n + 12345) == rx.workspace_size(n + 12345, chunk_len=k)   # same length bucket
    assert fresh.workspace_size(n) == rule_ws                                           # per handle
    want = serial.parse(compile_re(W.DNA_RE), host)
    cols, st, kind = rx.parse(t)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert np.array_equal(rx.decode(cols.cpu().numpy(), kind), want)
    # a workspace sized by the rule: the parse falls back to the rule's chunk length
    small = torch.empty(rule_ws, dtype=torch.uint8, device="cuda")
    cols2, st2, _ = rx.parse(t, workspace=small)
    torch.cuda.synchronize()
    assert int(st2.item()) == 0 and torch.equal(cols2, cols)


def test_recognizer_has_its_own_choice(lib):
    """The recognizer's chunk length is tuned and kept apart from the parse's
    (the key holds the mode), and recognizing with it gives the oracle's verdict."""
    Regex = lib
    n = 3 << 20
    host = W.dna_text(n, seed=42)
    t = torch.from_numpy(host).cuda()
    rx = Regex(W.DNA_RE)
    k_parse = rx.autotune(t)
    k_rec = rx.autotune(t, recognize_only=True)
    assert k_rec >= 256 and k_rec % 64 == 0
    assert rx.workspace_size(n) == rx.workspace_size(n, chunk_len=k_parse)
    assert rx.workspace_size(n, flags=1) == rx.workspace_size(n, chunk_len=k_rec, flags=1)
    want = serial.accepted(serial.parse(compile_re(W.DNA_RE), host))
    for h in (host, np.concatenate([host[:1000], np.frombuffer(b"X", dtype=np.uint8), host[1001:]])):
        tt = torch.from_numpy(np.ascontiguousarray(h)).cuda()
        _, st, _ = rx.parse(tt, recognize_only=True)
        torch.cuda.synchronize()
        expect = want if h is host else serial.accepted(serial.parse(compile_re(W.DNA_RE), h.tobytes()))
        assert int(st.item()) == (0 if expect else 1)


def test_autotune_chooses_a_reach_shape(lib):
    """The tuner searches reach shapes too; the (length, shape) it keeps is
    reported by re_tuned and the parse with it matches the oracle."""
    Regex = lib
    host = W.log_text(2 << 20, seed=43)
    t = torch.from_numpy(host).cuda()
    rx = Regex(W.LOG_RE)
    assert rx.tuned(len(host)) == (0, 0)
    k = rx.autotune(t)
    kt, shape = rx.tuned(len(host))
    assert kt == k and shape in (1, 2, 3, 4)
    ids, table = serial.parse_ids(compile_re(W.LOG_RE), host)
    cols, st, kind = rx.parse(t)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert np.array_equal(rx.decode(cols.cpu().numpy(), kind), table[ids])
