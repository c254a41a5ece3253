"""SLPF archives (App. C) rebuilt on the device.

The columns of a device parse are archived by the library's host encoder
(pinned against the oracle in ``test_oracle_slpf_dfa``) and rebuilt by
``re_slpf_dfa_decode``; the rebuilt bytes must equal the parse's, and the
parse's equal the oracle's.  Also: a rejected text, the empty text, every
checkpoint interval from 1 up, and an archive run over another text (the
table misses a pair: the status says so and nothing is read out of bounds).
"""
import numpy as np
import pytest

import workloads as W
from oracle import serial
from oracle.re_front import compile_re

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def native():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2503_06763_gb300 import native
    return native


def _parse(rx, host):
    t = torch.from_numpy(np.ascontiguousarray(host)).cuda()
    cols, st, kind = rx.parse(t)
    torch.cuda.synchronize()
    return t, cols, int(st.item()), kind


@pytest.mark.parametrize("case", ["log", "dna", "ab-dense", "rejected", "empty"])
@pytest.mark.parametrize("K", [1, 64, 4096])
def test_archive_round_trip(native, case, K):
    if case == "log":
        pattern, host = W.LOG_RE, W.log_text(300_000, seed=4)
    elif case == "dna":
        pattern, host = W.DNA_RE, W.dna_text(300_000, seed=4)
    elif case == "ab-dense":
        pattern, host = W.AB_RE, W.ab_text(100_001, seed=4)
    elif case == "rejected":
        pattern, host = W.LOG_RE, W.log_text(50_000, seed=5).copy()
        host[-1] = ord("x")
    else:
        pattern, host = W.AB_RE, np.zeros(0, dtype=np.uint8)
    rx = native.Regex(pattern)
    t, cols, st, kind = _parse(rx, host)
    assert kind in ("dict", "dense")
    want = serial.parse(compile_re(pattern), host.tobytes())
    assert np.array_equal(rx.decode(cols.cpu().numpy(), kind), want)
    cb = cols.element_size()
    arch = native.slpf_dfa_encode(cols.cpu().numpy().view({1: np.uint8, 2: np.uint16, 4: np.uint32}[cb]),
                                  host.tobytes(), K)
    got, status = native.slpf_dfa_decode(arch, t, cb)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert torch.equal(got.view(torch.uint8), cols.view(torch.uint8)), case


def test_archive_of_another_text_is_flagged(native):
    rx = native.Regex(W.AB_RE)
    a = W.ab_text(5000, seed=1)
    t, cols, st, _ = _parse(rx, a)
    arch = native.slpf_dfa_encode(cols.cpu().numpy().view(np.uint16), a.tobytes(), 256)
    other = torch.from_numpy(np.full(5000, ord("c"), dtype=np.uint8)).cuda()   # pairs (column, 'c') never occur
    got, status = native.slpf_dfa_decode(arch, other, 2)
    torch.cuda.synchronize()
    assert int(status.item()) == -9
