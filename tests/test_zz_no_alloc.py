"""re_parse_static (library-owned scratch, no allocation) against re_parse.

Collected last on purpose (file name): it must give the same bytes whether it
runs alone or after every other GPU test has used the device.  Each case makes
two re_parse_static calls in a row and compares both with re_parse on a
caller workspace.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2503_06763_gb300 import Regex, native
    return Regex, native


def reference(rx, text, chunk_len=0):
    cols, status, kind = rx.parse(text, chunk_len=chunk_len)
    torch.cuda.synchronize()
    return cols.cpu().numpy(), int(status.item()), kind


@pytest.mark.parametrize("pattern,make,n", [
    (W.DNA_RE, lambda n: W.dna_text(n, seed=11), 1 << 20),
    (W.AB_RE, lambda n: W.ab_text(n, seed=12), 300_001),
    (W.DNA_RE, lambda n: W.dna_text(n, seed=13), 4097),
])
def test_two_calls_match_re_parse(lib, pattern, make, n):
    Regex, _ = lib
    rx = Regex(pattern)
    text = torch.from_numpy(make(n)).cuda()
    want, wst, kind = reference(rx, text)
    for _ in range(2):
        cols, status, k2 = rx.parse_static(text)
        torch.cuda.synchronize()
        assert k2 == kind
        assert int(status.item()) == wst == 0
        assert np.array_equal(cols.cpu().numpy(), want)


def test_consecutive_different_texts(lib):
    """A second call on another text must not see the first call's scratch."""
    Regex, _ = lib
    rx = Regex(W.DNA_RE)
    a = torch.from_numpy(W.dna_text(200_000, seed=21)).cuda()
    b_host = W.dna_text(150_000, seed=22)
    b_host[77_777] = ord("N")                            # not in the alphabet: rejected text
    b = torch.from_numpy(b_host).cuda()
    wa, sa, _ = reference(rx, a)
    wb, sb, _ = reference(rx, b)
    assert (sa, sb) == (0, 1)
    ca, st_a, _ = rx.parse_static(a)
    cb, st_b, _ = rx.parse_static(b)
    torch.cuda.synchronize()
    assert int(st_a.item()) == 0 and int(st_b.item()) == 1
    assert np.array_equal(ca.cpu().numpy(), wa)
    assert np.array_equal(cb.cpu().numpy(), wb)


def test_text_beyond_scratch_is_refused(lib):
    Regex, native = lib
    rx = Regex(W.DNA_RE)
    n = 16 << 20                                         # automatic chunking needs > 64 MiB here
    assert rx.workspace_size(n) > native.RE_STATIC_SCRATCH_BYTES
    text = torch.from_numpy(W.dna_text(n, seed=31)).cuda()
    out = torch.zeros(n + 1, dtype=torch.int16, device="cuda")
    status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    with pytest.raises(native.ReError) as e:
        rx.parse_static(text, out=out, status=status)
    assert e.value.status == -8                          # RE_E_CAPACITY, nothing enqueued
    torch.cuda.synchronize()
    assert int(status.item()) == 7 and int(out.abs().sum().item()) == 0
