"""re_parse_static (library-owned scratch, no allocation) against re_parse.

The file name makes pytest collect it last, so a run that stops at the first
failure has run every other test before these.  No other test uses the
library's scratch: the cases here dirty it themselves, each call after the
first finding what the previous call left there.  Every case compares
re_parse_static with re_parse on a caller workspace, over calls in a row:
two calls on one text, two accepted texts of different lengths, a text after
a longer one under another RE, the recognizer mode, and a non-default stream.
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
    """Two accepted texts in a row, the second shorter, then a rejected one:
    no call may see what the call before it left in the scratch."""
    Regex, _ = lib
    rx = Regex(W.DNA_RE)
    a = torch.from_numpy(W.dna_text(200_000, seed=21)).cuda()
    b = torch.from_numpy(W.dna_text(150_000, seed=22)).cuda()
    c_host = W.dna_text(120_000, seed=23)
    c_host[77_777] = ord("N")                            # not in the alphabet: rejected text
    c = torch.from_numpy(c_host).cuda()
    want = [reference(rx, t) for t in (a, b, c)]
    assert [w[1] for w in want] == [0, 0, 1]
    got = [rx.parse_static(t) for t in (a, b, c)]
    torch.cuda.synchronize()
    for (cols, st, _), (wc, ws, _) in zip(got, want):
        assert int(st.item()) == ws
        assert np.array_equal(cols.cpu().numpy(), wc)


def test_after_a_longer_text_under_another_re(lib):
    """A log text of 162 segments fills much more of the scratch first (more
    slots, records and checkpoints); a shorter DNA text after it must still
    match re_parse, and so must the log text parsed again after that."""
    Regex, _ = lib
    rl, rd = Regex(W.LOG_RE), Regex(W.DNA_RE)
    big = torch.from_numpy(W.log_text(3 << 20, seed=24)).cuda()
    small = torch.from_numpy(W.dna_text(70_001, seed=25)).cuda()
    wl, sl, _ = reference(rl, big)
    wd, sd, _ = reference(rd, small)
    assert (sl, sd) == (0, 0)
    for rx, t, w in ((rl, big, wl), (rd, small, wd), (rl, big, wl)):
        cols, st, _ = rx.parse_static(t)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        assert np.array_equal(cols.cpu().numpy(), w)


def test_recognizer_and_side_stream(lib):
    """Recognizer mode through re_parse_static gives re_parse's status; a
    parse on a non-default stream gives its columns."""
    Regex, _ = lib
    rx = Regex(W.DNA_RE)
    good = torch.from_numpy(W.dna_text(90_000, seed=26)).cuda()
    bad_host = W.dna_text(90_000, seed=27)
    bad_host[123] = ord("N")
    bad = torch.from_numpy(bad_host).cuda()
    for t, want in ((good, 0), (bad, 1), (good, 0)):
        _, st, _ = rx.parse_static(t, recognize_only=True)
        torch.cuda.synchronize()
        assert int(st.item()) == want
    side = torch.cuda.Stream()
    want_cols, wst, _ = reference(rx, good)
    for _ in range(2):
        with torch.cuda.stream(side):
            cols, st, _ = rx.parse_static(good, stream=side)
        side.synchronize()
        assert int(st.item()) == wst == 0
        assert np.array_equal(cols.cpu().numpy(), want_cols)


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
