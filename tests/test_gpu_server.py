"""The library's request loop (re_server): results, admission, batching.

Every request served from a mixed stream must equal ``Regex.parse`` of its
text alone, byte for byte (the batch kernels compute each text
independently); a burst must be batched; a request too large for a slot must
be refused at submission; completions are reported once, with their times.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def native():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2503_06763_gb300 import native
    return native


def _alone(rx, host):
    t = torch.from_numpy(np.ascontiguousarray(host)).cuda()
    cols, st, kind = rx.parse(t)
    torch.cuda.synchronize()
    return cols.cpu().numpy(), int(st.item())


def _texts():
    out = []
    for j, n in enumerate([0, 1, 700, 5000, 70_000, 300_000, 2_000_000]):
        out.append((0, W.log_text(n, seed=40 + j)))
        out.append((1, W.dna_text(n, seed=40 + j)))
        out.append((2, W.ab_text(n, seed=40 + j)))
    bad = W.log_text(20_000, seed=7).copy()
    bad[-1] = ord("x")                                        # rejected
    out.append((0, bad))
    return out


def test_mixed_stream_equals_single_parses(native):
    rxs = [native.Regex(W.LOG_RE), native.Regex(W.DNA_RE), native.Regex(W.AB_RE)]
    srv = native.NativeServer(rxs, slots=3, arena_bytes=256 << 20)
    try:
        reqs = _texts() * 2
        tickets = [srv.submit(ri, host) for ri, host in reqs]
        for t in tickets:
            srv.wait(t, 60_000)
        done = srv.poll(cap=len(tickets) + 10)
        assert sorted(t for t, _ in done) == sorted(tickets)
        for (ri, host), t in zip(reqs, tickets):
            cols, st = srv.result(t)
            want, wst = _alone(rxs[ri], host)
            assert st == wst, (ri, len(host))
            assert np.array_equal(cols.view(np.uint8), want.view(np.uint8)), (ri, len(host))
        stats = srv.stats()
        assert stats["requests"] == len(reqs) and stats["max_batch"] > 1 and stats["max_inflight"] >= 2
    finally:
        srv.close()


def test_oversized_request_is_refused(native):
    rx = native.Regex(W.AB_RE)
    srv = native.NativeServer([rx], slots=1, arena_bytes=32 << 20)
    try:
        with pytest.raises(native.ReError) as e:
            srv.submit(0, W.ab_text(24 << 20, seed=1))
        assert e.value.status == -8
        t = srv.submit(0, W.ab_text(1000, seed=1))            # the server still serves
        srv.wait(t, 60_000)
        cols, st = srv.result(t)
        assert st == 0
    finally:
        srv.close()


def test_wait_errors_and_timeout(native):
    rx = native.Regex(W.AB_RE)
    srv = native.NativeServer([rx], slots=1, arena_bytes=64 << 20)
    try:
        with pytest.raises(native.ReError):
            srv.wait(12345, 10)                               # never issued
        t = srv.submit(0, W.ab_text(10, seed=2))
        srv.wait(t, 60_000)
        srv.wait(t, 0)                                        # already complete: returns at once
        assert srv.result(t)[1] == 0
    finally:
        srv.close()


def test_concurrent_submitters(native):
    """Four host threads submit at once (re_server_submit is thread-safe);
    every request still equals its parse alone."""
    import threading
    rxs = [native.Regex(W.LOG_RE), native.Regex(W.AB_RE)]
    srv = native.NativeServer(rxs, slots=4, arena_bytes=128 << 20)
    texts = [(j % 2, (W.log_text if j % 2 == 0 else W.ab_text)(1000 + 997 * j, seed=100 + j)) for j in range(64)]
    tickets = [None] * len(texts)
    errors = []

    def submit(lo):
        try:
            for j in range(lo, len(texts), 4):
                tickets[j] = srv.submit(texts[j][0], texts[j][1])
        except Exception as e:                           # surfaced below
            errors.append(e)

    threads = [threading.Thread(target=submit, args=(lo,)) for lo in range(4)]
    try:
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        assert not errors
        assert len(set(tickets)) == len(texts)
        for (ri, host), t in zip(texts, tickets):
            srv.wait(t, 60_000)
            cols, st = srv.result(t)
            want, wst = _alone(rxs[ri], host)
            assert st == wst and np.array_equal(cols.view(np.uint8), want.view(np.uint8)), (ri, len(host))
    finally:
        srv.close()
