"""re_parse_batch: many texts under several REs, one launch per phase and RE.

Each text's columns and status must be byte-identical to re_parse on the
same text alone (which the parity tests pin to the oracle); a few small
texts are also checked against the oracle directly.  Covers empty, tiny and
ragged texts, rejected texts, a 162-segment RE (three words per column),
recognizer mode, re-running the bound buffers after their bytes change, and
capture of the re-run in a CUDA graph.
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
    from paper_2503_06763_gb300 import Batch, Regex
    return Batch, Regex


def _texts(patterns):
    """(pattern index, host bytes) pairs of mixed sizes, seeded."""
    rng = np.random.Generator(np.random.PCG64(5))
    out = []
    sizes = [0, 1, 2, 63, 64, 65, 255, 1000, 4097, 20_000, 70_001, 300_000]
    for pi, (pat, make) in enumerate(patterns):
        for n in sizes:
            out.append((pi, make(n, int(rng.integers(1 << 30)))))
    return out


def _patterns():
    rp, tree, _ = W.random_re(41, 10, 60)
    log = W.log_text(400_000, seed=2)

    def log_slice(n, s):                    # a window of one generated log text
        off = s % (len(log) - n) if n < len(log) else 0
        return log[off:off + n].copy()

    return [
        (W.DNA_RE, lambda n, s: W.dna_text(n, seed=s)),
        (W.AB_RE, lambda n, s: W.ab_text(n, seed=s)),
        (rp, lambda n, s: np.frombuffer(W.sample_text(tree, n, s).tobytes()[:n], dtype=np.uint8).copy()),
        (W.LOG_RE, log_slice),
    ]


def _alone(rx, t, recognize=False):
    cols, st, _ = rx.parse(t, recognize_only=recognize)
    torch.cuda.synchronize()
    return (None if recognize else cols.cpu().numpy()), int(st.item())


def test_mixed_batch_matches_single_parses(lib):
    Batch, Regex = lib
    pats = _patterns()
    rxs = [Regex(p) for p, _ in pats]
    items = _texts(pats)
    # one rejected text per RE: a byte no RE here matches
    for pi in range(len(pats)):
        h = pats[pi][1](5000, 77 + pi)
        h[len(h) // 2] = 0xFF
        items.append((pi, h))
    texts = [torch.from_numpy(np.ascontiguousarray(h)).cuda() for _, h in items]
    b = Batch([rxs[pi] for pi, _ in items], [len(h) for _, h in items])
    outs, status, kinds = b.parse(texts)
    torch.cuda.synchronize()
    st = status.cpu().numpy()
    rejected = 0
    for j, ((pi, h), t) in enumerate(zip(items, texts)):
        want, wst = _alone(rxs[pi], t)
        assert st[j] == wst, (j, pi, len(h))
        assert np.array_equal(outs[j].cpu().numpy(), want), (j, pi, len(h), b.chunk_len(j))
        rejected += wst == 1
    assert rejected >= 3                               # the log RE accepts any byte in a line
    # small texts straight against the oracle
    for j, (pi, h) in enumerate(items):
        if len(h) <= 1000:
            c = compile_re(pats[pi][0])
            want = serial.parse(c, h.tobytes())
            got = rxs[pi].decode(outs[j].cpu().numpy(), kinds[j])
            assert np.array_equal(got, want)
            assert st[j] == (0 if serial.accepted(want) else 1)


def test_batch_rerun_after_text_change_and_graph_capture(lib):
    Batch, Regex = lib
    rx_d, rx_a = Regex(W.DNA_RE), Regex(W.AB_RE)
    hosts = [W.dna_text(100_000, seed=1), W.ab_text(33_333, seed=2), W.dna_text(7_777, seed=3)]
    texts = [torch.from_numpy(h).cuda() for h in hosts]
    b = Batch([rx_d, rx_a, rx_d], [len(h) for h in hosts])
    outs, status, _ = b.parse(texts)
    torch.cuda.synchronize()
    # new bytes in the same buffers, then run again (kernels only)
    new = [W.dna_text(100_000, seed=11), W.ab_text(33_333, seed=12), W.dna_text(7_777, seed=13)]
    for t, h in zip(texts, new):
        t.copy_(torch.from_numpy(h))
    b.run()
    torch.cuda.synchronize()
    for j, (rx, t) in enumerate(zip([rx_d, rx_a, rx_d], texts)):
        want, wst = _alone(rx, t)
        assert int(status[j].item()) == wst and np.array_equal(outs[j].cpu().numpy(), want)
    # the same re-run captured in a CUDA graph and replayed on fresh bytes
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        b.run(stream=side)                      # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        b.run()
    newer = [W.dna_text(100_000, seed=21), W.ab_text(33_333, seed=22), W.dna_text(7_777, seed=23)]
    for t, h in zip(texts, newer):
        t.copy_(torch.from_numpy(h))
    for o in outs:
        o.zero_()
    g.replay()
    torch.cuda.synchronize()
    for j, (rx, t) in enumerate(zip([rx_d, rx_a, rx_d], texts)):
        want, wst = _alone(rx, t)
        assert int(status[j].item()) == wst and np.array_equal(outs[j].cpu().numpy(), want)


def test_recognizer_batch(lib):
    Batch, Regex = lib
    rx = Regex(W.DNA_RE)
    hosts = [W.dna_text(n, seed=n) for n in (0, 10, 5000, 90_000)]
    bad = W.dna_text(40_000, seed=9)
    bad[123] = ord("x")
    hosts.append(bad)
    texts = [torch.from_numpy(h).cuda() for h in hosts]
    b = Batch([rx] * len(hosts), [len(h) for h in hosts], recognize_only=True)
    outs, status, _ = b.parse(texts)
    torch.cuda.synchronize()
    for j, t in enumerate(texts):
        _, wst = _alone(rx, t, recognize=True)
        assert int(status[j].item()) == wst
    assert int(status[len(hosts) - 1].item()) == 1


def test_fixed_chunk_length_and_only_empty_texts(lib):
    Batch, Regex = lib
    rx = Regex(W.AB_RE)
    e = [torch.empty(0, dtype=torch.uint8, device="cuda") for _ in range(3)]
    b = Batch([rx] * 3, [0, 0, 0])
    outs, status, kinds = b.parse(e)
    torch.cuda.synchronize()
    want, wst = _alone(rx, e[0])
    for j in range(3):
        assert int(status[j].item()) == wst and np.array_equal(outs[j].cpu().numpy(), want)
    hosts = [W.ab_text(n, seed=n) for n in (129, 4096, 10_001)]
    texts = [torch.from_numpy(h).cuda() for h in hosts]
    b2 = Batch([rx] * 3, [len(h) for h in hosts], chunk_len=128)
    assert all(b2.chunk_len(j) == 128 for j in range(3))
    outs, status, _ = b2.parse(texts)
    torch.cuda.synchronize()
    for j, t in enumerate(texts):
        want, wst = _alone(rx, t)
        assert int(status[j].item()) == wst and np.array_equal(outs[j].cpu().numpy(), want)


def test_pair_columns_in_a_batch(lib):
    """RE_SLPF_PAIRS through a batch (per-position-state groups and the
    checkpoint path alike): each text's pairs equal its single parse's, and
    decode to the oracle's columns."""
    Batch, Regex = lib
    pats = _patterns()
    rxs = [Regex(p) for p, _ in pats]
    items = [(pi, pats[pi][1](n, 300 + pi * 7 + n % 5)) for pi in range(len(pats)) for n in (0, 700, 9000, 200_001)]
    texts = [torch.from_numpy(np.ascontiguousarray(h)).cuda() for _, h in items]
    b = Batch([rxs[pi] for pi, _ in items], [len(h) for _, h in items], kind="pairs")
    outs, status, kinds = b.parse(texts)
    torch.cuda.synchronize()
    st = status.cpu().numpy()
    for j, ((pi, h), t) in enumerate(zip(items, texts)):
        cols, wst, _ = rxs[pi].parse(t, kind="pairs")
        torch.cuda.synchronize()
        assert kinds[j] == "pairs" and st[j] == int(wst.item())
        assert np.array_equal(outs[j].cpu().numpy(), cols.cpu().numpy()), (pi, len(h))
        if len(h) <= 9000:
            want = serial.parse(compile_re(pats[pi][0]), h.tobytes())
            assert np.array_equal(rxs[pi].decode(outs[j].cpu().numpy(), "pairs"), want), (pi, len(h))


def test_high_bytes_in_a_batch(lib):
    """Bytes >= 128 through the batch's byte-table reach, whose rows hold
    bytes below 128 only (each high byte replaced by an ASCII byte of its
    class first): log records with 2 % of their bytes set >= 128, and an RE
    whose class [\\x7f-\\xff] is mostly high bytes, against the oracle."""
    Batch, Regex = lib
    rng = np.random.default_rng(17)

    def log_high(n, s):
        h = W.log_text(n, seed=s).copy()
        hit = (rng.random(h.size) < 0.02) & (h != ord("\n"))
        h[hit] = rng.integers(128, 256, size=int(hit.sum()))
        return h

    def fold_tokens(n, s):
        r = np.random.default_rng(s)
        toks = [bytes([v, 97]) for v in range(127, 256)] + [b"b"] * 40
        return np.frombuffer(b"".join(toks[j] for j in r.integers(0, len(toks), size=n // 2)), dtype=np.uint8).copy()

    pats = [(W.LOG_RE, log_high), (r"([\x7f-\xff]a|b)*", fold_tokens)]
    rxs = [Regex(p) for p, _ in pats]
    assert all(rx.info["ascii_rows"] == 1 for rx in rxs)
    items = [(pi, pats[pi][1](n, 500 + 3 * pi + n % 7)) for pi in range(2) for n in (0, 900, 9000, 70_001, 300_000)]
    texts = [torch.from_numpy(np.ascontiguousarray(h)).cuda() for _, h in items]
    b = Batch([rxs[pi] for pi, _ in items], [len(h) for _, h in items])
    outs, status, kinds = b.parse(texts)
    torch.cuda.synchronize()
    st = status.cpu().numpy()
    for j, (pi, h) in enumerate(items):
        want = serial.parse(compile_re(pats[pi][0]), h.tobytes())
        assert st[j] == (0 if serial.accepted(want) else 1), (pi, len(h))
        assert np.array_equal(rxs[pi].decode(outs[j].cpu().numpy(), kinds[j]), want), (pi, len(h))
