"""A text longer than 4 GiB: byte offsets, chunk and column indices past 2^32.

The text is a 1 MiB block of (a|b|ab)* input (i.i.d. a/b, seed 0) repeated
4096 times plus a 17-byte ragged tail.  For this RE the DFA state after a
prefix is fixed by the prefix's last byte, and the reverse DFA state before a
suffix by its first byte, so column r depends only on the bytes around r.
Hence every column in the big text's interior equals the column at the same
offset in the middle period of a three-period text, and the columns near
either end equal those of a short text with the same start or end; the
oracle gives those short texts' columns.  Sampled columns -- all around
2^31 and 2^32 and the end, plus random ones -- are compared.
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
    from paper_2503_06763_gb300 import Regex
    return Regex


def test_text_over_4gib(lib):
    Regex = lib
    P = 1 << 20
    block = W.ab_text(P, seed=0)
    tail = block[:17]
    n = 4096 * P + len(tail)
    assert n > (1 << 32)
    rx = Regex(W.AB_RE)
    big = torch.empty(n, dtype=torch.uint8, device="cuda")
    blk = torch.from_numpy(block).cuda()
    big[:4096 * P].view(4096, P).copy_(blk.expand(4096, P))
    big[4096 * P:] = torch.from_numpy(tail).cuda()
    cols, st, kind = rx.parse(big)
    torch.cuda.synchronize()
    assert int(st.item()) == 0 and kind == "dense"
    assert cols.numel() == n + 1

    c = compile_re(W.AB_RE)
    mid = serial.parse(c, np.tile(block, 3))                       # middle period: offsets P .. 2P
    end = serial.parse(c, np.concatenate([np.tile(block, 2), tail]))
    n_end = 2 * P + len(tail)

    rng = np.random.Generator(np.random.PCG64(9))
    picks = [np.arange(0, 64), np.arange(P - 64, P + 64),
             np.arange((1 << 31) - 64, (1 << 31) + 64), np.arange((1 << 32) - 128, n + 1),
             np.arange(n - P - 64, n + 1), rng.integers(0, n + 1, size=20_000)]
    r = np.unique(np.concatenate(picks)).astype(np.int64)
    assert r.min() >= 0 and r.max() <= n                          # columns 0 .. n only
    # plain copy to the host, then index there: no device gather over a tensor of more than 2^32 elements
    host_cols = cols.cpu().numpy().view(np.uint16)
    del cols, big
    got = host_cols[r].astype(np.uint64)
    want = np.empty(len(r), dtype=np.uint64)
    for j, rr in enumerate(r.tolist()):
        if rr < P:
            want[j] = mid[rr, 0]                                   # same start as the 3-period text
        elif rr > n - P:
            want[j] = end[n_end - (n - rr), 0]                      # same end as the 2-period + tail text
        else:
            want[j] = mid[P + (rr % P), 0]
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, f"{bad.size} columns differ, first at r={r[bad[:5]].tolist()}"
