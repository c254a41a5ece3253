"""Serving loop: continuous batching gives every request the bytes it gets alone.

Requests of mixed lengths under several resident REs arrive as a Poisson
stream fast enough that batches mix texts and REs and several slots are on
the GPU at once; slot arenas are small so admission by device memory splits
the stream into many batches.  Each request's columns and status must equal
``Regex.parse`` of its text alone.
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
    from paper_2503_06763_gb300 import Regex, serve
    return Regex, serve


def _requests(serve, n, rate, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    trees = [W.random_re(500 + i, 20, 60)[1] for i in range(3)]
    pools = [W.PiecePool(t, 600 + i) for i, t in enumerate(trees)]
    pats = [W.random_re(500 + i, 20, 60)[0] for i in range(3)] + [W.DNA_RE, W.AB_RE]
    reqs, t = [], 0.0
    for j in range(n):
        t += rng.exponential(1.0 / rate)
        ri = int(rng.integers(0, len(pats)))
        ln = int(min(np.exp(rng.normal(np.log(4096), 1.5)), 1 << 20))
        if j % 37 == 0:
            ln = 0
        if ri < 3:
            txt = pools[ri].text(ln, seed=j)
        elif ri == 3:
            txt = W.dna_text(ln, seed=j)
        else:
            txt = W.ab_text(ln, seed=j)
        if j % 23 == 5 and len(txt) > 2:
            txt = txt.copy()
            txt[len(txt) // 2] = 0xFF                  # rejected text
        reqs.append(serve.Request(rid=j, re_index=ri, text=np.ascontiguousarray(txt), arrival=t))
    return pats, reqs


def _check_alone(Regex, pats, reqs):
    rxs = {}
    for r in reqs:
        rx = rxs.setdefault(r.re_index, Regex(pats[r.re_index]))
        t = torch.from_numpy(r.text).cuda()
        cols, st, _ = rx.parse(t)
        torch.cuda.synchronize()
        assert r.status == int(st.item()), r.rid
        want = cols.cpu().numpy()
        assert np.array_equal(r.cols.view(want.dtype), want), r.rid


def test_stream_mixes_and_matches_alone(lib):
    Regex, serve = lib
    pats, reqs = _requests(serve, 400, rate=20_000.0, seed=1)
    srv = serve.Server(pats, slots=3, arena_bytes=24 << 20)
    srv.run(reqs, realtime=True, keep_cols=True)
    stats = dict(srv.stats)
    srv.close()
    assert all(r.status in (0, 1) for r in reqs)
    assert any(r.status == 1 for r in reqs) and any(r.status == 0 for r in reqs)
    assert stats["max_batch"] > 1 and stats["batches"] > 3
    assert stats["max_inflight"] >= 2
    assert all(r.done >= r.arrival for r in reqs)
    _check_alone(Regex, pats, reqs)


def test_offline_burst_is_admitted_by_memory(lib):
    Regex, serve = lib
    pats, reqs = _requests(serve, 400, rate=1e9, seed=2)
    srv = serve.Server(pats, slots=2, arena_bytes=16 << 20)
    srv.run(reqs, realtime=False, keep_cols=True)
    stats = dict(srv.stats)
    srv.close()
    assert stats["batches"] > 2                      # the arena limit split the burst
    _check_alone(Regex, pats, reqs)


def test_oversized_request_is_refused(lib):
    Regex, serve = lib
    srv = serve.Server([W.DNA_RE], slots=1, arena_bytes=8 << 20)
    big = serve.Request(rid=0, re_index=0, text=W.dna_text(6 << 20, seed=3))
    with pytest.raises(ValueError):
        srv.run([big])
    srv.close()
