"""The sharded parse's exchange step on CPU (gloo, world size 2).

Each rank takes one slice of the text and computes its slice maps with the
oracle (Sect. 3.2: the ME-DFA / reverse ME-DFA run of Eq. reacher over the
slice, from every state of the library's automaton, read back as state ids
by their segment sets), the maps are all-gathered over gloo
(``shard.gather_maps``), and the library's host composition
(``re_shard_entry``, on a host-only handle) turns them into each slice's
entry states.  The checker is the oracle's parallel equations run with the
slices as chunks: the entry states must be its J at every slice start and its
Ĵ at every slice end, and the verdict the serial parser's.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _cases():
    import workloads as W
    log = W.log_text(900, seed=8).tobytes()
    dna = W.dna_text(700, seed=8, mean_gap=150).tobytes()
    bad = bytearray(dna)
    bad[123] = ord("N")                                    # rejected in the first slice
    return [(W.LOG_RE, log), (W.DNA_RE, dna), (W.DNA_RE, bytes(bad)), ("(aa)*", b"a" * 500),
            ("(aa)*", b"a" * 501), (W.AB_RE, W.ab_text(333, seed=9).tobytes())]


def _slice_maps(rx, c, piece: bytes):
    """This slice's maps computed with the oracle: forward / backward image of
    every classic-DFA state's segment set over the slice."""
    from oracle import parallel_equations as pe
    nf, nb = rx.shard_map_size()
    info = rx.info
    fwd_ids = {tuple(rx.state_bits(True, s).tolist()): s for s in range(info["fwd_states"] + 1)}
    bwd_ids = {tuple(rx.state_bits(False, s).tolist()): s for s in range(info["bwd_states"] + 1)}

    def as_set(v):
        return frozenset(q for q in range(c.ell) if (int(v[q >> 6]) >> (q & 63)) & 1)

    def as_id(ids, S):
        v = np.zeros(rx.words, dtype=np.uint64)
        for q in S:
            v[q >> 6] |= np.uint64(1) << np.uint64(q & 63)
        return ids[tuple(v.tolist())]

    out = np.zeros(nf + nb, dtype=np.uint8)
    for s in range(nf):
        out[s] = as_id(fwd_ids, pe.run(c, as_set(rx.state_bits(True, s)), piece))
    for s in range(nb):
        out[nf + s] = as_id(bwd_ids, pe.run(c, as_set(rx.state_bits(False, s)), piece, reverse=True))
    return out


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle.re_front import compile_re
    from paper_2503_06763_gb300 import shard
    from paper_2503_06763_gb300.native import Regex
    res = []
    for pattern, text in _cases():
        rx = Regex(pattern, host_only=True)
        c = compile_re(pattern)
        k = (len(text) + world - 1) // world                  # slice r = chunk r + 1 of length k
        piece = text[rank * k:(rank + 1) * k]
        maps = shard.gather_maps(_slice_maps(rx, c, piece))
        entry, entry_bwd, accepted = rx.shard_entry(maps)
        res.append((maps.shape[0], entry.tolist(), entry_bwd.tolist(), accepted))
    q.put((rank, res))
    dist.destroy_process_group()


def test_two_ranks_compose_slice_maps_into_the_joins_states():
    sys.path.insert(0, ROOT)
    try:
        from paper_2503_06763_gb300 import native
        native.load()
    except ImportError:
        import __graft_entry__
        __graft_entry__.build()
        from paper_2503_06763_gb300 import native
    from oracle import parallel_equations as pe
    from oracle import serial
    from oracle.re_front import compile_re
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get() for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert got[0] == got[1]                                    # every rank composes the same entries
    for (pattern, text), (ranks, entry, entry_bwd, accepted) in zip(_cases(), got[0]):
        assert ranks == world
        c = compile_re(pattern)
        rx = native.Regex(pattern, host_only=True)
        k = (len(text) + world - 1) // world
        _, tr = pe.parse_parallel(c, text, k)                  # the slices as chunks: J_i, Ĵ_i
        acc = serial.accepted(serial.parse(c, text))
        assert accepted == acc, pattern
        for r in range(world):
            fwd = frozenset(q for q in range(c.ell) if (int(rx.state_bits(True, entry[r])[q >> 6]) >> (q & 63)) & 1)
            bwd = frozenset(q for q in range(c.ell)
                            if (int(rx.state_bits(False, entry_bwd[r])[q >> 6]) >> (q & 63)) & 1)
            if acc:
                assert fwd == tr["J"][r], (pattern, r)         # J at the slice's start
            else:
                assert entry[r] == 0                          # a rejected text: every column empty
            assert bwd == tr["Jh"][r + 2], (pattern, r)        # Ĵ at the slice's end
