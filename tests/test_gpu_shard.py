"""The sharded parse on one GPU, slice after slice (Sect. 3.2: chunks meet
only in the join): every slice's maps on the device (re_shard_map), their
composition on the host (re_shard_entry), every slice parsed from its entry
states (re_parse_slice), the columns stitched.  The result must be the
oracle's SLPF of the whole text, column by column, for accepted and rejected
texts, 2-5 slices, slices shorter than a chunk, and (aa)* whose chunks never
converge.  A slice's device maps are also compared with the oracle's."""
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
    from paper_2503_06763_gb300 import Regex, shard
    return Regex, shard


def _want(pattern, host):
    ids, table = serial.parse_ids(compile_re(pattern), host)
    return table[ids]


CASES = [("log", W.LOG_RE, lambda: W.log_text(2 << 20, seed=51), 3),
         ("dna", W.DNA_RE, lambda: W.dna_text((1 << 20) + 33, seed=52), 4),
         ("ab", W.AB_RE, lambda: W.ab_text(300_001, seed=53), 5),
         ("aa-even", "(aa)*", lambda: np.full((1 << 20) + 2, ord("a"), dtype=np.uint8), 2),
         ("aa-odd", "(aa)*", lambda: np.full((1 << 20) + 1, ord("a"), dtype=np.uint8), 3),
         ("small", W.DNA_RE, lambda: W.dna_text(1000, seed=54, mean_gap=200), 4)]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_slices_stitch_into_the_whole_slpf(lib, case):
    Regex, shard = lib
    name, pattern, make, parts = CASES[case]
    rx = Regex(pattern)
    host = make()
    t = torch.from_numpy(host).cuda()
    cols, stats, accepted = shard.parse_in_slices(rx, t, parts)
    torch.cuda.synchronize()
    want = _want(pattern, host)
    acc = serial.accepted(want)
    assert accepted == acc, name
    assert (stats.cpu().numpy() == (0 if acc else 1)).all(), (name, stats.cpu().numpy().tolist())
    kind = rx.layout(1)[0]
    got = rx.decode(cols.cpu().numpy(), kind)
    assert got.shape == want.shape
    bad = np.nonzero(np.any(got != want, axis=1))[0]
    assert bad.size == 0, (name, bad[:5].tolist())


def test_rejected_text_gives_empty_slices(lib):
    Regex, shard = lib
    host = W.dna_text(400_000, seed=55)
    host[250_000] = ord("N")                              # in the second of three slices
    rx = Regex(W.DNA_RE)
    cols, stats, accepted = shard.parse_in_slices(rx, torch.from_numpy(host).cuda(), 3)
    torch.cuda.synchronize()
    assert not accepted
    assert (stats.cpu().numpy() == 1).all() and not cols.cpu().numpy().any()


def test_device_maps_equal_the_oracle(lib):
    """A middle slice's maps from the device equal the oracle's run of
    Eq. reacher over the slice, from every state that can stand at the
    slice's edge: forward, every classic-DFA state after the byte before the
    slice; backward, every reverse one after the byte after it (the slots a
    chunk speculates from are keyed by those bytes, so the maps are exact on
    the states a text can bring there)."""
    Regex, _ = lib
    from oracle import parallel_equations as pe
    pattern = W.LOG_RE
    host = W.log_text(300_000, seed=56)
    rx = Regex(pattern)
    c = compile_re(pattern)
    a, b = 64 * 1000, 64 * 1500
    t = torch.from_numpy(host).cuda()
    dev = rx.shard_map(t[a:b], True, True)
    nf, nb = rx.shard_map_size()
    piece = host[a:b].tobytes()

    def as_set(v):
        return frozenset(q for q in range(c.ell) if (int(v[q >> 6]) >> (q & 63)) & 1)

    fwd = {as_set(rx.state_bits(True, s)): s for s in range(rx.info["fwd_states"] + 1)}
    bwd = {as_set(rx.state_bits(False, s)): s for s in range(rx.info["bwd_states"] + 1)}
    edge_f = {pe.run(c, as_set(rx.state_bits(True, s)), host[a - 1:a].tobytes()) for s in range(nf)}
    edge_b = {pe.run(c, as_set(rx.state_bits(False, s)), host[b:b + 1].tobytes(), reverse=True) for s in range(nb)}
    assert len(edge_f) > 2 and len(edge_b) > 2
    for S in edge_f:
        assert as_set(rx.state_bits(True, int(dev[fwd[S]]))) == pe.run(c, S, piece), sorted(S)
    for S in edge_b:
        assert as_set(rx.state_bits(False, int(dev[nf + bwd[S]]))) == pe.run(c, S, piece, reverse=True), sorted(S)
