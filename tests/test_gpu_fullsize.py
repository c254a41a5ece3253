"""Parity at the workloads' full sizes, in the launch configuration the
benchmark uses (automatic chunk length, AUTO encoding).

* ab, 1 MiB (seed 0): every column against the serial oracle.
* DNA, 256 MiB (seed 1, the benchmark workload): every column against the
  serial oracle (one serial pass over the whole text on the host).
* log, 1 GiB (seed 2, the benchmark workload): every column against the
  oracle's interned serial pass (``serial.parse_ids``: one id per position,
  each distinct column stored once), compared as decoded columns.
* batch, 4096 texts under 8 random REs (seed 3): every status, every column
  of 48 sampled texts up to 256 KiB and of 6 texts of 1-4 MiB against the
  oracle.
"""
import hashlib
import json
import os

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
    from paper_2503_06763_gb300 import Batch, Regex, ReError
    return Batch, Regex, ReError


def golden_sha(name):
    """The oracle's SHA-256 of a benchmark text's canonical SLPF bytes
    (tests/golden/make_slpf_sha256.py)."""
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "slpf_sha256.json")) as f:
        return json.load(f)[name]


def assert_sha(cols, kind, name):
    g = golden_sha(name)
    assert kind == g["encoding"] and cols.dtype.itemsize == g["col_bytes"]
    assert hashlib.sha256(np.ascontiguousarray(cols).tobytes()).hexdigest() == g["sha256"], name


def gpu_parse(rx, host):
    t = torch.from_numpy(host).cuda()
    cols, st, kind = rx.parse(t)
    torch.cuda.synchronize()
    out = cols.cpu().numpy()
    del cols, t
    return out, int(st.item()), kind


def assert_columns_equal(rx, cols, kind, want):
    """Compare in chunks (decoded GPU columns vs the oracle's bitsets)."""
    step = 1 << 24
    for a in range(0, len(cols), step):
        got = rx.decode(cols[a:a + step], kind)
        bad = np.nonzero(np.any(got != want[a:a + step], axis=1))[0]
        assert bad.size == 0, f"{bad.size} columns differ from r={a + bad[0]}"


def test_ab_1mib(lib):
    _, Regex, _ = lib
    host = W.ab_text(1 << 20, seed=0)
    rx = Regex(W.AB_RE)
    cols, st, kind = gpu_parse(rx, host)
    want = serial.parse(compile_re(W.AB_RE), host)
    assert st == 0 and kind == "dense"
    assert_columns_equal(rx, cols, kind, want)
    assert_sha(cols, kind, "ab_1MiB_seed0")


def test_dna_256mib_every_column(lib):
    _, Regex, _ = lib
    host = W.dna_text(256 << 20, seed=1)
    rx = Regex(W.DNA_RE)
    cols, st, kind = gpu_parse(rx, host)
    want = serial.parse(compile_re(W.DNA_RE), host)
    assert st == (0 if serial.accepted(want) else 1) == 0
    assert_columns_equal(rx, cols, kind, want)
    assert_sha(cols, kind, "dna_256MiB_seed1")


def assert_interned_equal(rx, cols, kind, ids, table):
    """GPU DICT columns against the oracle's interned columns: every oracle
    column is looked up in the decoding table of the GPU encoding (the
    dictionary; index 0 is the empty column), then the GPU ids must equal the
    translated oracle ids at every position."""
    gdict = rx.dictionary()
    lookup = {tuple(row): d + 1 for d, row in enumerate(gdict.tolist())}
    lookup[tuple([0] * gdict.shape[1])] = 0
    want_id = np.array([lookup.get(tuple(row), -1) for row in table.tolist()], dtype=np.int64)
    missing = np.nonzero(want_id < 0)[0]
    if missing.size:                                      # an oracle column the GPU encoding cannot express
        used = np.isin(ids, missing)
        assert not used.any(), f"oracle column absent from the GPU encoding at r={np.nonzero(used)[0][:5].tolist()}"
    got = cols.view({1: np.uint8, 2: np.uint16, 4: np.uint32}[cols.dtype.itemsize])
    step = 1 << 26
    for a in range(0, len(got), step):
        exp = want_id[ids[a:a + step]]
        bad = np.nonzero(got[a:a + step] != exp)[0]
        assert bad.size == 0, f"{bad.size} columns differ from r={a + bad[0]}"


def test_log_1gib_every_column(lib):
    _, Regex, _ = lib
    c = compile_re(W.LOG_RE)
    rx = Regex(W.LOG_RE)
    host = W.log_text(1 << 30, seed=2)
    cols, st, kind = gpu_parse(rx, host)
    assert kind == "dict"
    ids, table = serial.parse_ids(c, host)
    accepted = bool(table[ids[0]].any())
    assert st == (0 if accepted else 1) == 0
    assert_interned_equal(rx, cols, kind, ids, table)
    assert_sha(cols, kind, "log_1GiB_seed2")


def test_batch_4096_texts_sampled(lib):
    Batch, Regex, ReError = lib
    res, seed = [], 3000
    while len(res) < 8:                                   # the benchmark's REs: next seed when the caps refuse one
        pat, tree, _ = W.random_re(seed, 10, 200)
        seed += 1
        try:
            res.append((pat, tree, Regex(pat)))
        except ReError:
            continue
    lens, which = W.batch_lengths(4096, seed=3)
    pools = [W.PiecePool(tree, 100 + i) for i, (_, tree, _) in enumerate(res)]
    hosts = [pools[w].text(int(n), seed=10_000 + j) for j, (n, w) in enumerate(zip(lens, which))]
    texts = [torch.from_numpy(h).cuda() for h in hosts]
    b = Batch([res[w][2] for w in which], [len(h) for h in hosts])
    outs, status, kinds = b.parse(texts)
    torch.cuda.synchronize()
    assert (status.cpu().numpy() == 0).all()             # every text is valid
    rng = np.random.Generator(np.random.PCG64(7))
    small = [j for j, h in enumerate(hosts) if len(h) <= (256 << 10)]
    compiled = {}
    for j in rng.choice(small, size=48, replace=False):
        w = int(which[j])
        c = compiled.setdefault(w, compile_re(res[w][0]))
        want = serial.parse(c, hosts[j])
        got = res[w][2].decode(outs[j].cpu().numpy(), kinds[j])
        assert np.array_equal(got, want), (j, len(hosts[j]))
    large = [j for j, h in enumerate(hosts) if (1 << 20) <= len(h) <= (4 << 20)]
    for j in rng.choice(large, size=6, replace=False):     # texts of 1-4 MiB, every column
        w = int(which[j])
        c = compiled.setdefault(w, compile_re(res[w][0]))
        ids, table = serial.parse_ids(c, hosts[j])
        got = res[w][2].decode(outs[j].cpu().numpy(), kinds[j])
        assert np.array_equal(got, table[ids]), (j, len(hosts[j]))
