"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no parsing arithmetic: it only draws texts and regular
expressions.  Random texts are drawn from random structure trees it builds
itself (a syntax tree is sampled top-down and its leaves emitted), never by
running an automaton.

Workloads (shapes follow the paper's benchmark families, Sect. 5.1, Tab.
benchmarks; all seeds fixed):
  * ``ab_text``      -- i.i.d. uniform {a, b} for the ambiguous RE (a|b|ab)*.
  * ``dna_text``     -- i.i.d. uniform ACGT with ORF-shaped motifs planted by
                        a Poisson process (stand-in for FASTA).
  * ``log_text``     -- web-server-like log lines, 2 % malformed (stand-in
                        for TRAFFIC), with ``LOG_RE``.
  * ``random_re`` / ``sample_text`` -- REgen-like random REs and valid texts
                        drawn from their structure trees (stand-in for REGEN).
"""
from __future__ import annotations

import numpy as np

AB_RE = "(a|b|ab)*"
DNA_RE = "([ACGT]|ATG([ACGT][ACGT][ACGT])*(TAA|TAG|TGA))*"

STOPS = [b"TAA", b"TAG", b"TGA"]
CODONS = [bytes([a, b, c]) for a in b"ACGT" for b in b"ACGT" for c in b"ACGT"]
NON_STOP = [c for c in CODONS if c not in STOPS]


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def ab_text(n: int, seed: int = 0) -> np.ndarray:
    """n bytes i.i.d. uniform over {a, b}."""
    return rng_for(seed).choice(np.frombuffer(b"ab", dtype=np.uint8), size=n)


def dna_text(n: int, seed: int = 1, mean_gap: int = 10_000, p_geom: float = 0.01,
             max_codons: int = 900) -> np.ndarray:
    """Uniform ACGT with planted ORFs: ATG + (L-2) non-stop codons + one stop,
    L ~ 30 + Geometric(p_geom) resampled above max_codons; ORF starts form a
    Poisson process of mean gap ``mean_gap`` bytes."""
    rng = rng_for(seed)
    x = rng.choice(np.frombuffer(b"ACGT", dtype=np.uint8), size=n)
    non_stop = np.frombuffer(b"".join(NON_STOP), dtype=np.uint8).reshape(-1, 3)
    stops = np.frombuffer(b"".join(STOPS), dtype=np.uint8).reshape(-1, 3)
    pos = 0
    while True:
        pos += int(rng.exponential(mean_gap)) + 1
        L = 30 + int(rng.geometric(p_geom))
        while L > max_codons:
            L = 30 + int(rng.geometric(p_geom))
        if pos + 3 * L > n:
            break
        orf = np.empty(3 * L, dtype=np.uint8)
        orf[:3] = np.frombuffer(b"ATG", dtype=np.uint8)
        orf[3:3 * (L - 1)] = non_stop[rng.integers(0, len(non_stop), size=L - 2)].reshape(-1)
        orf[3 * (L - 1):] = stops[rng.integers(0, 3)]
        x[pos:pos + 3 * L] = orf
        pos += 3 * L
    return x


# ----------------------------------------------------------------------------
# Web-server-like log records (stand-in for the TRAFFIC benchmark)
_OCTET = "[0-9][0-9]?[0-9]?"
_D2 = "[0-9][0-9]"
_MONTHS = ["Jan", "Feb", "Mar", "Apr", "May", "Jun", "Jul", "Aug", "Sep", "Oct", "Nov", "Dec"]
_METHODS = ["GET", "POST", "PUT", "DELETE", "HEAD"]
LOG_GOOD = (
    f"{_OCTET}\\.{_OCTET}\\.{_OCTET}\\.{_OCTET} - - \\["
    f"{_D2}/({'|'.join(_MONTHS)})/[0-9][0-9][0-9][0-9]:{_D2}:{_D2}:{_D2} [+\\-][0-9][0-9][0-9][0-9]\\] "
    f"\"({'|'.join(_METHODS)}) /[a-zA-Z0-9_./\\-]* HTTP/1\\.[01]\" [1-5][0-9][0-9] [0-9]+"
)
LOG_RE = f"(({LOG_GOOD}|[^\\n]*)\\n)*"


def _log_line(rng: np.random.Generator, vocab, zipf_cdf) -> bytes:
    ip = ".".join(str(int(v)) for v in rng.integers(0, 256, size=4))
    day = int(rng.integers(1, 29))
    mon = _MONTHS[int(rng.integers(0, 12))]
    year = int(rng.integers(1995, 2026))
    hh, mm, ss = (int(v) for v in rng.integers(0, 60, size=3))
    hh %= 24
    tz = ("+" if rng.random() < 0.5 else "-") + f"{int(rng.integers(0, 1300)):04d}"
    u = rng.random()
    method = "GET" if u < 0.80 else "POST" if u < 0.95 else _METHODS[2 + int(rng.integers(0, 3))]
    ntok = 1 + int(rng.integers(0, 3))
    toks = [vocab[int(np.searchsorted(zipf_cdf, rng.random()))] for _ in range(ntok)]
    path = "/" + "/".join(toks)
    status = 200 if rng.random() < 0.9 else int(rng.choice([301, 302, 304, 400, 403, 404, 500, 503]))
    size = str(int(rng.integers(1, 10)))
    size += "".join(str(int(d)) for d in rng.integers(0, 10, size=int(rng.integers(0, 7))))
    line = (f"{ip} - - [{day:02d}/{mon}/{year}:{hh:02d}:{mm:02d}:{ss:02d} {tz}] "
            f"\"{method} {path} HTTP/1.{int(rng.integers(0, 2))}\" {status} {size}")
    if rng.random() < 0.02:            # malformed: truncate, replace one char, or drop the closing quote
        kind = int(rng.integers(0, 3))
        if kind == 0:
            line = line[:int(rng.integers(1, len(line)))]
        elif kind == 1:
            j = int(rng.integers(0, len(line)))
            line = line[:j] + chr(int(rng.integers(32, 127))) + line[j + 1:]
        else:
            j = line.rfind('"')
            line = line[:j] + line[j + 1:]
    return line.encode("ascii") + b"\n"


def log_text(n: int, seed: int = 2, pool: int = 20_000) -> np.ndarray:
    """About n bytes of log lines (whole lines, cut to n at a line end).

    A pool of distinct lines is drawn from the field distributions (paths Zipf
    s = 1 over 10^5 tokens, status 200 w.p. 0.9, 2 % malformed lines) and the
    text is a uniform sample of pool lines, so long texts keep the same mix."""
    rng = rng_for(seed)
    letters = np.frombuffer(b"abcdefghijklmnopqrstuvwxyz0123456789_", dtype=np.uint8)
    vocab = ["".join(chr(c) for c in rng.choice(letters, size=int(rng.integers(3, 12)))) for _ in range(100_000)]
    w = 1.0 / np.arange(1, len(vocab) + 1)
    zipf_cdf = np.cumsum(w) / w.sum()
    lines = [_log_line(rng, vocab, zipf_cdf) for _ in range(pool)]
    blob = np.frombuffer(b"".join(lines), dtype=np.uint8)
    lens = np.array([len(s) for s in lines], dtype=np.int64)
    starts = np.concatenate([[0], np.cumsum(lens)[:-1]])
    mean = float(lens.mean())
    count = int(n / mean * 1.05) + 16
    pick = rng.integers(0, pool, size=count)
    plen = lens[pick]
    ends = np.cumsum(plen)
    keep = int(np.searchsorted(ends, n, side="right"))
    pick, plen = pick[:keep], plen[:keep]
    total = int(plen.sum())
    out = np.empty(total, dtype=np.uint8)
    dst = np.concatenate([[0], np.cumsum(plen)[:-1]])
    # gather: for every output byte, its source byte in the pool blob
    rep_src = np.repeat(starts[pick] - dst, plen)
    out[:] = blob[np.arange(total) + rep_src]
    return out


# ----------------------------------------------------------------------------
# Random REs (REgen-like, stand-in for the REGEN collection) and valid texts
class _Tree:
    __slots__ = ("kind", "kids", "chars")

    def __init__(self, kind, kids=(), chars=b""):
        self.kind, self.kids, self.chars = kind, list(kids), chars


def _nullable(t: _Tree) -> bool:
    if t.kind == "sym":
        return False
    if t.kind == "star":
        return True
    if t.kind == "cat":
        return all(_nullable(k) for k in t.kids)
    return any(_nullable(k) for k in t.kids)          # alt


def _gen(rng, budget: int, depth: int, star_h: int, alphabet: bytes) -> _Tree:
    if budget <= 1 or depth > 12:
        return _Tree("sym", chars=bytes([alphabet[int(rng.integers(0, len(alphabet)))]]))
    u = rng.random()
    if u < 0.3:
        kind = "alt"
    elif u < 0.8:
        kind = "cat"
    else:
        kind = "star" if star_h < 3 else "cat"
    if kind == "star":
        body = _gen(rng, budget - 1, depth + 1, star_h + 1, alphabet)
        tries = 0
        while _nullable(body) and tries < 20:
            body = _gen(rng, budget - 1, depth + 1, star_h + 1, alphabet)
            tries += 1
        if _nullable(body):
            return body
        return _Tree("star", [body])
    arity = int(rng.integers(2, 4))
    parts = np.maximum(1, (budget * rng.dirichlet(np.ones(arity))).astype(int))
    return _Tree(kind, [_gen(rng, int(b), depth + 1, star_h, alphabet) for b in parts])


def _positions(t: _Tree) -> int:
    return 1 if t.kind == "sym" else sum(_positions(k) for k in t.kids)


def _to_pattern(t: _Tree) -> str:
    if t.kind == "sym":
        c = t.chars.decode("latin-1")
        return "\\" + c if c in "|*+?()[].\\{}" else c
    if t.kind == "star":
        return "(" + _to_pattern(t.kids[0]) + ")*"
    sep = "|" if t.kind == "alt" else ""
    return "(" + sep.join(_to_pattern(k) for k in t.kids) + ")"


def random_re(seed: int, min_pos: int = 10, max_pos: int = 200, alphabet_size=None):
    """(pattern, tree, alphabet): a random RE with min_pos..max_pos positions,
    union / concat / star w.p. 0.3 / 0.5 / 0.2, star height <= 3, no
    iterated nullable sub-expression, wrapped as (R)* so texts of any length
    exist.  The alphabet has A ~ U{4..64} letters (lowercase, uppercase,
    digits, punctuation) unless given."""
    rng = rng_for(seed)
    pool = b"abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ0123456789!#%&,-/:;<=>@_~"
    while True:
        A = alphabet_size or int(rng.integers(4, 65))
        alphabet = bytes(rng.choice(np.frombuffer(pool, dtype=np.uint8), size=A, replace=False))
        target = int(rng.integers(min_pos, max_pos + 1))
        body = _gen(rng, target, 0, 1, alphabet)
        if _nullable(body) or not (min_pos <= _positions(body) <= max_pos):
            continue
        tree = _Tree("star", [body])
        return _to_pattern(tree), tree, alphabet


def _emit(t: _Tree, rng, out: list, limit: int):
    if len(out) > limit:
        return
    if t.kind == "sym":
        out.append(t.chars)
    elif t.kind == "cat":
        for k in t.kids:
            _emit(k, rng, out, limit)
    elif t.kind == "alt":
        _emit(t.kids[int(rng.integers(0, len(t.kids)))], rng, out, limit)
    else:  # star: geometric number of iterations (mean 1)
        while rng.random() < 0.5 and len(out) <= limit:
            _emit(t.kids[0], rng, out, limit)


def sample_text(tree: _Tree, n: int, seed: int) -> np.ndarray:
    """A text of L(tree) of about n bytes: whole iterations of the top-level
    star, each drawn from a random syntax tree of the body."""
    rng = rng_for(seed)
    body = tree.kids[0]
    pieces, total = [], 0
    while total < n:
        part: list = []
        _emit(body, rng, part, 1 << 20)
        s = b"".join(part)
        if total + len(s) > n and total > 0:
            break
        pieces.append(s)
        total += len(s)
    return np.frombuffer(b"".join(pieces), dtype=np.uint8).copy()


class PiecePool:
    """Valid iterations of the top-level star of a random RE (see random_re),
    drawn once from random syntax trees of its body; long valid texts are
    then random sequences of whole pieces, assembled with numpy."""

    def __init__(self, tree: _Tree, seed: int, count: int = 2048):
        rng = rng_for(seed)
        body = tree.kids[0]
        pieces = []
        for _ in range(count):
            part: list = []
            _emit(body, rng, part, 1 << 16)
            pieces.append(b"".join(part))
        self.lens = np.array([len(p) for p in pieces], dtype=np.int64)
        self.starts = np.concatenate([[0], np.cumsum(self.lens)[:-1]]).astype(np.int64)
        self.data = np.frombuffer(b"".join(pieces), dtype=np.uint8)

    def text(self, n: int, seed: int) -> np.ndarray:
        """A valid text of at most n bytes: whole pieces while they fit."""
        rng = rng_for(seed)
        mean = max(1.0, float(self.lens.mean()))
        idx = rng.integers(0, len(self.lens), size=int(n / mean * 1.2) + 16)
        ln = self.lens[idx]
        cum = np.cumsum(ln)
        while cum[-1] < n:                       # rare: draw more pieces
            more = rng.integers(0, len(self.lens), size=len(idx))
            idx = np.concatenate([idx, more])
            ln = self.lens[idx]
            cum = np.cumsum(ln)
        q = int(np.searchsorted(cum, n, side="right"))   # pieces 0..q-1 fit in n bytes
        idx, ln = idx[:q], ln[:q]
        total = int(ln.sum())
        if total == 0:
            return np.zeros(0, dtype=np.uint8)
        before = np.concatenate([[0], np.cumsum(ln)[:-1]])
        src = np.repeat(self.starts[idx] - before, ln) + np.arange(total, dtype=np.int64)
        return self.data[src]


def batch_lengths(n_texts: int, seed: int, lo: int = 1 << 10, hi: int = 4 << 20):
    """Text lengths log-uniform in [lo, hi] and an RE index in 0..7 per text."""
    rng = rng_for(seed)
    lens = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_texts)).astype(np.int64)
    which = rng.integers(0, 8, size=n_texts)
    return lens, which
