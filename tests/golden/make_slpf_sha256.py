"""Write tests/golden/slpf_sha256.json: SHA-256 of the canonical SLPF bytes
of the benchmark texts, computed by the oracle alone.

The canonical encodings are those the library's header defines: DENSE (bit
j of a column is segment j, little-endian in 1, 2, 4 or 8 bytes) and DICT
(the column's 1-based rank in the dictionary of every non-empty B ∩ B̂ over
pairs of DFA states reachable from I and reverse DFA states reachable from
F, ranked in lexicographic order of their ascending segment ids; 0 for the
empty column; 1 byte below 255 entries, 2 below 65535, else 4).  The
columns come from the oracle's interned serial parser (Fig. serialparser);
the dictionary from the oracle's powerset construction (Sect. 3.1).

Run from the repository root: python tests/golden/make_slpf_sha256.py
(a few minutes on one core: the 1 GiB log text dominates).
"""
import hashlib
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W                                      # noqa: E402
from oracle import parallel_equations as pe                # noqa: E402
from oracle import serial                                  # noqa: E402
from oracle.re_front import compile_re                     # noqa: E402


def canonical_bytes(pattern, host):
    c = compile_re(pattern)
    ids, table = serial.parse_ids(c, host)               # distinct columns as W-word bitsets
    cols = [serial.from_bits(row) for row in table]
    if c.ell <= 16:                                      # DENSE (the AUTO choice up to 16 segments)
        cb = 1 if c.ell <= 8 else 2
        vals = np.array([sum(1 << q for q in col) for col in cols], dtype=np.uint64)
        enc = vals.astype({1: np.uint8, 2: np.uint16}[cb])
        return "dense", cb, enc[ids].tobytes()
    fw, bw = pe.dfa_states(c), pe.dfa_states(c, reverse=True)
    dictionary = sorted({tuple(sorted(a & b)) for a in fw for b in bw if a & b})
    rank = {d: j + 1 for j, d in enumerate(dictionary)}
    cb = 1 if len(dictionary) < 255 else 2 if len(dictionary) < 65535 else 4
    idx = np.array([rank[tuple(sorted(col))] if col else 0 for col in cols], dtype=np.uint32)
    enc = idx.astype({1: np.uint8, 2: np.uint16, 4: np.uint32}[cb])
    return "dict", cb, enc[ids].tobytes()


def main():
    out = {"_about": "SHA-256 of the canonical SLPF column bytes of the benchmark texts, written by "
                     "tests/golden/make_slpf_sha256.py from the oracle alone (interned serial parser, "
                     "powerset dictionary)."}
    for name, pattern, make, n, seed in (("ab_1MiB_seed0", W.AB_RE, W.ab_text, 1 << 20, 0),
                                         ("dna_256MiB_seed1", W.DNA_RE, W.dna_text, 256 << 20, 1),
                                         ("log_1GiB_seed2", W.LOG_RE, W.log_text, 1 << 30, 2)):
        host = make(n, seed=seed)
        kind, cb, data = canonical_bytes(pattern, host)
        out[name] = {"text_bytes": int(host.size), "encoding": kind, "col_bytes": cb,
                     "sha256": hashlib.sha256(data).hexdigest()}
        print(name, out[name], flush=True)
    with open(os.path.join(ROOT, "tests", "golden", "slpf_sha256.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
