"""The seeded input generators are reproducible: pinned SHA-256 of their texts."""
import hashlib

import workloads as W


def sha(x):
    return hashlib.sha256(x.tobytes()).hexdigest()


def test_generator_texts_are_pinned():
    assert sha(W.ab_text(1 << 20, seed=0)) == "cae2cf93735161201bab417ffe99c23abcc5df44308414f7ece1629b9d4b4e5e"
    assert sha(W.dna_text(1 << 20, seed=1)) == "21a9bf10be0ea87434beea34cabe59cc019b0665578734846d769ff1ab616080"
    assert sha(W.log_text(1 << 20, seed=2)) == "a04a7f12cb125f233de32e9a60b325650ec84dd3e22dff4539516540a39d464a"
