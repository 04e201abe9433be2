"""Readers for the known-answer fixtures in tests/golden/ (written from the
oracle by tests/golden/make_golden.py)."""

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.rstrip("\n") for ln in f if ln.strip() and not ln.startswith("#")]


def engine_word_cases():
    """[(engine, seed, offset, words as uint32 array)]"""
    out = []
    for ln in _lines("engine_words.txt"):
        head, vals = ln.split(":")
        name, seed, off, n = head.split()
        w = np.array([int(v, 16) for v in vals.split()], dtype=np.uint32)
        assert w.size == int(n)
        out.append((0 if name == "philox" else 1, int(seed), int(off), w))
    return out


def transform_cases():
    """(words, [(name, kind, dtype, p0, p1, n, expected)]) with expected as
    uint32 / uint64 bit patterns for bits and uniforms, float64 values else."""
    words, cases = None, []
    for ln in _lines("transforms.txt"):
        head, vals = ln.split(":")
        parts = head.split()
        if parts[0] == "words":
            words = np.array([int(v, 16) for v in vals.split()], dtype=np.uint32)
            continue
        name, kind, dtype, p0, p1, n = parts
        kind, dtype, n = int(kind), int(dtype), int(n)
        if kind in (0, 1):
            exp = np.array([int(v, 16) for v in vals.split()],
                           dtype=np.uint64 if dtype == 2 else np.uint32)
        else:
            exp = np.array([float(v) for v in vals.split()], dtype=np.float64)
        assert exp.size == n
        cases.append((name, kind, dtype, float(p0), float(p1), n, exp))
    return words, cases
