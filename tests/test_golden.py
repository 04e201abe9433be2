"""The oracle against its stored known-answer vectors (tests/golden/).

The vectors were written by tests/golden/make_golden.py from the oracle; they
hold it to its definitions between changes (a change of the oracle's
arithmetic regenerates them, and its commit names the passage behind it)."""

import numpy as np

import oracle
from golden_fixtures import engine_word_cases, transform_cases


def test_engine_words_match_the_fixture():
    for eng, seed, off, w in engine_word_cases():
        got = oracle.words(eng, seed, off, w.size)
        assert np.array_equal(got.astype(np.uint32), w), (eng, seed, off)


def test_transforms_match_the_fixture():
    words, cases = transform_cases()
    for name, kind, dtype, p0, p1, n, exp in cases:
        got = oracle.transform_words(kind, dtype, p0, p1, n, words)
        if kind in (0, 1):
            got = got.view(np.uint64 if dtype == 2 else np.uint32)
        assert np.array_equal(got, exp), name
