"""The CUDA path against the stored known-answer vectors (tests/golden/):
engine words through the bits fill at their seeds and word offsets (Philox
counter carries across 2^64 and the 2^128 wrap, MRG32k3a jumps of 2^76 and
2^127), and every distribution variant through grng_transform_words."""

import numpy as np
import pytest

from golden_fixtures import engine_word_cases, transform_cases

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2109_01329_gb300 as grng

    return grng


def test_engine_words(g):
    for eng, seed, off, w in engine_word_cases():
        out = torch.empty(w.size, dtype=torch.int32, device="cuda")
        g.generate(g.Distribution.bits(), g.Engine(eng, seed, off), out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, w), (eng, seed, off)


def test_transforms(g):
    words, cases = transform_cases()
    w = torch.from_numpy(words.view(np.int32)).cuda()
    for name, kind, dtype, p0, p1, n, exp in cases:
        tdt = {0: torch.int32, 1: torch.float32, 2: torch.float64}[dtype]
        out = torch.empty(n, dtype=tdt, device="cuda")
        g.transform_words(g.Distribution(kind, dtype, p0, p1), w, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        if kind in (0, 1):
            assert np.array_equal(got.view(np.uint64 if dtype == 2 else np.uint32), exp), name
        else:
            tol = 2e-6 if dtype == 1 else 1e-14
            err = np.abs(got.astype(np.float64) - exp) / np.maximum(1.0, np.abs(exp))
            assert float(err.max()) <= tol, f"{name}: {err.max():.3e}"
