"""Writes the known-answer fixtures in this directory from the oracle alone.

    python tests/golden/make_golden.py

engine_words.txt: 32-bit engine words at chosen seeds and word offsets
(including block-counter carries across 2^64 and the 2^128 wrap for Philox,
and substream-sized jumps for MRG32k3a).  transforms.txt: every distribution
variant applied to fixed words.  Both are regression fixtures for the oracle
(a change to its definitions must come with regenerated files) and
known-answer vectors for the CUDA path.  Only oracle/ is called.
"""

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

WORD_CASES = [
    # (engine, seed, offset, n)
    (oracle.ENGINE_PHILOX, 2021, 0, 32),
    (oracle.ENGINE_PHILOX, 0x12345678, 0, 8),
    (oracle.ENGINE_PHILOX, 2021, (1 << 66) - 6, 12),
    (oracle.ENGINE_PHILOX, 2021, (1 << 128) - 6, 12),
    (oracle.ENGINE_PHILOX, (1 << 64) - 1, 3, 9),
    (oracle.ENGINE_MRG, 2021, 0, 32),
    (oracle.ENGINE_MRG, 2021, 1 << 76, 8),
    (oracle.ENGINE_MRG, 1, (1 << 127) + 5, 8),
    (oracle.ENGINE_MRG, 4294967086, 1000, 8),
]

TRANSFORM_CASES = [
    # (name, kind, dtype, p0, p1)
    ("bits_u32", 0, 0, 0.0, 0.0),
    ("uniform_f32", 1, 1, 0.0, 1.0),
    ("uniform_f32_m2.5_7", 1, 1, -2.5, 7.0),
    ("uniform_f64", 1, 2, 0.0, 1.0),
    ("uniform_f64_m1_1", 1, 2, -1.0, 1.0),
    ("uniform_f64_2_5", 1, 2, 2.0, 5.0),
    ("gaussian_f32", 2, 1, 0.0, 1.0),
    ("gaussian_f32_0.5_2", 2, 1, 0.5, 2.0),
    ("gaussian_f64", 2, 2, 0.0, 1.0),
    ("gaussian_f64_m1_0.5", 2, 2, -1.0, 0.5),
    ("lognormal_f32", 3, 1, 0.0, 1.0),
    ("lognormal_f64_0.25_0.75", 3, 2, 0.25, 0.75),
    ("icdf_gaussian_f32", 4, 1, 0.0, 1.0),
    ("icdf_gaussian_f64", 4, 2, 0.0, 1.0),
    ("icdf_lognormal_f32", 5, 1, 0.0, 1.0),
    ("icdf_lognormal_f64", 5, 2, 0.25, 0.5),
]
N_OUT = 10  # outputs per transform case (odd Box-Muller tails included)


def fmt_values(kind, vals):
    if kind in (0, 1):
        bits = vals.view(np.uint32 if vals.dtype.itemsize == 4 else np.uint64)
        return " ".join(f"{int(b):x}" for b in bits)
    return " ".join(repr(float(v)) for v in vals)


def main():
    with open(os.path.join(HERE, "engine_words.txt"), "w") as f:
        f.write("# 32-bit engine words (hex), from the oracle (oracle/grng_oracle.cpp):\n"
                "#   Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): key = (seed mod 2^32,\n"
                "#   seed >> 32), word g = lane g mod 4 of the block with counter floor(g/4);\n"
                "#   MRG32k3a (L'Ecuyer 1999): x1 = (1, 1, seed mod m1), x2 = (1, 1, 1),\n"
                "#   word n = (x1_n - x2_n) mod m1, word 0 after the first step.\n"
                "# Written by make_golden.py.  Line: engine seed offset n: words\n")
        for eng, seed, off, n in WORD_CASES:
            w = oracle.words(eng, seed, off, n)
            name = "philox" if eng == oracle.ENGINE_PHILOX else "mrg32k3a"
            f.write(f"{name} {seed} {off} {n}: " + " ".join(f"{int(x):08x}" for x in w) + "\n")
    words = oracle.words(oracle.ENGINE_PHILOX, 2021, 0, 64)
    with open(os.path.join(HERE, "transforms.txt"), "w") as f:
        f.write("# Every distribution variant on the first Philox4x32-10 words of seed 2021,\n"
                "# offset 0 (the first line of engine_words.txt, continued), from the oracle:\n"
                "# bits and uniforms as IEEE bit patterns (hex, exact), gaussian / lognormal\n"
                "# values as the oracle's long double result rounded to double (repr).\n"
                "# Written by make_golden.py.  Line: name kind dtype p0 p1 n: values\n")
        f.write("words 64: " + " ".join(f"{int(x):08x}" for x in words) + "\n")
        for name, kind, dtype, p0, p1 in TRANSFORM_CASES:
            vals = oracle.transform_words(kind, dtype, p0, p1, N_OUT, words)
            f.write(f"{name} {kind} {dtype} {p0!r} {p1!r} {N_OUT}: {fmt_values(kind, vals)}\n")


if __name__ == "__main__":
    main()
