"""Writes icdf64_tables.h: the piecewise polynomial of the FP64 inverse CDF.

Run from this directory: ``python gen_icdf64_tables.py > icdf64_tables.h``.

For p in (0, 1/2], t = -Phi^-1(p) is a smooth function of w = sqrt(-2 ln p),
w in [w0, sqrt(106 ln 2)] with w0 = sqrt(2 ln 2) (p = 1/2 ... 2^-53); t is
analytic at w0, where it vanishes.  With D = w - w0 the range is cut into 46
segments: width 1/16 for D < 3/4 (12), 1/8 for D < 5/2 (14), 1/4 beyond
(20).  On each segment t = c0 + c1 s + ... + c8 s^8, s in [0, 1) the
position inside it; the coefficients are least-squares fits on Chebyshev
nodes against mpmath at 200 bits (t = sqrt(2) erfinv(1 - 2p)), rounded to
integers in units of 2^-59.  The fits stay below 1e-17 of max(1, t).
"""

import mpmath as mp

mp.mp.prec = 200
DEG = 8
W0 = mp.sqrt(2 * mp.log(2))
WMAX = mp.sqrt(106 * mp.log(2))
REGIONS = [(mp.mpf(0), mp.mpf("0.75"), mp.mpf(1) / 16),
           (mp.mpf("0.75"), mp.mpf("2.5"), mp.mpf(1) / 8),
           (mp.mpf("2.5"), mp.mpf("7.5"), mp.mpf(1) / 4)]


def t_of_w(w):
    if w <= W0:
        return mp.mpf(0)
    p = mp.e ** (-(w * w) / 2)
    return mp.sqrt(2) * mp.erfinv(1 - 2 * p)


def fit(a, h):
    n = 3 * (DEG + 1)
    nodes = [mp.mpf(1) / 2 + mp.cos(mp.pi * (2 * k + 1) / (2 * n)) / 2 for k in range(n)]
    A = mp.matrix(n, DEG + 1)
    b = mp.matrix(n, 1)
    for r, s in enumerate(nodes):
        b[r] = t_of_w(a + h * s)
        for c in range(DEG + 1):
            A[r, c] = s ** c
    coef = mp.lu_solve(A.T * A, A.T * b)
    err = mp.mpf(0)
    for i in range(65):
        s = mp.mpf(i) / 64
        t = t_of_w(a + h * s)
        v = sum(coef[c] * s ** c for c in range(DEG + 1))
        err = max(err, abs(v - t) / max(1, t))
    return [int(mp.nint(c * mp.mpf(2) ** 59)) for c in coef], err


def main():
    rows, worst = [], mp.mpf(0)
    for lo, hi, h in REGIONS:
        d = lo
        while d < hi and W0 + d < WMAX:
            coef, err = fit(W0 + d, h)
            rows.append(coef)
            worst = max(worst, err)
            d += h
    assert len(rows) == 46, len(rows)
    out = ["// Generated by gen_icdf64_tables.py (mpmath, 200-bit); do not edit.",
           f"// {len(rows)} segments x {DEG + 1} coefficients (units 2^-59); worst fit error "
           f"{float(worst):.2e} of max(1, t).",
           "#pragma once",
           "#include <cstdint>",
           "namespace grng {",
           "namespace icdf64 {",
           f"constexpr uint64_t kW0_60 = {int(mp.nint(W0 * mp.mpf(2) ** 60))}ull;  // w0 2^60",
           f"#define GRNG_ICDF64_SEGS {len(rows)}",
           f"#define GRNG_ICDF64_DEG {DEG}",
           "#define GRNG_ICDF64_COEF { \\"]
    for r in rows:
        out.append("    " + ", ".join(f"{v}ll" for v in r) + ", \\")
    out.append("}")
    out.append("}  // namespace icdf64")
    out.append("}  // namespace grng")
    print("\n".join(out))


if __name__ == "__main__":
    main()
