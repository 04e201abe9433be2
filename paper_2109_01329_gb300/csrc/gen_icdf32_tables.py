"""Writes icdf32_tables.h: the polynomials of the FP32 inverse CDF.

Run from this directory: ``python gen_icdf32_tables.py > icdf32_tables.h``.

With x = 2u - 1 and v = -log2(1 - x^2) (symmetric in u and 1 - u),
z = Phi^-1(u) = sqrt(2) erfinv(x) = x P(v) (the form of M. Giles,
"Approximating the erfinv function", GPU Computing Gems, 2011, with the
logarithm in base 2 and fits of our own): P1(v) of degree 9 below
V1 = 5 / ln 2 and P2(sqrt(v) - sqrt(V1)) of degree 8 up to the v of
u = 2^-24.  Each is a weighted minimax fit (Lawson's iteration on 3000
Chebyshev nodes, weight x / max(1, |z|), so that the error of z relative to
max(1, |z|) is what is bounded) of values from mpmath at 100 bits, rounded to
float.
"""

import mpmath as mp
import numpy as np

mp.mp.prec = 100
D1, D2 = 9, 8
V1 = mp.mpf(5) / mp.log(2)
VMAX = -mp.log(4 * mp.mpf(2) ** -24 * (1 - mp.mpf(2) ** -24), 2)
NODES = 3000


def x_z(v):
    x = mp.sqrt(1 - mp.mpf(2) ** (-v))
    return x, mp.sqrt(2) * mp.erfinv(x)


def lawson(ts, fs, wts, deg, iters=30):
    t = np.array([float(v) for v in ts])
    f = np.array([float(v) for v in fs])
    wt = np.array([float(v) for v in wts])
    a = np.vander(t, deg + 1, increasing=True)
    lw = np.full(t.size, 1.0 / t.size)
    best = None
    for _ in range(iters):
        sw = np.sqrt(lw) * wt
        c = np.linalg.lstsq(a * sw[:, None], f * sw, rcond=None)[0]
        err = np.abs(a @ c - f) * wt
        if best is None or err.max() < best[0]:
            best = (err.max(), c)
        lw = lw * err
        lw /= lw.sum()
    return best[1].astype(np.float32)


def fit(t_of_k, v_of_t, deg):
    ts = [t_of_k(k) for k in range(NODES)]
    xz = [x_z(v_of_t(t)) for t in ts]
    c = lawson(ts, [z / x for x, z in xz], [x / max(1, z) for x, z in xz], deg)
    worst = max(abs(x * sum(mp.mpf(float(ci)) * t ** i for i, ci in enumerate(c)) - z) / max(1, z)
                for t, (x, z) in zip(ts[::10], xz[::10]))
    return c, worst


def horner(name, var, c):
    expr = f"{float(c[-1])!r}f"
    for ci in c[-2::-1]:
        expr = f"fmaf({expr}, ({var}), {float(ci)!r}f)"
    return [f"#define GRNG_ICDF32_{name}({var}) \\", "  " + expr]


def main():
    cheb = lambda k: (1 - mp.cos(mp.pi * (k + mp.mpf(0.5)) / NODES)) / 2
    c1, e1 = fit(lambda k: V1 * cheb(k), lambda v: v, D1)
    r0, r1 = mp.sqrt(V1), mp.sqrt(VMAX)
    c2, e2 = fit(lambda k: (r1 - r0) * cheb(k), lambda d: (d + r0) ** 2, D2)
    out = ["// Generated by gen_icdf32_tables.py (mpmath, 100-bit); do not edit.",
           "// z = x P1(v) for v < V1, x P2(sqrt(v) - sqrt(V1)) above; fit errors with",
           f"// float coefficients {float(e1):.1e} and {float(e2):.1e} of max(1, |z|).",
           "#pragma once",
           f"#define GRNG_ICDF32_V1 {float(np.float32(float(V1)))!r}f",
           f"#define GRNG_ICDF32_SQRT_V1 {float(np.float32(float(r0)))!r}f"]
    out += horner("P1", "v", c1)
    out += horner("P2", "d", c2)
    print("\n".join(out))


if __name__ == "__main__":
    main()
