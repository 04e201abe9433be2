"""Prints the polynomial coefficients of the FP32 Box-Muller (device_common.cuh).

Run from this directory: ``python gen_bm32_poly.py``.  Each fit is a weighted
least-squares fit on Chebyshev nodes, refined towards minimax by Lawson
reweighting, against mpmath values at 120 bits:
  sin(pi v / 4) / v      = S0 + S1 w + S2 w^2 + S3 w^3,  w = v^2, v in [0, 1]
  (cos(pi v / 4) - 1)/w  = C0 + C1 w + C2 w^2 + C3 w^3   (weighted by w)
  (ln(1 + t) - t) / t^2  = L0 + L1 t + ... + L7 t^7,   t in [sqrt(1/2) - 1, sqrt(2) - 1]
and each coefficient is rounded to the nearest float.
"""

import mpmath as mp
import numpy as np

mp.mp.prec = 120


def cheb_nodes(a, b, n):
    k = np.arange(n)
    return (a + b) / 2 + (b - a) / 2 * np.cos(np.pi * (2 * k + 1) / (2 * n))


def lawson(powers, x, target, weight, iters=60):
    A = np.stack([x ** p for p in powers], axis=1)
    w = np.ones_like(x)
    for _ in range(iters):
        sw = np.sqrt(w) * weight
        c, *_ = np.linalg.lstsq(A * sw[:, None], target * sw, rcond=None)
        err = np.abs(A @ c - target) * weight
        w = w * (err / err.max() + 1e-12)
        w /= w.sum()
    return c, float((np.abs(A @ c - target) * weight).max())


def main():
    v = cheb_nodes(0.0, 1.0, 4000)
    vm = [mp.mpf(float(x)) for x in v]
    ts = np.array([float(mp.sin(mp.pi * x / 4) / x) for x in vm])
    sc, se = lawson([0, 2, 4, 6], v, ts, np.ones_like(v))
    tc = np.array([float((mp.cos(mp.pi * x / 4) - 1) / (x * x)) for x in vm])
    cc, ce = lawson([0, 2, 4, 6], v, tc, v ** 2)
    a, b = float(mp.sqrt(0.5) - 1), float(mp.sqrt(2) - 1)
    t = cheb_nodes(a, b, 6000)
    t = t[np.abs(t) > 1e-9]
    tm = [mp.mpf(float(x)) for x in t]
    lg = np.array([float(mp.log1p(x)) for x in tm])
    tl = np.array([float((mp.log1p(x) - x) / (x * x)) for x in tm])
    lc, le = lawson(list(range(8)), t, tl, t ** 2 / np.abs(lg))
    for name, cs, err in (("S", sc, se), ("C", cc, ce), ("L", lc, le)):
        vals = ", ".join(f"{float(np.float32(c))!r}f" for c in cs)
        print(f"// {name}: max weighted error {err:.3e}")
        print(f"{name} = {{{vals}}}")


if __name__ == "__main__":
    main()
