"""Writes bm64_tables.h: constants of the integer FP64 Box-Muller transform.

Run from this directory: ``python gen_bm64_tables.py > bm64_tables.h``.
Values are computed with mpmath at 200 bits and rounded to nearest.

Tables (emitted as initializer macros)
  LT[i], i = 0..512:     (ln(c_i) * 2^64, c_i * 2^24) with c_i = floor(2^24 / (1 - i/1024))
                         / 2^24, the reduction factor for -ln(1 - delta) with delta in
                         [i/1024, (i+1)/1024)
  SC[j], j = 0..1024:    (sin, cos(2 pi j / 8192)) * 2^63
  kE58[e], e = 0..52:    e ln 2 * 2^58
  kExp2T[j], j = 0..256: 2^(j / 256) * 2^62
Scalars
  kLn2:    ln 2 * 2^64
  k2Pi61:  2 pi * 2^61
  kLog2e63: log2(e) * 2^63
  kInv2 .. kInv6: 2^64 / k (truncated)
"""

import mpmath as mp

mp.mp.prec = 200


def rnd(x):
    return int(mp.nint(x))


def main():
    out = []
    out.append("// Generated by gen_bm64_tables.py (mpmath, 200-bit); do not edit.")
    out.append("#pragma once")
    out.append("#include <cstdint>")
    out.append("namespace grng {")
    out.append("namespace bm64 {")
    two24 = mp.mpf(2) ** 24
    two63 = mp.mpf(2) ** 63
    two64 = mp.mpf(2) ** 64
    logc, logt = [], []
    for i in range(513):
        c = int(mp.floor(two24 / (1 - mp.mpf(i) / 1024)))
        logc.append(c)
        logt.append(rnd(mp.log(mp.mpf(c) / two24) * two64))
    assert logc[0] == 1 << 24 and logc[512] == 1 << 25
    assert all(t < 1 << 64 for t in logt)
    sint = [rnd(mp.sin(2 * mp.pi * j / 8192) * two63) for j in range(1025)]
    cost = [rnd(mp.cos(2 * mp.pi * j / 8192) * two63) for j in range(1025)]
    e58 = [rnd(e * mp.log(2) * mp.mpf(2) ** 58) for e in range(53)]
    assert all(v < 1 << 64 for v in e58)
    exp2t = [rnd(mp.mpf(2) ** (mp.mpf(j) / 256) * mp.mpf(2) ** 62) for j in range(257)]
    assert exp2t[0] == 1 << 62 and exp2t[256] == 1 << 63

    out.append(f"constexpr uint64_t kLn2 = {rnd(mp.log(2) * two64)}ull;")
    out.append(f"constexpr uint64_t k2Pi61 = {rnd(2 * mp.pi * mp.mpf(2) ** 61)}ull;")
    out.append(f"constexpr uint64_t kLog2e63 = {rnd(mp.log(mp.e, 2) * mp.mpf(2) ** 63)}ull;")
    for k in range(2, 7):
        out.append(f"constexpr uint64_t kInv{k} = {(1 << 64) // k}ull;")
    # interleaved pairs, one 16-byte load each: (sin, cos) and (ln c_i, c_i)
    for name, a, b in (("SC", sint, cost), ("LT", logt, logc)):
        out.append(f"#define GRNG_BM64_{name} {{ \\")
        for k in range(0, len(a), 2):
            out.append("    " + ", ".join(f"{{{a[i]}ull, {b[i]}ull}}" for i in range(k, min(k + 2, len(a)))) + ", \\")
        out.append("}")
    out.append(f"#define GRNG_BM64_LOGT_LEN {len(logt)}")
    out.append(f"#define GRNG_BM64_SINT_LEN {len(sint)}")
    # table bodies as macros: the device and host copies are declared where used
    for name, ctype, vals in [("E58", "uint64_t", e58), ("EXP2T", "uint64_t", exp2t)]:
        suffix = "ull" if "64" in ctype else "u"
        out.append(f"#define GRNG_BM64_{name}_LEN {len(vals)}")
        out.append(f"#define GRNG_BM64_{name} {{ \\")
        for k in range(0, len(vals), 4):
            out.append("    " + ", ".join(f"{v}{suffix}" for v in vals[k:k + 4]) + ", \\")
        out.append("}")
    out.append("}  // namespace bm64")
    out.append("}  // namespace grng")
    print("\n".join(out))


if __name__ == "__main__":
    main()
