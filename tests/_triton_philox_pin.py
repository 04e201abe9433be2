"""Runs Triton's own Philox4x32-10 (``tl.philox``) in Triton's CPU interpreter.

Used by test_oracle_philox.py as an independent implementation of the
published Philox4x32-10 algorithm: the oracle's blocks must equal these.
Reads an (N, 6) uint32 array of (c0, c1, c2, c3, k0, k1) rows from argv[1]
and writes the (N, 4) output blocks to argv[2].  Must run in its own process
because the interpreter is selected by an environment variable at import.
"""

import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _philox_rows(out_ptr, c0_ptr, c1_ptr, c2_ptr, c3_ptr, seed, N: tl.constexpr):
    i = tl.arange(0, N)
    r0, r1, r2, r3 = tl.philox(seed, tl.load(c0_ptr + i), tl.load(c1_ptr + i),
                               tl.load(c2_ptr + i), tl.load(c3_ptr + i))
    tl.store(out_ptr + 4 * i + 0, r0)
    tl.store(out_ptr + 4 * i + 1, r1)
    tl.store(out_ptr + 4 * i + 2, r2)
    tl.store(out_ptr + 4 * i + 3, r3)


def main():
    rows = np.load(sys.argv[1]).astype(np.uint32)
    out = np.empty((rows.shape[0], 4), dtype=np.uint32)
    # one launch per distinct key (the seed is a scalar argument)
    keys = {}
    for idx, r in enumerate(rows):
        keys.setdefault((int(r[4]), int(r[5])), []).append(idx)
    for (k0, k1), idxs in keys.items():
        sel = rows[idxs]
        n = 1
        while n < len(idxs):
            n *= 2
        cols = []
        for j in range(4):
            col = np.zeros(n, dtype=np.uint32)
            col[: len(idxs)] = sel[:, j]
            cols.append(torch.from_numpy(col.view(np.int32)))
        o = torch.empty(4 * n, dtype=torch.int32)
        seed = k0 | (k1 << 32)
        if seed >= 1 << 63:
            seed -= 1 << 64  # passed as int64; Triton reinterprets it as uint64
        _philox_rows[(1,)](o, cols[0], cols[1], cols[2], cols[3], seed, N=n)
        out[idxs] = o.numpy().view(np.uint32).reshape(n, 4)[: len(idxs)]
    np.save(sys.argv[2], out)


if __name__ == "__main__":
    main()
