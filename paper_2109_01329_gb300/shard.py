"""Partition of one fill across ranks (one process per GPU).

A fill of n outputs is data parallel over word indices and needs no exchange:
rank r of `world` writes elements [start, start + count) from word offset
base + words_for(start), and the concatenation over ranks equals the
unsharded fill bit for bit.  Boundaries fall on multiples of 4 elements, so
they are whole Box-Muller pairs and (for 16-byte aligned buffers) 16-byte
boundaries.
"""

from __future__ import annotations

_WPO = {0: 1, 1: 1, 2: 2}  # words per output by dtype (U32, F32, F64)


def _boundary(r: int, world: int, n: int) -> int:
    if r >= world:
        return n
    b = (r * n) // world
    return min(n, (b // 4) * 4)


def shard_range(rank: int, world: int, n: int, kind: int, dtype: int):
    """(start element, element count, word offset of start) for one rank."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("bad rank / world / n")
    start = _boundary(rank, world, n)
    stop = _boundary(rank + 1, world, n)
    # start is a multiple of 4, hence of a Box-Muller pair: words_for(start)
    # is simply start words per output.
    return start, stop - start, start * _WPO[dtype]
