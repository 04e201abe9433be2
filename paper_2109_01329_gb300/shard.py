"""Partition of one fill across ranks (one process per GPU).

A fill of n outputs is data parallel over word indices and needs no exchange:
rank r of `world` writes elements [start, start + count) from word offset
base + words_for(start), and the concatenation over ranks equals the
unsharded fill bit for bit.  Boundaries fall on multiples of 4 elements, so
they are whole Box-Muller pairs and (for 16-byte aligned buffers) 16-byte
boundaries.  The word offset comes from the library's consumption rule
(grng_words_for), not from a copy of it here.
"""

from __future__ import annotations

from . import _binding


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
    # (0, 1) are valid parameters of every distribution; the word count
    # depends only on the kind, the dtype and the element count
    dist = _binding.Distribution(kind, dtype, 0.0, 1.0)
    return start, stop - start, _binding.words_for(dist, start)
