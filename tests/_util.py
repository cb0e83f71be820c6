"""Test helpers: index permutations between the oracle's row-major levels
and the library's Morton order (index work only, no method arithmetic)."""
import numpy as np


def _compact(x):
    x = x & 0x55555555
    x = (x | (x >> 1)) & 0x33333333
    x = (x | (x >> 2)) & 0x0F0F0F0F
    x = (x | (x >> 4)) & 0x00FF00FF
    x = (x | (x >> 8)) & 0x0000FFFF
    return x


def morton_perm(n):
    """perm[code] = row-major index of the cell with that Morton code."""
    code = np.arange(1 << (2 * n), dtype=np.int64)
    i = _compact(code)
    j = _compact(code >> 1)
    return j * (1 << n) + i


def rm_to_morton(a, n):
    return np.asarray(a).reshape(-1)[morton_perm(n)]


def level_slice(n):
    s = ((1 << (2 * n)) - 1) // 3
    return slice(s, s + (1 << (2 * n)))
