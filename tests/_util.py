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


def word_off(n):
    """First 32-bit word of level n in a significance bit array (levels
    0..2 take one word each, level n >= 3 takes 4^n/32 words)."""
    if n <= 3:
        return n
    return 3 + ((1 << (2 * n)) - 64) // 96


def pack_bits(S, L):
    """The oracle's flags (bytes, level-major, row-major in a level) -> the
    library's bit words (bit b of word w of level n is the cell with Morton
    code 32 (w - word_off(n)) + b)."""
    S = np.asarray(S, dtype=np.uint8)
    out = np.zeros(max(word_off(L), 1), dtype=np.uint32)
    for n in range(L):
        bits = rm_to_morton(S[level_slice(n)], n).astype(np.uint8)
        if bits.size < 32:
            bits = np.concatenate([bits, np.zeros(32 - bits.size, np.uint8)])
        words = np.packbits(bits, bitorder="little").view("<u4")
        out[word_off(n): word_off(n) + words.size] = words
    return out
