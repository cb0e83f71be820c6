"""The CUDA path's layout arithmetic (csrc/common.cuh) over the whole accepted
range of levels, up to L = 14: level offsets aligned and non-overlapping,
significance-word offsets, Morton codes and same-level neighbour steps,
checked on the host against plain 64-bit formulas (no GPU; the helpers are
__host__ __device__).  Compiled with nvcc into the package's git-ignored
build folder."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2206_05761_gb300", "csrc")
OUT = os.path.join(ROOT, "paper_2206_05761_gb300", "_build", "layout_check")

PROGRAM = r"""
#include <cstdio>
#include "common.cuh"
using namespace hwfv1;

static int fails = 0;
#define CHECK(c, ...) do { if (!(c)) { if (fails++ < 10) std::printf(__VA_ARGS__); } } while (0)

// bit interleave written out bit by bit (x to the even bits, y to the odd)
static uint64_t interleave(uint64_t x, uint64_t y) {
    uint64_t m = 0;
    for (int b = 0; b < 32; ++b) m |= ((x >> b) & 1ull) << (2 * b) | ((y >> b) & 1ull) << (2 * b + 1);
    return m;
}

int main() {
    // hierarchy levels 0..kMaxL+1: 64-element aligned, each holding 4^n cells
    for (int n = 0; n <= kMaxL; ++n) {
        const uint64_t a = lvl_off(n), b = lvl_off(n + 1), cells = 1ull << (2 * n);
        CHECK(a % 64 == 0, "level %d offset %llu not 64-aligned\n", n, (unsigned long long)a);
        CHECK(b >= a + cells, "level %d overlaps level %d\n", n, n + 1);
        CHECK(b - a < cells + 64 + 64, "level %d leaves a gap of more than one alignment step\n", n);
    }
    CHECK(hier_size(kMaxL) == lvl_off(kMaxL + 1), "hier_size\n");
    // significance words: level n (0..L-1) holds 4^n bits, no word shared
    for (int n = 0; n < kMaxL; ++n) {
        const uint64_t w0 = word_off(n), w1 = word_off(n + 1), need = ((1ull << (2 * n)) + 31) / 32;
        CHECK(w1 >= w0 + need, "bit level %d overlaps\n", n);
    }
    CHECK((uint64_t)bits_words(kMaxL) < (1ull << 32), "bit words overflow\n");
    // packed leaves: level in the top 4 bits, a 28-bit Morton code below
    const uint32_t side = 1u << kMaxL;
    CHECK(morton2(side - 1, side - 1) == kCodeMask, "largest code\n");
    CHECK(((uint64_t)kMaxL << kLeafShift | kCodeMask) < (1ull << 32), "packed leaf overflow\n");
    // Morton codes and neighbour steps on a lattice of (i, j) with the edges
    uint64_t r = 0x9E3779B97F4A7C15ull;
    for (int k = 0; k < 200000; ++k) {
        r ^= r << 13; r ^= r >> 7; r ^= r << 17;
        uint32_t i = (uint32_t)(r & (side - 1)), j = (uint32_t)((r >> 20) & (side - 1));
        if (k < 4) { i = (k & 1) ? side - 1 : 0; j = (k & 2) ? side - 1 : 0; }
        const uint32_t c = morton2(i, j);
        CHECK((uint64_t)c == interleave(i, j), "morton2(%u, %u)\n", i, j);
        CHECK(compact16(c) == i && compact16(c >> 1) == j, "compact16 of (%u, %u)\n", i, j);
        if (i + 1 < side) CHECK(mort_xp(c) == morton2(i + 1, j), "x+ of (%u, %u)\n", i, j);
        if (i > 0) CHECK(mort_xm(c) == morton2(i - 1, j), "x- of (%u, %u)\n", i, j);
        if (j + 1 < side) CHECK(mort_yp(c) == morton2(i, j + 1), "y+ of (%u, %u)\n", i, j);
        if (j > 0) CHECK(mort_ym(c) == morton2(i, j - 1), "y- of (%u, %u)\n", i, j);
        // the ancestor at level m is the code shifted by 2 (L - m)
        const int m = (int)(r >> 40) % (kMaxL + 1);
        CHECK((c >> (2 * (kMaxL - m))) == morton2(i >> (kMaxL - m), j >> (kMaxL - m)), "ancestor\n");
    }
    std::printf(fails ? "FAILED %d\n" : "OK\n", fails);
    return fails ? 1 : 0;
}
"""


def test_layout_arithmetic_up_to_the_largest_level():
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc")
    if not nvcc:
        pytest.skip("nvcc not found")
    os.makedirs(OUT, exist_ok=True)
    src = os.path.join(OUT, "layout_check.cu")
    exe = os.path.join(OUT, "layout_check")
    with open(src, "w") as fh:
        fh.write(PROGRAM)
    b = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O1", "-std=c++17", "-I" + CSRC,
                        "-o", exe, src], capture_output=True, text=True)
    assert b.returncode == 0, b.stderr[-2000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "OK", r.stdout
