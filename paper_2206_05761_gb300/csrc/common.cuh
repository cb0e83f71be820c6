// common.cuh -- layout of the Morton-ordered hierarchy and small device
// helpers shared by the HWFV1 kernels.
//
// Hierarchy layout (one array per quantity): level n (0..L) holds the 4^n
// cells of the 2^n x 2^n grid in Morton order (the Z-order indexing of
// Sec. 2.2.1, Fig. 5-6), so the four children of a parent are four
// consecutive elements.  The paper numbers the cells of level n from
// (4^n-1)/3; here every level starts on a multiple of 64 elements instead
// (A(n) below) so that sibling groups and whole tiles are aligned for
// 128-bit loads.
//
// Significance bits: level n (0..L-1) holds 4^n bits in Morton order,
// starting at word W(n) (a level never shares a word with another).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hwfv1 {

constexpr int kMaxL = 14;
constexpr int kLeafShift = 28;              // packed leaf: level << 28 | code
constexpr uint32_t kCodeMask = (1u << kLeafShift) - 1u;

// element offset of level n in a hierarchy array
__host__ __device__ inline uint64_t lvl_off(int n) {
    if (n <= 3) return 64ull * (uint64_t)n;
    return 192ull + (((1ull << (2 * n)) - 64ull) / 3ull);
}
// element count of a hierarchy with levels 0..L
__host__ __device__ inline uint64_t hier_size(int L) { return lvl_off(L + 1); }

// word offset of level n in a significance bit array
__host__ __device__ inline uint32_t word_off(int n) {
    if (n <= 3) return (uint32_t)n;
    return 3u + (uint32_t)(((1ull << (2 * n)) - 64ull) / 96ull);
}
__host__ __device__ inline uint32_t bits_words(int L) { return word_off(L); }

// Morton code <-> (i, j): bit b of i -> bit 2b, bit b of j -> bit 2b+1
__host__ __device__ inline uint32_t spread16(uint32_t x) {
    x &= 0xFFFFu;
    x = (x | (x << 8)) & 0x00FF00FFu;
    x = (x | (x << 4)) & 0x0F0F0F0Fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}
__host__ __device__ inline uint32_t compact16(uint32_t x) {
    x &= 0x55555555u;
    x = (x | (x >> 1)) & 0x33333333u;
    x = (x | (x >> 2)) & 0x0F0F0F0Fu;
    x = (x | (x >> 4)) & 0x00FF00FFu;
    x = (x | (x >> 8)) & 0x0000FFFFu;
    return x;
}
__host__ __device__ inline uint32_t morton2(uint32_t i, uint32_t j) {
    return spread16(i) | (spread16(j) << 1);
}

// significance bit (n, code)
__device__ __forceinline__ uint32_t sig_bit(const uint32_t* __restrict__ b, int n, uint32_t code) {
    return (__ldg(b + word_off(n) + (code >> 5)) >> (code & 31u)) & 1u;
}

// 8 bits -> 32 bits, each bit repeated 4 times (parent flags -> children)
__host__ __device__ inline uint32_t expand4x8(uint32_t x) {
    x &= 0xFFu;
    x = (x | (x << 12)) & 0x000F000Fu;
    x = (x | (x << 6)) & 0x03030303u;
    x = (x | (x << 3)) & 0x11111111u;
    return x * 0xFu;
}

// ordered bits of a non-negative double (min/max by integer atomics)
__device__ __forceinline__ unsigned long long obits(double x) {
    return (unsigned long long)__double_as_longlong(x);
}
__device__ __forceinline__ double from_obits(unsigned long long b) {
    return __longlong_as_double((long long)b);
}
constexpr unsigned long long kInfBits = 0x7FF0000000000000ull;

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w < v ? w : v;
    }
    return v;
}
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// Block-wide min (IS_MAX = false) or max of a uint64 followed by one
// atomic on `dst`.  Every thread of the block must call it.
template <bool IS_MAX>
__device__ __forceinline__ void block_atomic_u64(unsigned long long v, unsigned long long* dst) {
    __shared__ unsigned long long red[32];
    v = IS_MAX ? warp_max_u64(v) : warp_min_u64(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        v = lane < nw ? red[lane] : (IS_MAX ? 0ull : ~0ull);
        v = IS_MAX ? warp_max_u64(v) : warp_min_u64(v);
        if (lane == 0) {
            if (IS_MAX) atomicMax(dst, v);
            else atomicMin(dst, v);
        }
    }
}

// Exclusive block scan of one uint32 per thread (blockDim <= 1024).
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* total) {
    __shared__ uint32_t ws[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        uint32_t s = lane < nw ? ws[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        ws[lane] = s;   // inclusive prefix of warp sums
    }
    __syncthreads();
    const uint32_t before = warp ? ws[warp - 1] : 0u;
    if (total) *total = ws[((blockDim.x + 31) >> 5) - 1];
    return before + x - v;
}

// Device-side state of one simulation (all scalars the step needs, so that
// a captured step graph replays without host input).
struct DevState {
    double t, dt, dt_use, t_end;
    double Qdt;                       // Q(t) * dt_use of the current step
    double smax[4];                   // s_max of h, qx, qy, z
    unsigned long long rmin_bits;     // min CFL bound over updated leaves
    unsigned long long max_bits[3];   // max |h|, |qx|, |qy| of the new state
    long long step;
    uint32_t M;                       // leaves of the last traversal
    uint32_t active;                  // t < t_end
    uint32_t cur;                     // which state buffer holds the state
    uint32_t err;                     // latched device error bits
    double thr[kMaxL * 3];            // eps*2^(n-L)*s_max,q for h, qx, qy
    float thrf[kMaxL * 3];            // same, float arithmetic (32-bit path)
};

enum : uint32_t { kErrNonFinite = 1u };

}  // namespace hwfv1
