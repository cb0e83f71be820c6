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

// The bit pattern of a double and back, by register moves the compiler
// cannot see through.  Integer tests written on __double_as_longlong are
// recognised as floating-point operations (x == 0, |x|, x < y) and issued
// on the FP64 pipe, the bottleneck of this GPU; on these patterns they stay
// integer instructions.
__device__ __forceinline__ long long dbits(double x) {
    long long b;
    asm("mov.b64 %0, %1;" : "=l"(b) : "d"(x));
    return b;
}
__device__ __forceinline__ double dval(long long b) {
    double x;
    asm("mov.b64 %0, %1;" : "=d"(x) : "l"(b));
    return x;
}

constexpr int kMaxL = 14;
constexpr int kLeafShift = 28;              // packed leaf: level << 28 | code
constexpr uint32_t kCodeMask = (1u << kLeafShift) - 1u;

// element offset of level n in a hierarchy array
// (32-bit arithmetic: 4^n < 2^32 for n <= 15 = kMaxL + 1, and a 32-bit
// division by a constant is two instructions where the 64-bit one is a chain)
__host__ __device__ inline uint64_t lvl_off(int n) {
    if (n <= 3) return 64ull * (uint64_t)n;
    return (uint64_t)(192u + (((1u << (2 * n)) - 64u) / 3u));
}
// element count of a hierarchy with levels 0..L
__host__ __device__ inline uint64_t hier_size(int L) { return lvl_off(L + 1); }

// word offset of level n in a significance bit array
__host__ __device__ inline uint32_t word_off(int n) {
    if (n <= 3) return (uint32_t)n;
    return 3u + (((1u << (2 * n)) - 64u) / 96u);
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

// Same-level neighbours in the interleaved (Morton) domain: x occupies the
// even bits, y the odd bits.  Adding 1 to the x bits alone = set the y bits
// so that the carry runs through them, add, keep the x bits.
constexpr uint32_t kXBits = 0x55555555u, kYBits = 0xAAAAAAAAu;
__host__ __device__ inline uint32_t mort_xp(uint32_t c) { return (((c | kYBits) + 1u) & kXBits) | (c & kYBits); }
__host__ __device__ inline uint32_t mort_xm(uint32_t c) { return (((c & kXBits) - 1u) & kXBits) | (c & kYBits); }
__host__ __device__ inline uint32_t mort_yp(uint32_t c) { return (((c | kXBits) + 2u) & kYBits) | (c & kXBits); }
__host__ __device__ inline uint32_t mort_ym(uint32_t c) { return (((c & kYBits) - 2u) & kYBits) | (c & kXBits); }

// Programmatic dependent launch.  A kernel of the step launched with the
// programmatic-serialisation attribute may be scheduled before the kernel
// ahead of it in the stream has finished; pdl_wait, its first statement,
// blocks until that kernel has completed and its writes are visible (an
// ordinary launch returns at once).  pdl_launch_next lets the next kernel
// be scheduled once every CTA of this grid has issued it or exited; every
// CTA has then been placed, so the waiting CTAs of the next kernel only take
// slots this grid no longer needs.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

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

// ordered bits of |x| (sign cleared with an integer op)
__device__ __forceinline__ unsigned long long abs_obits(double x) {
    return (unsigned long long)dbits(x) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ unsigned long long abs_obits(float x) {
    // |x| widened to double is exact; its bits order like the value
    return (unsigned long long)dbits((double)__int_as_float(__float_as_int(x) & 0x7FFFFFFF));
}

// ordered bits of a non-negative double (min/max by integer atomics)
__device__ __forceinline__ unsigned long long obits(double x) {
    return (unsigned long long)dbits(x);
}
__device__ __forceinline__ double from_obits(unsigned long long b) {
    return dval((long long)b);
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

// Block-wide max of three uint64 values, then one atomicMax each into
// dst[0..2].  Every thread of the block must call it.
__device__ __forceinline__ void block_max3_u64(unsigned long long a, unsigned long long b,
                                               unsigned long long c, unsigned long long* dst) {
    __shared__ unsigned long long red3[3][32];
    __syncthreads();          // a previous call's readers are done with red3
    a = warp_max_u64(a);
    b = warp_max_u64(b);
    c = warp_max_u64(c);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red3[0][warp] = a;
        red3[1][warp] = b;
        red3[2][warp] = c;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        a = lane < nw ? red3[0][lane] : 0ull;
        b = lane < nw ? red3[1][lane] : 0ull;
        c = lane < nw ? red3[2][lane] : 0ull;
        a = warp_max_u64(a);
        b = warp_max_u64(b);
        c = warp_max_u64(c);
        if (lane == 0) {
            if (a) atomicMax(dst, a);
            if (b) atomicMax(dst + 1, b);
            if (c) atomicMax(dst + 2, c);
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
    double fric_k;                    // ((dt_use * g) * n) * n: the friction term's step factor
    float fric_kf;                    // the same in float arithmetic (float32 path)
    double smax[4];                   // s_max of h, qx, qy, z
    unsigned long long rmin_bits;     // min CFL bound over updated leaves
    unsigned long long speed_bits[3]; // max |u|+sqrt(gh), |v|+sqrt(gh) over updated wet leaves
                                      // (float64 updates; the bound is formed in the finish)
    unsigned long long max_bits[3];   // max |h|, |qx|, |qy| of the new state
    long long step;
    uint32_t active;                  // t < t_end
    uint32_t cur;                     // which state buffer holds the state
    uint32_t err;                     // latched device error bits
    unsigned long long ticket;        // running tile ticket of the traversal
    uint32_t nwet;                    // leaves queued for the full FV1 update
    uint32_t ndec;                    // tiles listed for the decode kernel
    uint32_t Mall;                    // leaves of the last traversal, skipped tiles included
    uint32_t M;                       // leaves in the step's list (processed tiles)
    uint32_t nact;                    // tiles in the traversal's work list; ndec, Mall, M and
                                      // nact are adjacent (cleared together)
    double rx0, ry0;                  // dt_use/lx, dt_use/ly (dt/dx_n = rx0 * 2^n)
    float rx0f, ry0f;                 // same, float arithmetic
    double thr[kMaxL * 3];            // eps*2^(n-L)*s_max,q for h, qx, qy
    float thrf[kMaxL * 3];            // same, float arithmetic (32-bit path)
    double thr4[kMaxL * 3];           // 4 * thr where thr >= 2^-1020, else -1
    float thr4f[kMaxL * 3];           // 4 * thrf where thrf >= 2^-124, else -1
    float thr4lo[kMaxL * 3];          // thr4 rounded down / up to float where thr4 >= 2^-100,
    float thr4hi[kMaxL * 3];          // else -1 (the float pre-check of the encode)
    unsigned long long leaf_updates;  // leaves updated, summed over the steps taken
    unsigned long long wet_updates;   // of them, leaves that took the full FV1 update
    unsigned long long act_updates;   // of them, leaves outside skipped (quiescent) tiles
    uint32_t epoch;                   // completed steps (never reset; tags the face stamps)
    uint32_t enc_ticket;              // finished CTAs of the fused last encode passes
    uint32_t dec_ticket;              // finished CTAs of the fused decode + finish
    uint32_t ntodo;                   // tiles the first encode pass works on (listed by the
                                      // clear kernel, reset by the encode's last CTA)
};

enum : uint32_t { kErrNonFinite = 1u, kErrTimeout = 2u };

// a double that is +0 or -0 (integer test, no FP64 instruction)
__device__ __forceinline__ bool is_zero(double x) { return (dbits(x) << 1) == 0; }
__device__ __forceinline__ bool is_zero(float x) { return (__float_as_int(x) << 1) == 0; }

// x >= y decided on the bit patterns.  Equal to the IEEE comparison for
// every x (negative, NaN and inf included) when y > 0, and when y == +0 for
// every x except -0 (callers use it with y > 0, or with x never -0).
__device__ __forceinline__ bool ge_nonneg(double x, double y) {
    const long long bx = dbits(x);
    return bx >= dbits(y) && bx <= 0x7FF0000000000000ll;
}
__device__ __forceinline__ bool ge_nonneg(float x, float y) {
    const int bx = __float_as_int(x);
    return bx >= __float_as_int(y) && bx <= 0x7F800000;
}

}  // namespace hwfv1
