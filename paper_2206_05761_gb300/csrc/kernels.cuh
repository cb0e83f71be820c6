// kernels.cuh -- HWFV1 device kernels, templated on the arithmetic type T
// (double: the parity path; float: the 32-bit path).
//
// Every kernel that belongs to a timestep reads its scalars (timestep,
// thresholds, leaf count, which state buffer is current) from DevState in
// device memory, so one step can be captured in a CUDA graph and replayed.
// The double instantiation evaluates the method in the operation order of
// the readings documented in the design notes (no FMA contraction: the
// library is compiled with --fmad=false); where a cheaper form is used it
// is equal for every finite input (noted at the spot).
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace hwfv1 {

template <typename T> struct Vec4;
template <> struct Vec4<double> {
    static __device__ __forceinline__ void load(const double* p, double& a, double& b, double& c,
                                                double& d) {
        const double2 u = __ldg(reinterpret_cast<const double2*>(p));
        const double2 v = __ldg(reinterpret_cast<const double2*>(p) + 1);
        a = u.x; b = u.y; c = v.x; d = v.y;
    }
    static __device__ __forceinline__ void store(double* p, double a, double b, double c, double d) {
        reinterpret_cast<double2*>(p)[0] = make_double2(a, b);
        reinterpret_cast<double2*>(p)[1] = make_double2(c, d);
    }
    // through L2 only: for data other CTAs of the same kernel wrote
    static __device__ __forceinline__ void load_cg(const double* p, double& a, double& b, double& c,
                                                   double& d) {
        const double2 u = __ldcg(reinterpret_cast<const double2*>(p));
        const double2 v = __ldcg(reinterpret_cast<const double2*>(p) + 1);
        a = u.x; b = u.y; c = v.x; d = v.y;
    }
};
template <> struct Vec4<float> {
    static __device__ __forceinline__ void load(const float* p, float& a, float& b, float& c,
                                                float& d) {
        const float4 u = __ldg(reinterpret_cast<const float4*>(p));
        a = u.x; b = u.y; c = u.z; d = u.w;
    }
    static __device__ __forceinline__ void load_cg(const float* p, float& a, float& b, float& c, float& d) {
        const float4 u = __ldcg(reinterpret_cast<const float4*>(p));
        a = u.x; b = u.y; c = u.z; d = u.w;
    }
    static __device__ __forceinline__ void store(float* p, float a, float b, float c, float d) {
        *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
    }
};

struct Vec4u {
    // leaves pos..pos+3 = (L << 28) | (m0 + e); pos need not be aligned
    static __device__ __forceinline__ void store(uint32_t* p, uint32_t tag_m0, uint32_t) {
#pragma unroll
        for (uint32_t e = 0; e < 4u; ++e) p[e] = tag_m0 + e;
    }
};

template <> struct Vec4<uint32_t> {
    // p[0..3] = v + 0..3; one 128-bit store when p is 16-byte aligned
    static __device__ __forceinline__ void store_u(uint32_t* p, uint32_t v) {
        if ((reinterpret_cast<uintptr_t>(p) & 15u) == 0u) {
            *reinterpret_cast<uint4*>(p) = make_uint4(v, v + 1u, v + 2u, v + 3u);
        } else {
#pragma unroll
            for (uint32_t e = 0; e < 4u; ++e) p[e] = v + e;
        }
    }
};

template <typename T> __device__ __forceinline__ bool same4(T a, T b, T c, T d);
template <> __device__ __forceinline__ bool same4<double>(double a, double b, double c, double d) {
    const long long x = dbits(a);
    // equal bit patterns and |a| < 2^1022 (so 4a does not overflow)
    return x == dbits(b) && x == dbits(c) &&
           x == dbits(d) && ((x >> 52) & 0x7FF) < 0x7FD;
}
template <> __device__ __forceinline__ bool same4<float>(float a, float b, float c, float d) {
    const int x = __float_as_int(a);
    return x == __float_as_int(b) && x == __float_as_int(c) && x == __float_as_int(d) &&
           ((x >> 23) & 0xFF) < 0xFD;
}

// |x| by clearing the sign bit (no FP64 instruction)
__device__ __forceinline__ double absval(double x) {
    return dval(dbits(x) & 0x7FFFFFFFFFFFFFFFll);
}
__device__ __forceinline__ float absval(float x) { return __int_as_float(__float_as_int(x) & 0x7FFFFFFF); }

// ---------------------------------------------------------------------------
// Exact replacements of FP64 (FP32) instructions by integer ones, on a GPU
// whose FP64 pipe is the bottleneck.  Each returns the bits the IEEE
// operation returns (NaN inputs aside, which the state checks report).
// ---------------------------------------------------------------------------
// x * 2^k for k in {-2, -1, 1}: an exponent step when input and result are
// normal numbers; otherwise the IEEE product (inline PTX, so that it is not
// executed when the integer path applies).
template <int K>
__device__ __forceinline__ double pow2_scale(double x) {
    const long long b = dbits(x);
    const int e = (int)((b >> 52) & 0x7FF);
    if (e + K >= 1 && e + K <= 0x7FE && e >= 1 && e <= 0x7FE) return dval(b + ((long long)K << 52));
    double r;
    if (K == -2) asm volatile("mul.rn.f64 %0, %1, 0d3FD0000000000000;" : "=d"(r) : "d"(x));
    else if (K == -1) asm volatile("mul.rn.f64 %0, %1, 0d3FE0000000000000;" : "=d"(r) : "d"(x));
    else asm volatile("mul.rn.f64 %0, %1, 0d4000000000000000;" : "=d"(r) : "d"(x));
    return r;
}
template <int K>
__device__ __forceinline__ float pow2_scale(float x) {
    const int b = __float_as_int(x);
    const int e = (b >> 23) & 0xFF;
    if (e + K >= 1 && e + K <= 0xFE && e >= 1 && e <= 0xFE) return __int_as_float(b + (K << 23));
    float r;
    if (K == -2) asm volatile("mul.rn.f32 %0, %1, 0f3E800000;" : "=f"(r) : "f"(x));
    else if (K == -1) asm volatile("mul.rn.f32 %0, %1, 0f3F000000;" : "=f"(r) : "f"(x));
    else asm volatile("mul.rn.f32 %0, %1, 0f40000000;" : "=f"(r) : "f"(x));
    return r;
}
// x * 2^n for 0 <= n <= 30: an exponent step when x and the result are
// normal numbers, otherwise the IEEE product (the same bits either way).
__device__ __forceinline__ double mul_pow2(double x, int n) {
    const long long b = dbits(x);
    const int e = (int)((b >> 52) & 0x7FF);
    if (e >= 1 && e + n <= 0x7FE) return dval(b + ((long long)n << 52));
    return x * (double)(1u << n);
}
__device__ __forceinline__ float mul_pow2(float x, int n) {
    const int b = __float_as_int(x);
    const int e = (b >> 23) & 0xFF;
    if (e >= 1 && e + n <= 0xFE) return __int_as_float(b + (n << 23));
    return x * (float)(1u << n);
}
template <typename T> __device__ __forceinline__ T quarter(T x) { return pow2_scale<-2>(x); }
template <typename T> __device__ __forceinline__ T half(T x) { return pow2_scale<-1>(x); }
template <typename T> __device__ __forceinline__ T twice(T x) { return pow2_scale<1>(x); }

// Integer key with the order of the IEEE comparison (+0 and -0 equal).
__device__ __forceinline__ long long ord_key(double x) {
    const long long b = dbits(x);
    return b >= 0 ? b : -(b & 0x7FFFFFFFFFFFFFFFll);
}
__device__ __forceinline__ int ord_key(float x) {
    const int b = __float_as_int(x);
    return b >= 0 ? b : -(b & 0x7FFFFFFF);
}
// a < b ? a : b and a > b ? a : b (the IEEE selections, which pick b on ties)
template <typename T> __device__ __forceinline__ T sel_min(T a, T b) { return ord_key(a) < ord_key(b) ? a : b; }
template <typename T> __device__ __forceinline__ T sel_max(T a, T b) { return ord_key(a) > ord_key(b) ? a : b; }
// x >= 0 and x <= 0 (true for either zero)
template <typename T> __device__ __forceinline__ bool ge_zero(T x) { return ord_key(x) >= 0; }
template <typename T> __device__ __forceinline__ bool le_zero(T x) { return ord_key(x) <= 0; }
// x is finite (not inf or NaN)
__device__ __forceinline__ bool finite_bits(double x) {
    return (dbits(x) & 0x7FF0000000000000ll) != 0x7FF0000000000000ll;
}
__device__ __forceinline__ bool finite_bits(float x) { return (__float_as_int(x) & 0x7F800000) != 0x7F800000; }
// x > 0, false for NaN as in IEEE
__device__ __forceinline__ bool gt_zero(double x) {
    const long long b = dbits(x);
    return b > 0 && b <= 0x7FF0000000000000ll;
}
__device__ __forceinline__ bool gt_zero(float x) {
    const int b = __float_as_int(x);
    return b > 0 && b <= 0x7F800000;
}

// A block of a (possibly batched) launch: its index among the blocks given
// to one domain and their number.  Single-domain launches use blockIdx.x and
// gridDim.x; batched launches (batch.cuh) map a flat grid onto domains.
struct Blk {
    uint32_t id, n;
};
__device__ __forceinline__ Blk this_blk() { return Blk{blockIdx.x, gridDim.x}; }

// Haar parent (Eq. 3a) and the largest detail magnitude (Eq. 3b-3d) of four
// children [0]=(2i,2j) [1]=(2i+1,2j) [2]=(2i,2j+1) [3]=(2i+1,2j+1).
// dmax = 0.25*max(|d+e|, |a-b|, |d-e|) equals max(|0.25(d+e)|, ...) because
// scaling by 0.25 and rounding commute with max.  Four equal children give
// s = c0 and dmax = 0 in every arithmetic, so that case skips the sums.
template <typename T>
__device__ __forceinline__ void haar4(T c0, T c1, T c2, T c3, T& s, T& dmax4) {
    if (same4<T>(c0, c1, c2, c3)) {
        s = c0;
        dmax4 = T(0);
        return;
    }
    const T a = c0 + c2, b = c1 + c3, d = c0 - c2, e = c1 - c3;
    s = quarter(a + b);
    const T da = absval(d + e), db = absval(a - b), dg = absval(d - e);
    // the largest |detail| times 4: details are a quarter of these sums, an
    // exact scaling that passes_thr compares against 4 * threshold
    dmax4 = sel_max(sel_max(da, db), dg);
}

// max|d| >= thr for the three details d = m4/4 of a parent: compared as
// m4 >= thr4 = 4 thr when thr >= 2^-1020 (then m4/4 is exact, or both
// sides of the original comparison are below thr); thr4 < 0 marks the
// other thresholds, compared as written.
template <typename T>
__device__ __forceinline__ bool passes_thr(T m4, T thr, T thr4) {
    if (ge_zero(thr4)) return ge_nonneg(m4, thr4);      // m4 is never -0
    return ge_nonneg(T(0.25) * m4, thr);
}

// A float near a double, by integer instructions alone (a conversion
// instruction would take the FP64 pipe): the significand truncated to 23
// bits, so |f - x| <= 2^-23 |x| and |f| <= |x| in the normal float range;
// +-0 when |x| < 2^-126; an infinity when |x| >= 2^128, or x is not finite.
__device__ __forceinline__ float trunc_float(double x) {
    const unsigned long long b = (unsigned long long)dbits(x);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const uint32_t sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
    uint32_t f;
    if (e <= 0) f = sign;
    else if (e >= 255) f = sign | 0x7F800000u;
    else f = sign | ((uint32_t)e << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    return __int_as_float((int)f);
}

// The parent of four doubles and its threshold decision, the details
// decided in float where that is conclusive.  With c' = trunc_float(c) and
// S = sum |c'|, the float m4' of the same sums satisfies
// |m4' - m4| <= 2^-20 S + 2^-120: the inputs are off by at most 2^-23 |c|
// (<= 2^-23 (1 + 2^-22) S in total) or 2^-126 each below the float range,
// the float sums add two roundings of at most 2^-24 S each, the double side
// two of 2^-53 S (about 2^-22 S + 2^-124 in all, with room to spare).
// Compared with directed roundings against thr4 rounded down and up, a
// decision taken in float is the one the double comparison m4 >= thr4
// takes; otherwise (or for values outside the float range) the details are
// computed in double.
__device__ __forceinline__ bool float_finite(float x) { return (__float_as_int(x) & 0x7F800000) != 0x7F800000; }
__device__ __forceinline__ void haar4_pre(double c0, double c1, double c2, double c3, double thr, double thr4,
                                          float lo, float hi, double& s, bool& flag) {
    if (same4<double>(c0, c1, c2, c3)) {
        s = c0;
        flag = passes_thr(0.0, thr, thr4);
        return;
    }
    const double a = c0 + c2, b = c1 + c3;
    s = quarter(a + b);
    if (lo >= 0.0f) {
        const float f0 = trunc_float(c0), f1 = trunc_float(c1), f2 = trunc_float(c2), f3 = trunc_float(c3);
        const float af = f0 + f2, bf = f1 + f3, df = f0 - f2, ef = f1 - f3;
        const float m = fmaxf(fmaxf(fabsf(df + ef), fabsf(af - bf)), fabsf(df - ef));
        const float S = __fadd_ru(__fadd_ru(fabsf(f0), fabsf(f1)), __fadd_ru(fabsf(f2), fabsf(f3)));
        const float E = __fadd_ru(__fmul_ru(S, 0x1p-20f), 0x1p-120f);
        if (float_finite(m) && float_finite(E)) {
            if (__fsub_rd(m, E) >= hi) { flag = true; return; }
            if (__fadd_ru(m, E) < lo) { flag = false; return; }
        }
    }
    const double d = c0 - c2, e = c1 - c3;
    const double m4 = sel_max(sel_max(absval(d + e), absval(a - b)), absval(d - e));
    flag = passes_thr(m4, thr, thr4);
}


// Write the per-thread flag of `cnt` consecutive parents (codes base..) of
// level n.  Full words are stored; a partial word (cnt < 32) is OR-ed into
// a word cleared before the pass.  Called by every thread of the block.
__device__ __forceinline__ uint32_t put_bits(uint32_t* bits, int n, uint32_t base, uint32_t cnt,
                                             bool flag) {
    const uint32_t ballot = __ballot_sync(0xffffffffu, flag);
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    if (cnt >= 32u) {
        if (lane == 0 && warp * 32u < cnt) bits[word_off(n) + (base >> 5) + warp] = ballot;
    } else if (threadIdx.x == 0 && ballot) {
        atomicOr(bits + word_off(n) + (base >> 5), ballot << (base & 31u));
    }
    return ballot;
}

// ---------------------------------------------------------------------------
// Encoding + threshold flags + closure (Eq. 3, Algorithm 1)
// ---------------------------------------------------------------------------
template <typename T, int NF>
struct EncodeArgs {
    T* f[2][NF];          // hierarchy of each quantity, per state buffer
    const T* thr;         // threshold of level n, quantity q at thr[n*NF + q]
    const T* thr4;        // 4 * thr where exact comparisons allow it, else -1
    const float* thr4lo = nullptr;   // float bounds of thr4 for the pre-check (NULL: none)
    const float* thr4hi = nullptr;
    uint32_t* Tb;         // threshold flags
    uint32_t* Cb;         // upward closure of the threshold flags
    const DevState* st;   // NULL: buffer 0, always active
    int L, ls, k;         // source level ls; produces levels ls-1 .. ls-k
    int span = 0;         // a CTA covers 4^span cells of level ls (0: 4^k)
    // Quiescent tiles (first pass only, its tiles are the traversal's):
    // zf[b][t] = 1 when every value of buffer b in tile t, levels ls-k..ls,
    // is +0.  NULL: no skipping.
    uint8_t* zf[2] = {nullptr, nullptr};
    // the first pass's tiles (k_encode_tiles): list[0 .. st->ntodo)
    const uint32_t* list = nullptr;
};

// The thresholds of one level and quantity (thr, 4 thr, and 4 thr's float
// bounds, lo < 0 when the float pre-check is off).
template <typename T>
struct Thr {
    T thr, thr4;
    float lo, hi;
};

// Parent coefficient of one quantity and its part of the parent's threshold
// flag tf (an OR over the quantities).  Once tf is set the remaining
// quantities need their parent only.
template <typename T>
__device__ __forceinline__ void parent_coef(const Thr<T>& h, T c0, T c1, T c2, T c3, T& s, bool& tf) {
    if constexpr (sizeof(T) == 8) {
        // haar4_pre with lo < 0 is haar4 + passes_thr
        if (tf) {
            s = same4<T>(c0, c1, c2, c3) ? c0 : quarter((c0 + c2) + (c1 + c3));
            return;
        }
        haar4_pre(c0, c1, c2, c3, h.thr, h.thr4, h.lo, h.hi, s, tf);
        return;
    }
    T dm;
    haar4<T>(c0, c1, c2, c3, s, dm);
    tf = tf || passes_thr(dm, h.thr, h.thr4);
}

// The parents of all NF quantities of one cell and its threshold flag.  In
// float64 the sums of every quantity come first (independent of one
// another, so the FP64 pipe takes them back to back instead of one
// quantity's chain after the other's), then the threshold decisions in
// quantity order, with the float pre-check of haar4_pre and the same
// shortcut: once a quantity has flagged the parent the others need their
// parent only.  Every value is formed by the same operations as in
// haar4_pre.
template <typename T, int NF>
__device__ __forceinline__ void parents_all(const Thr<T>* th, const T (&c)[NF][4], T (&s)[NF], bool& tf) {
    if constexpr (sizeof(T) == 8) {
        bool eq[NF];
        T sa[NF], sb[NF];
#pragma unroll
        for (int q = 0; q < NF; ++q) {
            eq[q] = same4<T>(c[q][0], c[q][1], c[q][2], c[q][3]);
            sa[q] = T(0);
            sb[q] = T(0);
            if (!eq[q]) {
                sa[q] = c[q][0] + c[q][2];
                sb[q] = c[q][1] + c[q][3];
            }
        }
#pragma unroll
        for (int q = 0; q < NF; ++q) s[q] = eq[q] ? c[q][0] : quarter(sa[q] + sb[q]);
#pragma unroll
        for (int q = 0; q < NF; ++q) {
            if (tf) break;
            const Thr<T>& h = th[q];
            if (eq[q]) {
                tf = passes_thr(T(0), h.thr, h.thr4);
                continue;
            }
            const T c0 = c[q][0], c1 = c[q][1], c2 = c[q][2], c3 = c[q][3];
            bool decided = false;
            if (h.lo >= 0.0f) {
                const float f0 = trunc_float(c0), f1 = trunc_float(c1), f2 = trunc_float(c2), f3 = trunc_float(c3);
                const float af = f0 + f2, bf = f1 + f3, df = f0 - f2, ef = f1 - f3;
                const float m = fmaxf(fmaxf(fabsf(df + ef), fabsf(af - bf)), fabsf(df - ef));
                const float S = __fadd_ru(__fadd_ru(fabsf(f0), fabsf(f1)), __fadd_ru(fabsf(f2), fabsf(f3)));
                const float E = __fadd_ru(__fmul_ru(S, 0x1p-20f), 0x1p-120f);
                if (float_finite(m) && float_finite(E)) {
                    if (__fsub_rd(m, E) >= h.hi) {
                        tf = true;
                        decided = true;
                    } else if (__fadd_ru(m, E) < h.lo) {
                        decided = true;
                    }
                }
            }
            if (!decided) {
                const T d = c0 - c2, e = c1 - c3;
                const T m4 = sel_max(sel_max(absval(d + e), absval(sa[q] - sb[q])), absval(d - e));
                tf = passes_thr(m4, h.thr, h.thr4);
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < NF; ++q) parent_coef(th[q], c[q][0], c[q][1], c[q][2], c[q][3], s[q], tf);
    }
}

// Hierarchy of quantity q in the current state buffer (selects, so that the
// parameter array is not indexed at run time).
template <typename T, int NF>
__device__ __forceinline__ T* quantity_ptr(const EncodeArgs<T, NF>& a, int par, uint32_t q) {
    T* r = par ? a.f[1][0] : a.f[0][0];
#pragma unroll
    for (int k = 1; k < NF; ++k)
        if (q == (uint32_t)k) r = par ? a.f[1][k] : a.f[0][k];
    return r;
}

// the value is +0 (all bits clear)
__device__ __forceinline__ bool pos_zero(double x) { return dbits(x) == 0ll; }
__device__ __forceinline__ bool pos_zero(float x) { return __float_as_int(x) == 0; }

// R-decode's free surface and finest depths with the FP64 work a flat bed
// does not need: x + (+0) = x for x != -0 and x - (+0) = x for every x are
// exact, and four beds of one bit pattern give four equal differences.
// eta_of: hl + zl for a wet leaf (hl >= tol > 0).
template <typename T>
__device__ __forceinline__ T eta_of(T hl, T zl) { return pos_zero(zl) ? hl : hl + zl; }
__device__ __forceinline__ bool bits_eq4(double a, double b, double c, double d) {
    const long long x = dbits(a);
    return x == dbits(b) && x == dbits(c) && x == dbits(d);
}
__device__ __forceinline__ bool bits_eq4(float a, float b, float c, float d) {
    const int x = __float_as_int(a);
    return x == __float_as_int(b) && x == __float_as_int(c) && x == __float_as_int(d);
}
// hf[k] = max(0, eta - z_k) as (eta - z_k > 0 ? eta - z_k : 0)
template <typename T>
__device__ __forceinline__ void restore4(T eta, T z0, T z1, T z2, T z3, T (&hf)[4]) {
    if (bits_eq4(z0, z1, z2, z3)) {
        const T d = pos_zero(z0) ? eta : eta - z0;
        hf[0] = hf[1] = hf[2] = hf[3] = gt_zero(d) ? d : T(0);
        return;
    }
    const T d0 = eta - z0, d1 = eta - z1, d2 = eta - z2, d3 = eta - z3;
    hf[0] = gt_zero(d0) ? d0 : T(0);
    hf[1] = gt_zero(d1) ? d1 : T(0);
    hf[2] = gt_zero(d2) ? d2 : T(0);
    hf[3] = gt_zero(d3) ? d3 : T(0);
}

// One CTA encodes one tile: the 4^k cells of level ls under one level-(ls-k)
// cell, k <= 5 levels in one pass.  The first level reads four children
// per thread with 128-bit loads; the next levels work from shared memory.
// CG: read the source level and the closure bits through L2 only (the tail
// pass reads what other CTAs of the same launch wrote).
template <typename T, int NF, bool CG = false>
__device__ __forceinline__ void encode_body(const EncodeArgs<T, NF>& a, int ls, int kk, uint32_t bid) {
    if (a.st && !a.st->active) return;
    const int par = a.st ? (int)a.st->cur : 0;
    // A tile known to hold only +0 encodes to +0 with no significant detail
    // (thresholds are > 0 whenever skipping is on): what is stored is
    // already the result, and the cleared flag words stay clear.
    const bool quiet = a.zf[0] != nullptr && ls == a.L;
    uint8_t* const zfp = par ? a.zf[1] : a.zf[0];   // (no dynamic index into parameters)
    if (quiet && zfp[bid]) return;
    __shared__ T sv0[NF][256];        // level ls-1 (and ls-3, ls-5)
    __shared__ T sv1[NF][64];         // level ls-2 (and ls-4)
    __shared__ uint32_t sc[2][8];
    __shared__ Thr<T> sthr[5][NF];    // thresholds of the pass's levels (one load each)
    const uint32_t tile = bid, tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    // parents of level ls-1 under the CTA (its block of 4^span cells of
    // level ls; a pass may stop short of the block's top level)
    const int span = (ls == a.ls && a.span > kk) ? a.span : kk;
    uint32_t cnt = 1u << (2 * (span - 1));
    int n = ls - 1;
    {   // level ls-1
        const bool act = tid < cnt;
        const uint32_t p = tile * cnt + tid;
        bool tf = false, nz = false;
        uint32_t cchild = 0;
        T s[NF];
#pragma unroll
        for (int q = 0; q < NF; ++q) s[q] = T(0);
        // every load first (the stores below could alias them for the
        // compiler, which would then serialise load, compute and store per
        // quantity), with the thresholds of all the pass's levels, then the
        // parents, then the stores
        T c[NF][4];
        if (act) {
#pragma unroll
            for (int q = 0; q < NF; ++q) {
                const T* fq = par ? a.f[1][q] : a.f[0][q];
                if (CG) Vec4<T>::load_cg(fq + lvl_off(ls) + 4ull * p, c[q][0], c[q][1], c[q][2], c[q][3]);
                else Vec4<T>::load(fq + lvl_off(ls) + 4ull * p, c[q][0], c[q][1], c[q][2], c[q][3]);
            }
            if (ls < a.L) {
                const uint32_t cb = 4u * p;
                const uint32_t* cw = a.Cb + word_off(ls) + (cb >> 5);
                cchild = ((CG ? __ldcg(cw) : __ldg(cw)) >> (cb & 31u)) & 0xFu;
            }
        }
        if (tid < (uint32_t)(kk * NF)) {
            const int j = tid / NF, q = tid - j * NF, idx = (ls - 1 - j) * NF + q;
            Thr<T> h;
            h.thr = a.thr[idx];
            h.thr4 = a.thr4[idx];
            h.lo = a.thr4lo ? a.thr4lo[idx] : -1.0f;
            h.hi = a.thr4hi ? a.thr4hi[idx] : -1.0f;
            sthr[j][q] = h;
        }
        __syncthreads();
        if (act) {
#pragma unroll
            for (int q = 0; q < NF; ++q)
                nz = nz || !(pos_zero(c[q][0]) && pos_zero(c[q][1]) && pos_zero(c[q][2]) && pos_zero(c[q][3]));
            parents_all<T, NF>(sthr[0], c, s, tf);
#pragma unroll
            for (int q = 0; q < NF; ++q) {
                T* fq = par ? a.f[1][q] : a.f[0][q];
                fq[lvl_off(n) + p] = s[q];
            }
        }
        const bool cf = act && (tf || cchild);
        put_bits(a.Tb, n, tile * cnt, cnt, act && tf);
        const uint32_t cball = put_bits(a.Cb, n, tile * cnt, cnt, cf);
#pragma unroll
        for (int q = 0; q < NF; ++q) sv0[q][tid] = s[q];
        if (lane == 0) sc[0][warp] = cball;
        if (quiet) {   // all finest values +0 => every coarser value written is +0
            const int any = __syncthreads_or(nz ? 1 : 0);
            if (tid == 0) zfp[tile] = any ? 0 : 1;
        }
    }
    // Levels of at most 64 parents: one warp per quantity, each through the
    // levels on its own, with no block barrier between them.  A parent's
    // threshold flag is the OR of its quantities' flags, and its upward
    // closure the OR of per-quantity closures that start from the full
    // closure of the pass's first level.  Every warp ORs its words into the
    // flag words, which were cleared before the pass.
    if (kk < 2) return;
    __syncthreads();                 // the first level's values and closure words
    if (warp >= (uint32_t)NF) return;
    const uint32_t q = warp;
    T* const fq = quantity_ptr(a, par, q);
    uint32_t cprev0 = 0u, cprev1 = 0u;   // this warp's closure bits of the level below (<= 64)
    for (int j = 2; j <= kk; ++j) {
        n = ls - j;
        cnt >>= 2;
        const int rbuf = (j - 2) & 1, wbuf = (j - 1) & 1;   // level j-1 wrote buffer (j-2)&1
        const T* const r = rbuf ? sv1[q] : sv0[q];
        T* const w = wbuf ? sv1[q] : sv0[q];
        uint32_t cnow0 = 0u, cnow1 = 0u;
        for (uint32_t k = 0u; k * 32u < cnt; ++k) {        // cnt <= 64: at most two rounds
            const uint32_t pp = k * 32u + lane;
            const bool act = pp < cnt;
            bool f = false;
            uint32_t cchild = 0u;
            if (act) {
                const T c0 = r[4 * pp], c1 = r[4 * pp + 1], c2 = r[4 * pp + 2], c3 = r[4 * pp + 3];
                T sp = T(0);
                parent_coef(sthr[j - 1][q], c0, c1, c2, c3, sp, f);
                fq[lvl_off(n) + tile * cnt + pp] = sp;
                w[pp] = sp;
                const uint32_t cb = 4u * pp;                  // the first child's bit
                const uint32_t cw = j == 2 ? sc[0][cb >> 5] : ((cb >> 5) ? cprev1 : cprev0);
                cchild = (cw >> (cb & 31u)) & 0xFu;
            }
            const uint32_t tb = __ballot_sync(0xffffffffu, act && f);
            const uint32_t cbl = __ballot_sync(0xffffffffu, act && (f || cchild != 0u));
            if (k == 0u) cnow0 = cbl;
            else cnow1 = cbl;
            if (lane == 0u) {
                const uint32_t base = tile * cnt + k * 32u;
                if (tb) atomicOr(a.Tb + word_off(n) + (base >> 5), tb << (base & 31u));
                if (cbl) atomicOr(a.Cb + word_off(n) + (base >> 5), cbl << (base & 31u));
            }
        }
        cprev0 = cnow0;
        cprev1 = cnow1;
        __syncwarp();                // this level's values before the next level reads them
    }
}

template <typename T, int NF>
static __global__ void __launch_bounds__(256) k_encode(EncodeArgs<T, NF> a) {
    pdl_wait();
    encode_body<T, NF>(a, a.ls, a.k, blockIdx.x);
}

// A pass followed, in its last CTA to finish, by the final one-CTA pass
// (levels ls2-1 .. 0), saving a launch; ticket counts the finished CTAs and
// is reset by the last one.
template <typename T, int NF>
static __global__ void __launch_bounds__(256) k_encode_tail(EncodeArgs<T, NF> a, int ls2, int k2,
                                                            uint32_t* ticket) {
    pdl_wait();
    encode_body<T, NF>(a, a.ls, a.k, blockIdx.x);
    __threadfence();                     // this CTA's coefficients and bits are visible
    __syncthreads();
    __shared__ bool last;
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1u;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x == 0) {
        *ticket = 0u;
        // the tile list of the pass before (k_encode_tiles, done) starts
        // empty next step
        if (a.list) const_cast<DevState*>(a.st)->ntodo = 0u;
    }
    encode_body<T, NF, true>(a, ls2, k2, 0u);
}

// The same pass with a fixed grid when quiescent tiles are skipped: the
// tiles that are not marked quiescent were listed by k_clear_words, and CTA
// b encodes list entries b, b + grid, ...: a step's active tiles, which
// cluster where the water is, spread one per CTA.
template <typename T, int NF>
static __global__ void __launch_bounds__(256) k_encode_tiles(EncodeArgs<T, NF> a) {
    pdl_wait();
    if (!a.st->active) return;
    const uint32_t n = *(volatile const uint32_t*)&a.st->ntodo;
    for (uint32_t e = blockIdx.x; e < n; e += gridDim.x) {
        encode_body<T, NF>(a, a.ls, a.k, __ldg(a.list + e));
        __syncthreads();                 // shared memory is reused by the next tile
    }
}

// Clear bit arrays before an encode (the partial words are OR-ed into),
// and with `list`, list the tiles of the current state buffer that are not
// marked quiescent (st->ntodo counts them; it is 0 on entry).
__device__ __forceinline__ void clear_body(uint32_t* w, uint32_t nwords, const DevState* st, Blk B) {
    if (st && !st->active) return;
    for (uint32_t i = B.id * blockDim.x + threadIdx.x; i < nwords; i += B.n * blockDim.x) w[i] = 0u;
}
static __global__ void k_clear_words(uint32_t* w, uint32_t nwords, DevState* st, const uint8_t* zf0,
                                     const uint8_t* zf1, uint32_t ntiles, uint32_t* list, uint32_t* zero4) {
    pdl_wait();
    // the traversal's four counters (ndec, Mall, M, nact), for the step's
    // traversal (no kernel in between uses them)
    if (zero4 && blockIdx.x == 0 && threadIdx.x < 4u && st->active) zero4[threadIdx.x] = 0u;
    clear_body(w, nwords, st, this_blk());
    if (!list || !st->active) return;
    const uint8_t* zf = st->cur ? zf1 : zf0;
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t lane = threadIdx.x & 31u;
    for (uint32_t t0 = blockIdx.x * blockDim.x; t0 < ntiles; t0 += stride) {   // whole warps
        const uint32_t t = t0 + threadIdx.x;
        const bool todo = t < ntiles && !zf[t];
        const uint32_t m = __ballot_sync(0xffffffffu, todo);
        if (m == 0u) continue;
        uint32_t base = 0u;
        if (lane == 0) base = atomicAdd(&st->ntodo, (uint32_t)__popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (todo) list[base + __popc(m & ((1u << lane) - 1u))] = t;
    }
}

// ---------------------------------------------------------------------------
// Regularised significance, word-parallel:
//   S(n,c) = Sbase(n,c) | (close ? C(n,c) : T(n,c)) | (predict ? T(n-1,c/4) : 0)
// ---------------------------------------------------------------------------
struct FlagArgs {
    const uint32_t *Tb, *Cb, *Sbase;
    uint32_t* Sb;
    int L, predict, close;
    DevState* st;
};

// Word lw of level n of S (the inputs are read-only in the caller).
__device__ __forceinline__ uint32_t reg_word(const uint32_t* __restrict__ Tb, const uint32_t* __restrict__ Cb,
                                             const uint32_t* __restrict__ Sbase, int n, uint32_t lw, int predict,
                                             int close) {
    const uint32_t w = word_off(n) + lw;
    uint32_t s = close ? __ldg(Cb + w) : __ldg(Tb + w);
    if (Sbase) s |= __ldg(Sbase + w);
    if (predict && n >= 1) {
        uint32_t pb;
        if (n >= 3) {
            pb = expand4x8(__ldg(Tb + word_off(n - 1) + (lw >> 2)) >> (8u * (lw & 3u)));
        } else if (n == 2) {   // 16 cells, parents are the 4 cells of level 1
            pb = expand4x8(__ldg(Tb + word_off(1)) & 0xFu);
        } else {               // level 1: the root's four children
            pb = (__ldg(Tb + word_off(0)) & 1u) ? 0xFu : 0u;
        }
        s |= pb;
    }
    if (n <= 2) s &= (n == 0 ? 1u : (n == 1 ? 0xFu : 0xFFFFu));
    return s;
}

__device__ __forceinline__ void flag_body(const uint32_t* __restrict__ Tb, const uint32_t* __restrict__ Cb,
                                          const uint32_t* __restrict__ Sbase, uint32_t* __restrict__ Sb,
                                          int L, int predict, int close, const DevState* st, Blk B) {
    if (st && !st->active) return;
    const uint32_t total = bits_words(L);
    for (uint32_t w = B.id * blockDim.x + threadIdx.x; w < total; w += B.n * blockDim.x) {
        int n = 0;
        while (n + 1 < L && word_off(n + 1) <= w) ++n;
        Sb[w] = reg_word(Tb, Cb, Sbase, n, w - word_off(n), predict, close);
    }
}

// Where a kernel reads S: the words k_flag wrote (Sb), or, with Sb NULL,
// each word formed on the spot from the words k_flag would read.
struct SigSrc {
    const uint32_t* Sb = nullptr;
    const uint32_t *Tb = nullptr, *Cb = nullptr, *Sbase = nullptr;
    int predict = 1, close = 1;
};
__device__ __forceinline__ uint32_t s_word(const SigSrc& s, int n, uint32_t lw) {
    return s.Sb ? __ldg(s.Sb + word_off(n) + lw) : reg_word(s.Tb, s.Cb, s.Sbase, n, lw, s.predict, s.close);
}
__device__ __forceinline__ uint32_t sig_bit(const SigSrc& s, int n, uint32_t code) {
    return (s_word(s, n, code >> 5) >> (code & 31u)) & 1u;
}
// One bit of S formed without a branch on the level (lanes asking for
// different levels issue the same loads together): Sbase(n,c) | (close ? C
// : T)(n,c) | (predict ? T(n-1, c/4) : 0), the bit of reg_word's word.
__device__ __forceinline__ uint32_t sig_bit_flat(const SigSrc& s, int n, uint32_t c) {
    if (s.Sb) return (__ldg(s.Sb + word_off(n) + (c >> 5)) >> (c & 31u)) & 1u;
    const uint32_t* cw = s.close ? s.Cb : s.Tb;
    const uint32_t a = __ldg(cw + word_off(n) + (c >> 5));
    const uint32_t z = s.Sbase ? __ldg(s.Sbase + word_off(n) + (c >> 5)) : 0u;
    const bool par = s.predict && n >= 1;
    const uint32_t p = par ? __ldg(s.Tb + word_off(par ? n - 1 : 0) + ((c >> 2) >> 5)) : 0u;
    return ((((a | z) >> (c & 31u)) | (p >> ((c >> 2) & 31u))) & 1u);
}
// The bits S(n, tile >> 2(Lr-n)) of the root path of a tile, levels
// 0..Lr, bit n of the result.  Formed on the spot, every word is loaded
// before any is used: S(n,c) = Sbase(n,c) | (close ? C : T)(n,c) |
// (predict ? T(n-1, c/4) : 0), the bit of reg_word's word.
__device__ __forceinline__ uint32_t root_bits(const SigSrc& s, int Lr, uint32_t tile) {
    uint32_t r = 0u;
    if (s.Sb) {
#pragma unroll
        for (int n = 0; n < kMaxL; ++n)
            if (n <= Lr) r |= sig_bit(s, n, tile >> (2 * (Lr - n))) << n;
        return r;
    }
    const uint32_t* cw = s.close ? s.Cb : s.Tb;
    uint32_t a[kMaxL], z[kMaxL], p[kMaxL];
#pragma unroll
    for (int n = 0; n < kMaxL; ++n) {
        a[n] = z[n] = p[n] = 0u;
        if (n <= Lr) {
            const uint32_t c = tile >> (2 * (Lr - n));
            a[n] = __ldg(cw + word_off(n) + (c >> 5));
            if (s.Sbase) z[n] = __ldg(s.Sbase + word_off(n) + (c >> 5));
            if (s.predict && n >= 1) p[n] = __ldg(s.Tb + word_off(n - 1) + ((c >> 2) >> 5));
        }
    }
#pragma unroll
    for (int n = 0; n < kMaxL; ++n) {
        if (n <= Lr) {
            const uint32_t c = tile >> (2 * (Lr - n));
            const uint32_t b = (((a[n] | z[n]) >> (c & 31u)) | (p[n] >> ((c >> 2) & 31u))) & 1u;
            r |= b << n;
        }
    }
    return r;
}
// zero4: the traversal's four counters (ndec, Mall, M, nact), cleared here
// for the traversal that follows (NULL: none).
static __global__ void k_flag(const uint32_t* __restrict__ Tb, const uint32_t* __restrict__ Cb,
                              const uint32_t* __restrict__ Sbase, uint32_t* __restrict__ Sb, int L,
                              int predict, int close, const DevState* st, uint32_t* zero4 = nullptr) {
    pdl_wait();
    if (zero4 && blockIdx.x == 0 && threadIdx.x < 4u) zero4[threadIdx.x] = 0u;
    flag_body(Tb, Cb, Sbase, Sb, L, predict, close, st, this_blk());
}

// OR of two bit arrays (threshold flags of h, qx, qy with those of z).
static __global__ void k_or_words(const uint32_t* a, const uint32_t* b, uint32_t* out, uint32_t n) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = a[i] | b[i];
}

// ---------------------------------------------------------------------------
// Leaf identification (Algorithm 5) and compaction (Sec. 2.2.3).
// A tile is the 4^kt finest cells under one level-(L-kt) cell; thread t owns
// the four finest cells 4t..4t+3 of the tile (one level-(L-1) parent).
// ---------------------------------------------------------------------------
struct TileWalk {
    int l;          // leaf level of the thread's four cells (common ancestor path)
    uint32_t m0;    // first finest Morton code of the thread
    bool act;
};

// Level at which the walk from the root towards the tile stops (<= L-kt), or
// L-kt+1 if every cell on the path is significant.  Run by one thread.
__device__ __forceinline__ int walk_root(const uint32_t* Sb, int Lr, uint32_t tile) {
    for (int n = 0; n <= Lr; ++n)
        if (!sig_bit(Sb, n, tile >> (2 * (Lr - n)))) return n;
    return Lr + 1;
}

__device__ __forceinline__ TileWalk walk_tile(const uint32_t* Sb, int L, int kt, uint32_t tile,
                                              int l0) {
    TileWalk w;
    const int Lr = L - kt;
    w.act = threadIdx.x < (1u << (2 * (kt - 1)));
    w.m0 = (tile << (2 * kt)) + 4u * threadIdx.x;
    if (!w.act) {            // threads past the tile touch no memory
        w.l = L;
        return w;
    }
    if (l0 <= Lr) {
        w.l = l0;
    } else {
        w.l = L;
        for (int n = Lr + 1; n <= L - 1; ++n)
            if (!sig_bit(Sb, n, w.m0 >> (2 * (L - n)))) { w.l = n; break; }
    }
    return w;
}

// number of leaves whose first finest cell is among the thread's 4 cells
__device__ __forceinline__ uint32_t heads_of(const TileWalk& w, int L) {
    if (!w.act) return 0u;
    if (w.l == L) return 4u;
    const uint32_t mask = (1u << (2 * (L - w.l))) - 1u;
    return (w.m0 & mask) == 0u ? 1u : 0u;
}

static __global__ void __launch_bounds__(256) k_trav_count_walk(const uint32_t* __restrict__ Sb,
                                                    uint32_t* __restrict__ counts, int L, int kt,
                                                    const DevState* st) {
    if (st && !st->active) return;
    __shared__ int s_l0;
    const uint32_t tile = blockIdx.x;
    if (threadIdx.x == 0) s_l0 = walk_root(Sb, L - kt, tile);
    __syncthreads();
    const TileWalk w = walk_tile(Sb, L, kt, tile, s_l0);
    uint32_t total;
    block_excl_scan(heads_of(w, L), &total);
    if (threadIdx.x == 0) counts[tile] = total;
}

// ---------------------------------------------------------------------------
// Traversal + compaction in three deterministic passes (count, scan, write).
// Each CTA stages its tile's significance bits in shared memory (the root
// path is read by 32 threads at once), then finds the leaf of every group of
// four finest cells from shared memory.
// ---------------------------------------------------------------------------
struct TileBits {
    uint32_t w[12];   // levels Lr+1..Lr+4 under the tile: j=1 w[0], j=2 w[1], j=3 w[2..3], j=4 w[4..11]
    int l0;           // leaf level if a cell on the root path (levels 0..Lr) is insignificant, else Lr+1
};

__device__ __forceinline__ int tb_slot(int j) { return j == 1 ? 0 : (j == 2 ? 1 : (j == 3 ? 2 : 4)); }

// Called by the whole block; ends with __syncthreads.
__device__ __forceinline__ void load_tile_bits(const SigSrc& Sb, int L, int kt, uint32_t tile, TileBits& tb) {
    const int Lr = L - kt;
    const int t = threadIdx.x;
    if (t < 32) {
        bool zero = false;
        if (t <= Lr) zero = sig_bit_flat(Sb, t, tile >> (2 * (Lr - t))) == 0u;
        const uint32_t z = __ballot_sync(0xffffffffu, zero);
        if (t == 0) tb.l0 = z ? (__ffs(z) - 1) : Lr + 1;
    } else if (t < 44) {
        const int k = t - 32;                       // word slot 0..11
        int j, idx;
        if (k == 0) { j = 1; idx = 0; }
        else if (k == 1) { j = 2; idx = 0; }
        else if (k < 4) { j = 3; idx = k - 2; }
        else { j = 4; idx = k - 4; }
        uint32_t v = 0u;
        if (j <= kt - 1) {
            const int n = Lr + j;
            const uint32_t cnt = 1u << (2 * j);
            const uint32_t first = tile * cnt;        // first code of the tile at level n
            if (cnt < 32u) {
                v = (s_word(Sb, n, first >> 5) >> (first & 31u)) & ((1u << cnt) - 1u);
            } else if ((uint32_t)idx * 32u < cnt) {
                v = s_word(Sb, n, (first >> 5) + idx);
            }
        }
        tb.w[k] = v;
    }
    __syncthreads();
}
__device__ __forceinline__ void load_tile_bits(const uint32_t* __restrict__ Sb, int L, int kt, uint32_t tile,
                                               TileBits& tb) {
    SigSrc s;
    s.Sb = Sb;
    load_tile_bits(s, L, kt, tile, tb);
}

// leaf level of the thread's group of four finest cells (local group g)
__device__ __forceinline__ int group_level(const TileBits& tb, int L, int kt, uint32_t g) {
    const int Lr = L - kt;
    if (tb.l0 <= Lr) return tb.l0;
    for (int j = 1; j <= kt - 1; ++j) {
        const uint32_t c = (4u * g) >> (2 * (kt - j));    // local code at level Lr+j
        if (!((tb.w[tb_slot(j) + (c >> 5)] >> (c & 31u)) & 1u)) return Lr + j;
    }
    return L;
}

// Leaves of up to 16 finest cells (levels L-1, L-2) are decoded by the FV1
// kernels themselves; larger ones by k_decode over the tiles listed here.
__device__ __forceinline__ bool needs_decode_kernel(int l, int L) { return l < L - 2; }

// One warp per tile.  Lane t reads bit t of the root path (levels 0..Lr) and
// word slot t of the tile's own levels; group_level then works from the
// warp's copy in shared memory.  Lane t owns the groups 8t..8t+7 (32
// consecutive finest cells), so its leaves are consecutive in Z-order.
constexpr int kTilesPerCta = 8;
constexpr int kGroupsPerLane = 8;

__device__ __forceinline__ void warp_tile_bits(const uint32_t* __restrict__ Sb, int L, int kt,
                                               uint32_t tile, TileBits& tb) {
    const int Lr = L - kt;
    const int t = threadIdx.x & 31;
    bool zero = false;
    if (t <= Lr) zero = sig_bit(Sb, t, tile >> (2 * (Lr - t))) == 0u;
    const uint32_t z = __ballot_sync(0xffffffffu, zero);
    if (t < 12) {
        int j, idx;
        if (t == 0) { j = 1; idx = 0; }
        else if (t == 1) { j = 2; idx = 0; }
        else if (t < 4) { j = 3; idx = t - 2; }
        else { j = 4; idx = t - 4; }
        uint32_t v = 0u;
        if (j <= kt - 1) {
            const int n = Lr + j;
            const uint32_t cnt = 1u << (2 * j);
            const uint32_t first = tile * cnt;
            if (cnt < 32u) {
                v = (__ldg(Sb + word_off(n) + (first >> 5)) >> (first & 31u)) & ((1u << cnt) - 1u);
            } else if ((uint32_t)idx * 32u < cnt) {
                v = __ldg(Sb + word_off(n) + (first >> 5) + idx);
            }
        }
        tb.w[t] = v;
    }
    if (t == 0) tb.l0 = z ? (__ffs(z) - 1) : Lr + 1;
    __syncwarp();
}

// Leaf heads of the lane's groups: returns the count; level of group e in lv[e].
__device__ __forceinline__ uint32_t lane_heads(const TileBits& tb, int L, int kt, uint32_t tile,
                                               int lv[kGroupsPerLane]) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t ngroups = 1u << (2 * (kt - 1));
    uint32_t cnt = 0u;
#pragma unroll
    for (int e = 0; e < kGroupsPerLane; ++e) {
        const uint32_t g = lane * kGroupsPerLane + e;
        lv[e] = -1;
        if (g < ngroups) {
            const int l = group_level(tb, L, kt, g);
            lv[e] = l;
            const uint32_t m0 = (tile << (2 * kt)) + 4u * g;
            cnt += l == L ? 4u : ((m0 & ((1u << (2 * (L - l))) - 1u)) == 0u ? 1u : 0u);
        }
    }
    return cnt;
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ uint32_t warp_excl(uint32_t v) {
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (uint32_t)o) x += y;
    }
    return x - v;
}

// Quiescent-tile skipping.  A traversal tile (level L-kt) is skipped in a
// step when every h, qx, qy value of both state buffers in it (levels
// L-kt..L) is +0, the same holds in the current buffer for its four edge
// neighbours, no inflow cell lies in it and no leaf coarser than the tile
// covers it.  Every leaf of such a tile then sees depth +0 at itself and at
// its same-level neighbours, so the update gives (+0, +0, +0) -- which the
// destination buffer already holds, at every level of the tile.  Its leaves
// are counted but not listed, updated or decoded, and its encode is a no-op.
// A tile covered by a coarser leaf is processed (act = kActCovered) but
// keeps its zf mark of the destination buffer: the decode kernel skips its
// writes when that leaf's new value is +0 and clears the mark otherwise.
struct Quiet {
    uint8_t* zf[2] = {nullptr, nullptr};   // per state buffer and tile: all +0 (NULL: off)
    const uint8_t* inlet = nullptr;        // tiles holding inflow cells
    uint8_t* act = nullptr;                // per tile: 0 skipped, kActOwn or kActCovered
};
constexpr uint8_t kActOwn = 1, kActCovered = 2;

// Traversal, pass 1: leaves per CTA (8 tiles) -- those of processed tiles
// into csum, all of them into *mall (if given); tiles holding a leaf of more
// than 16 finest cells are listed for the decode kernel (if dlist is given).
__device__ __forceinline__ void trav_count_body(const uint32_t* __restrict__ Sb, uint32_t* __restrict__ csum,
                                                uint32_t* __restrict__ dlist, int L, int kt, uint32_t ntiles,
                                                DevState* st, Blk B, uint32_t* mall, const Quiet& q) {
    if (!st->active) return;
    __shared__ TileBits tbs[kTilesPerCta];
    __shared__ uint32_t wsum[kTilesPerCta], wall[kTilesPerCta];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const uint32_t tile = B.id * kTilesPerCta + warp;
    uint32_t total = 0u, total_all = 0u;
    if (tile < ntiles) {
        TileBits& tb = tbs[warp];
        warp_tile_bits(Sb, L, kt, tile, tb);
        bool skip = false;
        if (q.zf[0] != nullptr) {
            if (lane == 0) {
                const int Lr = L - kt;
                const uint32_t cur = st->cur;
                const uint8_t* X = cur ? q.zf[1] : q.zf[0];
                uint8_t* Y = cur ? q.zf[0] : q.zf[1];
                const bool covered = tb.l0 < Lr;
                skip = !covered && X[tile] && Y[tile] && !q.inlet[tile];
                if (skip) {
                    const uint32_t lm = (1u << (2 * Lr)) - 1u;
                    const uint32_t xs = tile & kXBits & lm, ys = tile & kYBits & lm;
                    if (xs != 0u) skip = skip && X[mort_xm(tile)];
                    if (xs != (kXBits & lm)) skip = skip && X[mort_xp(tile)];
                    if (ys != 0u) skip = skip && X[mort_ym(tile)];
                    if (ys != (kYBits & lm)) skip = skip && X[mort_yp(tile)];
                }
                q.act[tile] = skip ? 0 : (covered ? kActCovered : kActOwn);
                if (!skip && !covered && Y[tile]) Y[tile] = 0;     // the step writes into it
            }
            skip = __shfl_sync(0xffffffffu, skip ? 1 : 0, 0) != 0;
        }
        int lv[kGroupsPerLane];
        const uint32_t c = lane_heads(tb, L, kt, tile, lv);
        bool big = false;
#pragma unroll
        for (int e = 0; e < kGroupsPerLane; ++e) big = big || (lv[e] >= 0 && needs_decode_kernel(lv[e], L));
        total_all = warp_sum(c);
        total = skip ? 0u : total_all;
        if (dlist && !skip && __any_sync(0xffffffffu, big) && lane == 0) {
            const uint32_t pos = atomicAdd(&st->ndec, 1u);
            dlist[pos] = tile;           // one entry per tile at most
        }
    }
    if (lane == 0) {
        wsum[warp] = total;
        wall[warp] = total_all;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0u, sa = 0u;
        for (int w = 0; w < kTilesPerCta; ++w) {
            s += wsum[w];
            sa += wall[w];
        }
        csum[B.id] = s;
        if (mall && sa) atomicAdd(mall, sa);
    }
}
static __global__ void __launch_bounds__(256) k_trav_count(const uint32_t* __restrict__ Sb,
                                                           uint32_t* __restrict__ csum,
                                                           uint32_t* __restrict__ dlist, int L, int kt,
                                                           uint32_t ntiles, DevState* st, uint32_t* mall,
                                                           Quiet q) {
    trav_count_body(Sb, csum, dlist, L, kt, ntiles, st, this_blk(), mall, q);
}

// Traversal, pass 2: exclusive scan of the per-CTA counts (one CTA); the
// total goes to *total_out.
__device__ __forceinline__ void trav_scan_body(const uint32_t* __restrict__ counts, uint32_t* __restrict__ offs,
                                               uint32_t n, DevState* st, uint32_t* total_out) {
    if (!st->active) return;
    const uint32_t per = (n + blockDim.x - 1) / blockDim.x;
    const uint32_t b = threadIdx.x * per, e = min(n, b + per);
    uint32_t sum = 0;
    for (uint32_t i = b; i < e; ++i) sum += counts[i];
    uint32_t total;
    uint32_t run = block_excl_scan(sum, &total);
    for (uint32_t i = b; i < e; ++i) {
        offs[i] = run;
        run += counts[i];
    }
    if (threadIdx.x == 0) *total_out = total;
}
static __global__ void __launch_bounds__(1024) k_trav_scan(const uint32_t* __restrict__ counts,
                                                           uint32_t* __restrict__ offs, uint32_t n,
                                                           DevState* st, uint32_t* total_out) {
    trav_scan_body(counts, offs, n, st, total_out);
}

// Traversal, pass 3: each warp writes its tile's leaves in Z-order, 32
// consecutive groups per round (lane t takes group 32r + t), so the stores
// of a round are contiguous.  With `act`, only the processed tiles.
__device__ __forceinline__ void trav_write_body(const uint32_t* __restrict__ Sb, const uint32_t* __restrict__ coffs,
                                                uint32_t* __restrict__ leaves, int L, int kt, uint32_t ntiles,
                                                const DevState* st, Blk B, const uint8_t* act) {
    if (!st->active) return;
    __shared__ TileBits tbs[kTilesPerCta];
    __shared__ uint32_t wsum[kTilesPerCta];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const uint32_t tile = B.id * kTilesPerCta + warp;
    const bool on = tile < ntiles && (act == nullptr || act[tile] != 0);
    uint32_t total = 0u;
    if (on) {
        TileBits& tb = tbs[warp];
        warp_tile_bits(Sb, L, kt, tile, tb);
        int lv[kGroupsPerLane];
        total = warp_sum(lane_heads(tb, L, kt, tile, lv));
    }
    if (lane == 0) wsum[warp] = total;
    __syncthreads();
    if (!on) return;
    const TileBits& tb = tbs[warp];
    uint32_t base = __ldg(coffs + B.id);
    for (uint32_t w = 0; w < warp; ++w) base += wsum[w];
    const uint32_t ngroups = 1u << (2 * (kt - 1));
    for (uint32_t r = 0; r * 32u < ngroups; ++r) {
        const uint32_t g = r * 32u + lane;
        int l = L;
        uint32_t c = 0u;
        const uint32_t m0 = (tile << (2 * kt)) + 4u * g;
        if (g < ngroups) {
            l = group_level(tb, L, kt, g);
            c = l == L ? 4u : ((m0 & ((1u << (2 * (L - l))) - 1u)) == 0u ? 1u : 0u);
        }
        const uint32_t pos = base + warp_excl(c);
        if (c == 4u) {
            Vec4<uint32_t>::store_u(leaves + pos, ((uint32_t)L << kLeafShift) | m0);
        } else if (c == 1u) {
            leaves[pos] = ((uint32_t)l << kLeafShift) | (m0 >> (2 * (L - l)));
        }
        base += warp_sum(c);
    }
}
static __global__ void __launch_bounds__(256) k_trav_write(const uint32_t* __restrict__ Sb,
                                                           const uint32_t* __restrict__ coffs,
                                                           uint32_t* __restrict__ leaves, int L, int kt,
                                                           uint32_t ntiles, const DevState* st,
                                                           const uint8_t* act) {
    trav_write_body(Sb, coffs, leaves, L, kt, ntiles, st, this_blk(), act);
}

// Leaf count of every tile when its root cell is significant and its own
// levels hold only the bed's static flags (what a skipped tile holds in the
// plain step): one warp per tile, run once after the bed is flagged.
static __global__ void __launch_bounds__(256) k_static_counts(const uint32_t* __restrict__ Sz, int L, int kt,
                                                              uint32_t ntiles, uint32_t* __restrict__ out) {
    __shared__ TileBits tbs[kTilesPerCta];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const uint32_t tile = blockIdx.x * kTilesPerCta + warp;
    if (tile >= ntiles) return;                  // whole warp
    TileBits& tb = tbs[warp];
    warp_tile_bits(Sz, L, kt, tile, tb);
    if (lane == 0) tb.l0 = L - kt + 1;
    __syncwarp();
    int lv[kGroupsPerLane];
    const uint32_t c = warp_sum(lane_heads(tb, L, kt, tile, lv));
    if (lane == 0) out[tile] = c;
}

// Traversal in one pass (the step's own list; get_leaves lists in Z-order
// with the three kernels above): a warp per tile, a fixed grid striding over
// the tiles.  Per tile: the skip decision, its leaf count into *mall (for a
// skipped tile from scount when given), its decode-list entry, and -- if it
// is processed -- its leaves, appended at a position taken with one atomic
// on st->M.  The list is therefore in Z-order within a tile only; nothing
// downstream depends on the order (every leaf's update is independent and
// the reductions are integer min/max).
__device__ __forceinline__ void trav_fused_body(const uint32_t* __restrict__ Sb, uint32_t* __restrict__ dlist,
                                                uint32_t* __restrict__ leaves, int L, int kt, uint32_t ntiles,
                                                DevState* st, const Quiet& q, const uint32_t* scount) {
    if (!st->active) return;
    __shared__ TileBits tbs[kTilesPerCta];
    __shared__ uint32_t wall[kTilesPerCta];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const int Lr = L - kt;
    const uint32_t cur = st->cur;
    const uint8_t* X = cur ? q.zf[1] : q.zf[0];
    uint8_t* Y = cur ? q.zf[0] : q.zf[1];
    const uint32_t lm = (1u << (2 * Lr)) - 1u;
    uint32_t sum_all = 0u;
    for (uint32_t tile = blockIdx.x * kTilesPerCta + warp; tile < ntiles; tile += gridDim.x * kTilesPerCta) {
        TileBits& tb = tbs[warp];
        __syncwarp();                            // tb reused across tiles
        warp_tile_bits(Sb, L, kt, tile, tb);
        bool skip = false;
        if (X != nullptr) {
            // the seven marks of the decision, one per lane, read together
            const uint32_t xs = tile & kXBits & lm, ys = tile & kYBits & lm;
            bool ok = true;
            if (lane == 0) ok = X[tile] != 0;
            else if (lane == 1) ok = Y[tile] != 0;
            else if (lane == 2) ok = q.inlet[tile] == 0;
            else if (lane == 3) ok = xs == 0u || X[mort_xm(tile)] != 0;
            else if (lane == 4) ok = xs == (kXBits & lm) || X[mort_xp(tile)] != 0;
            else if (lane == 5) ok = ys == 0u || X[mort_ym(tile)] != 0;
            else if (lane == 6) ok = ys == (kYBits & lm) || X[mort_yp(tile)] != 0;
            const uint32_t b = __ballot_sync(0xffffffffu, ok);
            const bool covered = tb.l0 < Lr;
            skip = !covered && (b & 0x7Fu) == 0x7Fu;
            if (lane == 0) {
                q.act[tile] = skip ? 0 : (covered ? kActCovered : kActOwn);
                if (!skip && !covered && (b & 2u)) Y[tile] = 0;     // the step writes into it
            }
        }
        if (skip && scount) {                    // uniform over the warp
            sum_all += tb.l0 == Lr ? 1u : __ldg(scount + tile);
            continue;
        }
        int lv[kGroupsPerLane];
        const uint32_t c = lane_heads(tb, L, kt, tile, lv);
        const uint32_t total = warp_sum(c);
        sum_all += total;
        if (skip) continue;
        bool big = false;
#pragma unroll
        for (int e = 0; e < kGroupsPerLane; ++e) big = big || (lv[e] >= 0 && needs_decode_kernel(lv[e], L));
        if (__any_sync(0xffffffffu, big) && lane == 0) dlist[atomicAdd(&st->ndec, 1u)] = tile;
        uint32_t base = 0u;
        if (lane == 0 && total) base = atomicAdd(&st->M, total);
        base = __shfl_sync(0xffffffffu, base, 0);
        const uint32_t ngroups = 1u << (2 * (kt - 1));
        for (uint32_t r = 0; r * 32u < ngroups; ++r) {
            const uint32_t g = r * 32u + lane;
            int l = L;
            uint32_t cc = 0u;
            const uint32_t m0 = (tile << (2 * kt)) + 4u * g;
            if (g < ngroups) {
                l = group_level(tb, L, kt, g);
                cc = l == L ? 4u : ((m0 & ((1u << (2 * (L - l))) - 1u)) == 0u ? 1u : 0u);
            }
            const uint32_t pos = base + warp_excl(cc);
            if (cc == 4u) {
                Vec4<uint32_t>::store_u(leaves + pos, ((uint32_t)L << kLeafShift) | m0);
            } else if (cc == 1u) {
                leaves[pos] = ((uint32_t)l << kLeafShift) | (m0 >> (2 * (L - l)));
            }
            base += warp_sum(cc);
        }
    }
    if (lane == 0) wall[warp] = sum_all;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0u;
        for (int w = 0; w < kTilesPerCta; ++w) s += wall[w];
        if (s) atomicAdd(&st->Mall, s);
    }
}
static __global__ void __launch_bounds__(256) k_trav_fused(const uint32_t* __restrict__ Sb,
                                                           uint32_t* __restrict__ dlist,
                                                           uint32_t* __restrict__ leaves, int L, int kt,
                                                           uint32_t ntiles, DevState* st, Quiet q,
                                                           const uint32_t* scount) {
    pdl_wait();
    trav_fused_body(Sb, dlist, leaves, L, kt, ntiles, st, q, scount);
}

// The traversal in two launches, for quiescent tiles: k_trav_classify
// decides every tile with one thread (its root path and marks loaded at
// once), counts a skipped tile from scount, and lists the others for
// k_trav_list, which treats them one warp per tile as k_trav_fused does.
// A list entry with bit 31 set is a skipped tile that is only counted (no
// scount: the learned look-ahead's flags).
static __global__ void __launch_bounds__(256) k_trav_classify(SigSrc Sb, int L, int kt,
                                                              uint32_t ntiles, DevState* st, Quiet q,
                                                              const uint32_t* scount, uint32_t* work) {
    pdl_wait();
    if (!st->active) return;
    const int Lr = L - kt;
    const uint32_t cur = st->cur;
    const uint8_t* X = cur ? q.zf[1] : q.zf[0];
    uint8_t* Y = cur ? q.zf[0] : q.zf[1];
    const uint32_t lm = (1u << (2 * Lr)) - 1u;
    uint32_t counted = 0u;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x) {
        // first insignificant cell on the root path (levels 0..Lr), else Lr+1
        const uint32_t rb = root_bits(Sb, Lr, t);
        const uint32_t zmask = ~rb & ((2u << Lr) - 1u);
        const int l0 = zmask ? (__ffs(zmask) - 1) : Lr + 1;
        const bool covered = l0 < Lr;
        const uint32_t xs = t & kXBits & lm, ys = t & kYBits & lm;
        const bool xw = xs == 0u || X[mort_xm(t)], xe = xs == (kXBits & lm) || X[mort_xp(t)];
        const bool ysn = ys == 0u || X[mort_ym(t)], yn = ys == (kYBits & lm) || X[mort_yp(t)];
        const bool yset = Y[t] != 0;
        const bool skip = !covered && X[t] && yset && !q.inlet[t] && xw && xe && ysn && yn;
        q.act[t] = skip ? 0 : (covered ? kActCovered : kActOwn);
        if (!skip && !covered && yset) Y[t] = 0;          // the step writes into it
        if (skip && scount) {
            counted += l0 == Lr ? 1u : __ldg(scount + t);
        } else {
            // warp-aggregated append to the work list
            const uint32_t m = __activemask();
            const uint32_t lane = threadIdx.x & 31u, leader = __ffs(m) - 1u;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(&st->nact, (uint32_t)__popc(m));
            base = __shfl_sync(m, base, leader);
            work[base + __popc(m & ((1u << lane) - 1u))] = t | (skip ? 0x80000000u : 0u);
        }
    }
    // leaves of the skipped tiles: one atomic per block
    __shared__ uint32_t red[8];
    uint32_t v = warp_sum(counted);
    if ((threadIdx.x & 31u) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0u;
        for (uint32_t w = 0; w < blockDim.x / 32u; ++w) s += red[w];
        if (s) atomicAdd(&st->Mall, s);
    }
}

// One CTA per listed tile, one thread per 4-cell group: its leaf count, a
// block scan for the positions, one atomic on st->M for the tile's base.
static __global__ void __launch_bounds__(256) k_trav_list(SigSrc Sb,
                                                          uint32_t* __restrict__ dlist,
                                                          uint32_t* __restrict__ leaves, int L, int kt,
                                                          DevState* st, const uint32_t* __restrict__ work) {
    pdl_wait();
    if (!st->active) return;
    __shared__ TileBits tb;
    __shared__ uint32_t sbase;
    const uint32_t nact = st->nact;
    const uint32_t g = threadIdx.x;
    const uint32_t ngroups = 1u << (2 * (kt - 1));
    uint32_t sum_all = 0u;                        // thread 0's running count
    for (uint32_t e = blockIdx.x; e < nact; e += gridDim.x) {
        const uint32_t item = __ldg(work + e);
        const uint32_t tile = item & 0x7FFFFFFFu;
        const bool count_only = (item >> 31) != 0u;
        __syncthreads();                          // tb and sbase reused across tiles
        load_tile_bits(Sb, L, kt, tile, tb);
        int l = L;
        uint32_t c = 0u;
        const uint32_t m0 = (tile << (2 * kt)) + 4u * g;
        if (g < ngroups) {
            l = group_level(tb, L, kt, g);
            c = l == L ? 4u : ((m0 & ((1u << (2 * (L - l))) - 1u)) == 0u ? 1u : 0u);
        }
        const bool big = g < ngroups && needs_decode_kernel(l, L);
        uint32_t total;
        const uint32_t pos = block_excl_scan(c, &total);
        const int anybig = __syncthreads_or(big ? 1 : 0);
        if (threadIdx.x == 0) {
            sum_all += total;
            if (!count_only) {
                sbase = total ? atomicAdd(&st->M, total) : 0u;
                if (anybig) dlist[atomicAdd(&st->ndec, 1u)] = tile;
            }
        }
        if (count_only) continue;                 // uniform over the CTA
        __syncthreads();
        const uint32_t p = sbase + pos;
        if (c == 4u) {
            Vec4<uint32_t>::store_u(leaves + p, ((uint32_t)L << kLeafShift) | m0);
        } else if (c == 1u) {
            leaves[p] = ((uint32_t)l << kLeafShift) | (m0 >> (2 * (L - l)));
        }
    }
    if (threadIdx.x == 0 && sum_all) atomicAdd(&st->Mall, sum_all);
}

// ---------------------------------------------------------------------------
// FV1 update of one cell (Eq. 1-2; the L_c reading: hydrostatic
// reconstruction, HLL, Audusse bed source, Manning friction)
// ---------------------------------------------------------------------------
template <typename T>
struct Cell { T h, qx, qy, z; };

template <typename T>
struct Phys {
    T g, tol, nM, cfl, dxL, dyL;
    T hg;                    // g / 2 (exact): the first product of every g h^2 / 2
};

template <typename T>
__device__ __forceinline__ void velocity(const Cell<T>& c, T tol, T& u, T& v) {
    if (ge_nonneg(c.h, tol)) {                         // h >= tol (tol > 0)
        const T rh = T(1) / c.h;
        u = c.qx * rh;
        v = c.qy * rh;
    } else {
        u = T(0);
        v = T(0);
    }
}

// HLL flux across a face with normal from L to R; F = (mass, normal
// momentum, tangential momentum), hLs/hRs the reconstructed depths.
//
// Every comparison, selection and power-of-two scaling below is done on the
// bit patterns (is_zero, ge_nonneg, sel_min/sel_max, ge_zero/le_zero,
// half/quarter/twice): the same results as the IEEE operations the oracle
// performs, without occupying the FP64 pipe.
template <typename T>
__device__ __forceinline__ void hll_face(T g, T hg, T tol, T hL, T zL, T unL, T utL, T hR, T zR, T unR,
                                         T utR, T F[3], T& hLs_o, T& hRs_o) {
    const T zf = sel_max(zR, zL);                       // zL > zR ? zL : zR
    // on a +0 bed both sides are exact: (h + 0) - 0 = h for h != -0, and a
    // -0 depth gives +0 where the shortcut gives -0, both below tol
    const bool bed0 = pos_zero(zL) && pos_zero(zR);
    const T dL = bed0 ? hL : (hL + zL) - zf;
    const T dR = bed0 ? hR : (hR + zR) - zf;
    const T hLs = ge_nonneg(dL, tol) ? dL : T(0);        // tol > 0
    const T hRs = ge_nonneg(dR, tol) ? dR : T(0);
    hLs_o = hLs;
    hRs_o = hRs;
    if (is_zero(hLs) && is_zero(hRs)) {
        F[0] = F[1] = F[2] = T(0);
        return;
    }
    const T aL = sqrt(g * hLs), aR = sqrt(g * hRs);
    T SL, SR;
    if (!is_zero(hLs) && !is_zero(hRs)) {
        const T us = half(unL + unR) + aL - aR;
        const T as = half(aL + aR) + quarter(unL - unR);
        const T a1 = unL - aL, a2 = us - as;
        const T b1 = unR + aR, b2 = us + as;
        SL = sel_min(a1, a2);
        SR = sel_max(b1, b2);
    } else if (is_zero(hLs)) {
        SL = unR - twice(aR);
        SR = unR + aR;
    } else {
        SL = unL - aL;
        SR = unL + twice(aL);
    }
    const T qnL = hLs * unL, qtL = hLs * utL;
    const T qnR = hRs * unR, qtR = hRs * utR;
    const T FL0 = qnL, FL1 = qnL * unL + hg * hLs * hLs, FL2 = qnL * utL;
    const T FR0 = qnR, FR1 = qnR * unR + hg * hRs * hRs, FR2 = qnR * utR;
    if (ge_zero(SL)) {
        F[0] = FL0; F[1] = FL1; F[2] = FL2;
    } else if (le_zero(SR)) {
        F[0] = FR0; F[1] = FR1; F[2] = FR2;
    } else {
        const T inv = T(1) / (SR - SL);
        F[0] = (SR * FL0 - SL * FR0 + SL * SR * (hRs - hLs)) * inv;
        F[1] = (SR * FL1 - SL * FR1 + SL * SR * (qnR - qnL)) * inv;
        F[2] = (SR * FL2 - SL * FR2 + SL * SR * (qtR - qtL)) * inv;
    }
}

template <typename T>
__device__ __forceinline__ void cell_update_faces(const Phys<T>& P, T rx, T ry, T fk, const Cell<T>& C,
                                                  const T FW[3], const T FE[3], const T GS[3], const T GN[3],
                                                  T hW_R, T hE_L, T hS_R, T hN_L, bool inlet, T dh, T out[3],
                                                  T* rh_out = nullptr);

// New (h, qx, qy) of a cell of size dx x dy: rx = dt/dx, ry = dt/dy.
template <typename T>
__device__ __forceinline__ void cell_update(const Phys<T>& P, T rx, T ry, T fk, const Cell<T>& C,
                                            const Cell<T>& W, const Cell<T>& E, const Cell<T>& S,
                                            const Cell<T>& N, bool inlet, T dh, T out[3]) {
    const T g = P.g, hg = P.hg, tol = P.tol;
    T FW[3], FE[3], GS[3], GN[3];
    T hW_R, hE_L, hS_R, hN_L, dummy;
    if (is_zero(C.h) && is_zero(W.h) && is_zero(E.h) && is_zero(S.h) && is_zero(N.h)) {
        // all five cells dry with zero depth: every reconstructed depth is 0
        // and every face flux is 0 (what the general path computes)
#pragma unroll
        for (int k = 0; k < 3; ++k) FW[k] = FE[k] = GS[k] = GN[k] = T(0);
        hW_R = hE_L = hS_R = hN_L = T(0);
    } else {
        T uC, vC, uW, vW, uE, vE, uS, vS, uN, vN;
        velocity(C, tol, uC, vC);
        velocity(W, tol, uW, vW);
        velocity(E, tol, uE, vE);
        velocity(S, tol, uS, vS);
        velocity(N, tol, uN, vN);
        hll_face(g, hg, tol, W.h, W.z, uW, vW, C.h, C.z, uC, vC, FW, dummy, hW_R);
        hll_face(g, hg, tol, C.h, C.z, uC, vC, E.h, E.z, uE, vE, FE, hE_L, dummy);
        hll_face(g, hg, tol, S.h, S.z, vS, uS, C.h, C.z, vC, uC, GS, dummy, hS_R);
        hll_face(g, hg, tol, C.h, C.z, vC, uC, N.h, N.z, vN, uN, GN, hN_L, dummy);
    }
    cell_update_faces(P, rx, ry, fk, C, FW, FE, GS, GN, hW_R, hE_L, hS_R, hN_L, inlet, dh, out);
}

// The friction term's per-step factor ((dt * g) * n) * n (formed once per
// step by the finish, in the arithmetic of T).
template <typename T> __device__ __forceinline__ T fric_k_of(const DevState* st);
template <> __device__ __forceinline__ double fric_k_of<double>(const DevState* st) { return st->fric_k; }
template <> __device__ __forceinline__ float fric_k_of<float>(const DevState* st) { return st->fric_kf; }

// h^(-1/3) of a double h whose float truncation is a normal number: the
// float inverse cube root as the seed, then one Newton step for
// f(r) = r^-3 - h, r <- r + r (1 - h r^3) / 3, which squares the seed's
// relative error (below 2^-21) up to a factor 2: about 2^-41 in all, where
// the double cube root and a division cost some 20 FP64 additions' worth of
// the FP64 pipe.  Not correctly rounded; the friction term is the one use.
__device__ __forceinline__ double rcbrt_newton(float hf, double h) {
    const float rf = rcbrtf(hf);
    // the float widened to a double by integer operations (exact)
    const uint32_t b = (uint32_t)__float_as_int(rf);
    const long long e = (long long)((b >> 23) & 0xFFu) - 127 + 1023;
    const double r = dval((e << 52) | ((long long)(b & 0x7FFFFFu) << 29));
    const double r3 = (r * r) * r;
    const double d = __fma_rn(-h, r3, 1.0);
    return __fma_rn(r * d, 1.0 / 3.0, r);
}

// x / (h cbrt(h)) = x h^(-4/3) of Manning's friction term for a wet cell
// (h >= tol > 0, rh = 1/h).  float64: x (1/h) h^(-1/3) with the Newton
// inverse cube root, within some 2^-40 relative of the quotient as written
// (the friction factor 1 + this term then within 2^-40 (D - 1)/D); outside
// the float range the quotient as written.  float32: the quotient as written.
__device__ __forceinline__ double friction_term(double x, double h, double rh) {
    const float hf = trunc_float(h);
    const uint32_t eb = ((uint32_t)__float_as_int(hf) >> 23) & 0xFFu;
    if (eb != 0u && eb != 0xFFu) return (x * rh) * rcbrt_newton(hf, h);
    return x / (h * cbrt(h));
}
__device__ __forceinline__ float friction_term(float x, float h, float /*rh*/) { return x / (h * cbrtf(h)); }

// The update from the four face fluxes and the squares of the cell's own
// reconstructed depths at them (hW2, hE2, hS2, hN2: the bed source term's
// face values).  rh_out (if given) receives 1/h of the new depth when the
// friction step formed it, else 0.
template <typename T>
__device__ __forceinline__ void cell_update_faces_sq(const Phys<T>& P, T rx, T ry, T fk, const Cell<T>& C,
                                                     const T FW[3], const T FE[3], const T GS[3], const T GN[3],
                                                     T hW2, T hE2, T hS2, T hN2, bool inlet, T dh, T out[3],
                                                     T* rh_out = nullptr) {
    if (rh_out) *rh_out = T(0);
    const T hg = P.hg, tol = P.tol;
    const T bx = hg * (hW2 - hE2);
    const T by = hg * (hS2 - hN2);
    T h = C.h - rx * (FE[0] - FW[0]) - ry * (GN[0] - GS[0]);
    T qx = C.qx - rx * ((FE[1] - FW[1]) + bx) - ry * (GN[2] - GS[2]);
    T qy = C.qy - rx * (FE[2] - FW[2]) - ry * ((GN[1] - GS[1]) + by);
    if (inlet) h = h + dh;
    h = gt_zero(h) ? h : T(0);
    if (!ge_nonneg(h, tol)) {                           // h < tol (tol > 0)
        qx = T(0);
        qy = T(0);
    } else if (P.nM > T(0)) {
        const T rh = T(1) / h;
        if (rh_out) *rh_out = rh;
        const T u = qx * rh, v = qy * rh;
        const T speed = sqrt(u * u + v * v);
        const T D = T(1) + friction_term(fk * speed, h, rh);
        const T rD = T(1) / D;
        qx = qx * rD;
        qy = qy * rD;
    }
    out[0] = h;
    out[1] = qx;
    out[2] = qy;
}

// The update of cell_update from its four face fluxes and its own
// reconstructed depths at them (hW_R, hE_L, hS_R, hN_L).
template <typename T>
__device__ __forceinline__ void cell_update_faces(const Phys<T>& P, T rx, T ry, T fk, const Cell<T>& C,
                                                  const T FW[3], const T FE[3], const T GS[3], const T GN[3],
                                                  T hW_R, T hE_L, T hS_R, T hN_L, bool inlet, T dh, T out[3],
                                                  T* rh_out) {
    cell_update_faces_sq(P, rx, ry, fk, C, FW, FE, GS, GN, hW_R * hW_R, hE_L * hE_L, hS_R * hS_R, hN_L * hN_L,
                         inlet, dh, out, rh_out);
}

// CFL bound of an updated cell: min(dx/(|u|+a), dy/(|v|+a)), +inf if dry
template <typename T>
__device__ __forceinline__ T cfl_bound(const Phys<T>& P, T h, T qx, T qy) {
    if (!ge_nonneg(h, P.tol)) return T(INFINITY);      // h < tol (tol > 0)
    const T rh = T(1) / h;
    const T u = absval(qx * rh), v = absval(qy * rh);
    const T a = sqrt(P.g * h);
    const T rx = P.dxL / (u + a), ry = P.dyL / (v + a);
    return sel_min(rx, ry);
}

template <typename T>
struct StepArgs {
    T* f[2][3];              // h, qx, qy hierarchies of the two state buffers
    const T* z;              // bed hierarchy
    const uint32_t* leaves;
    uint32_t* wet;           // packed leaves that need the full update
    DevState* st;
    Phys<T> P;
    T lx, ly;
    int L;
    int bc_ref[4];           // 1: the side reflects (closed or inflow)
    int inflow_side;         // -1: none
    int a0, a1;
    // shared faces (k_fv1_faces / k_fv1_update): 12 arrays of fcap values
    // (east face F0..F2, h*_L, h*_R, then the north face's, then the
    // leaf's velocities u, v, written by k_fv1_dry), and a stamp per
    // hierarchy cell ((epoch + 1) << 32 | queue slot)
    T* face = nullptr;
    uint32_t fcap = 0;
    unsigned long long* mark = nullptr;
    // matched fluxes at resolution changes (k_fv1_match): the regularised
    // significance bits, which tell a refined same-level neighbour
    const uint32_t* Sb = nullptr;
    int fm = 0;
    // 1: every leaf writes its own cell only (the learned skip's decode
    // kernel forms the stored cells below coarser leaves)
    int own_slot = 0;
};

template <typename T>
struct CellSrc { const T *h, *qx, *qy, *z; };

template <typename T>
__device__ __forceinline__ Cell<T> fetch(const CellSrc<T>& a, uint64_t idx) {
    Cell<T> c;
    c.h = __ldg(a.h + idx);
    c.qx = __ldg(a.qx + idx);
    c.qy = __ldg(a.qy + idx);
    c.z = __ldg(a.z + idx);
    return c;
}

template <typename T>
__device__ __forceinline__ Cell<T> ghost(const Cell<T>& c, bool reflect, bool xside) {
    Cell<T> g = c;
    if (reflect) {
        if (xside) g.qx = -g.qx;
        else g.qy = -g.qy;
    }
    return g;
}

// Inlet test of leaf (n, i, j): whether it touches the inflow range, and
// the covered range of finest cells.
template <typename T>
__device__ __forceinline__ bool inlet_range(const StepArgs<T>& a, int n, uint32_t i, uint32_t j,
                                            uint32_t last, int64_t& lo, int64_t& hi) {
    const int s = a.inflow_side;
    if (s < 0) return false;
    const bool touch = (s == 0 && i == 0) || (s == 1 && i == last) || (s == 2 && j == 0) ||
                       (s == 3 && j == last);
    if (!touch) return false;
    const int64_t w = 1ll << (a.L - n);
    const int64_t pos = (s <= 1) ? (int64_t)j : (int64_t)i;
    lo = pos * w;
    hi = lo + w;
    if (lo < a.a0) lo = a.a0;
    if (hi > a.a1) hi = a.a1;
    return hi > lo;
}

template <typename T> __device__ __forceinline__ T rx0_of(const DevState* st);
template <> __device__ __forceinline__ double rx0_of<double>(const DevState* st) { return st->rx0; }
template <> __device__ __forceinline__ float rx0_of<float>(const DevState* st) { return st->rx0f; }
template <typename T> __device__ __forceinline__ T ry0_of(const DevState* st);
template <> __device__ __forceinline__ double ry0_of<double>(const DevState* st) { return st->ry0; }
template <> __device__ __forceinline__ float ry0_of<float>(const DevState* st) { return st->ry0f; }

// FV1, first kernel: every leaf whose own and four same-level neighbour
// depths are exactly zero and that has no inflow gets (+0, +0, +0) -- what
// the full update computes for it (all reconstructed depths and fluxes are
// 0, its CFL bound is infinite) -- decided on the depth bits alone.  Every
// other leaf is queued for k_fv1_wet.  Needs few registers, so many warps
// hide the gather latency.
// Neighbour depth addresses of a leaf from its packed id (Morton-domain
// arithmetic; ghosts read the leaf itself).
struct DryProbe {
    uint64_t iC, iW, iE, iS, iN;
    uint32_t code;
    int n;
};
__device__ __forceinline__ DryProbe dry_probe(uint32_t pk) {
    DryProbe d;
    d.n = (int)(pk >> kLeafShift);
    d.code = pk & kCodeMask;
    const uint64_t base = lvl_off(d.n);
    const uint32_t lm = (1u << (2 * d.n)) - 1u;
    const uint32_t xs = d.code & kXBits & lm, ys = d.code & kYBits;
    d.iC = base + d.code;
    d.iW = xs != 0u ? base + mort_xm(d.code) : d.iC;
    d.iE = xs != (kXBits & lm) ? base + mort_xp(d.code) : d.iC;
    d.iS = ys != 0u ? base + mort_ym(d.code) : d.iC;
    d.iN = ys != (kYBits & lm) ? base + mort_yp(d.code) : d.iC;
    return d;
}

// Whether a same-level neighbour of the leaf is refined (significant after
// the upward closure, so smaller leaves lie behind that face).
__device__ __forceinline__ bool refined_nbr(const uint32_t* __restrict__ Sb, const DryProbe& d, int L) {
    if (d.n >= L) return false;
    const uint64_t base = lvl_off(d.n);
    return (d.iW != d.iC && sig_bit(Sb, d.n, (uint32_t)(d.iW - base))) ||
           (d.iE != d.iC && sig_bit(Sb, d.n, (uint32_t)(d.iE - base))) ||
           (d.iS != d.iC && sig_bit(Sb, d.n, (uint32_t)(d.iS - base))) ||
           (d.iN != d.iC && sig_bit(Sb, d.n, (uint32_t)(d.iN - base)));
}

template <typename T>
__device__ __forceinline__ bool dry5(const T* __restrict__ h, const DryProbe& d) {
    const T a = __ldg(h + d.iC), b = __ldg(h + d.iW), c = __ldg(h + d.iE), e = __ldg(h + d.iS),
            f = __ldg(h + d.iN);
    return is_zero(a) && is_zero(b) && is_zero(c) && is_zero(e) && is_zero(f);
}

// FV1, first kernel: every leaf whose own and four same-level neighbour
// depths are exactly zero and that has no inflow gets (+0, +0, +0) -- what
// the full update computes for it (all reconstructed depths and fluxes are
// 0, its CFL bound is infinite) -- decided on the depth bits alone.  Every
// other leaf is queued for k_fv1_wet.  Few registers and two leaves per
// iteration, so many independent loads are in flight.
template <typename T>
__device__ __forceinline__ void dry_finish(const StepArgs<T>& a, DevState* st, T* oh, T* oqx, T* oqy,
                                           const DryProbe& d, bool dry, uint32_t pk, const CellSrc<T>& src,
                                           unsigned long long stamp) {
    if (dry && a.inflow_side >= 0) {
        int64_t lo, hi;
        dry = !inlet_range(a, d.n, compact16(d.code), compact16(d.code >> 1), (1u << d.n) - 1u, lo, hi);
    }
    if (dry) {
        if (d.n == a.L || needs_decode_kernel(d.n, a.L) || a.own_slot) {
            oh[d.iC] = T(0);
            oqx[d.iC] = T(0);
            oqy[d.iC] = T(0);
        } else {                              // 4 or 16 finest cells: decode here
            const uint64_t fo = lvl_off(a.L) + ((uint64_t)d.code << (2 * (a.L - d.n)));
            const uint32_t cnt = 1u << (2 * (a.L - d.n));
            for (uint32_t e = 0; e < cnt; e += 4) {
                Vec4<T>::store(oh + fo + e, T(0), T(0), T(0), T(0));
                Vec4<T>::store(oqx + fo + e, T(0), T(0), T(0), T(0));
                Vec4<T>::store(oqy + fo + e, T(0), T(0), T(0), T(0));
            }
        }
    } else {
        // warp-aggregated append to the queue of full updates
        const uint32_t m = __activemask();
        const uint32_t lane = threadIdx.x & 31u;
        const uint32_t leader = __ffs(m) - 1u;
        uint32_t base_pos = 0;
        if (lane == leader) base_pos = atomicAdd(&st->nwet, (uint32_t)__popc(m));
        base_pos = __shfl_sync(m, base_pos, leader);
        const uint32_t w = base_pos + __popc(m & ((1u << lane) - 1u));
        a.wet[w] = pk;                                            // the packed leaf
        // float64 with shared faces: the leaf's velocities (the operations
        // of velocity() in k_fv1_faces, which reads them here instead of
        // forming them for the leaf and for the two neighbours whose west
        // and south faces it is) and its stamp, once per queued leaf
        if (sizeof(T) == 8 && a.face != nullptr && !a.fm && w < a.fcap) {
            Cell<T> C;
            C.h = __ldg(src.h + d.iC);
            C.qx = __ldg(src.qx + d.iC);
            C.qy = __ldg(src.qy + d.iC);
            T u, v;
            velocity(C, a.P.tol, u, v);
            a.face[10 * (size_t)a.fcap + w] = u;
            a.face[11 * (size_t)a.fcap + w] = v;
            a.mark[d.iC] = stamp | w;
        }
    }
}

template <typename T>
__device__ __forceinline__ void fv1_dry_body(const StepArgs<T>& a, Blk B) {
    DevState* st = a.st;
    if (!st->active) return;
    const int par = (int)st->cur, nxt = par ^ 1;
    const uint32_t M = st->M;
    const T* __restrict__ hsrc = par ? a.f[1][0] : a.f[0][0];
    CellSrc<T> src;
    src.h = hsrc;
    src.qx = par ? a.f[1][1] : a.f[0][1];
    src.qy = par ? a.f[1][2] : a.f[0][2];
    src.z = a.z;
    const unsigned long long stamp = (unsigned long long)(st->epoch + 1u) << 32;
    T* const oh = nxt ? a.f[1][0] : a.f[0][0];
    T* const oqx = nxt ? a.f[1][1] : a.f[0][1];
    T* const oqy = nxt ? a.f[1][2] : a.f[0][2];
    const uint32_t stride = B.n * blockDim.x;
    for (uint32_t k = B.id * blockDim.x + threadIdx.x; k < M; k += 2u * stride) {
        const uint32_t k2 = k + stride;
        const bool two = k2 < M;
        const uint32_t p1 = __ldg(a.leaves + k), p2 = two ? __ldg(a.leaves + k2) : 0u;
        const DryProbe d1 = dry_probe(p1);
        const DryProbe d2 = dry_probe(p2);
        bool y1 = dry5(hsrc, d1);
        bool y2 = two && dry5(hsrc, d2);
        if (a.fm) {
            // with matched fluxes a face toward a refined neighbour averages
            // finer faces: such a leaf takes the full update
            y1 = y1 && !refined_nbr(a.Sb, d1, a.L);
            y2 = y2 && !refined_nbr(a.Sb, d2, a.L);
        }
        dry_finish(a, st, oh, oqx, oqy, d1, y1, p1, src, stamp);
        if (two) dry_finish(a, st, oh, oqx, oqy, d2, y2, p2, src, stamp);
    }
}
template <typename T>
static __global__ void __launch_bounds__(256) k_fv1_dry(StepArgs<T> a) {
    pdl_wait();
    fv1_dry_body<T>(a, this_blk());
}

// CFL bound, write-back (with the prolongation of leaves of 4 or 16 finest
// cells) and reductions of one updated wet leaf.
template <typename T>
__device__ __forceinline__ void wet_leaf_store(const StepArgs<T>& a, DevState* st, const T* z, T* oh, T* oqx,
                                               T* oqy, int n, uint32_t code, uint64_t iC, const Cell<T>& C,
                                               const T out[3], unsigned long long& rmin, unsigned long long& mh,
                                               unsigned long long& mqx, unsigned long long& mqy,
                                               unsigned long long* spd = nullptr, T rh_known = T(0)) {
    if (sizeof(T) == 8 && spd != nullptr) {
        // float64: the CFL speeds of the leaf (the divisions are formed once
        // per step from their maxima, finish_body); the same operations as
        // cfl_bound up to the division, reusing the friction step's 1/h
        if (ge_nonneg(out[0], a.P.tol)) {
            const T rh = is_zero(rh_known) ? T(1) / out[0] : rh_known;
            const T u = absval(out[1] * rh), v = absval(out[2] * rh);
            const T aa = sqrt(a.P.g * out[0]);
            const unsigned long long bx = abs_obits(u + aa), by = abs_obits(v + aa);
            spd[0] = bx > spd[0] ? bx : spd[0];
            spd[1] = by > spd[1] ? by : spd[1];
        }
    } else {
        const T r = cfl_bound(a.P, out[0], out[1], out[2]);
        const unsigned long long rb = obits((double)r);
        rmin = rb < rmin ? rb : rmin;
    }
    if (n == a.L || needs_decode_kernel(n, a.L) || a.own_slot) {
        oh[iC] = out[0];
        oqx[iC] = out[1];
        oqy[iC] = out[2];
        if (n == a.L) {
            const unsigned long long b0 = abs_obits(out[0]);
            mh = b0 > mh ? b0 : mh;
            const unsigned long long b1 = abs_obits(out[1]);
            mqx = b1 > mqx ? b1 : mqx;
            const unsigned long long b2 = abs_obits(out[2]);
            mqy = b2 > mqy ? b2 : mqy;
        }
    } else {
        // decode-back of a leaf of 4 or 16 finest cells (as k_decode does)
        const uint64_t fo = lvl_off(a.L) + ((uint64_t)code << (2 * (a.L - n)));
        const uint32_t cnt = 1u << (2 * (a.L - n));
        const T hl = out[0];
        const bool restore = ge_nonneg(hl, a.P.tol);
        const T eta = restore ? eta_of(hl, C.z) : T(0);
        for (uint32_t e = 0; e < cnt; e += 4) {
            T hf[4];
            if (restore) {
                T z0, z1, z2, z3;
                Vec4<T>::load(z + fo + e, z0, z1, z2, z3);
                restore4(eta, z0, z1, z2, z3, hf);
            } else {
                hf[0] = hf[1] = hf[2] = hf[3] = hl;
            }
            Vec4<T>::store(oh + fo + e, hf[0], hf[1], hf[2], hf[3]);
            Vec4<T>::store(oqx + fo + e, out[1], out[1], out[1], out[1]);
            Vec4<T>::store(oqy + fo + e, out[2], out[2], out[2], out[2]);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const unsigned long long b = abs_obits(hf[q]);
                mh = b > mh ? b : mh;
            }
        }
        const unsigned long long b1 = abs_obits(out[1]);
        mqx = b1 > mqx ? b1 : mqx;
        const unsigned long long b2 = abs_obits(out[2]);
        mqy = b2 > mqy ? b2 : mqy;
    }
    if (!(finite_bits(out[0]) && finite_bits(out[1]) && finite_bits(out[2])))
        atomicOr(&st->err, kErrNonFinite);
}

// FV1, second kernel: the full update (Eq. 2 with the L_c reading) of every
// queued leaf, with the CFL and s_max reductions.
template <typename T>
__device__ __forceinline__ void fv1_wet_body(const StepArgs<T>& a, Blk B) {
    DevState* st = a.st;
    if (!st->active) return;
    const uint32_t nq = st->nwet;
    if (B.id * blockDim.x >= nq) return;          // whole block idle
    const int par = (int)st->cur, nxt = par ^ 1;
    const T fk = fric_k_of<T>(st);
    const T rx0 = rx0_of<T>(st), ry0 = ry0_of<T>(st);
    const T Qdt = (T)st->Qdt;
    CellSrc<T> src;
    src.h = par ? a.f[1][0] : a.f[0][0];
    src.qx = par ? a.f[1][1] : a.f[0][1];
    src.qy = par ? a.f[1][2] : a.f[0][2];
    src.z = a.z;
    T* const oh = nxt ? a.f[1][0] : a.f[0][0];
    T* const oqx = nxt ? a.f[1][1] : a.f[0][1];
    T* const oqy = nxt ? a.f[1][2] : a.f[0][2];
    unsigned long long rmin = kInfBits, mh = 0, mqx = 0, mqy = 0, spd[2] = {0ull, 0ull};
    for (uint32_t w = B.id * blockDim.x + threadIdx.x; w < nq; w += B.n * blockDim.x) {
        const uint32_t pk = a.wet[w];            // the queue holds packed leaves
        const int n = (int)(pk >> kLeafShift);
        const uint32_t code = pk & kCodeMask;
        const uint32_t i = compact16(code), j = compact16(code >> 1);
        const uint32_t last = (1u << n) - 1u;
        const uint64_t base = lvl_off(n);
        const uint64_t iC = base + code;
        const Cell<T> C = fetch(src, iC);
        const Cell<T> W = i > 0 ? fetch(src, base + morton2(i - 1, j)) : ghost(C, a.bc_ref[0], true);
        const Cell<T> E = i < last ? fetch(src, base + morton2(i + 1, j)) : ghost(C, a.bc_ref[1], true);
        const Cell<T> S = j > 0 ? fetch(src, base + morton2(i, j - 1)) : ghost(C, a.bc_ref[2], false);
        const Cell<T> N = j < last ? fetch(src, base + morton2(i, j + 1)) : ghost(C, a.bc_ref[3], false);
        const T rx = mul_pow2(rx0, n), ry = mul_pow2(ry0, n);   // rx0 * 2^n, exact
        int64_t lo = 0, hi = 0;
        const bool inlet = inlet_range(a, n, i, j, last, lo, hi);
        T dh = T(0);
        if (inlet) {
            const T scale = (T)(1u << n);
            const T frac = (T)(hi - lo) / (T)(a.a1 - a.a0);
            const T inv2n = T(1) / scale;
            const T dxn = a.lx * inv2n, dyn = a.ly * inv2n;
            dh = (Qdt * frac) / (dxn * dyn);
        }
        T out[3];
        cell_update(a.P, rx, ry, fk, C, W, E, S, N, inlet, dh, out);
        wet_leaf_store(a, st, src.z, oh, oqx, oqy, n, code, iC, C, out, rmin, mh, mqx, mqy, spd);
    }
    block_atomic_u64<false>(rmin, &st->rmin_bits);
    block_max3_u64(mh, mqx, mqy, st->max_bits);
    block_max3_u64(spd[0], spd[1], 0ull, st->speed_bits);
}
template <typename T>
static __global__ void __launch_bounds__(256) k_fv1_wet(StepArgs<T> a) {
    pdl_wait();
    fv1_wet_body<T>(a, this_blk());
}

// ---------------------------------------------------------------------------
// Matched fluxes at resolution changes (the conservative variant): a face of
// a leaf whose same-level neighbour is refined takes, for its flux and for
// the square of the leaf's own reconstructed depth, the average
// half(first + second) of its two halves one level finer, recursively, down
// to the half faces whose neighbour cell is not refined; such a half face
// is evaluated between the two same-level cells that touch it -- the call
// the smaller leaf on the other side makes for the same face, so both sides
// carry one flux.
// ---------------------------------------------------------------------------

// One face of a cell seen from the cell: side s (0 W, 1 E, 2 S, 3 N) between
// its state C and the state X across the face.  F in the order of
// cell_update (x faces (h, qx, qy), y faces (h, qy, qx)), own2 the square of
// the cell's own reconstructed depth at the face.
template <typename T>
__device__ __forceinline__ void face_of(const Phys<T>& P, int s, const Cell<T>& C, const Cell<T>& X, T F[3],
                                        T& own2) {
    T uC, vC, uX, vX, hl, hr;
    velocity(C, P.tol, uC, vC);
    velocity(X, P.tol, uX, vX);
    if (s == 0) {
        hll_face(P.g, P.hg, P.tol, X.h, X.z, uX, vX, C.h, C.z, uC, vC, F, hl, hr);
        own2 = hr * hr;
    } else if (s == 1) {
        hll_face(P.g, P.hg, P.tol, C.h, C.z, uC, vC, X.h, X.z, uX, vX, F, hl, hr);
        own2 = hl * hl;
    } else if (s == 2) {
        hll_face(P.g, P.hg, P.tol, X.h, X.z, vX, uX, C.h, C.z, vC, uC, F, hl, hr);
        own2 = hr * hr;
    } else {
        hll_face(P.g, P.hg, P.tol, C.h, C.z, vC, uC, X.h, X.z, vX, uX, F, hl, hr);
        own2 = hl * hl;
    }
}

// The face on side s of the leaf (n, i, j) whose same-level neighbour is
// refined.  Depth first over the halves (first half: lower j on x faces,
// lower i on y faces): half r of level m lies between the own-side cell and
// the neighbour cell of level m that touch it; a finished second half is
// averaged with the pending first half of its level, one level up, until
// the face itself is reached.  The walk visits each half face of the finite
// tree once.
template <typename T>
__device__ __noinline__ void matched_face(const StepArgs<T>& a, const CellSrc<T>& src, int s, int n, uint32_t i,
                                          uint32_t j, T F[3], T& own2) {
    T pend[kMaxL][4];                     // pending first halves, by level - n - 1
    int m = n + 1;
    uint32_t r = 0u;
    for (;;) {
        const bool xf = s <= 1;
        uint32_t oi, oj, ni, nj;
        for (;;) {
            const int k = m - n;
            if (xf) {
                oi = s == 0 ? (i << k) : ((i + 1u) << k) - 1u;
                ni = s == 0 ? (i << k) - 1u : ((i + 1u) << k);
                oj = nj = (j << k) + r;
            } else {
                oj = s == 2 ? (j << k) : ((j + 1u) << k) - 1u;
                nj = s == 2 ? (j << k) - 1u : ((j + 1u) << k);
                oi = ni = (i << k) + r;
            }
            if (m >= a.L || !sig_bit(a.Sb, m, morton2(ni, nj))) break;
            ++m;                                  // the neighbour cell is refined: split
            r <<= 1;
        }
        const uint64_t base = lvl_off(m);
        T v[4];
        face_of(a.P, s, fetch(src, base + morton2(oi, oj)), fetch(src, base + morton2(ni, nj)), v, v[3]);
        while (r & 1u) {                          // a second half: close its pair
            const T* p = pend[m - n - 1];
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = half(p[q] + v[q]);
            --m;
            r >>= 1;
        }
        if (m == n) {
            F[0] = v[0];
            F[1] = v[1];
            F[2] = v[2];
            own2 = v[3];
            return;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) pend[m - n - 1][q] = v[q];
        r += 1u;                                  // on to its second half
    }
}

// One face of a queued leaf: the ghost at the domain edge, the matched face
// toward a refined neighbour, else the same-level neighbour.
template <typename T>
__device__ __forceinline__ void leaf_face(const StepArgs<T>& a, const CellSrc<T>& src, int s, int n, uint32_t i,
                                          uint32_t j, uint32_t last, const Cell<T>& C, T F[3], T& own2) {
    const bool edge = (s == 0 && i == 0u) || (s == 1 && i == last) || (s == 2 && j == 0u) ||
                      (s == 3 && j == last);
    if (edge) {
        face_of(a.P, s, C, ghost(C, a.bc_ref[s], s <= 1), F, own2);
        return;
    }
    const uint32_t ni = s == 0 ? i - 1u : (s == 1 ? i + 1u : i);
    const uint32_t nj = s == 2 ? j - 1u : (s == 3 ? j + 1u : j);
    const uint32_t nc = morton2(ni, nj);
    if (n < a.L && sig_bit(a.Sb, n, nc)) {
        matched_face(a, src, s, n, i, j, F, own2);
        return;
    }
    face_of(a.P, s, C, fetch(src, lvl_off(n) + nc), F, own2);
}

// FV1 with matched fluxes: the full update of every queued leaf.
template <typename T>
__device__ __forceinline__ void fv1_match_body(const StepArgs<T>& a, Blk B) {
    DevState* st = a.st;
    if (!st->active) return;
    const uint32_t nq = st->nwet;
    if (B.id * blockDim.x >= nq) return;          // whole block idle
    const int par = (int)st->cur, nxt = par ^ 1;
    const T fk = fric_k_of<T>(st);
    const T rx0 = rx0_of<T>(st), ry0 = ry0_of<T>(st);
    const T Qdt = (T)st->Qdt;
    CellSrc<T> src;
    src.h = par ? a.f[1][0] : a.f[0][0];
    src.qx = par ? a.f[1][1] : a.f[0][1];
    src.qy = par ? a.f[1][2] : a.f[0][2];
    src.z = a.z;
    T* const oh = nxt ? a.f[1][0] : a.f[0][0];
    T* const oqx = nxt ? a.f[1][1] : a.f[0][1];
    T* const oqy = nxt ? a.f[1][2] : a.f[0][2];
    unsigned long long rmin = kInfBits, mh = 0, mqx = 0, mqy = 0, spd[2] = {0ull, 0ull};
    for (uint32_t w = B.id * blockDim.x + threadIdx.x; w < nq; w += B.n * blockDim.x) {
        const uint32_t pk = a.wet[w];
        const int n = (int)(pk >> kLeafShift);
        const uint32_t code = pk & kCodeMask;
        const uint32_t i = compact16(code), j = compact16(code >> 1);
        const uint32_t last = (1u << n) - 1u;
        const uint64_t iC = lvl_off(n) + code;
        const Cell<T> C = fetch(src, iC);
        T FW[3], FE[3], GS[3], GN[3], w2, e2, s2, n2;
        leaf_face(a, src, 0, n, i, j, last, C, FW, w2);
        leaf_face(a, src, 1, n, i, j, last, C, FE, e2);
        leaf_face(a, src, 2, n, i, j, last, C, GS, s2);
        leaf_face(a, src, 3, n, i, j, last, C, GN, n2);
        const T rx = mul_pow2(rx0, n), ry = mul_pow2(ry0, n);   // rx0 * 2^n, exact
        int64_t lo = 0, hi = 0;
        const bool inlet = inlet_range(a, n, i, j, last, lo, hi);
        T dh = T(0);
        if (inlet) {
            const T scale = (T)(1u << n);
            const T frac = (T)(hi - lo) / (T)(a.a1 - a.a0);
            const T inv2n = T(1) / scale;
            const T dxn = a.lx * inv2n, dyn = a.ly * inv2n;
            dh = (Qdt * frac) / (dxn * dyn);
        }
        T out[3], rh;
        cell_update_faces_sq(a.P, rx, ry, fk, C, FW, FE, GS, GN, w2, e2, s2, n2, inlet, dh, out, &rh);
        wet_leaf_store(a, st, src.z, oh, oqx, oqy, n, code, iC, C, out, rmin, mh, mqx, mqy, spd, rh);
    }
    block_atomic_u64<false>(rmin, &st->rmin_bits);
    block_max3_u64(mh, mqx, mqy, st->max_bits);
    block_max3_u64(spd[0], spd[1], 0ull, st->speed_bits);
}
template <typename T>
static __global__ void __launch_bounds__(256) k_fv1_match(StepArgs<T> a) {
    pdl_wait();
    fv1_match_body<T>(a, this_blk());
}

// The same update in two kernels that compute every face between two queued
// leaves of one level once.  Phase 1: each queued leaf computes its east and
// north faces (it is their left side) and stamps its cell.  Phase 2: a
// queued leaf whose west (south) same-level neighbour carries this step's
// stamp takes that neighbour's east (north) face -- the same call with the
// same operands, so the same bits -- and computes only its other faces.
// The velocities k_fv1_dry formed for the queued leaf at hierarchy index
// idx, if that cell holds one this step (its stamp is this step's).
template <typename T>
__device__ __forceinline__ bool queued_velocity(const StepArgs<T>& a, unsigned long long stamp, uint64_t idx,
                                                T& u, T& v) {
    const unsigned long long m = __ldg(a.mark + idx);
    if ((m >> 32) != (stamp >> 32)) return false;
    const uint32_t wn = (uint32_t)m;
    u = a.face[10 * (size_t)a.fcap + wn];
    v = a.face[11 * (size_t)a.fcap + wn];
    return true;
}

template <typename T, bool FM = false>
__device__ __forceinline__ void fv1_faces_body(const StepArgs<T>& a, Blk B) {
    DevState* st = a.st;
    if (!st->active) return;
    const uint32_t nq = st->nwet;
    if (nq > a.fcap || B.id * blockDim.x >= nq) return;
    const int par = (int)st->cur;
    CellSrc<T> src;
    src.h = par ? a.f[1][0] : a.f[0][0];
    src.qx = par ? a.f[1][1] : a.f[0][1];
    src.qy = par ? a.f[1][2] : a.f[0][2];
    src.z = a.z;
    const T g = a.P.g, hg = a.P.hg, tol = a.P.tol;
    const unsigned long long stamp = (unsigned long long)(st->epoch + 1u) << 32;
    const uint32_t cap = a.fcap;
    for (uint32_t w = B.id * blockDim.x + threadIdx.x; w < nq; w += B.n * blockDim.x) {
        const uint32_t pk = a.wet[w];
        const int n = (int)(pk >> kLeafShift);
        const uint32_t code = pk & kCodeMask;
        const uint32_t i = compact16(code), j = compact16(code >> 1);
        const uint32_t last = (1u << n) - 1u;
        const uint64_t base = lvl_off(n);
        const uint64_t iC = base + code;
        const Cell<T> C = fetch(src, iC);
        T FE[3], GN[3], hEL2, hER2 = T(0), hNL2, hNR2 = T(0);
        // with matched fluxes, a face toward a refined neighbour is the walk
        // over its finer halves (its other side belongs to no leaf)
        const bool mE = FM && i < last && n < a.L && sig_bit(a.Sb, n, morton2(i + 1, j));
        const bool mN = FM && j < last && n < a.L && sig_bit(a.Sb, n, morton2(i, j + 1));
        if (FM && (mE || mN)) {
            if (mE) matched_face(a, src, 1, n, i, j, FE, hEL2);
            if (mN) matched_face(a, src, 3, n, i, j, GN, hNL2);
        }
        if (!(mE && mN)) {
            const Cell<T> E = i < last ? fetch(src, base + morton2(i + 1, j)) : ghost(C, a.bc_ref[1], true);
            const Cell<T> N = j < last ? fetch(src, base + morton2(i, j + 1)) : ghost(C, a.bc_ref[3], false);
            T uC, vC, uE, vE, uN, vN;
            // velocities formed by k_fv1_dry for every queued leaf (the
            // leaf's own, and a same-level neighbour's when it is queued:
            // its stamp is this step's), else formed here
            if (!FM) {
                uC = a.face[10 * (size_t)cap + w];
                vC = a.face[11 * (size_t)cap + w];
            } else {
                velocity(C, tol, uC, vC);
            }
            if (!mE) {
                if (!(!FM && i < last && queued_velocity(a, stamp, base + morton2(i + 1, j), uE, vE)))
                    velocity(E, tol, uE, vE);
                T hEL, hER;
                hll_face(g, hg, tol, C.h, C.z, uC, vC, E.h, E.z, uE, vE, FE, hEL, hER);
                hEL2 = hEL * hEL;
                hER2 = hER * hER;
            }
            if (!mN) {
                if (!(!FM && j < last && queued_velocity(a, stamp, base + morton2(i, j + 1), uN, vN)))
                    velocity(N, tol, uN, vN);
                T hNL, hNR;
                hll_face(g, hg, tol, C.h, C.z, vC, uC, N.h, N.z, vN, uN, GN, hNL, hNR);
                hNL2 = hNL * hNL;
                hNR2 = hNR * hNR;
            }
        }
        // the face of both sides: flux, then the squares of the two
        // reconstructed depths (the bed source terms of the two cells)
        T* f = a.face + w;
        f[0 * (size_t)cap] = FE[0];
        f[1 * (size_t)cap] = FE[1];
        f[2 * (size_t)cap] = FE[2];
        f[3 * (size_t)cap] = hEL2;
        f[4 * (size_t)cap] = hER2;
        f[5 * (size_t)cap] = GN[0];
        f[6 * (size_t)cap] = GN[1];
        f[7 * (size_t)cap] = GN[2];
        f[8 * (size_t)cap] = hNL2;
        f[9 * (size_t)cap] = hNR2;
        if (FM) a.mark[iC] = stamp | w;      // (k_fv1_dry stamped the leaf otherwise)
    }
}
template <typename T, bool FM = false>
static __global__ void __launch_bounds__(256) k_fv1_faces(StepArgs<T> a) {
    pdl_wait();
    fv1_faces_body<T, FM>(a, this_blk());
}

template <typename T, bool FM = false>
__device__ __forceinline__ void fv1_update_body(const StepArgs<T>& a, Blk B) {
    DevState* st = a.st;
    if (!st->active) return;
    const uint32_t nq = st->nwet;
    if (nq > a.fcap) {                            // no room for the faces: one pass
        if (FM) fv1_match_body<T>(a, B);
        else fv1_wet_body<T>(a, B);
        return;
    }
    if (B.id * blockDim.x >= nq) return;          // whole block idle
    const int par = (int)st->cur, nxt = par ^ 1;
    const T fk = fric_k_of<T>(st);
    const T rx0 = rx0_of<T>(st), ry0 = ry0_of<T>(st);
    const T Qdt = (T)st->Qdt;
    CellSrc<T> src;
    src.h = par ? a.f[1][0] : a.f[0][0];
    src.qx = par ? a.f[1][1] : a.f[0][1];
    src.qy = par ? a.f[1][2] : a.f[0][2];
    src.z = a.z;
    T* const oh = nxt ? a.f[1][0] : a.f[0][0];
    T* const oqx = nxt ? a.f[1][1] : a.f[0][1];
    T* const oqy = nxt ? a.f[1][2] : a.f[0][2];
    const T g = a.P.g, hg = a.P.hg, tol = a.P.tol;
    const uint32_t tag = st->epoch + 1u;
    const uint32_t cap = a.fcap;
    const T* F = a.face;
    unsigned long long rmin = kInfBits, mh = 0, mqx = 0, mqy = 0, spd[2] = {0ull, 0ull};
    for (uint32_t w = B.id * blockDim.x + threadIdx.x; w < nq; w += B.n * blockDim.x) {
        const uint32_t pk = a.wet[w];
        const int n = (int)(pk >> kLeafShift);
        const uint32_t code = pk & kCodeMask;
        const uint32_t i = compact16(code), j = compact16(code >> 1);
        const uint32_t last = (1u << n) - 1u;
        const uint64_t base = lvl_off(n);
        const uint64_t iC = base + code;
        const Cell<T> C = fetch(src, iC);
        // squares of the reconstructed depths of the cell at its faces
        T FE[3], GN[3], FW[3], GS[3], hE2, hN2, hW2, hS2;
        FE[0] = F[0 * (size_t)cap + w];
        FE[1] = F[1 * (size_t)cap + w];
        FE[2] = F[2 * (size_t)cap + w];
        hE2 = F[3 * (size_t)cap + w];
        GN[0] = F[5 * (size_t)cap + w];
        GN[1] = F[6 * (size_t)cap + w];
        GN[2] = F[7 * (size_t)cap + w];
        hN2 = F[8 * (size_t)cap + w];
        bool haveW = false, haveS = false;
        if (i > 0) {
            const unsigned long long m = __ldg(a.mark + base + morton2(i - 1, j));
            if ((uint32_t)(m >> 32) == tag) {
                const uint32_t v = (uint32_t)m;
                FW[0] = F[0 * (size_t)cap + v];
                FW[1] = F[1 * (size_t)cap + v];
                FW[2] = F[2 * (size_t)cap + v];
                hW2 = F[4 * (size_t)cap + v];
                haveW = true;
            }
        }
        if (j > 0) {
            const unsigned long long m = __ldg(a.mark + base + morton2(i, j - 1));
            if ((uint32_t)(m >> 32) == tag) {
                const uint32_t v = (uint32_t)m;
                GS[0] = F[5 * (size_t)cap + v];
                GS[1] = F[6 * (size_t)cap + v];
                GS[2] = F[7 * (size_t)cap + v];
                hS2 = F[9 * (size_t)cap + v];
                haveS = true;
            }
        }
        if (FM && !haveW && i > 0 && n < a.L && sig_bit(a.Sb, n, morton2(i - 1, j))) {
            matched_face(a, src, 0, n, i, j, FW, hW2);
            haveW = true;
        }
        if (FM && !haveS && j > 0 && n < a.L && sig_bit(a.Sb, n, morton2(i, j - 1))) {
            matched_face(a, src, 2, n, i, j, GS, hS2);
            haveS = true;
        }
        if (!(haveW && haveS)) {
            T uC, vC, dummy;
            velocity(C, tol, uC, vC);
            if (!haveW) {
                const Cell<T> W = i > 0 ? fetch(src, base + morton2(i - 1, j)) : ghost(C, a.bc_ref[0], true);
                T uW, vW, hW_R;
                velocity(W, tol, uW, vW);
                hll_face(g, hg, tol, W.h, W.z, uW, vW, C.h, C.z, uC, vC, FW, dummy, hW_R);
                hW2 = hW_R * hW_R;
            }
            if (!haveS) {
                const Cell<T> S = j > 0 ? fetch(src, base + morton2(i, j - 1)) : ghost(C, a.bc_ref[2], false);
                T uS, vS, hS_R;
                velocity(S, tol, uS, vS);
                hll_face(g, hg, tol, S.h, S.z, vS, uS, C.h, C.z, vC, uC, GS, dummy, hS_R);
                hS2 = hS_R * hS_R;
            }
        }
        const T rx = mul_pow2(rx0, n), ry = mul_pow2(ry0, n);   // rx0 * 2^n, exact
        int64_t lo = 0, hi = 0;
        const bool inlet = inlet_range(a, n, i, j, last, lo, hi);
        T dh = T(0);
        if (inlet) {
            const T scale = (T)(1u << n);
            const T frac = (T)(hi - lo) / (T)(a.a1 - a.a0);
            const T inv2n = T(1) / scale;
            const T dxn = a.lx * inv2n, dyn = a.ly * inv2n;
            dh = (Qdt * frac) / (dxn * dyn);
        }
        T out[3], rh;
        cell_update_faces_sq(a.P, rx, ry, fk, C, FW, FE, GS, GN, hW2, hE2, hS2, hN2, inlet, dh, out, &rh);
        wet_leaf_store(a, st, src.z, oh, oqx, oqy, n, code, iC, C, out, rmin, mh, mqx, mqy, spd, rh);
    }
    block_atomic_u64<false>(rmin, &st->rmin_bits);
    block_max3_u64(mh, mqx, mqy, st->max_bits);
    block_max3_u64(spd[0], spd[1], 0ull, st->speed_bits);
}
template <typename T, bool FM = false>
static __global__ void __launch_bounds__(256) k_fv1_update(StepArgs<T> a) {
    pdl_wait();
    fv1_update_body<T, FM>(a, this_blk());
}

// Uniform FV1 (every finest cell a leaf): the fixed leaf list in Z-order ...
static __global__ void k_fill_finest_leaves(uint32_t* leaves, int L, uint64_t N) {
    for (uint64_t m = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; m < N; m += (uint64_t)gridDim.x * blockDim.x)
        leaves[m] = ((uint32_t)L << kLeafShift) | (uint32_t)m;
}
// ... and the step's list counts (no tile is skipped, none needs decoding).
static __global__ void k_set_uniform(DevState* st, uint32_t N) {
    pdl_wait();
    if (threadIdx.x != 0 || !st->active) return;
    st->M = N;
    st->Mall = N;
    st->ndec = 0u;
}

// ---------------------------------------------------------------------------
// Decode-back (Eq. 4 with zero details below leaves, free surface restored
// on wet coarse leaves), tile-parallel like the traversal.
// ---------------------------------------------------------------------------
template <typename T>
struct DecodeArgs {
    T* f[2][3];
    const T* z;
    SigSrc Sb;                // the step's regularised flags
    const uint32_t* dlist;    // tiles holding a leaf of more than 16 finest cells
    DevState* st;
    T tol;
    int L, kt;
    Quiet q;                  // quiescent-tile marks (zf NULL: off)
};

// Decode-back of the leaves of more than 16 finest cells, over the tiles the
// traversal listed (smaller leaves were decoded by the FV1 kernels): every
// finest cell takes the leaf's discharges and free surface (R-decode).
template <typename T>
__device__ __forceinline__ void decode_body(const DecodeArgs<T>& a, Blk B) {
    DevState* st = a.st;
    // the state is read through L2 only: k_decode_finish's last CTA reads
    // what the other CTAs' atomics wrote and must not find stale L1 lines
    if (!__ldcg(&st->active)) return;
    const uint32_t nd = __ldcg(&st->ndec);
    if (B.id >= nd) return;                   // whole block idle
    const int nxt = (int)__ldcg(&st->cur) ^ 1;
    __shared__ TileBits tb;
    T* const fh = nxt ? a.f[1][0] : a.f[0][0];
    T* const fqx = nxt ? a.f[1][1] : a.f[0][1];
    T* const fqy = nxt ? a.f[1][2] : a.f[0][2];
    unsigned long long mh = 0, mqx = 0, mqy = 0;
    const uint32_t g = threadIdx.x;
    const bool act = g < (1u << (2 * (a.kt - 1)));
    for (uint32_t d = B.id; d < nd; d += B.n) {
        const uint32_t tile = a.dlist[d];
        __syncthreads();                            // tb reused across tiles
        load_tile_bits(a.Sb, a.L, a.kt, tile, tb);
        if (a.q.zf[0] != nullptr && a.q.act[tile] == kActCovered) {
            // one coarser leaf covers the whole tile: when its new value is
            // (+0, +0, +0) and the tile already holds +0, nothing changes
            const int lc = group_level(tb, a.L, a.kt, 0);
            const uint64_t sc = lvl_off(lc) + (((uint64_t)tile << (2 * a.kt)) >> (2 * (a.L - lc)));
            const bool zero = pos_zero(fh[sc]) && pos_zero(fqx[sc]) && pos_zero(fqy[sc]);
            uint8_t* Y = nxt ? a.q.zf[1] : a.q.zf[0];
            if (zero && Y[tile]) continue;           // uniform over the CTA
            __syncthreads();                         // every thread has read Y[tile]
            if (threadIdx.x == 0) Y[tile] = 0;
        }
        const int l = act ? group_level(tb, a.L, a.kt, g) : a.L;
        if (!needs_decode_kernel(l, a.L)) continue;
        const uint32_t m0 = (tile << (2 * a.kt)) + 4u * g;
        const uint64_t slot = lvl_off(l) + (m0 >> (2 * (a.L - l)));
        const T hl = fh[slot], qxl = fqx[slot], qyl = fqy[slot];
        const bool restore = ge_nonneg(hl, a.tol);      // hl >= tol (tol > 0)
        const uint64_t fo = lvl_off(a.L) + m0;
        T hf[4];
        if (restore) {
            const T eta = eta_of(hl, __ldg(a.z + slot));
            T z0, z1, z2, z3;
            Vec4<T>::load(a.z + fo, z0, z1, z2, z3);
            restore4(eta, z0, z1, z2, z3, hf);
        } else {
            hf[0] = hf[1] = hf[2] = hf[3] = hl;
        }
        Vec4<T>::store(fh + fo, hf[0], hf[1], hf[2], hf[3]);
        Vec4<T>::store(fqx + fo, qxl, qxl, qxl, qxl);
        Vec4<T>::store(fqy + fo, qyl, qyl, qyl, qyl);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const unsigned long long b = abs_obits(hf[e]);
            mh = b > mh ? b : mh;
        }
        const unsigned long long bx = abs_obits(qxl), by = abs_obits(qyl);
        mqx = bx > mqx ? bx : mqx;
        mqy = by > mqy ? by : mqy;
    }
    block_max3_u64(mh, mqx, mqy, st->max_bits);
}
template <typename T>
static __global__ void __launch_bounds__(256) k_decode(DecodeArgs<T> a) {
    decode_body<T>(a, this_blk());
}

// ---------------------------------------------------------------------------
// Time advance and next-step scalars (Algorithm 3: t += dt, new CFL dt)
// ---------------------------------------------------------------------------
struct FinishArgs {
    const double* inflow_t;
    const double* inflow_Q;
    int inflow_n;
    int L;
    double eps, cfl, dt_max, lx, ly;
    double g, manning_n;
};

__device__ inline double inflow_Q(const FinishArgs& a, double t) {
    const int n = a.inflow_n;
    if (n <= 0) return 0.0;
    if (t <= a.inflow_t[0]) return a.inflow_Q[0];
    if (t >= a.inflow_t[n - 1]) return a.inflow_Q[n - 1];
    int k = 0;
    while (!(t >= a.inflow_t[k] && t < a.inflow_t[k + 1])) k++;
    const double w = (t - a.inflow_t[k]) / (a.inflow_t[k + 1] - a.inflow_t[k]);
    return a.inflow_Q[k] + (a.inflow_Q[k + 1] - a.inflow_Q[k]) * w;
}

// Thresholds, timestep clamp and inflow volume of the step about to run.
// Called by every thread of a one-block launch after s_max is final; the
// (level, quantity) thresholds are spread over the threads.
// 4 thr for passes_thr when the comparison against it is exact, else -1
__device__ __forceinline__ double thr4_of(double t) { return t >= 0x1p-1020 ? ldexp(t, 2) : -1.0; }
__device__ __forceinline__ float thr4_of(float t) { return t >= 0x1p-124f ? ldexpf(t, 2) : -1.0f; }

// With t, t_end, dt and s_max given (no reload of what the caller holds).
__device__ inline void prepare_vals(DevState* st, const FinishArgs& a, double t, double t_end, double dt,
                                    const double* smax) {
    for (int k = threadIdx.x; k < 3 * a.L; k += blockDim.x) {
        const int n = k / 3, q = k - 3 * n;
        const double td = ldexp(a.eps, n - a.L) * smax[q];
        const float tf = ldexpf((float)a.eps, n - a.L) * (float)smax[q];
        st->thr[n * 3 + q] = td;
        st->thrf[n * 3 + q] = tf;
        const double t4 = thr4_of(td);
        st->thr4[n * 3 + q] = t4;
        st->thr4f[n * 3 + q] = thr4_of(tf);
        const bool pre = t4 >= 0x1p-100;
        st->thr4lo[n * 3 + q] = pre ? __double2float_rd(t4) : -1.0f;
        st->thr4hi[n * 3 + q] = pre ? __double2float_ru(t4) : -1.0f;
    }
    // the scalars: four independent tasks on lane 0 of different warps (a
    // double division holds the FP64 pipe of its sub-partition for hundreds
    // of cycles), each forming dt_use itself
    if ((threadIdx.x & 31u) != 0u) return;
    const int warp = (int)(threadIdx.x >> 5), nw = (int)((blockDim.x + 31u) >> 5);
    double dt_use = dt;
    if (t + dt_use > t_end) dt_use = t_end - t;
    for (int task = warp; task < 4; task += nw) {
        if (task == 0) {
            st->active = t < t_end ? 1u : 0u;
            st->dt_use = dt_use;
            st->rx0f = (float)dt_use / (float)a.lx;
            st->ry0f = (float)dt_use / (float)a.ly;
            st->nwet = 0u;
            st->rmin_bits = kInfBits;
            st->max_bits[0] = st->max_bits[1] = st->max_bits[2] = 0ull;
            st->speed_bits[0] = st->speed_bits[1] = st->speed_bits[2] = 0ull;
            // the friction term's product with dt, in the operation order of
            // dt * g * n * n * |u| (the leaf's part follows in the update)
            st->fric_k = ((dt_use * a.g) * a.manning_n) * a.manning_n;
            st->fric_kf = (((float)dt_use * (float)a.g) * (float)a.manning_n) * (float)a.manning_n;
        } else if (task == 1) {
            st->rx0 = dt_use / a.lx;            // dt/dx_n = (dt/lx) * 2^n exactly
        } else if (task == 2) {
            st->ry0 = dt_use / a.ly;
        } else {
            st->Qdt = inflow_Q(a, t) * dt_use;
        }
    }
}
__device__ inline void prepare_step(DevState* st, const FinishArgs& a) {
    const double smax[3] = {st->smax[0], st->smax[1], st->smax[2]};
    prepare_vals(st, a, st->t, st->t_end, st->dt, smax);
}

// next timestep: CFL * (min CFL bound), capped at dt_max (+inf when dry)
__device__ inline double dt_from(const FinishArgs& a, double r) {
    const double dt = a.cfl * r;
    return dt < a.dt_max ? dt : a.dt_max;
}

__device__ inline double smax_of(unsigned long long bits) {
    const double m = from_obits(bits);
    return 1.0 > m ? 1.0 : m;
}

// One block advances the scalars, then prepares the next step.  The
// independent parts run on lane 0 of different warps: the time and the
// counters, the two CFL quotients (one division each), the three s_max;
// then the timestep.  The step's CFL bound is the min of the bounds reduced
// as such and of dx_L / max(|u|+sqrt(gh)) and dy_L / max(|v|+sqrt(gh)) over
// the wet leaves whose speeds were reduced instead: a correctly rounded
// division is monotone in its divisor, so dx_L divided by the largest speed
// is exactly the smallest of the per-leaf quotients (Sec. 2.1.3 CFL).
__device__ __forceinline__ void finish_body(DevState* st, const FinishArgs& a) {
    if (!st->active) return;
    __syncthreads();                 // every thread has read `active`
    // values handed between the parts through shared memory, so that
    // nothing written here is read back from global memory
    __shared__ double s_q[2], s_t, s_tend, s_dt, s_r, s_smax[3];
    const int warp = (int)(threadIdx.x >> 5), nw = (int)((blockDim.x + 31u) >> 5);
    const bool speeds = st->speed_bits[0] != 0ull;
    if ((threadIdx.x & 31u) == 0u) {
        for (int task = warp; task < 4; task += nw) {
            if (task == 0) {
                const double t = st->t + st->dt_use;
                st->t = t;
                s_t = t;
                s_tend = st->t_end;
                st->step += 1;
                st->epoch += 1u;
                st->leaf_updates += st->Mall;
                st->act_updates += st->M;
                st->wet_updates += st->nwet;
                st->cur ^= 1u;
            } else if (task == 1) {
                if (speeds) s_q[0] = ldexp(a.lx, -a.L) / __longlong_as_double((long long)st->speed_bits[0]);
                s_r = from_obits(st->rmin_bits);
            } else if (task == 2) {
                if (speeds) s_q[1] = ldexp(a.ly, -a.L) / __longlong_as_double((long long)st->speed_bits[1]);
            } else {
                for (int q = 0; q < 3; ++q) {
                    const double m = smax_of(st->max_bits[q]);
                    st->smax[q] = m;
                    s_smax[q] = m;
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = s_r;
        if (speeds) {
            const double rx = s_q[0], ry = s_q[1];
            const double rr = rx < ry ? rx : ry;
            r = rr < r ? rr : r;
        }
        const double dt = dt_from(a, r);
        st->dt = dt;
        s_dt = dt;
        if (!isfinite(dt) || !isfinite(s_smax[0]) || !isfinite(s_smax[1]) || !isfinite(s_smax[2]))
            st->err |= kErrNonFinite;
    }
    __syncthreads();
    prepare_vals(st, a, s_t, s_tend, s_dt, s_smax);
}

// Decode-back followed, in its last CTA to finish, by the time advance (one
// launch instead of two).  decode_body reads the state through L2 only, so
// the last CTA sees every other CTA's reductions after the fence.
//
// Only the first min(ndec, grid) CTAs (at least one) take part: the others
// have no tile to decode (decode_body strides over the list by the grid)
// and leave at once, so a short decode list costs few fences and ticket
// atomics.  ndec is fixed from the traversal to the next step's clear.
template <typename T>
static __global__ void __launch_bounds__(256) k_decode_finish(DecodeArgs<T> a, FinishArgs fa) {
    pdl_wait();
    const uint32_t nd = __ldcg(&a.st->ndec);
    const uint32_t parts = nd < gridDim.x ? (nd > 0u ? nd : 1u) : gridDim.x;
    if (blockIdx.x >= parts) return;
    decode_body<T>(a, this_blk());
    __threadfence();
    __syncthreads();
    __shared__ bool last;
    if (threadIdx.x == 0) last = atomicAdd(&a.st->dec_ticket, 1u) == parts - 1u;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x == 0) a.st->dec_ticket = 0u;
    finish_body(a.st, fa);
}

// Set t_end (hwfv1_advance) and recompute the step scalars.
__device__ __forceinline__ void set_tend_body(DevState* st, const FinishArgs& a, double t_end) {
    if (threadIdx.x == 0) st->t_end = t_end;
    __syncthreads();
    prepare_step(st, a);
}
static __global__ void k_set_tend(DevState* st, FinishArgs a, double t_end) {
    set_tend_body(st, a, t_end);
}

// State from the reductions of the initial (or reloaded) fields:
// s_max from max_bits[0..2], and, if set_dt, dt from rmin_bits.
static __global__ void k_init_state(DevState* st, FinishArgs a, int set_dt) {
    if (threadIdx.x == 0) {
        for (int q = 0; q < 3; ++q) st->smax[q] = smax_of(st->max_bits[q]);
        // a NaN or inf anywhere in the fields shows up in its maximum
        for (int q = 0; q < 3; ++q)
            if (!isfinite(st->smax[q])) st->err |= kErrNonFinite;
        if (set_dt) st->dt = dt_from(a, from_obits(st->rmin_bits));
    }
    __syncthreads();
    prepare_step(st, a);
}

// z thresholds for the one-off bed encode
static __global__ void k_z_thresholds(const unsigned long long* zmax_bits, double* thr_d, float* thr_f,
                                      double* thr4_d, float* thr4_f, double* smax_z, int L, double eps,
                                      DevState* st) {
    if (threadIdx.x != 0) return;
    const double s = smax_of(*zmax_bits);
    *smax_z = s;
    if (!isfinite(s)) st->err |= kErrNonFinite;
    for (int n = 0; n < L; ++n) {
        thr_d[n] = ldexp(eps, n - L) * s;
        thr_f[n] = ldexpf((float)eps, n - L) * (float)s;
        thr4_d[n] = thr4_of(thr_d[n]);
        thr4_f[n] = thr4_of(thr_f[n]);
    }
}

// ---------------------------------------------------------------------------
// Reductions over the finest grid (initial state)
// ---------------------------------------------------------------------------
template <typename T>
static __global__ void __launch_bounds__(256) k_maxabs(const T* __restrict__ x, uint64_t n,
                                                unsigned long long* dst) {
    unsigned long long m = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long b = abs_obits(x[i]);
        m = b > m ? b : m;
    }
    block_atomic_u64<true>(m, dst);
}

template <typename T>
static __global__ void __launch_bounds__(256) k_cfl_finest(const T* __restrict__ h, const T* __restrict__ qx,
                                                    const T* __restrict__ qy, uint64_t n, Phys<T> P,
                                                    unsigned long long* dst) {
    unsigned long long m = kInfBits;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long b = obits((double)cfl_bound(P, h[i], qx[i], qy[i]));
        m = b < m ? b : m;
    }
    block_atomic_u64<false>(m, dst);
}

// Reductions into DevState over the finest level of the current buffer
// (set_fields / load / init).
static __global__ void k_reset_red(DevState* st) {
    if (threadIdx.x != 0) return;
    st->rmin_bits = kInfBits;
    st->max_bits[0] = st->max_bits[1] = st->max_bits[2] = 0ull;
    st->speed_bits[0] = st->speed_bits[1] = st->speed_bits[2] = 0ull;
}

template <typename T>
static __global__ void __launch_bounds__(256) k_maxabs_cur(const T* __restrict__ x0, const T* __restrict__ x1,
                                                    DevState* st, uint64_t n, int q) {
    const T* x = st->cur ? x1 : x0;
    unsigned long long m = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long b = abs_obits(x[i]);
        m = b > m ? b : m;
    }
    block_atomic_u64<true>(m, &st->max_bits[q]);
}

template <typename T>
static __global__ void __launch_bounds__(256) k_cfl_cur(const T* h0, const T* h1, const T* qx0, const T* qx1,
                                                 const T* qy0, const T* qy1, DevState* st, uint64_t n,
                                                 Phys<T> P) {
    const bool c = st->cur != 0;
    const T* h = c ? h1 : h0;
    const T* qx = c ? qx1 : qx0;
    const T* qy = c ? qy1 : qy0;
    unsigned long long m = kInfBits;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long b = obits((double)cfl_bound(P, h[i], qx[i], qy[i]));
        m = b < m ? b : m;
    }
    block_atomic_u64<false>(m, &st->rmin_bits);
}

// ---------------------------------------------------------------------------
// Layout conversion: row-major (j*2^L + i, float64) <-> Morton (type T)
// ---------------------------------------------------------------------------
template <typename T>
static __global__ void k_rm_to_morton(const double* __restrict__ src, T* __restrict__ dst, int L) {
    const uint64_t N = 1ull << (2 * L);
    for (uint64_t m = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; m < N;
         m += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t i = compact16((uint32_t)m), j = compact16((uint32_t)(m >> 1));
        dst[m] = (T)src[((uint64_t)j << L) + i];
    }
}

// dst_rm[j*2^L+i] = src[Morton(i,j)]; src chosen by the current buffer when
// `src2` is given (src = buffer 0, src2 = buffer 1)
template <typename T>
static __global__ void k_morton_to_rm(const T* __restrict__ src, const T* __restrict__ src2,
                               const DevState* st, double* __restrict__ dst, int L) {
    const T* s = (src2 && st && st->cur) ? src2 : src;
    const uint64_t N = 1ull << (2 * L);
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < N;
         r += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t i = (uint32_t)(r & ((1ull << L) - 1)), j = (uint32_t)(r >> L);
        dst[r] = (double)s[morton2(i, j)];
    }
}

template <typename T>
static __global__ void k_copy_level(const T* __restrict__ src, const T* __restrict__ src2,
                             const DevState* st, double* __restrict__ dst, uint64_t n) {
    const T* s = (src2 && st && st->cur) ? src2 : src;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        dst[i] = (double)s[i];
}

// into the current buffer (set_fields / load)
template <typename T>
static __global__ void k_rm_to_morton_cur(const double* __restrict__ src, T* dst0, T* dst1,
                                   const DevState* st, int L) {
    T* dst = st->cur ? dst1 : dst0;
    const uint64_t N = 1ull << (2 * L);
    for (uint64_t m = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; m < N;
         m += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t i = compact16((uint32_t)m), j = compact16((uint32_t)(m >> 1));
        dst[m] = (T)src[((uint64_t)j << L) + i];
    }
}


// ---------------------------------------------------------------------------
// Learned look-ahead (subtree CNN).  A subtree is one cell of level
// Ls = L - 4 (16 x 16 finest cells).
// ---------------------------------------------------------------------------

// CNN input: the level-Ls coefficients of h, qx, qy (current buffer) and z,
// each over its s_max, as bf16 channels-last pixels (row j, column i).
template <typename T>
static __global__ void k_features(const T* h0, const T* h1, const T* qx0, const T* qx1, const T* qy0,
                                  const T* qy1, const T* z, const DevState* st, const double* smax_z, int Ls,
                                  __nv_bfloat16* out) {
    const bool c1 = st->cur != 0;
    const T* h = c1 ? h1 : h0;
    const T* qx = c1 ? qx1 : qx0;
    const T* qy = c1 ? qy1 : qy0;
    const uint32_t n = 1u << (2 * Ls), S = 1u << Ls;
    const uint64_t o = lvl_off(Ls);
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const uint32_t pix = compact16(c >> 1) * S + compact16(c);
        out[4 * pix + 0] = __float2bfloat16((float)((double)h[o + c] / st->smax[0]));
        out[4 * pix + 1] = __float2bfloat16((float)((double)qx[o + c] / st->smax[1]));
        out[4 * pix + 2] = __float2bfloat16((float)((double)qy[o + c] / st->smax[2]));
        out[4 * pix + 3] = __float2bfloat16((float)((double)z[o + c] / *smax_z));
    }
}

// Training label of every subtree: 1 + the deepest level (>= Ls) holding a
// closed threshold flag (C | Cz) in the subtree, minus Ls; 0 if none.  One
// byte per pixel, row-major.
static __global__ void k_labels(const uint32_t* __restrict__ Cb, const uint32_t* __restrict__ Cz, int L, int Ls,
                                uint8_t* __restrict__ out) {
    const uint32_t n = 1u << (2 * Ls), S = 1u << Ls;
    for (uint32_t sub = blockIdx.x * blockDim.x + threadIdx.x; sub < n; sub += gridDim.x * blockDim.x) {
        int deepest = -1;
        for (int lv = Ls; lv < L; ++lv) {
            const uint32_t cnt = 1u << (2 * (lv - Ls)), first = sub * cnt;
            bool any = false;
            if (cnt < 32u) {
                const uint32_t w = word_off(lv) + (first >> 5);
                const uint32_t m = ((Cb[w] | Cz[w]) >> (first & 31u)) & ((1u << cnt) - 1u);
                any = m != 0u;
            } else {
                for (uint32_t k = 0; k < cnt / 32u && !any; ++k) {
                    const uint32_t w = word_off(lv) + (first >> 5) + k;
                    any = (Cb[w] | Cz[w]) != 0u;
                }
            }
            if (any) deepest = lv;
        }
        const int lab = deepest < 0 ? 0 : deepest + 1 - Ls;
        out[compact16(sub >> 1) * S + compact16(sub)] = (uint8_t)lab;
    }
}

// Predicted deepest level per subtree (Morton order): the smallest class
// whose cumulative probability reaches 1 - margin (so levels are only cut
// where the network is confident); margin < 0 keeps every level (L).
static __global__ void k_predict(const float* __restrict__ logits, int Ls, float margin, uint8_t* __restrict__ phat) {
    const uint32_t n = 1u << (2 * Ls), S = 1u << Ls;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        int cls = 4;
        if (margin >= 0.f) {
            const uint32_t pix = compact16(c >> 1) * S + compact16(c);
            float z[5], m = -INFINITY;
            for (int o = 0; o < 5; ++o) {
                z[o] = logits[(size_t)pix * 16 + o];
                m = fmaxf(m, z[o]);
            }
            float se = 0.f;
            for (int o = 0; o < 5; ++o) se += expf(z[o] - m);
            float cum = 0.f;
            for (int o = 0; o < 4; ++o) {
                cum += expf(z[o] - m) / se;
                if (cum >= 1.f - margin) {
                    cls = o;
                    break;
                }
            }
        }
        phat[c] = (uint8_t)(Ls + cls);
    }
}

}  // namespace hwfv1
