// skip.cuh -- the learned subtree skip: every level-(L-4) subtree is
// encoded, flagged and stored only down to a predicted level (a layer the
// project adds on top of Algorithm 3; the paper has no learned part).
//
// The subtree s (Morton code s at level Ls = L - 4, 16 x 16 finest cells)
// keeps its state at a storage level m_s in [Ls, L]: its level-m_s cells
// (m_s = L after the start and after every plain step).  A skip step is given
// a predicted level p_s per subtree and
//   1. keeps s down to P_s = max(p_s, p of the subtrees sharing an edge with
//      s), so that a leaf next to s finds its same-level neighbour in s;
//   2. takes its thresholds from s_max over the stored state (the previous
//      step's decode reduced it over the cells it stored);
//   3. forms the level-P_s cells of s from its level-m_s cells when
//      P_s > m_s, as the decode-back forms the cells under a leaf;
//   4. encodes s from level E_s = max(m_s, P_s) up to Ls (k_skip_encode),
//      then levels Ls-1 .. 0 (the plain encode passes from level Ls);
//   5./6. flags a parent of s only at levels below p_s, with the bed's
//      details of those levels, regularises (R1, R2) and keeps no cell of
//      s significant at a level >= p_s (k_skip_flag);
//   7. lists and updates the leaves as the plain step does, each leaf
//      writing its own cell only;
//   8. stores s at level P_s: every level-P_s cell takes its covering
//      leaf's value, with the decode-back's free surface against z^(P_s)
//      (k_skip_decode, which then advances the time).
// A plain step (the exact audit) first brings every subtree to level L
// (k_skip_finest).  The same steps, written out plainly, are the CPU
// oracle's orc_skip_step.
#pragma once
#include "kernels.cuh"

namespace hwfv1 {

// P_s: the largest predicted level of s and of its edge neighbours
// (predictions in Morton order over level Ls).
__device__ __forceinline__ int skip_store_level(const uint8_t* __restrict__ phat, int Ls, uint32_t s) {
    const uint32_t last = (1u << Ls) - 1u;
    const uint32_t i = compact16(s), j = compact16(s >> 1);
    int v = phat[s];
    if (i > 0u) v = max(v, (int)phat[mort_xm(s)]);
    if (i < last) v = max(v, (int)phat[mort_xp(s)]);
    if (j > 0u) v = max(v, (int)phat[mort_ym(s)]);
    if (j < last) v = max(v, (int)phat[mort_yp(s)]);
    return v;
}

// Depth of a cell under a coarser cell (the decode-back's rule, reading
// R-decode): a wet coarse cell hands down its free surface, the finer cell
// takes max(0, eta - z_fine); a dry one hands down its depth.
template <typename T>
__device__ __forceinline__ T redecode_h(T hl, T zl, T zc, T tol) {
    if (!ge_nonneg(hl, tol)) return hl;
    const T eta = eta_of(hl, zl);                    // hl + zl (exact shortcuts on a +0 bed)
    const T d = pos_zero(zc) ? eta : eta - zc;
    return gt_zero(d) ? d : T(0);
}

template <typename T>
struct SkipArgs {
    T* f[2][3];               // h, qx, qy hierarchies of the two state buffers
    const T* z;               // bed hierarchy
    const T* thr;             // thresholds per (level, quantity), as the plain encode
    const T* thr4;
    const float* thr4lo = nullptr;
    const float* thr4hi = nullptr;
    const uint32_t* Tz;       // the bed's threshold flags (static)
    uint32_t* Tb;             // threshold flags (bed included at levels >= Ls)
    uint32_t* Cb;             // their upward closure
    const uint8_t* phat;      // predicted level per subtree
    const uint8_t* mlev;      // storage level per subtree as the step starts
    uint8_t* plev;            // storage level per subtree after the step (P_s)
    const uint8_t* flat = nullptr;   // exact store: 1 where the subtree's bed is flat (NULL: the learned skip)
    DevState* st;
    T tol;
    int L, Ls;
};

// Steps 1, 3 and 4 inside the subtrees: one warp per subtree, eight
// subtrees per CTA, a grid striding over the subtrees.  Every level the
// encode forms is written to the current state buffer (neighbouring leaves
// and the FV1 update read them there); threshold and closure bits are OR-ed
// into words the clear kernel zeroed.  The level chain of a subtree runs in
// its warp alone (warp barriers only), so many subtrees are in flight per SM.
// The chain is bound by load latency, so the loads a level needs are issued
// ahead of it: the thresholds of the subtree levels sit in shared memory,
// the bed's flag words of a subtree are read with its levels, and the
// level-P cells are formed four warp rounds at a time, loads first.
template <typename T>
static __global__ void __launch_bounds__(256, 3) k_skip_encode(SkipArgs<T> a) {
    pdl_wait();
    if (!a.st->active) return;
    const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
    const int par = (int)a.st->cur;
    T* const fh = par ? a.f[1][0] : a.f[0][0];
    T* const fqx = par ? a.f[1][1] : a.f[0][1];
    T* const fqy = par ? a.f[1][2] : a.f[0][2];
    const int Ls = a.Ls;
    const uint32_t nsub = 1u << (2 * Ls);
    __shared__ T sv[8][3][64];               // the level just formed, per warp
    __shared__ uint8_t scl[8][64];           // its closure bits
    __shared__ Thr<T> sth[4][3];             // thresholds of levels Ls .. Ls+3
    if (threadIdx.x < 12u) {
        const int d = (int)threadIdx.x / 3, q = (int)threadIdx.x % 3, idx = (Ls + d) * 3 + q;
        sth[d][q].thr = a.thr[idx];
        sth[d][q].thr4 = a.thr4[idx];
        sth[d][q].lo = a.thr4lo ? a.thr4lo[idx] : -1.0f;
        sth[d][q].hi = a.thr4hi ? a.thr4hi[idx] : -1.0f;
    }
    __syncthreads();
    for (uint32_t s = blockIdx.x * 8u + wib; s < nsub; s += gridDim.x * 8u) {
        // the bed's flag words of the parents of s: lane d < 3 holds level
        // Ls+d's word (at most 16 parents, one word), lanes 3 and 4 the two
        // words of level Ls+3's 64 parents
        uint32_t tzw = 0u;
        if (lane < 5u) {
            const int d = lane < 3u ? (int)lane : 3;
            const uint32_t pc = (s << (2 * d)) + (lane == 4u ? 32u : 0u);
            tzw = __ldg(a.Tz + word_off(Ls + d) + (pc >> 5));
        }
        const int p = a.phat[s];
        const int P = skip_store_level(a.phat, Ls, s);
        const int m = a.mlev[s];
        if (lane == 0u) a.plev[s] = (uint8_t)P;
        const int E = P > m ? P : m;
        if (P > m) {                         // step 3: level P from level m
            const uint32_t cnt = 1u << (2 * (P - Ls));
            const uint64_t b = (uint64_t)s << (2 * (P - Ls));
            // the exact store keeps a flat subtree's stored cells as the
            // finest cells they stand for: formed by copying
            const bool copy = a.flat != nullptr && a.flat[s] != 0;
#pragma unroll 1
            for (uint32_t k0 = 0u; k0 < cnt; k0 += 64u) {
                T hl[2], zl[2], zc[2], ql[2], rl[2];
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const uint32_t k = k0 + 32u * j + lane;
                    if (k < cnt) {
                        const uint64_t c = b + k, ia = lvl_off(m) + (c >> (2 * (P - m))), ic = lvl_off(P) + c;
                        hl[j] = __ldcg(fh + ia);
                        ql[j] = __ldcg(fqx + ia);
                        rl[j] = __ldcg(fqy + ia);
                        if (!copy) {
                            zl[j] = __ldg(a.z + ia);
                            zc[j] = __ldg(a.z + ic);
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const uint32_t k = k0 + 32u * j + lane;
                    if (k < cnt) {
                        const uint64_t ic = lvl_off(P) + b + k;
                        fh[ic] = copy ? hl[j] : redecode_h(hl[j], zl[j], zc[j], a.tol);
                        fqx[ic] = ql[j];
                        fqy[ic] = rl[j];
                    }
                }
            }
            __syncwarp();                    // the warp reads level P below
        }
        // step 4: levels E-1 .. Ls; a parent is flagged only below p (step 5).
        // The first level reads its children from the state (up to 64
        // parents, two rounds of the warp); the others from shared memory.
        for (int n = E - 1; n >= Ls; --n) {
            const uint32_t cnt = 1u << (2 * (n - Ls));
            const bool first = n == E - 1;
#pragma unroll 1
            for (uint32_t t0 = 0u; t0 < (first ? cnt : 32u); t0 += 32u) {   // warp-uniform rounds
                const uint32_t t = t0 + lane;
                const bool act = t < cnt;
                const uint64_t pc = ((uint64_t)s << (2 * (n - Ls))) + t;
                const uint32_t tz = __shfl_sync(0xffffffffu, tzw, n - Ls < 3 ? (uint32_t)(n - Ls) : 3u + (t0 >> 5));
                T c[3][4];
                bool cch = false;
                T sq[3] = {T(0), T(0), T(0)};
                bool cf = false, tt = false;
                if (act) {
                    if (first) {
                        Vec4<T>::load_cg(fh + lvl_off(n + 1) + 4ull * pc, c[0][0], c[0][1], c[0][2], c[0][3]);
                        Vec4<T>::load_cg(fqx + lvl_off(n + 1) + 4ull * pc, c[1][0], c[1][1], c[1][2], c[1][3]);
                        Vec4<T>::load_cg(fqy + lvl_off(n + 1) + 4ull * pc, c[2][0], c[2][1], c[2][2], c[2][3]);
                    } else {
#pragma unroll
                        for (int q = 0; q < 3; ++q)
#pragma unroll
                            for (int e = 0; e < 4; ++e) c[q][e] = sv[wib][q][4 * t + e];
                        cch = (scl[wib][4 * t] | scl[wib][4 * t + 1] | scl[wib][4 * t + 2] | scl[wib][4 * t + 3]) != 0;
                    }
                    bool tf = false;
                    parents_all<T, 3>(sth[n - Ls], c, sq, tf);
                    fh[lvl_off(n) + pc] = sq[0];
                    fqx[lvl_off(n) + pc] = sq[1];
                    fqy[lvl_off(n) + pc] = sq[2];
                    tt = n < p && (tf || (tz & (1u << (pc & 31u))) != 0u);
                    cf = tt || cch;
                }
                // one OR per word: a round's parents are consecutive codes
                // within one word (aligned to their count, or to 32)
                const uint32_t tb = __ballot_sync(0xffffffffu, act && tt);
                const uint32_t cb = __ballot_sync(0xffffffffu, act && cf);
                if (lane == 0u && (tb | cb)) {
                    const uint64_t pc0 = ((uint64_t)s << (2 * (n - Ls))) + t0;
                    const uint32_t w0 = word_off(n) + (uint32_t)(pc0 >> 5), sh = (uint32_t)(pc0 & 31u);
                    if (tb) atomicOr(a.Tb + w0, tb << sh);
                    if (cb) atomicOr(a.Cb + w0, cb << sh);
                }
                // the first level writes slots no lane reads in this level;
                // the others overwrite what the warp has just read
                if (!first) __syncwarp();
                if (act) {
#pragma unroll
                    for (int q = 0; q < 3; ++q) sv[wib][q][t] = sq[q];
                    scl[wib][t] = cf ? 1 : 0;
                }
            }
            __syncwarp();
        }
    }
}

// Steps 5 and 6 as words of the regularised flags S: above the subtrees
//   S = C | Cz' | R1 of (T | Tz)          (Cz': closure of the bed's flags
//                                          of levels < Ls, static)
// and at levels n >= Ls
//   S = (C | R1) & [n < p of the cell's subtree]
// where T, C already hold the bed's flags there (k_skip_encode).
static __global__ void k_skip_flag(const uint32_t* __restrict__ Tb, const uint32_t* __restrict__ Cb,
                                   const uint32_t* __restrict__ Tz, const uint32_t* __restrict__ Czu,
                                   uint32_t* __restrict__ Sb, const uint8_t* __restrict__ phat, int L, int Ls,
                                   const DevState* st) {
    pdl_wait();
    if (!st->active) return;
    const uint32_t total = bits_words(L);
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < total; w += gridDim.x * blockDim.x) {
        int n = 0;
        while (n + 1 < L && word_off(n + 1) <= w) ++n;
        const uint32_t lw = w - word_off(n);
        uint32_t s = Cb[w];
        if (n < Ls) s |= Czu[w];
        if (n >= 1) {                       // R1: children of the parent level's flags
            const bool bed = n - 1 < Ls;     // above the subtrees T lacks the bed's flags
            uint32_t pb;
            if (n >= 3) {
                const uint32_t pw = word_off(n - 1) + (lw >> 2);
                pb = expand4x8((Tb[pw] | (bed ? Tz[pw] : 0u)) >> (8u * (lw & 3u)));
            } else if (n == 2) {
                pb = expand4x8((Tb[word_off(1)] | (bed ? Tz[word_off(1)] : 0u)) & 0xFu);
            } else {
                pb = ((Tb[word_off(0)] | (bed ? Tz[word_off(0)] : 0u)) & 1u) ? 0xFu : 0u;
            }
            s |= pb;
        }
        if (n >= Ls) {
            const int sh = 2 * (n - Ls);
            const uint32_t nb = n < 3 ? (1u << (2 * n)) : 32u;     // cells in this word
            uint32_t allow = 0u;
            for (uint32_t b = 0; b < nb; ++b)
                if (n < (int)phat[(32u * lw + b) >> sh]) allow |= 1u << b;
            s &= allow;
        }
        if (n <= 2) s &= (n == 0 ? 1u : (n == 1 ? 0xFu : 0xFFFFu));
        Sb[w] = s;
    }
}

template <typename T>
struct SkipDecodeArgs {
    T* f[2][3];
    const T* z;
    const uint32_t* Sb;       // the step's regularised flags
    const uint8_t* plev;      // P_s
    uint8_t* mlev;            // set to the level the subtree is stored at
    const uint8_t* flat = nullptr;   // exact store (see k_skip_decode)
    DevState* st;
    T tol;
    int L, Ls;
};

// Step 8 and the time advance: every level-P_s cell of every subtree takes
// its covering leaf's new value (the leaf found by the walk of Algorithm 5
// over S), with the free surface restored against z^(P_s) below a wet
// coarser leaf; the s_max reductions run over every stored cell.  64
// threads per subtree, four subtrees per CTA; a subtree's flag bits on its
// root path and at its own levels are read once into shared memory.  The
// last CTA to finish advances the time (as k_decode_finish).
template <typename T>
static __global__ void __launch_bounds__(256) k_skip_decode(SkipDecodeArgs<T> a, FinishArgs fa) {
    pdl_wait();
    DevState* st = a.st;
    unsigned long long mh = 0, mqx = 0, mqy = 0;
    __shared__ int s_l0[4];
    __shared__ unsigned long long s_bits[4][4];   // S of the subtree's levels Ls .. Ls+3
    const bool run = __ldcg(&st->active) != 0u;
    const int Ls = a.Ls;
    const uint32_t nsub = 1u << (2 * Ls);
    const uint32_t g = threadIdx.x >> 6, t = threadIdx.x & 63u;
    const int nxt = (int)__ldcg(&st->cur) ^ 1;
    T* const fh = nxt ? a.f[1][0] : a.f[0][0];
    T* const fqx = nxt ? a.f[1][1] : a.f[0][1];
    T* const fqy = nxt ? a.f[1][2] : a.f[0][2];
    // uniform trip count over the CTA (barriers below)
    const uint32_t rounds = run ? (nsub + gridDim.x * 4u - 1u) / (gridDim.x * 4u) : 0u;
    for (uint32_t r = 0; r < rounds; ++r) {
        const uint32_t s = (r * gridDim.x + blockIdx.x) * 4u + g;
        const bool have = s < nsub;
        const int P = have ? (int)a.plev[s] : Ls;
        __syncthreads();                          // the previous round's readers are done
        if (t < 32u) {                            // the group's first warp, warp-uniform
            // the leaf on the root path that covers the subtree: the first
            // level n <= Ls whose cell over s is not significant (Ls + 1:
            // none), its bits loaded by lane n, all at once
            const bool clear = have && (int)t <= Ls && !sig_bit(a.Sb, (int)t, s >> (2 * (Ls - (int)t)));
            const uint32_t cb = __ballot_sync(0xffffffffu, clear);
            if (have && t == 0u) s_l0[g] = cb ? __ffs((int)cb) - 1 : Ls + 1;
        }
        if (have && t >= 1u && t <= 3u && Ls + (int)t < P) {     // levels Ls+1 .. Ls+3
            const int n = Ls + (int)t;
            const uint32_t cnt = 1u << (2 * t), first = s << (2 * t);
            const uint32_t* w = a.Sb + word_off(n) + (first >> 5);
            unsigned long long v;
            if (cnt >= 32u) v = (unsigned long long)__ldg(w) | ((unsigned long long)__ldg(w + 1) << 32);
            else v = (__ldg(w) >> (first & 31u)) & ((1u << cnt) - 1u);
            s_bits[g][t] = v;
        }
        __syncthreads();
        if (!have) continue;
        const int l0 = s_l0[g];
        // the level the subtree is stored at: P_s, or with the exact store
        // on a flat bed its deepest leaf level (every finest cell below a
        // stored cell then holds that cell's value), where a wet leaf at the
        // stored level also takes the free surface the finest cells get
        const bool exact = a.flat != nullptr && a.flat[s] != 0;
        int tgt = P;
        if (exact) {
            tgt = Ls;
            if (l0 > Ls) {
                tgt = Ls + 1;
                for (int d = 1; d <= 3 && Ls + d < P; ++d)
                    if (s_bits[g][d] != 0ull) tgt = Ls + d + 1;
            }
        }
        const uint32_t cnt = 1u << (2 * (tgt - Ls));
        const uint64_t b = (uint64_t)s << (2 * (tgt - Ls));
        for (uint32_t k = t; k < cnt; k += 64u) {
            const uint64_t c = b + k;
            int l = l0;
            if (l0 > Ls) {
                l = tgt;
                for (int n = Ls + 1; n < tgt; ++n) {
                    const uint32_t idx = k >> (2 * (tgt - n));
                    if (!((s_bits[g][n - Ls] >> idx) & 1ull)) {
                        l = n;
                        break;
                    }
                }
            }
            const uint64_t il = lvl_off(l) + (c >> (2 * (tgt - l))), ic = lvl_off(tgt) + c;
            // the leaf's values and the two bed values in one round of loads
            const bool fill = l < tgt || (exact && tgt < a.L);
            const T hl = fh[il], qxl = fqx[il], qyl = fqy[il];
            T zl = T(0), zc = T(0);
            if (fill) {
                zl = __ldg(a.z + il);
                zc = __ldg(a.z + ic);
            }
            T hf = hl;
            if (fill) {
                hf = redecode_h(hl, zl, zc, a.tol);
                fh[ic] = hf;
                fqx[ic] = qxl;
                fqy[ic] = qyl;
            }
            const unsigned long long bh = abs_obits(hf), bx = abs_obits(qxl), by = abs_obits(qyl);
            mh = bh > mh ? bh : mh;
            mqx = bx > mqx ? bx : mqx;
            mqy = by > mqy ? by : mqy;
        }
        if (t == 0u) a.mlev[s] = (uint8_t)tgt;
    }
    block_max3_u64(mh, mqx, mqy, st->max_bits);
    __threadfence();
    __syncthreads();
    __shared__ bool last;
    if (threadIdx.x == 0) last = atomicAdd(&st->dec_ticket, 1u) == gridDim.x - 1u;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x == 0) st->dec_ticket = 0u;
    finish_body(st, fa);
}

// Every subtree brought to level L (step 3 with P = L).  mode 0: into the
// other buffer's finest level, for reading the fields (the current state
// stays as it is stored); 1: in place before a plain step, whose storage
// levels then become L (nothing when the step will not run); 2: in place
// whatever the time (leaving the skip, checkpoints).
template <typename T>
struct SkipFinestArgs {
    T* f[2][3];
    const T* z;
    uint8_t* mlev;
    const uint8_t* flat = nullptr;   // exact store: flat subtrees are copied down
    DevState* st;
    T tol;
    int L, Ls;
    int mode;
};
template <typename T>
static __global__ void __launch_bounds__(256) k_skip_finest(SkipFinestArgs<T> a) {
    pdl_wait();
    if (a.mode == 1 && !a.st->active) return;
    const bool in_place = a.mode != 0;
    const int par = (int)a.st->cur, dst = in_place ? par : par ^ 1;
    const T* const sh = par ? a.f[1][0] : a.f[0][0];
    const T* const sqx = par ? a.f[1][1] : a.f[0][1];
    const T* const sqy = par ? a.f[1][2] : a.f[0][2];
    T* const dh = dst ? a.f[1][0] : a.f[0][0];
    T* const dqx = dst ? a.f[1][1] : a.f[0][1];
    T* const dqy = dst ? a.f[1][2] : a.f[0][2];
    const int L = a.L, Ls = a.Ls;
    const uint32_t nsub = 1u << (2 * Ls);
    const uint32_t g = threadIdx.x >> 6, t = threadIdx.x & 63u;
    for (uint32_t s = blockIdx.x * 4u + g; s < nsub; s += gridDim.x * 4u) {
        const int m = a.mlev[s];
        if (m == L && in_place) continue;
        const bool copy = a.flat != nullptr && a.flat[s] != 0;
        const uint64_t b = (uint64_t)s << (2 * (L - Ls));
        for (uint32_t k = t; k < (1u << (2 * (L - Ls))); k += 64u) {
            const uint64_t c = b + k, ic = lvl_off(L) + c;
            if (m == L) {
                dh[ic] = sh[ic];
                dqx[ic] = sqx[ic];
                dqy[ic] = sqy[ic];
            } else {
                const uint64_t ia = lvl_off(m) + (c >> (2 * (L - m)));
                dh[ic] = copy ? sh[ia] : redecode_h(sh[ia], __ldg(a.z + ia), __ldg(a.z + ic), a.tol);
                dqx[ic] = sqx[ia];
                dqy[ic] = sqy[ia];
            }
        }
        if (in_place && t == 0u) a.mlev[s] = (uint8_t)L;
    }
}

// The exact leaf-value store's levels: a subtree whose bed is flat holds
// after a step the same value in every finest cell below each cell of its
// stored level m (its deepest leaf level), so none of its details at levels
// >= m is significant (eps > 0) and its next leaves are no finer than m + 1;
// p = m + 1 keeps exactly the plain step's tree.  Other subtrees keep L.
static __global__ void k_exact_levels(const uint8_t* __restrict__ mlev, const uint8_t* __restrict__ flat,
                                      uint8_t* __restrict__ phat, int L, int Ls, const DevState* st) {
    pdl_wait();
    if (!st->active) return;
    const uint32_t n = 1u << (2 * Ls);
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const int m = mlev[s];
        phat[s] = (uint8_t)(flat[s] ? (m + 1 < L ? m + 1 : L) : L);
    }
}

// 1 where every finest bed value of the subtree is the same (bit for bit);
// then so is every coarser bed coefficient inside it.
template <typename T>
static __global__ void k_flat_subtrees(const T* __restrict__ zL, int L, int Ls, uint8_t* __restrict__ flat) {
    const uint32_t n = 1u << (2 * Ls), cells = 1u << (2 * (L - Ls));
    const uint32_t lane = threadIdx.x & 31u;
    for (uint32_t s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < n; s += (gridDim.x * blockDim.x) >> 5) {
        const T z0 = zL[(uint64_t)s * cells];
        bool same = true;
        for (uint32_t k = lane; k < cells; k += 32u) same = same && zL[(uint64_t)s * cells + k] == z0;
        same = __all_sync(0xffffffffu, same);
        if (lane == 0u) flat[s] = same ? 1 : 0;
    }
}

}  // namespace hwfv1
