// skipnet.cu -- the subtree CNN on the tensor cores: forward, backward and
// Adam, each convolution an implicit GEMM issued with tcgen05.mma (BF16
// operands staged in shared memory, FP32 accumulators in TMEM).
//
//   forward       Z[p][o]  = b[o] + sum_k Xcol[p][k] W[o][k]      M=128 pixels, N=16, K=48|144
//   grad input    dXcol    = dZ W  -> scattered back (col2im)      M=128 pixels, N=K, K=16
//   grad weights  dW[k][o] = sum_p Xcol[p][k] dZ[p][o]            M=128 k-rows, N=16, K=128 pixels
//
// k = tap * cin + c with tap = 3*(di+1) + (dj+1): the im2col of a 3x3 window
// with zero padding over channels-last images.  Parameters are kept in FP32
// (the CPU oracle's layout [cout][cin][3][3]) and packed to BF16 operand
// tiles after every update.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/hwfv1.h"
#include "skipnet.h"
#include "tcgen05.cuh"

namespace hwfv1 {
namespace {

using bf16 = __nv_bfloat16;

struct Layer {
    int cin, kpad, cout, offw, offb;
};
constexpr Layer kLayers[3] = {
    {4, 48, 16, 0, 576},
    {16, 144, 16, 592, 2896},
    {16, 144, 5, 2912, 3632},
};
__constant__ Layer c_layers[3] = {
    {4, 48, 16, 0, 576},
    {16, 144, 16, 592, 2896},
    {16, 144, 5, 2912, 3632},
};
constexpr uint32_t kWaitLimit = 1u << 24;   // polls of an mbarrier before giving up

__device__ __forceinline__ void put_bf16(uint8_t* base, uint32_t off, bf16 v) {
    *reinterpret_cast<bf16*>(base + off) = v;
}

__device__ __forceinline__ uint32_t tmem_cols_for(int n) {
    uint32_t c = 32;
    while ((int)c < n) c <<= 1;
    return c;
}

// ---------------------------------------------------------------------------
// Weight packing: FP32 [cout][cin][3][3] -> the B tiles of the forward GEMM
// (N = 16 rows of cout, K = kpad) and of the input-gradient GEMM (N = kpad
// rows, K = 16 cout), both in the core-matrix layout.
// ---------------------------------------------------------------------------
__global__ void k_pack(const float* __restrict__ params, bf16* __restrict__ wf, bf16* __restrict__ wt) {
    const Layer ly = c_layers[blockIdx.y];
    bf16* f = wf + blockIdx.y * (16 * 144);
    bf16* t = wt + blockIdx.y * (144 * 16);
    for (int idx = threadIdx.x; idx < 16 * ly.kpad; idx += blockDim.x) {
        const int o = idx / ly.kpad, k = idx % ly.kpad;
        float v = 0.f;
        if (o < ly.cout && k < 9 * ly.cin) {
            const int tap = k / ly.cin, c = k % ly.cin;
            v = params[ly.offw + (o * ly.cin + c) * 9 + tap];
        }
        const bf16 b = __float2bfloat16(v);
        f[tc::core_off(o, k, ly.kpad / 8) / 2] = b;
        t[tc::core_off(k, o, 2) / 2] = b;
    }
}

// im2col value (pixel p, k) of a channels-last image batch
struct Img {
    int B, H, W, cin;
};
__device__ __forceinline__ bf16 xcol(const bf16* __restrict__ X, const Img& g, int p, int k) {
    const int npix = g.B * g.H * g.W;
    if (p >= npix || k >= 9 * g.cin) return __float2bfloat16(0.f);
    const int tap = k / g.cin, c = k % g.cin;
    const int b = p / (g.H * g.W), rem = p % (g.H * g.W);
    const int y = rem / g.W + tap / 3 - 1, x = rem % g.W + tap % 3 - 1;
    if (y < 0 || y >= g.H || x < 0 || x >= g.W) return __float2bfloat16(0.f);
    return X[((size_t)(b * g.H + y) * g.W + x) * g.cin + c];
}

// The im2col row of pixel p (k = tap * cin + c over the 3x3 taps, zero
// outside the image and for k >= 9 cin) written to row `row` of the
// core-matrix operand: the pixel's position is formed once, and each tap's
// channels move as one 16-byte (cin % 8 == 0) or 8-byte (cin == 4) vector.
__device__ __forceinline__ void im2col_row(const bf16* __restrict__ X, const Img& g, int p, uint32_t row,
                                           uint8_t* sA, int kpad) {
    const uint32_t kb = (uint32_t)kpad / 8u;
    const int npix = g.B * g.H * g.W;
    if (g.cin % 8 != 0 && g.cin != 4) {
        for (int k = 0; k < kpad; ++k) put_bf16(sA, tc::core_off(row, k, kb), xcol(X, g, p, k));
        return;
    }
    const bool inside = p < npix;
    int b = 0, y = 0, x = 0;
    if (inside) {
        b = p / (g.H * g.W);
        const int rem = p % (g.H * g.W);
        y = rem / g.W;
        x = rem % g.W;
    }
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
        const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
        const bool ok = inside && yy >= 0 && yy < g.H && xx >= 0 && xx < g.W;
        const size_t at = ok ? ((size_t)(b * g.H + yy) * g.W + xx) * g.cin : 0;
        if (g.cin == 4) {
            const uint2 v = ok ? __ldg(reinterpret_cast<const uint2*>(X + at)) : make_uint2(0u, 0u);
            *reinterpret_cast<uint2*>(sA + tc::core_off(row, tap * 4, kb)) = v;
        } else {
            for (int cb = 0; cb < g.cin / 8; ++cb) {
                const uint4 v = ok ? __ldg(reinterpret_cast<const uint4*>(X + at) + cb) : make_uint4(0u, 0u, 0u, 0u);
                *reinterpret_cast<uint4*>(sA + tc::core_off(row, tap * g.cin + cb * 8, kb)) = v;
            }
        }
    }
    for (int k = 9 * g.cin; k < kpad; ++k) put_bf16(sA, tc::core_off(row, k, kb), __float2bfloat16(0.f));
}

// Shared TMEM/mbarrier bookkeeping of one CTA (128 threads).
struct TcCta {
    uint64_t bar;
    uint32_t tmem;
};

__device__ __forceinline__ void tc_begin(TcCta& s, uint32_t ncols) {
    if (threadIdx.x < 32) {
        tc::tmem_alloc(&s.tmem, ncols);
        tc::tmem_relinquish();
    }
    if (threadIdx.x == 0) {
        tc::mbar_init(&s.bar, 1);
        tc::fence_mbar_init();
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

// Wait for the committed MMAs (bounded); on timeout flag the error and wait
// once more (bounded) so that TMEM is not freed under a running MMA.
__device__ __forceinline__ void tc_wait(TcCta& s, int* err) {
    if (!tc::mbar_wait_bounded(&s.bar, 0, kWaitLimit)) {
        if (threadIdx.x == 0) atomicOr(err, 1);
        tc::mbar_wait_bounded(&s.bar, 0, kWaitLimit);
    }
    tc::fence_after_sync();
}

__device__ __forceinline__ void tc_end(TcCta& s, uint32_t ncols) {
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc::fence_after_sync();
        tc::tmem_dealloc(s.tmem, ncols);
    }
}

// ---------------------------------------------------------------------------
// Forward convolution: 128 pixels per CTA.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_conv_fwd(const bf16* __restrict__ X, Img g,
                                                  const bf16* __restrict__ wf, int kpad,
                                                  const float* __restrict__ bias, int cout,
                                                  float* __restrict__ Z, bf16* __restrict__ A, int relu,
                                                  int* err) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ TcCta s;
    uint8_t* sA = smem;                        // 128 x kpad
    uint8_t* sB = smem + 256 * kpad;           // 16 x kpad
    const int kb = kpad / 8;
    const int t = threadIdx.x;
    const int p = blockIdx.x * 128 + t;
    im2col_row(X, g, p, (uint32_t)t, sA, kpad);
    const uint4* src = reinterpret_cast<const uint4*>(wf);
    for (int i = t; i < 2 * kpad; i += 128) reinterpret_cast<uint4*>(sB)[i] = src[i];
    tc_begin(s, 32);
    if (t == 0) {
        const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sB);
        for (int kk = 0; kk < kpad / 16; ++kk)
            tc::mma_bf16(s.tmem, tc::sdesc(a0 + kk * 256, 128, kb * 128), tc::sdesc(b0 + kk * 256, 128, kb * 128),
                         tc::idesc_bf16(128, 16), kk > 0);
        tc::mma_commit(&s.bar);
    }
    tc_wait(s, err);
    float v[16];
    tc::tmem_ld16(s.tmem + ((uint32_t)(32 * (t >> 5)) << 16), v);
    const int npix = g.B * g.H * g.W;
    if (p < npix) {
#pragma unroll
        for (int o = 0; o < 16; ++o) {
            const float z = o < cout ? v[o] + bias[o] : 0.f;
            Z[(size_t)p * 16 + o] = z;
            if (A) A[(size_t)p * 16 + o] = __float2bfloat16(relu ? fmaxf(z, 0.f) : z);
        }
    }
    tc_end(s, 32);
}

// ---------------------------------------------------------------------------
// Input gradient: dXcol = dZ W (K = 16 output channels) into dcol [pix][kpad];
// k_col2im then sums each input cell's nine taps in a fixed order (no float
// atomics: the same gradients on every run).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_conv_bwd_data(const bf16* __restrict__ dZ, Img g,
                                                       const bf16* __restrict__ wt, int kpad,
                                                       float* __restrict__ dcol, int* err) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ TcCta s;
    uint8_t* sA = smem;                        // 128 x 16
    uint8_t* sB = smem + 4096;                 // kpad x 16
    const int t = threadIdx.x;
    const int p = blockIdx.x * 128 + t;
    const int npix = g.B * g.H * g.W;
    for (int o = 0; o < 16; ++o)
        put_bf16(sA, tc::core_off(t, o, 2), p < npix ? dZ[(size_t)p * 16 + o] : __float2bfloat16(0.f));
    const uint4* src = reinterpret_cast<const uint4*>(wt);
    for (int i = t; i < 2 * kpad; i += 128) reinterpret_cast<uint4*>(sB)[i] = src[i];
    const uint32_t ncols = tmem_cols_for(kpad);
    tc_begin(s, ncols);
    if (t == 0) {
        tc::mma_bf16(s.tmem, tc::sdesc(tc::smem_addr(sA), 128, 256), tc::sdesc(tc::smem_addr(sB), 128, 256),
                     tc::idesc_bf16(128, kpad), 0);
        tc::mma_commit(&s.bar);
    }
    tc_wait(s, err);
    for (int c0 = 0; c0 < kpad; c0 += 16) {
        float v[16];
        tc::tmem_ld16(s.tmem + ((uint32_t)(32 * (t >> 5)) << 16) + c0, v);
        if (p < npix) {
#pragma unroll
            for (int j = 0; j < 16; ++j) dcol[(size_t)p * kpad + c0 + j] = v[j];
        }
    }
    tc_end(s, ncols);
}

// dX[b][y][x][c] = sum over the taps (0..8, in order) of the column entry of
// the output cell that the tap maps onto (b, y, x): the transpose of the
// forward's im2col.
__global__ void k_col2im(const float* __restrict__ dcol, Img g, int kpad, float* __restrict__ dX) {
    const int64_t n = (int64_t)g.B * g.H * g.W * g.cin;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % g.cin);
        const int64_t q = i / g.cin;
        const int x = (int)(q % g.W), y = (int)((q / g.W) % g.H), b = (int)(q / ((int64_t)g.W * g.H));
        float acc = 0.f;
        for (int tap = 0; tap < 9; ++tap) {
            const int ys = y - (tap / 3 - 1), xs = x - (tap % 3 - 1);     // the output cell of this tap
            if (ys < 0 || ys >= g.H || xs < 0 || xs >= g.W) continue;
            acc += dcol[((size_t)(b * g.H + ys) * g.W + xs) * kpad + tap * g.cin + c];
        }
        dX[i] = acc;
    }
}

// ---------------------------------------------------------------------------
// Weight gradient of 128 pixels: D[k][o] = sum_p Xcol[p][k] dZ[p][o] and
// sum_p dZ[p][o], this block's part (part + blockIdx.x * (16 kpad + 16):
// [o][k] then [o]); k_sum_parts adds the blocks' parts in block order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_conv_bwd_weight(const bf16* __restrict__ X, Img g,
                                                         const bf16* __restrict__ dZ, int kpad, int cout,
                                                         float* __restrict__ part, int* err) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ TcCta s;
    const int mt = (kpad + 127) / 128;         // 128-row tiles of k
    uint8_t* sA = smem;                        // mt*128 x 128 (rows k, K = pixels)
    uint8_t* sB = smem + mt * 32768;           // 16 x 128 (rows o)
    const int t = threadIdx.x;
    const int p = blockIdx.x * 128 + t;
    const int npix = g.B * g.H * g.W;
    for (int k = 0; k < mt * 128; ++k) put_bf16(sA, tc::core_off(k, t, 16), xcol(X, g, p, k));
    float dzv[16];
#pragma unroll
    for (int o = 0; o < 16; ++o) {
        const bf16 d = p < npix ? dZ[(size_t)p * 16 + o] : __float2bfloat16(0.f);
        dzv[o] = __bfloat162float(d);
        put_bf16(sB, tc::core_off(o, t, 16), d);
    }
    tc_begin(s, 32);
    if (t == 0) {
        const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sB);
        for (int m = 0; m < mt; ++m)
            for (int kk = 0; kk < 8; ++kk)
                tc::mma_bf16(s.tmem + 16 * m, tc::sdesc(a0 + m * 32768 + kk * 256, 128, 2048),
                             tc::sdesc(b0 + kk * 256, 128, 2048), tc::idesc_bf16(128, 16), kk > 0);
        tc::mma_commit(&s.bar);
    }
    tc_wait(s, err);
    float* const pw = part + (size_t)blockIdx.x * (16 * kpad + 16);
    for (int m = 0; m < mt; ++m) {
        float v[16];
        tc::tmem_ld16(s.tmem + ((uint32_t)(32 * (t >> 5)) << 16) + 16 * m, v);
        const int k = m * 128 + t;
        if (k < kpad) {
#pragma unroll
            for (int o = 0; o < 16; ++o) pw[(size_t)o * kpad + k] = (o < cout && k < 9 * g.cin) ? v[o] : 0.f;
        }
    }
    // bias gradient: warp sums, then the four warps' sums in order
    __shared__ float sdb[4][16];
#pragma unroll
    for (int o = 0; o < 16; ++o) {
        float x = dzv[o];
        for (int off = 16; off; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        if ((t & 31) == 0) sdb[t >> 5][o] = x;
    }
    __syncthreads();
    if (t < 16) pw[16 * kpad + t] = t < cout ? ((sdb[0][t] + sdb[1][t]) + sdb[2][t]) + sdb[3][t] : 0.f;
    tc_end(s, 32);
}

// dW[o][k] and db[o]: the nb blocks' parts added in a fixed order, one warp
// per entry (lane l adds blocks l, l + 32, ... in turn, then a fixed
// shuffle tree adds the lanes' sums).
__global__ void k_sum_parts(const float* __restrict__ part, int nb, int kpad, float* __restrict__ dW,
                            float* __restrict__ db) {
    const int per = 16 * kpad + 16;
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < per; e += nw) {
        float acc = 0.f;
        for (int b = lane; b < nb; b += 32) acc += part[(size_t)b * per + e];
        for (int off = 16; off; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
        if (lane == 0) {
            if (e < 16 * kpad) dW[e] = acc;
            else db[e - 16 * kpad] = acc;
        }
    }
}

// softmax cross-entropy over the 5 classes of every pixel
__global__ void k_xent(const float* __restrict__ Z3, const uint8_t* __restrict__ labels, int npix,
                       float inv_npix, bf16* __restrict__ dZ3, double* loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (p < npix) {
        float z[kSkipCls], m = -INFINITY;
        for (int o = 0; o < kSkipCls; ++o) {
            z[o] = Z3[(size_t)p * 16 + o];
            m = fmaxf(m, z[o]);
        }
        float se = 0.f;
        for (int o = 0; o < kSkipCls; ++o) se += expf(z[o] - m);
        const int y = labels[p];
        for (int o = 0; o < 16; ++o) {
            float d = 0.f;
            if (o < kSkipCls) d = (expf(z[o] - m) / se - (o == y ? 1.f : 0.f)) * inv_npix;
            dZ3[(size_t)p * 16 + o] = __float2bfloat16(d);
        }
        l = (double)(logf(se) + m - z[y < kSkipCls ? y : 0]);
    }
    for (int off = 16; off; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, l);
}

// dZ = dA * (Z > 0), to bf16
__global__ void k_relu_bwd(const float* __restrict__ dA, const float* __restrict__ Z, int64_t n,
                           bf16* __restrict__ dZ) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dZ[i] = __float2bfloat16(Z[i] > 0.f ? dA[i] : 0.f);
}

// dW [cout][kpad] (k = tap*cin + c) + db -> the flat FP32 gradient layout
__global__ void k_unpack_grads(const float* __restrict__ dWl, const float* __restrict__ dbl, int layer,
                               float* __restrict__ grads) {
    const Layer ly = c_layers[layer];
    for (int idx = threadIdx.x; idx < ly.cout * ly.cin * 9; idx += blockDim.x) {
        const int o = idx / (ly.cin * 9), r = idx % (ly.cin * 9), c = r / 9, tap = r % 9;
        grads[ly.offw + idx] = dWl[(size_t)o * ly.kpad + tap * ly.cin + c];
    }
    for (int o = threadIdx.x; o < ly.cout; o += blockDim.x) grads[ly.offb + o] = dbl[o];
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        m[i] = b1 * m[i] + (1.f - b1) * g[i];
        v[i] = b2 * v[i] + (1.f - b2) * g[i] * g[i];
        w[i] -= lr * (m[i] / c1) / (sqrtf(v[i] / c2) + eps);
    }
}

template <typename P>
bool dalloc(P** p, size_t bytes) {
    if (cudaMalloc(reinterpret_cast<void**>(p), bytes) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

size_t smem_fwd(int kpad) { return 288u * kpad; }
size_t smem_bwd_data(int kpad) { return 4096u + 32u * kpad; }
size_t smem_bwd_weight(int kpad) { return ((kpad + 127) / 128) * 32768u + 4096u; }

}  // namespace

struct SkipNet {
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    bf16 *wf = nullptr, *wt = nullptr;      // 3 layers x (16 x 144) and (144 x 16)
    float *dW = nullptr, *db = nullptr;     // per-layer weight/bias gradient scratch [16][144], [16]
    // training scratch of the fixed-order reductions: the input gradient's
    // columns [pix][144] and the weight gradient's per-block parts
    float *dcol = nullptr, *part = nullptr;
    int64_t dcol_cap = 0, part_cap = 0;
    int* err = nullptr;
    double* loss = nullptr;
    int64_t adam_t = 0;
    SkipWork work;
};

static void pack(SkipNet* n, cudaStream_t st) {
    k_pack<<<dim3(1, 3), 256, 0, st>>>(n->params, n->wf, n->wt);
}

SkipNet* skipnet_create(uint32_t seed) {
    static bool attrs = false;
    if (!attrs) {
        cudaFuncSetAttribute(k_conv_bwd_weight, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bwd_weight(144));
        attrs = true;
    }
    SkipNet* n = new SkipNet;
    bool ok = dalloc(&n->params, sizeof(float) * kSkipParams) && dalloc(&n->grads, sizeof(float) * kSkipParams) &&
              dalloc(&n->m, sizeof(float) * kSkipParams) && dalloc(&n->v, sizeof(float) * kSkipParams) &&
              dalloc(&n->wf, sizeof(bf16) * 3 * 16 * 144) && dalloc(&n->wt, sizeof(bf16) * 3 * 144 * 16) &&
              dalloc(&n->dW, sizeof(float) * 16 * 144) && dalloc(&n->db, sizeof(float) * 16) &&
              dalloc(&n->err, sizeof(int)) && dalloc(&n->loss, sizeof(double));
    if (!ok) {
        skipnet_destroy(n);
        return nullptr;
    }
    cudaMemset(n->m, 0, sizeof(float) * kSkipParams);
    cudaMemset(n->v, 0, sizeof(float) * kSkipParams);
    cudaMemset(n->err, 0, sizeof(int));
    // He initialisation from a seeded xorshift + Box-Muller on the host
    std::vector<float> h(kSkipParams, 0.f);
    uint64_t s = 0x9E3779B97F4A7C15ull ^ seed;
    auto uni = [&]() {
        s ^= s << 13;
        s ^= s >> 7;
        s ^= s << 17;
        return ((s >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    };
    for (const Layer& ly : kLayers) {
        const double sd = std::sqrt(2.0 / (9.0 * ly.cin));
        for (int i = 0; i < ly.cout * ly.cin * 9; ++i) {
            const double u1 = uni(), u2 = uni();
            h[ly.offw + i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
        }
    }
    skipnet_set_params(n, h.data(), kSkipParams);
    return n;
}

void skipnet_destroy(SkipNet* n) {
    if (!n) return;
    for (void* p : {(void*)n->params, (void*)n->grads, (void*)n->m, (void*)n->v, (void*)n->wf, (void*)n->wt,
                    (void*)n->dW, (void*)n->db, (void*)n->err, (void*)n->loss, (void*)n->dcol, (void*)n->part})
        if (p) cudaFree(p);
    skipwork_free(&n->work);
    delete n;
}

bool skipnet_set_params(SkipNet* n, const float* host, int64_t cnt) {
    if (cnt != kSkipParams) return false;
    if (cudaMemcpy(n->params, host, sizeof(float) * kSkipParams, cudaMemcpyHostToDevice) != cudaSuccess) return false;
    pack(n, 0);
    return cudaDeviceSynchronize() == cudaSuccess;
}

bool skipnet_get_params(const SkipNet* n, float* host, int64_t cnt) {
    if (cnt != kSkipParams) return false;
    return cudaMemcpy(host, n->params, sizeof(float) * kSkipParams, cudaMemcpyDeviceToHost) == cudaSuccess;
}

int* skipnet_err(SkipNet* n) { return n->err; }

bool skipwork_reserve(SkipWork* w, int64_t npix) {
    if (w->cap >= npix) return true;
    skipwork_free(w);
    const size_t nf = sizeof(float) * 16 * npix, nb = sizeof(bf16) * 16 * npix;
    bool ok = dalloc(&w->A1, nb) && dalloc(&w->A2, nb) && dalloc(&w->Z1, nf) && dalloc(&w->Z2, nf) &&
              dalloc(&w->Z3, nf) && dalloc(&w->dZ1, nb) && dalloc(&w->dZ2, nb) && dalloc(&w->dZ3, nb) &&
              dalloc(&w->dA1, nf) && dalloc(&w->dA2, nf);
    if (!ok) {
        skipwork_free(w);
        return false;
    }
    w->cap = npix;
    return true;
}

void skipwork_free(SkipWork* w) {
    for (void* p : {(void*)w->A1, (void*)w->A2, (void*)w->Z1, (void*)w->Z2, (void*)w->Z3, (void*)w->dZ1,
                    (void*)w->dZ2, (void*)w->dZ3, (void*)w->dA1, (void*)w->dA2})
        if (p) cudaFree(p);
    *w = SkipWork();
}

cudaError_t skipnet_forward(const SkipNet* n, const bf16* x, int nimg, int H, int W, SkipWork* w,
                            cudaStream_t st) {
    const int npix = nimg * H * W;
    if (w->cap < npix) return cudaErrorInvalidValue;
    const int nb = (npix + 127) / 128;
    Img g{nimg, H, W, 4};
    k_conv_fwd<<<nb, 128, smem_fwd(48), st>>>(x, g, n->wf, 48, n->params + kLayers[0].offb, 16, w->Z1, w->A1, 1,
                                              n->err);
    g.cin = 16;
    k_conv_fwd<<<nb, 128, smem_fwd(144), st>>>(w->A1, g, n->wf + 16 * 144, 144, n->params + kLayers[1].offb, 16,
                                               w->Z2, w->A2, 1, n->err);
    k_conv_fwd<<<nb, 128, smem_fwd(144), st>>>(w->A2, g, n->wf + 2 * 16 * 144, 144, n->params + kLayers[2].offb,
                                               5, w->Z3, nullptr, 0, n->err);
    return cudaGetLastError();
}

// Forward + loss + backward; gradients (flat FP32) in n->grads, loss in n->loss.
static cudaError_t skipnet_backprop(SkipNet* n, const bf16* x, const uint8_t* labels, int nimg, int H, int W,
                                    cudaStream_t st) {
    SkipWork* w = &n->work;
    const int npix = nimg * H * W;
    if (!skipwork_reserve(w, npix)) return cudaErrorMemoryAllocation;
    const int64_t nb_all = (npix + 127) / 128;
    if (n->dcol_cap < npix) {
        if (n->dcol) cudaFree(n->dcol);
        n->dcol = nullptr;
        n->dcol_cap = 0;
        if (!dalloc(&n->dcol, sizeof(float) * 144 * (size_t)npix)) return cudaErrorMemoryAllocation;
        n->dcol_cap = npix;
    }
    if (n->part_cap < nb_all) {
        if (n->part) cudaFree(n->part);
        n->part = nullptr;
        n->part_cap = 0;
        if (!dalloc(&n->part, sizeof(float) * (16 * 144 + 16) * (size_t)nb_all)) return cudaErrorMemoryAllocation;
        n->part_cap = nb_all;
    }
    cudaError_t e = skipnet_forward(n, x, nimg, H, W, w, st);
    if (e != cudaSuccess) return e;
    const int nb = (npix + 127) / 128;
    cudaMemsetAsync(n->loss, 0, sizeof(double), st);
    k_xent<<<(npix + 255) / 256, 256, 0, st>>>(w->Z3, labels, npix, 1.f / npix, w->dZ3, n->loss);
    const bf16* acts[3] = {x, w->A1, w->A2};
    bf16* dZ[3] = {w->dZ1, w->dZ2, w->dZ3};
    float* dA[3] = {nullptr, w->dA1, w->dA2};
    const float* Zs[3] = {w->Z1, w->Z2, nullptr};
    for (int l = 2; l >= 0; --l) {
        const Layer ly = kLayers[l];
        Img g{nimg, H, W, ly.cin};
        k_conv_bwd_weight<<<nb, 128, smem_bwd_weight(ly.kpad), st>>>(acts[l], g, dZ[l], ly.kpad, ly.cout, n->part,
                                                                     n->err);
        k_sum_parts<<<(16 * ly.kpad + 16 + 7) / 8, 256, 0, st>>>(n->part, nb, ly.kpad, n->dW, n->db);
        k_unpack_grads<<<1, 256, 0, st>>>(n->dW, n->db, l, n->grads);
        if (l > 0) {
            // gradient w.r.t. this layer's input = the previous layer's activation
            k_conv_bwd_data<<<nb, 128, smem_bwd_data(ly.kpad), st>>>(dZ[l], g, n->wt + l * 144 * 16, ly.kpad,
                                                                     n->dcol, n->err);
            k_col2im<<<(int)std::min<int64_t>(((int64_t)npix * g.cin + 255) / 256, 4096), 256, 0, st>>>(
                n->dcol, g, ly.kpad, dA[l]);
            k_relu_bwd<<<(npix * 16 + 255) / 256, 256, 0, st>>>(dA[l], Zs[l - 1], (int64_t)npix * 16, dZ[l - 1]);
        }
    }
    return cudaGetLastError();
}

}  // namespace hwfv1

// ---------------------------------------------------------------------------
// C ABI of the network (include/hwfv1.h)
// ---------------------------------------------------------------------------
namespace {
hwfv1_status net_status(hwfv1::SkipNet* n, cudaError_t e) {
    if (e != cudaSuccess) return HWFV1_ERR_CUDA;
    int err = 0;
    if (cudaMemcpy(&err, hwfv1::skipnet_err(n), sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return HWFV1_ERR_CUDA;
    return err ? HWFV1_ERR_TIMEOUT : HWFV1_OK;
}
bool image_ok(int nimg, int H, int W) {
    return nimg >= 1 && H >= 1 && W >= 1 && (int64_t)nimg * H * W <= (1ll << 28);
}
}  // namespace

extern "C" {

int32_t hwfv1_skipnet_num_params(void) { return hwfv1::kSkipParams; }

hwfv1_status hwfv1_skipnet_create(uint32_t seed, hwfv1_skipnet** out) {
    if (!out) return HWFV1_ERR_INVALID_SPEC;
    *out = nullptr;
    hwfv1::SkipNet* n = hwfv1::skipnet_create(seed);
    if (!n) return HWFV1_ERR_OOM;
    *out = new hwfv1_skipnet{n};
    return cudaDeviceSynchronize() == cudaSuccess ? HWFV1_OK : HWFV1_ERR_CUDA;
}

hwfv1_status hwfv1_skipnet_set_params(hwfv1_skipnet* s, const float* host, int64_t n) {
    if (!s || !host) return HWFV1_ERR_INVALID_SPEC;
    return hwfv1::skipnet_set_params(s->net, host, n) ? HWFV1_OK : HWFV1_ERR_INVALID_SPEC;
}

hwfv1_status hwfv1_skipnet_get_params(hwfv1_skipnet* s, float* host, int64_t n) {
    if (!s || !host) return HWFV1_ERR_INVALID_SPEC;
    return hwfv1::skipnet_get_params(s->net, host, n) ? HWFV1_OK : HWFV1_ERR_INVALID_SPEC;
}

hwfv1_status hwfv1_skipnet_forward(hwfv1_skipnet* s, const uint16_t* x, int32_t nimg, int32_t H, int32_t W,
                                   float* logits) {
    if (!s || !x || !logits || !image_ok(nimg, H, W)) return HWFV1_ERR_INVALID_SPEC;
    hwfv1::SkipNet* n = s->net;
    const int64_t npix = (int64_t)nimg * H * W;
    if (!hwfv1::skipwork_reserve(&n->work, npix)) return HWFV1_ERR_OOM;
    cudaError_t e = hwfv1::skipnet_forward(n, reinterpret_cast<const __nv_bfloat16*>(x), nimg, H, W, &n->work, 0);
    if (e == cudaSuccess)
        e = cudaMemcpy(logits, n->work.Z3, sizeof(float) * 16 * npix, cudaMemcpyDeviceToDevice);
    return net_status(n, e);
}

hwfv1_status hwfv1_skipnet_gradients(hwfv1_skipnet* s, const uint16_t* x, const uint8_t* labels, int32_t nimg,
                                     int32_t H, int32_t W, double* loss, float* grads_host) {
    if (!s || !x || !labels || !image_ok(nimg, H, W)) return HWFV1_ERR_INVALID_SPEC;
    hwfv1::SkipNet* n = s->net;
    cudaError_t e = hwfv1::skipnet_backprop(n, reinterpret_cast<const __nv_bfloat16*>(x), labels, nimg, H, W, 0);
    if (e == cudaSuccess && loss) {
        double l = 0;
        e = cudaMemcpy(&l, n->loss, sizeof(double), cudaMemcpyDeviceToHost);
        *loss = l / ((double)nimg * H * W);
    }
    if (e == cudaSuccess && grads_host)
        e = cudaMemcpy(grads_host, n->grads, sizeof(float) * hwfv1::kSkipParams, cudaMemcpyDeviceToHost);
    return net_status(n, e);
}

hwfv1_status hwfv1_skipnet_train(hwfv1_skipnet* s, const uint16_t* x, const uint8_t* labels, int32_t nimg,
                                 int32_t H, int32_t W, int32_t batch, int32_t epochs, float lr, uint32_t seed,
                                 double* last_loss) {
    if (!s || !x || !labels || !image_ok(nimg, H, W) || batch < 1 || batch > nimg || epochs < 0 || !(lr > 0.f))
        return HWFV1_ERR_INVALID_SPEC;
    hwfv1::SkipNet* n = s->net;
    const int nbatch = nimg / batch;
    const int64_t per = (int64_t)batch * H * W;
    std::vector<int> order(nbatch);
    uint64_t r = 0x2545F4914F6CDD1Dull ^ seed;
    cudaError_t e = cudaSuccess;
    double ls = 0.0;
    for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
        for (int i = 0; i < nbatch; ++i) order[i] = i;
        for (int i = nbatch - 1; i > 0; --i) {          // Fisher-Yates with xorshift
            r ^= r << 13;
            r ^= r >> 7;
            r ^= r << 17;
            const int j = (int)(r % (uint64_t)(i + 1));
            std::swap(order[i], order[j]);
        }
        for (int bi = 0; bi < nbatch && e == cudaSuccess; ++bi) {
            const int b = order[bi];
            const __nv_bfloat16* xb = reinterpret_cast<const __nv_bfloat16*>(x) + (size_t)b * per * 4;
            e = hwfv1::skipnet_backprop(n, xb, labels + (size_t)b * per, batch, H, W, 0);
            n->adam_t++;
            const float b1 = 0.9f, b2 = 0.999f;
            const float c1 = 1.f - std::pow(b1, (float)n->adam_t), c2 = 1.f - std::pow(b2, (float)n->adam_t);
            hwfv1::k_adam<<<(hwfv1::kSkipParams + 255) / 256, 256>>>(n->params, n->grads, n->m, n->v,
                                                                    hwfv1::kSkipParams, lr, b1, b2, 1e-8f, c1, c2);
            hwfv1::pack(n, 0);
            if (e == cudaSuccess) e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess && last_loss) {
        e = cudaMemcpy(&ls, n->loss, sizeof(double), cudaMemcpyDeviceToHost);
        *last_loss = ls / (double)per;
    }
    return net_status(n, e);
}

void hwfv1_skipnet_destroy(hwfv1_skipnet* s) {
    if (!s) return;
    hwfv1::skipnet_destroy(s->net);
    delete s;
}

}  // extern "C"
