// skipnet.h -- host interface of the subtree CNN (skipnet.cu) used by the
// engine's learned step: a 3-layer 3x3 convolutional network (4 -> 16 -> 16
// -> 5 channels, ReLU between) over the level-(L-4) coefficients, BF16
// weights and activations, FP32 accumulation on the tensor cores.
#pragma once
#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace hwfv1 {

constexpr int kSkipIn = 4;        // h, qx, qy, z
constexpr int kSkipCh = 16;       // hidden channels
constexpr int kSkipCls = 5;       // max level L-4 .. L
constexpr int kSkipParams = 16 * 4 * 9 + 16 + 16 * 16 * 9 + 16 + 5 * 16 * 9 + 5;   // 3637

struct SkipNet;                   // weights, gradients, optimiser state (device)

// Activations of one forward/backward pass for up to `cap` pixels.
struct SkipWork {
    int64_t cap = 0;
    __nv_bfloat16 *A1 = nullptr, *A2 = nullptr;           // post-ReLU, [pix][16]
    float *Z1 = nullptr, *Z2 = nullptr, *Z3 = nullptr;     // pre-activations, [pix][16]
    __nv_bfloat16 *dZ1 = nullptr, *dZ2 = nullptr, *dZ3 = nullptr;
    float *dA1 = nullptr, *dA2 = nullptr;
};

SkipNet* skipnet_create(uint32_t seed);
void skipnet_destroy(SkipNet* net);
bool skipnet_set_params(SkipNet* net, const float* host, int64_t n);
bool skipnet_get_params(const SkipNet* net, float* host, int64_t n);
bool skipwork_reserve(SkipWork* w, int64_t npix);
void skipwork_free(SkipWork* w);
int* skipnet_err(SkipNet* net);

// logits [nimg*H*W][16] (classes 0..4 valid) of the images x [nimg][H][W][4]
// (bf16, channels last); asynchronous on `stream`, capturable.
cudaError_t skipnet_forward(const SkipNet* net, const __nv_bfloat16* x, int nimg, int H, int W,
                            SkipWork* work, cudaStream_t stream);

}  // namespace hwfv1

// the C ABI's opaque network handle
struct hwfv1_skipnet {
    hwfv1::SkipNet* net = nullptr;
};
