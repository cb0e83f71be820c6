// noalloc.cu -- hwfv1_traverse_noalloc: the leaf traversal and compaction
// for callers that cannot allocate device memory.
//
// The regular path (hwfv1_traverse) keeps its per-tile counts and offsets in
// buffers that hwfv1_init allocates.  Some callers cannot call cudaMalloc at
// all: a host application whose own pool allocator owns the whole device
// memory budget, a fixed-footprint deployment that must not grow after
// start-up, or a latency-bound loop that cannot afford the device-wide
// synchronisation cudaMalloc may imply.  For them this entry point takes the
// significance bits and output buffers from the caller and keeps its only
// scratch (the per-tile counts and offsets) in a file-scope __device__ array
// of fixed size.  Every GPU that loads the library holds that array
// (kMaxTiles * 2 * 4 bytes = 128 KiB) until the process exits.
#include <mutex>

#include "../../include/hwfv1.h"
#include "kernels.cuh"

namespace hwfv1 {
namespace {

constexpr int kNoAllocMaxL = 12;
constexpr int kNoAllocKt = 5;                                  // tile = 4^5 finest cells
constexpr uint32_t kMaxTiles = 1u << (2 * (kNoAllocMaxL - kNoAllocKt));   // 16384

// Scratch shared by every call on a device: counts at [0, kMaxTiles),
// offsets at [kMaxTiles, 2*kMaxTiles).  Host code must not pass this name
// to a kernel: on the host it is only a stand-in for the symbol, so its
// device address is looked up (below) and passed instead.
static __device__ __align__(256) uint32_t g_scratch[2 * kMaxTiles];

// Last address looked up per device, used only while the caller's stream
// is capturing a graph (a symbol lookup is not made during a capture).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint32_t* g_scratch_ptr[kMaxDevices] = {};

// exclusive scan of the tile counts into offsets, total to *num_leaves
__global__ void __launch_bounds__(1024) k_scan_noalloc(const uint32_t* __restrict__ counts,
                                                       uint32_t* __restrict__ offs, uint32_t ntiles,
                                                       uint32_t* __restrict__ num_leaves) {
    const uint32_t per = (ntiles + blockDim.x - 1) / blockDim.x;
    const uint32_t b = threadIdx.x * per, e = min(ntiles, b + per);
    uint32_t sum = 0;
    for (uint32_t i = b; i < e; ++i) sum += counts[i];
    uint32_t total;
    uint32_t run = block_excl_scan(sum, &total);
    for (uint32_t i = b; i < e; ++i) {
        offs[i] = run;
        run += counts[i];
    }
    if (threadIdx.x == 0) *num_leaves = total;
}

// leaves of each tile at its offset; entries past `cap` are not written
__global__ void __launch_bounds__(256) k_write_noalloc(const uint32_t* __restrict__ Sb,
                                                       const uint32_t* __restrict__ offs,
                                                       uint32_t* __restrict__ leaves, uint64_t cap,
                                                       int L, int kt) {
    __shared__ int s_l0;
    const uint32_t tile = blockIdx.x;
    if (threadIdx.x == 0) s_l0 = walk_root(Sb, L - kt, tile);
    __syncthreads();
    const TileWalk w = walk_tile(Sb, L, kt, tile, s_l0);
    const uint32_t hc = heads_of(w, L);
    const uint64_t pos = (uint64_t)offs[tile] + block_excl_scan(hc, nullptr);
    if (hc == 4u) {
        for (uint32_t e = 0; e < 4u; ++e)
            if (pos + e < cap) leaves[pos + e] = ((uint32_t)L << kLeafShift) | (w.m0 + e);
    } else if (hc == 1u && pos < cap) {
        leaves[pos] = ((uint32_t)w.l << kLeafShift) | (w.m0 >> (2 * (L - w.l)));
    }
}

// Device address of g_scratch in the current context.  Outside a stream
// capture it is looked up on every call (a host-side query that allocates
// nothing), so a context that was reset or replaced since the last call is
// never handed a stale address.  During a capture the last address looked
// up on this device is used; a capture needs one earlier uncaptured call.
cudaError_t scratch_address(cudaStream_t st, uint32_t** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<uint32_t*>(p);
    } else if (!g_scratch_ptr[dev]) {
        return cudaErrorStreamCaptureUnsupported;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace hwfv1

extern "C" hwfv1_status hwfv1_traverse_noalloc(const uint32_t* sig_bits, int32_t L, uint32_t* leaves,
                                               int64_t cap, uint32_t* num_leaves, void* stream) {
    using namespace hwfv1;
    if (!sig_bits || !leaves || !num_leaves || cap < 0) return HWFV1_ERR_INVALID_SPEC;
    if (L < 1 || L > kNoAllocMaxL) return HWFV1_ERR_INVALID_SPEC;   // scratch holds L <= 12
    // an error left pending by an earlier, unrelated call stays pending for
    // its owner: this call launches nothing and reports HWFV1_ERR_CUDA
    if (cudaPeekAtLastError() != cudaSuccess) return HWFV1_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t* scratch = nullptr;
    if (scratch_address(st, &scratch) != cudaSuccess) return HWFV1_ERR_CUDA;
    const int kt = L < kNoAllocKt ? L : kNoAllocKt;
    const uint32_t ntiles = 1u << (2 * (L - kt));
    uint32_t* counts = scratch;
    uint32_t* offs = scratch + kMaxTiles;
    // every count and offset the call reads is written by the call itself
    k_trav_count_walk<<<ntiles, 256, 0, st>>>(sig_bits, counts, L, kt, nullptr);
    if (cudaGetLastError() != cudaSuccess) return HWFV1_ERR_CUDA;
    k_scan_noalloc<<<1, 1024, 0, st>>>(counts, offs, ntiles, num_leaves);
    if (cudaGetLastError() != cudaSuccess) return HWFV1_ERR_CUDA;
    k_write_noalloc<<<ntiles, 256, 0, st>>>(sig_bits, offs, leaves, (uint64_t)cap, L, kt);
    return cudaGetLastError() == cudaSuccess ? HWFV1_OK : HWFV1_ERR_CUDA;
}
