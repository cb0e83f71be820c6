// engine_iface.h -- the interface between the C ABI (api.cu) and the
// per-precision engines (engine_f64.cu, engine_f32.cu).
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "../../include/hwfv1.h"

namespace hwfv1 {

struct SkipNet;

class Engine {
   public:
    virtual ~Engine() {}
    virtual hwfv1_status init(const double* z, const double* h, const double* qx,
                              const double* qy) = 0;
    virtual hwfv1_status encode() = 0;
    virtual hwfv1_status flag() = 0;
    virtual hwfv1_status traverse(int64_t* num_leaves) = 0;
    virtual hwfv1_status step() = 0;
    virtual hwfv1_status decode() = 0;
    virtual hwfv1_status advance(double t_end, int64_t max_steps) = 0;
    virtual hwfv1_status advance_uniform(double t_end, int64_t max_steps) = 0;
    virtual hwfv1_status get_fields(double* h, double* qx, double* qy) = 0;
    virtual hwfv1_status set_fields(const double* h, const double* qx, const double* qy) = 0;
    virtual hwfv1_status get_leaves(uint32_t* out, int64_t cap, int64_t* n) = 0;
    virtual hwfv1_status get_flags(int which, uint32_t* out, int64_t cap_words) = 0;
    virtual hwfv1_status get_level(int field, int level, double* out) = 0;
    virtual hwfv1_status get_time(double* t, double* dt, int64_t* step) = 0;
    virtual hwfv1_status set_time(double t, double dt) = 0;
    virtual hwfv1_status get_stats(int64_t* M, double* smax3) = 0;
    virtual hwfv1_status profile_step(float* ms, const char** names, int32_t cap, int32_t* n) = 0;
    virtual hwfv1_status profile_update(int32_t reps, float* ms) = 0;
    virtual hwfv1_status get_counters(int64_t* steps, int64_t* leaf_updates, int64_t* active_updates,
                                      int64_t* wet_updates, int64_t* kernels_per_step) = 0;
    virtual hwfv1_status save(void* buf, size_t cap, size_t* used) = 0;
    virtual hwfv1_status load(const void* buf, size_t n) = 0;
    // learned subtree skip with the network's levels (skipnet.cu); net ==
    // nullptr turns it off
    virtual hwfv1_status set_skipnet(SkipNet* net, int audit_K, float margin, int predict_every) = 0;
    // learned subtree skip with the caller's levels (host, row-major over
    // level L-4); levels == nullptr turns it off
    virtual hwfv1_status set_skip_levels(const uint8_t* levels, int audit_K) = 0;
    virtual hwfv1_status get_skip_levels(int which, uint8_t* out, int64_t cap) = 0;
    // exact leaf-value store on (1) or off (0)
    virtual hwfv1_status set_leaf_store(int on) = 0;
    virtual hwfv1_status get_features(uint16_t* out, int64_t cap) = 0;
    virtual hwfv1_status get_labels(uint8_t* out, int64_t cap) = 0;
    std::string err;
};

Engine* make_engine_f64(const hwfv1_problem& spec, cudaStream_t stream);
Engine* make_engine_f32(const hwfv1_problem& spec, cudaStream_t stream);

// Many domains advanced together (batch.cuh).
class Batch {
   public:
    virtual ~Batch() {}
    virtual hwfv1_status init(const double* const* z, const double* const* h, const double* const* qx,
                              const double* const* qy) = 0;
    virtual hwfv1_status advance(double t_end, int64_t max_steps) = 0;
    virtual hwfv1_status autotune(int64_t trial_steps, int32_t* choice) = 0;
    virtual Engine* member(int d) = 0;
    virtual int size() const = 0;
    virtual int64_t launches_per_step() const = 0;
    std::string err;
};

Batch* make_batch_f64(const hwfv1_problem* specs, int n, cudaStream_t stream);
Batch* make_batch_f32(const hwfv1_problem* specs, int n, cudaStream_t stream);

struct SaveHeader {
    uint64_t magic;
    int32_t L, precision;
    double t, dt;
    int64_t step;
};
constexpr uint64_t kSaveMagic = 0x31564657484D5248ull;   // "HRMHWFV1"

}  // namespace hwfv1
