// api.cu -- the extern "C" boundary of the HWFV1 library (include/hwfv1.h):
// argument validation, handle bookkeeping, dispatch to the 64- or 32-bit
// engine.
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "engine_iface.h"
#include "skipnet.h"

struct hwfv1_handle {
    hwfv1::Engine* eng = nullptr;
    std::string msg;
    bool borrowed = false;       // a member view of a batch: the batch owns the engine
};

struct hwfv1_batch {
    hwfv1::Batch* b = nullptr;
    std::vector<hwfv1_handle*> views;
    std::string msg;
};

namespace {

hwfv1_status spec_error(const char* why, std::string* msg) {
    if (msg) *msg = why;
    return HWFV1_ERR_INVALID_SPEC;
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

// Validate a problem description before any device work.
hwfv1_status validate(const hwfv1_problem* s, std::string* msg) {
    if (!s) return spec_error("spec is NULL", msg);
    if (s->L < 1 || s->L > 14) return spec_error("L must be in 1..14", msg);
    if (!finite_pos(s->lx) || !finite_pos(s->ly)) return spec_error("lx, ly must be > 0", msg);
    if (!std::isfinite(s->x0) || !std::isfinite(s->y0)) return spec_error("x0, y0 must be finite", msg);
    if (!(s->eps == 0.0 || (s->eps >= 1e-200 && s->eps <= 1e300)))
        return spec_error("eps must be 0 or in [1e-200, 1e300]", msg);
    if (!(std::isfinite(s->cfl) && s->cfl > 0.0 && s->cfl <= 1.0)) return spec_error("cfl must be in (0, 1]", msg);
    if (!finite_pos(s->g)) return spec_error("g must be > 0", msg);
    if (!(std::isfinite(s->manning_n) && s->manning_n >= 0.0)) return spec_error("manning_n must be >= 0", msg);
    if (!finite_pos(s->tol_h)) return spec_error("tol_h must be > 0", msg);
    if (!finite_pos(s->dt_max)) return spec_error("dt_max must be > 0", msg);
    if (s->precision != 64 && s->precision != 32) return spec_error("precision must be 64 or 32", msg);
    if (s->flags & ~(HWFV1_REG_PREDICT | HWFV1_REG_CLOSE | HWFV1_FULL_SWEEP | HWFV1_FLUX_MATCH))
        return spec_error("unknown flags", msg);
    if ((s->flags & HWFV1_FLUX_MATCH) && !(s->flags & HWFV1_REG_CLOSE))
        return spec_error("HWFV1_FLUX_MATCH needs HWFV1_REG_CLOSE", msg);
    int inflow_sides = 0;
    for (int k = 0; k < 4; ++k) {
        if (s->bc[k] < HWFV1_BC_CLOSED || s->bc[k] > HWFV1_BC_INFLOW) return spec_error("bad boundary kind", msg);
        if (s->bc[k] == HWFV1_BC_INFLOW) inflow_sides++;
    }
    if (inflow_sides > 1) return spec_error("at most one inflow side", msg);
    if (inflow_sides == 1) {
        if (s->inflow_n < 1 || !s->inflow_t || !s->inflow_Q)
            return spec_error("inflow side needs inflow_n >= 1 and the hydrograph arrays", msg);
        if (s->inflow_n > 4096) return spec_error("inflow_n must be <= 4096", msg);
        for (int k = 0; k < s->inflow_n; ++k) {
            if (!std::isfinite(s->inflow_t[k]) || !std::isfinite(s->inflow_Q[k]))
                return spec_error("hydrograph values must be finite", msg);
            if (k && !(s->inflow_t[k] > s->inflow_t[k - 1]))
                return spec_error("hydrograph times must increase", msg);
        }
        const int64_t side = 1ll << s->L;
        if (s->inflow_a0 < 0 || s->inflow_a1 > side || s->inflow_a0 >= s->inflow_a1)
            return spec_error("inflow range must satisfy 0 <= a0 < a1 <= 2^L", msg);
    }
    return HWFV1_OK;
}

hwfv1_status from_engine(hwfv1_handle* hd, hwfv1_status s) {
    if (s != HWFV1_OK) hd->msg = hd->eng->err;
    return s;
}

}  // namespace

extern "C" {

int32_t hwfv1_version(void) { return 1; }

hwfv1_status hwfv1_init(const hwfv1_problem* spec, const double* z, const double* h,
                        const double* qx, const double* qy, void* stream, hwfv1_handle** out) {
    if (!out) return HWFV1_ERR_INVALID_SPEC;
    *out = nullptr;
    std::string msg;
    hwfv1_status s = validate(spec, &msg);
    if (s != HWFV1_OK) return s;
    if (!z || !h || !qx || !qy) return HWFV1_ERR_INVALID_SPEC;
    hwfv1_handle* hd = new (std::nothrow) hwfv1_handle;
    if (!hd) return HWFV1_ERR_OOM;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    hd->eng = spec->precision == 64 ? hwfv1::make_engine_f64(*spec, st)
                                    : hwfv1::make_engine_f32(*spec, st);
    s = hd->eng->init(z, h, qx, qy);
    if (s != HWFV1_OK) {
        delete hd->eng;
        delete hd;
        return s;
    }
    *out = hd;
    return HWFV1_OK;
}

#define HWFV1_CHECK_HANDLE(hd) \
    if (!(hd) || !(hd)->eng) return HWFV1_ERR_STATE

hwfv1_status hwfv1_encode(hwfv1_handle* hd) {
    HWFV1_CHECK_HANDLE(hd);
    return from_engine(hd, hd->eng->encode());
}
hwfv1_status hwfv1_flag(hwfv1_handle* hd) {
    HWFV1_CHECK_HANDLE(hd);
    return from_engine(hd, hd->eng->flag());
}
hwfv1_status hwfv1_traverse(hwfv1_handle* hd, int64_t* num_leaves) {
    HWFV1_CHECK_HANDLE(hd);
    return from_engine(hd, hd->eng->traverse(num_leaves));
}
hwfv1_status hwfv1_step(hwfv1_handle* hd) {
    HWFV1_CHECK_HANDLE(hd);
    return from_engine(hd, hd->eng->step());
}
hwfv1_status hwfv1_decode(hwfv1_handle* hd) {
    HWFV1_CHECK_HANDLE(hd);
    return from_engine(hd, hd->eng->decode());
}
hwfv1_status hwfv1_advance(hwfv1_handle* hd, double t_end, int64_t max_steps) {
    HWFV1_CHECK_HANDLE(hd);
    if (std::isnan(t_end)) return HWFV1_ERR_INVALID_SPEC;
    return from_engine(hd, hd->eng->advance(t_end, max_steps));
}
hwfv1_status hwfv1_advance_uniform(hwfv1_handle* hd, double t_end, int64_t max_steps) {
    HWFV1_CHECK_HANDLE(hd);
    if (std::isnan(t_end)) return HWFV1_ERR_INVALID_SPEC;
    return from_engine(hd, hd->eng->advance_uniform(t_end, max_steps));
}
hwfv1_status hwfv1_get_fields(hwfv1_handle* hd, double* h, double* qx, double* qy) {
    HWFV1_CHECK_HANDLE(hd);
    return from_engine(hd, hd->eng->get_fields(h, qx, qy));
}
hwfv1_status hwfv1_set_fields(hwfv1_handle* hd, const double* h, const double* qx, const double* qy) {
    HWFV1_CHECK_HANDLE(hd);
    return from_engine(hd, hd->eng->set_fields(h, qx, qy));
}
hwfv1_status hwfv1_get_leaves(hwfv1_handle* hd, uint32_t* packed, int64_t cap, int64_t* n) {
    HWFV1_CHECK_HANDLE(hd);
    return from_engine(hd, hd->eng->get_leaves(packed, cap, n));
}
hwfv1_status hwfv1_get_flags(hwfv1_handle* hd, int32_t which, uint32_t* bits, int64_t cap_words) {
    HWFV1_CHECK_HANDLE(hd);
    if (!bits) return HWFV1_ERR_INVALID_SPEC;
    return from_engine(hd, hd->eng->get_flags(which, bits, cap_words));
}
hwfv1_status hwfv1_get_level(hwfv1_handle* hd, int32_t field, int32_t level, double* out) {
    HWFV1_CHECK_HANDLE(hd);
    if (!out) return HWFV1_ERR_INVALID_SPEC;
    return from_engine(hd, hd->eng->get_level(field, level, out));
}
hwfv1_status hwfv1_get_time(hwfv1_handle* hd, double* t, double* dt, int64_t* step) {
    HWFV1_CHECK_HANDLE(hd);
    return from_engine(hd, hd->eng->get_time(t, dt, step));
}
hwfv1_status hwfv1_set_time(hwfv1_handle* hd, double t, double dt) {
    HWFV1_CHECK_HANDLE(hd);
    if (!std::isfinite(t) || !(std::isfinite(dt) && dt > 0.0)) return HWFV1_ERR_INVALID_SPEC;
    return from_engine(hd, hd->eng->set_time(t, dt));
}
hwfv1_status hwfv1_get_stats(hwfv1_handle* hd, int64_t* num_leaves, double* smax3) {
    HWFV1_CHECK_HANDLE(hd);
    return from_engine(hd, hd->eng->get_stats(num_leaves, smax3));
}
hwfv1_status hwfv1_profile_step(hwfv1_handle* hd, float* ms, const char** names, int32_t cap, int32_t* n) {
    HWFV1_CHECK_HANDLE(hd);
    if (cap < 0) return HWFV1_ERR_INVALID_SPEC;
    return from_engine(hd, hd->eng->profile_step(ms, names, cap, n));
}

hwfv1_status hwfv1_profile_update(hwfv1_handle* hd, int32_t reps, float* ms) {
    HWFV1_CHECK_HANDLE(hd);
    if (reps < 1 || !ms) return HWFV1_ERR_INVALID_SPEC;
    return from_engine(hd, hd->eng->profile_update(reps, ms));
}
hwfv1_status hwfv1_get_counters(hwfv1_handle* hd, int64_t* steps, int64_t* leaf_updates,
                                int64_t* active_updates, int64_t* wet_updates, int64_t* kernels_per_step) {
    HWFV1_CHECK_HANDLE(hd);
    return from_engine(hd, hd->eng->get_counters(steps, leaf_updates, active_updates, wet_updates,
                                                 kernels_per_step));
}
hwfv1_status hwfv1_save(hwfv1_handle* hd, void* host_buf, size_t cap, size_t* used) {
    HWFV1_CHECK_HANDLE(hd);
    return from_engine(hd, hd->eng->save(host_buf, cap, used));
}
hwfv1_status hwfv1_load(hwfv1_handle* hd, const void* host_buf, size_t n) {
    HWFV1_CHECK_HANDLE(hd);
    return from_engine(hd, hd->eng->load(host_buf, n));
}
const char* hwfv1_last_error(hwfv1_handle* hd) {
    if (!hd) return "NULL handle";
    return hd->msg.c_str();
}
void hwfv1_destroy(hwfv1_handle* hd) {
    if (!hd || hd->borrowed) return;      // member views are freed with their batch
    delete hd->eng;
    delete hd;
}

hwfv1_status hwfv1_set_skipnet(hwfv1_handle* hd, hwfv1_skipnet* net, int32_t audit_K, float margin,
                               int32_t predict_every) {
    HWFV1_CHECK_HANDLE(hd);
    if (predict_every < 1) return HWFV1_ERR_INVALID_SPEC;
    return from_engine(hd, hd->eng->set_skipnet(net ? net->net : nullptr, audit_K, margin, predict_every));
}
hwfv1_status hwfv1_set_skip_levels(hwfv1_handle* hd, const uint8_t* levels, int32_t audit_K) {
    HWFV1_CHECK_HANDLE(hd);
    if (levels && audit_K < 1) return HWFV1_ERR_INVALID_SPEC;
    return from_engine(hd, hd->eng->set_skip_levels(levels, audit_K));
}
hwfv1_status hwfv1_get_skip_levels(hwfv1_handle* hd, int32_t which, uint8_t* out, int64_t cap) {
    HWFV1_CHECK_HANDLE(hd);
    if (!out) return HWFV1_ERR_INVALID_SPEC;
    return from_engine(hd, hd->eng->get_skip_levels(which, out, cap));
}
hwfv1_status hwfv1_set_leaf_store(hwfv1_handle* hd, int32_t on) {
    HWFV1_CHECK_HANDLE(hd);
    return from_engine(hd, hd->eng->set_leaf_store(on ? 1 : 0));
}
hwfv1_status hwfv1_get_features(hwfv1_handle* hd, uint16_t* out, int64_t cap) {
    HWFV1_CHECK_HANDLE(hd);
    if (!out) return HWFV1_ERR_INVALID_SPEC;
    return from_engine(hd, hd->eng->get_features(out, cap));
}
hwfv1_status hwfv1_get_labels(hwfv1_handle* hd, uint8_t* out, int64_t cap) {
    HWFV1_CHECK_HANDLE(hd);
    if (!out) return HWFV1_ERR_INVALID_SPEC;
    return from_engine(hd, hd->eng->get_labels(out, cap));
}

// ---------------------------------------------------------------------------
// Batched ensembles
// ---------------------------------------------------------------------------
hwfv1_status hwfv1_batch_init(const hwfv1_problem* specs, int32_t n, const double* const* z,
                              const double* const* h, const double* const* qx, const double* const* qy,
                              void* stream, hwfv1_batch** out) {
    if (!out) return HWFV1_ERR_INVALID_SPEC;
    *out = nullptr;
    if (!specs || n < 1 || n > 4096 || !z || !h || !qx || !qy) return HWFV1_ERR_INVALID_SPEC;
    for (int d = 0; d < n; ++d) {
        std::string msg;
        const hwfv1_status s = validate(specs + d, &msg);
        if (s != HWFV1_OK) return s;
        if (specs[d].precision != specs[0].precision) return HWFV1_ERR_INVALID_SPEC;
        if (specs[d].flags & HWFV1_FLUX_MATCH) return HWFV1_ERR_INVALID_SPEC;
        if (!z[d] || !h[d] || !qx[d] || !qy[d]) return HWFV1_ERR_INVALID_SPEC;
    }
    hwfv1_batch* bt = new (std::nothrow) hwfv1_batch;
    if (!bt) return HWFV1_ERR_OOM;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    bt->b = specs[0].precision == 64 ? hwfv1::make_batch_f64(specs, n, st) : hwfv1::make_batch_f32(specs, n, st);
    const hwfv1_status s = bt->b->init(z, h, qx, qy);
    if (s != HWFV1_OK) {
        delete bt->b;
        delete bt;
        return s;
    }
    for (int d = 0; d < n; ++d) {
        hwfv1_handle* v = new hwfv1_handle;
        v->eng = bt->b->member(d);
        v->borrowed = true;
        bt->views.push_back(v);
    }
    *out = bt;
    return HWFV1_OK;
}

hwfv1_status hwfv1_batch_advance(hwfv1_batch* bt, double t_end, int64_t max_steps) {
    if (!bt || !bt->b) return HWFV1_ERR_STATE;
    if (std::isnan(t_end)) return HWFV1_ERR_INVALID_SPEC;
    const hwfv1_status s = bt->b->advance(t_end, max_steps);
    if (s != HWFV1_OK) bt->msg = bt->b->err;
    return s;
}

hwfv1_status hwfv1_batch_autotune(hwfv1_batch* bt, int64_t trial_steps, int32_t* choice) {
    if (!bt || !bt->b) return HWFV1_ERR_STATE;
    const hwfv1_status s = bt->b->autotune(trial_steps, choice);
    if (s != HWFV1_OK) bt->msg = bt->b->err;
    return s;
}

hwfv1_status hwfv1_batch_member(hwfv1_batch* bt, int32_t d, hwfv1_handle** view) {
    if (!bt || !bt->b || !view) return HWFV1_ERR_STATE;
    if (d < 0 || d >= (int32_t)bt->views.size()) return HWFV1_ERR_INVALID_SPEC;
    *view = bt->views[d];
    return HWFV1_OK;
}

int64_t hwfv1_batch_launches_per_step(hwfv1_batch* bt) {
    return (bt && bt->b) ? bt->b->launches_per_step() : 0;
}

const char* hwfv1_batch_last_error(hwfv1_batch* bt) {
    if (!bt) return "NULL batch";
    return bt->msg.c_str();
}

}  // extern "C"

namespace {
// Eight independent chains of dependent double additions per thread: the
// sub-partitions' FP64 units stay busy, nothing else is issued in between.
__global__ void k_fp64_add_loop(double* out, int iters) {
    const double c = 1.0000000001;
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-3 + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = __dadd_rn(x[k], c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s = __dadd_rn(s, x[k]);
    out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}
}  // namespace

extern "C" {

hwfv1_status hwfv1_fp64_throughput(double* tflops) {
    if (!tflops) return HWFV1_ERR_INVALID_SPEC;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return HWFV1_ERR_CUDA;
    const int threads = 256, blocks = nsm * 8, iters = 2048;
    double* out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * (size_t)threads * blocks) != cudaSuccess) {
        cudaGetLastError();
        return HWFV1_ERR_OOM;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int r = 0; r < 4; ++r) {            // the first launch warms up
        cudaEventRecord(e0);
        k_fp64_add_loop<<<blocks, threads>>>(out, iters);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0 && ms < best) best = ms;
    }
    const cudaError_t e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return HWFV1_ERR_CUDA;
    *tflops = (double)blocks * threads * iters * 8.0 / (best * 1e-3) / 1e12;
    return HWFV1_OK;
}

void hwfv1_batch_destroy(hwfv1_batch* bt) {
    if (!bt) return;
    for (hwfv1_handle* v : bt->views) delete v;
    delete bt->b;
    delete bt;
}

}  // extern "C"
