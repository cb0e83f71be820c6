// engine.cuh -- host side of one HWFV1 simulation: device buffers, the
// launch sequence of a timestep, CUDA-graph replay, checkpoints, host field
// transfers (and k_quiet_tiles, a kernel only the initialisation launches).
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "engine_iface.h"
#include "kernels.cuh"
#include "skip.cuh"
#include "skipnet.h"

namespace hwfv1 {

// Quiescence marks of an initial state, one field at a time: zf[t] (set to
// 1 beforehand) is cleared where the finest values of field x in tile t
// (4^kt consecutive Morton codes) are not all +0.  The tiles' coarser levels
// were cleared beforehand, so a mark left at 1 holds for them too.  One warp
// per tile.
template <typename T>
static __global__ void k_quiet_tiles(const T* __restrict__ x, uint8_t* __restrict__ zf, uint32_t ntiles, int kt) {
    const uint32_t lane = threadIdx.x & 31u, cells = 1u << (2 * kt);
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < ntiles; t += nw) {   // warp-uniform
        const uint64_t b = (uint64_t)t * cells;
        bool nz = false;
        for (uint32_t i = lane; i < cells; i += 32u) nz |= !pos_zero(x[b + i]);
        nz = __any_sync(0xffffffffu, nz);
        if (lane == 0u && nz) zf[t] = 0;
    }
}

// Kernel nodes of a captured graph (memset and copy nodes are not counted).
inline int64_t count_kernel_nodes(cudaGraph_t g) {
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return 0;
    std::vector<cudaGraphNode_t> nodes(n);
    if (n && cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return 0;
    int64_t k = 0;
    for (size_t i = 0; i < n; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

template <typename T>
class EngineT final : public Engine {
   public:
    // batched: a member of a BatchT, whose own kernels run its steps (no
    // shared-face buffers)
    EngineT(const hwfv1_problem& s, cudaStream_t stream, bool batched = false)
        : spec_(s), stream_(stream), batched_(batched) {
        L_ = s.L;
        N_ = 1ull << (2 * L_);
        H_ = hier_size(L_);
        kt_ = L_ < 5 ? L_ : 5;
        ntiles_ = 1u << (2 * (L_ - kt_));
        words_ = bits_words(L_);
        if (s.inflow_n > 0 && s.inflow_t) {
            it_.assign(s.inflow_t, s.inflow_t + s.inflow_n);
            iq_.assign(s.inflow_Q, s.inflow_Q + s.inflow_n);
        }
    }
    ~EngineT() override {
        if (exec_) cudaGraphExecDestroy(exec_);
        if (exec_multi_) cudaGraphExecDestroy(exec_multi_);
        drop_skip_graphs();
        if (exec_uniform_) cudaGraphExecDestroy(exec_uniform_);
        skipwork_free(&skw_);
        if (ev_fork_) cudaEventDestroy(ev_fork_);
        if (ev_join_) cudaEventDestroy(ev_join_);
        if (side_) cudaStreamDestroy(side_);
        for (cudaEvent_t& e : hev_)
            if (e) cudaEventDestroy(e);
        if (cstream_) cudaStreamDestroy(cstream_);
        for (void* p : allocs_)
            if (cudaFreeAsync(p, stream_) != cudaSuccess) {     // (a stream the caller destroyed)
                cudaGetLastError();
                cudaFree(p);
            }
        if (own_stream_) cudaStreamDestroy(stream_);
    }

    // The staging area of a host transfer.  Whatever way the call leaves,
    // no copy of the caller's buffers is still in flight and the area goes
    // back to the pool (ordered after every kernel that reads it).
    struct Staging {
        EngineT* e;
        double* p = nullptr;
        ~Staging() {
            if (!p) return;
            cudaStreamSynchronize(e->cstream_);
            cudaFreeAsync(p, e->stream_);
        }
    };

    hwfv1_status init(const double* z, const double* h, const double* qx,
                      const double* qy) override {
        if (!stream_) {
            if (cudaStreamCreate(&stream_) != cudaSuccess) return fail(HWFV1_ERR_CUDA, "stream");
            own_stream_ = true;
        }
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm_, cudaDevAttrMultiProcessorCount, dev);
        for (int b = 0; b < 2; ++b)
            for (int q = 0; q < 3; ++q)
                if (!alloc(&f_[b][q], H_ * sizeof(T))) return oom();
        if (!alloc(&z_, H_ * sizeof(T))) return oom();
        // Fields in host memory (pinned or pageable) are copied in on the copy
        // stream through two staging slots, in the order z, h, qx, qy: the
        // bed is converted and encoded while h, qx and qy are on their way.
        // Events 0-3: field k copied in; 4-7: field k converted (its slot free).
        const double* src[4] = {z, h, qx, qy};
        bool hostp[4];
        bool any_host = false;
        for (int k = 0; k < 4; ++k) any_host |= (hostp[k] = on_host(src[k]));
        Staging stg{this};
        if (any_host) {
            if (hwfv1_status r = host_io_ready(); r != HWFV1_OK) return r;
            if (hwfv1_status r = stage_alloc(&stg.p); r != HWFV1_OK) return r;
        }
        double* const stage = stg.p;
        auto copy_in = [&](int k) -> bool {
            if (!hostp[k]) return true;
            if (k >= 2 && hostp[k - 2]) cudaStreamWaitEvent(cstream_, hev_[4 + k - 2], 0);
            if (cudaMemcpyAsync(stage + (size_t)(k & 1) * N_, src[k], N_ * sizeof(double), cudaMemcpyHostToDevice,
                                cstream_) != cudaSuccess)
                return false;
            return cudaEventRecord(hev_[k], cstream_) == cudaSuccess;
        };
        auto field = [&](int k) -> const double* {          // on stream_: field k on the device
            if (!hostp[k]) return src[k];
            cudaStreamWaitEvent(stream_, hev_[k], 0);
            return stage + (size_t)(k & 1) * N_;
        };
        auto converted = [&](int k) {
            if (hostp[k]) cudaEventRecord(hev_[4 + k], stream_);
        };
        if (!copy_in(0) || !copy_in(1)) return fail(HWFV1_ERR_CUDA, "init: copy of a host field");
        if (!alloc(&bits_, (size_t)words_ * 6 * sizeof(uint32_t))) return oom();
        Tb_ = bits_;
        Cb_ = bits_ + words_;
        Tz_ = bits_ + 2 * words_;
        Cz_ = bits_ + 3 * words_;
        Sz_ = bits_ + 4 * words_;
        Sb_ = bits_ + 5 * words_;
        if (!alloc(&leaves_, N_ * sizeof(uint32_t))) return oom();
        if (!alloc(&wet_, N_ * sizeof(uint32_t))) return oom();
        // tile counters: counts and offsets of the ordered traversal, the
        // decode list after them (one spare word: get_leaves keeps its
        // 2 nct + 1 words below the decode list for every tile count)
        if (!alloc(&counts_, ((size_t)ntiles_ * 3 + 1) * sizeof(uint32_t))) return oom();
        offs_ = counts_ + ntiles_;
        dlist_ = counts_ + 2 * ntiles_ + 1;
        // shared faces of the wet-leaf update: 10 values per queued leaf and
        // its two velocities, a stamp per hierarchy cell.  Float64 only: in
        // float32 the arithmetic saved costs less than the extra launch and
        // face traffic.
        if (sizeof(T) == 8) {
            fcap_ = (uint32_t)std::min<uint64_t>(N_, 1ull << 22);
            if (!alloc(&face_, (size_t)fcap_ * 12 * sizeof(T))) return oom();
            if (!alloc(&mark_, H_ * sizeof(unsigned long long))) return oom();
            cudaMemsetAsync(mark_, 0, H_ * sizeof(unsigned long long), stream_);
        }
        // quiescent-tile bookkeeping: zf (two buffers), inlet, act
        if (!alloc(&tilebytes_, (size_t)ntiles_ * 4)) return oom();
        if (!alloc(&work_, (size_t)ntiles_ * sizeof(uint32_t))) return oom();
        cudaMemsetAsync(tilebytes_, 0, (size_t)ntiles_ * 4, stream_);
        quiet_on_ = !(spec_.flags & HWFV1_FULL_SWEEP) && spec_.eps >= 1e-30;
        // With quiescent tiles on, the first step starts from marks as a
        // later step does: both buffers are cleared (buffer 0 below its
        // finest level, which the fields fill) and the tiles of +0 marked
        // once the fields are in (k_quiet_tiles), so that the first encode,
        // traversal and decode skip them as well.
        if (quiet_on_)
            for (int q = 0; q < 3; ++q) {
                cudaMemsetAsync(f_[0][q], 0, lvl_off(L_) * sizeof(T), stream_);
                cudaMemsetAsync(f_[1][q], 0, H_ * sizeof(T), stream_);
            }
        pdl_ = std::getenv("HWFV1_NO_PDL") == nullptr;
        {
            std::vector<uint8_t> inl(ntiles_, 0);
            const int side = step_args().inflow_side;
            if (side >= 0) {
                const uint32_t last = (1u << (L_ - kt_)) - 1u;
                for (int64_t pos = spec_.inflow_a0; pos < spec_.inflow_a1; ++pos) {
                    const uint32_t tp = (uint32_t)(pos >> kt_);
                    const uint32_t ti = side == 0 ? 0u : side == 1 ? last : tp;
                    const uint32_t tj = side == 2 ? 0u : side == 3 ? last : tp;
                    inl[morton2(ti, tj)] = 1;
                }
            }
            cudaMemcpyAsync(tilebytes_ + 2 * ntiles_, inl.data(), ntiles_, cudaMemcpyHostToDevice, stream_);
            cudaStreamSynchronize(stream_);
        }
        if (!alloc(&st_, sizeof(DevState))) return oom();
        if (!alloc(&zaux_, kZauxBytes)) return oom();
        cudaMemsetAsync(zaux_, 0, kZauxBytes, stream_);      // zmax is a max-reduction target
        if (!it_.empty()) {
            if (!alloc(&it_d_, it_.size() * sizeof(double))) return oom();
            if (!alloc(&iq_d_, iq_.size() * sizeof(double))) return oom();
            cudaMemcpyAsync(it_d_, it_.data(), it_.size() * sizeof(double), cudaMemcpyHostToDevice, stream_);
            cudaMemcpyAsync(iq_d_, iq_.data(), iq_.size() * sizeof(double), cudaMemcpyHostToDevice, stream_);
        }
        cudaMemsetAsync(bits_, 0, (size_t)words_ * 6 * sizeof(uint32_t), stream_);
        {   // t = 0, no end time until hwfv1_advance sets one, buffer 0 current
            DevState s0;
            std::memset(&s0, 0, sizeof s0);
            s0.t_end = HUGE_VAL;
            s0.active = 1u;
            cudaMemcpyAsync(st_, &s0, sizeof s0, cudaMemcpyHostToDevice, stream_);
            cudaStreamSynchronize(stream_);
        }
        // finest fields into the Morton hierarchy, the bed's first
        const int g = grid_for(N_);
        k_rm_to_morton<T><<<g, 256, 0, stream_>>>(field(0), z_ + lvl_off(L_), L_);
        converted(0);
        if (!copy_in(2)) return fail(HWFV1_ERR_CUDA, "init: copy of a host field");
        // bed: s_max, thresholds, one-off encode and its static flags
        unsigned long long* zmax = reinterpret_cast<unsigned long long*>(zaux_);
        double* smax_z = reinterpret_cast<double*>(zaux_ + 8);
        double* thr_zd = reinterpret_cast<double*>(zaux_ + kZThrD);
        float* thr_zf = reinterpret_cast<float*>(zaux_ + kZThrF);
        k_maxabs<T><<<g, 256, 0, stream_>>>(z_ + lvl_off(L_), N_, zmax);
        k_z_thresholds<<<1, 32, 0, stream_>>>(zmax, thr_zd, thr_zf, reinterpret_cast<double*>(zaux_ + kZThr4D),
                                              reinterpret_cast<float*>(zaux_ + kZThr4F), smax_z, L_, spec_.eps,
                                              st_);
        {
            EncodeArgs<T, 1> a;
            a.f[0][0] = a.f[1][0] = z_;
            a.thr = thr_z();
            a.thr4 = thr4_z();
            a.Tb = Tz_;
            a.Cb = Cz_;
            a.st = nullptr;
            a.L = L_;
            encode_passes(a);
        }
        lk(k_flag, grid_for(words_), 256, Tz_, Cz_, nullptr, Sz_, L_, predict(), close(),
           (const DevState*)nullptr, (uint32_t*)nullptr);
        // leaf count of each tile holding the bed's flags alone (skipped tiles)
        if (!alloc(&scount_, (size_t)ntiles_ * sizeof(uint32_t))) return oom();
        k_static_counts<<<(ntiles_ + kTilesPerCta - 1) / kTilesPerCta, 256, 0, stream_>>>(Sz_, L_, kt_, ntiles_,
                                                                                       scount_);
        // h, qx, qy: each field's share of the initial scalars (its s_max)
        // and of the quiescence marks is taken as soon as it is in, so that
        // only the last field's and the CFL pass follow the last copy
        if (quiet_on_) cudaMemsetAsync(tilebytes_, 1, (size_t)ntiles_ * 2, stream_);   // both buffers +0 so far
        k_reset_red<<<1, 32, 0, stream_>>>(st_);
        for (int q = 0; q < 3; ++q) {
            T* const x = f_[0][q] + lvl_off(L_);
            k_rm_to_morton<T><<<g, 256, 0, stream_>>>(field(1 + q), x, L_);
            converted(1 + q);
            if (q == 0 && !copy_in(3)) return fail(HWFV1_ERR_CUDA, "init: copy of a host field");
            k_maxabs_cur<T><<<g, 256, 0, stream_>>>(x, f_[1][q] + lvl_off(L_), st_, N_, q);
            if (quiet_on_)
                k_quiet_tiles<T><<<grid_for((uint64_t)ntiles_ * 32), 256, 0, stream_>>>(x, tilebytes_, ntiles_, kt_);
        }
        // initial state scalars: the CFL step over the three fields
        k_cfl_cur<T><<<g, 256, 0, stream_>>>(f_[0][0] + lvl_off(L_), f_[1][0] + lvl_off(L_), f_[0][1] + lvl_off(L_),
                                              f_[1][1] + lvl_off(L_), f_[0][2] + lvl_off(L_), f_[1][2] + lvl_off(L_),
                                              st_, N_, phys());
        k_init_state<<<1, 64, 0, stream_>>>(st_, fin_args(), 1);
        // the plain step's graphs, captured while the device initialises
        // (capturing runs nothing), so that the first hwfv1_advance does not
        // pay for them; a batch member is stepped by its batch
        if (!batched_ && std::getenv("HWFV1_NO_GRAPH") == nullptr) {
            if (hwfv1_status r = check("init"); r != HWFV1_OK) return r;
            if (capture(&exec_, kStepPlain) != HWFV1_OK) return HWFV1_ERR_CUDA;
            if (capture(&exec_multi_, kStepPlain, kMultiSteps) != HWFV1_OK) return HWFV1_ERR_CUDA;
        }
        return check("init", true);
    }

    // The phases one by one are those of the plain step: with the learned
    // skip on, the stored state may be above level L, so they are refused.
    hwfv1_status phase_guard(const char* what) {
        if (skipmode_) return fail(HWFV1_ERR_STATE, std::string(what) + ": the learned skip is on (use hwfv1_advance)");
        return HWFV1_OK;
    }
    hwfv1_status encode() override {
        if (hwfv1_status r = phase_guard("encode"); r != HWFV1_OK) return r;
        launch_encode();
        return check("encode");
    }
    hwfv1_status flag() override {
        if (hwfv1_status r = phase_guard("flag"); r != HWFV1_OK) return r;
        launch_flag();
        sb_valid_ = true;
        return check("flag");
    }
    hwfv1_status traverse(int64_t* num_leaves) override {
        if (hwfv1_status r = phase_guard("traverse"); r != HWFV1_OK) return r;
        cudaMemsetAsync(&st_->ndec, 0, 4 * sizeof(uint32_t), stream_);     // ndec, Mall, M, nact
        launch_traverse();
        if (num_leaves) {
            DevState s;
            if (read_state(&s) != HWFV1_OK) return HWFV1_ERR_CUDA;
            *num_leaves = s.Mall;
        }
        return check("traverse");
    }
    hwfv1_status step() override {
        if (hwfv1_status r = phase_guard("step"); r != HWFV1_OK) return r;
        launch_fv1();
        return check("step");
    }
    hwfv1_status decode() override {
        if (hwfv1_status r = phase_guard("decode"); r != HWFV1_OK) return r;
        launch_decode();
        return check("decode");
    }

    hwfv1_status advance(double t_end, int64_t max_steps) override {
        if (max_steps < 0) return fail(HWFV1_ERR_INVALID_SPEC, "max_steps < 0");
        k_set_tend<<<1, 64, 0, stream_>>>(st_, fin_args(), t_end);
        if (max_steps == 0) return check("advance");
        const bool use_graph = std::getenv("HWFV1_NO_GRAPH") == nullptr;
        if (use_graph && !skipmode_ && !exec_ && capture(&exec_, kStepPlain) != HWFV1_OK) return HWFV1_ERR_CUDA;
        int64_t s = 0;
        if (use_graph && !skipmode_ && max_steps >= kMultiSteps) {
            // kMultiSteps plain steps per graph launch: the kernels of
            // consecutive steps follow each other as inside one step, without
            // the gap between two graph launches.  A step after t_end does
            // nothing, as with single-step launches.
            if (!exec_multi_ && capture(&exec_multi_, kStepPlain, kMultiSteps) != HWFV1_OK) return HWFV1_ERR_CUDA;
            for (; s + kMultiSteps <= max_steps; s += kMultiSteps)
                if (cudaGraphLaunch(exec_multi_, stream_) != cudaSuccess) return fail(HWFV1_ERR_CUDA, "graph launch");
        }
        int kind = kStepPlain;
        for (; s < max_steps; ++s) {
            kind = skipmode_ ? skip_kind(lstep_++) : kStepPlain;
            if (use_graph) {
                cudaGraphExec_t* g = kind == kStepPlain ? &exec_ : &exec_skip_[kind - kStepAudit];
                if (!*g && capture(g, kind) != HWFV1_OK) return HWFV1_ERR_CUDA;
                if (cudaGraphLaunch(*g, stream_) != cudaSuccess) return fail(HWFV1_ERR_CUDA, "graph launch");
            } else {
                launch_step(kind);
            }
        }
        // a plain last step formed S on the spot: Sb_ is materialised on demand
        sb_valid_ = kind == kStepSkip || kind == kStepSkipPredict || !onfly_flags();
        return check("advance");
    }

    // Uniform FV1 on the finest grid (eps plays no part): the comparison
    // solver of the paper's Sec. 3 (GPU-FV1), on the same kernels.
    hwfv1_status advance_uniform(double t_end, int64_t max_steps) override {
        if (max_steps < 0) return fail(HWFV1_ERR_INVALID_SPEC, "max_steps < 0");
        if (!uniform_leaves_) {
            if (!alloc(&uniform_leaves_, N_ * sizeof(uint32_t))) return oom();
            k_fill_finest_leaves<<<grid_for(N_), 256, 0, stream_>>>(uniform_leaves_, L_, N_);
        }
        // uniform steps keep no quiescence marks: forget them for later
        // adaptive steps; with the learned skip on, the state is brought to
        // level L first
        if (skipmode_) launch_skip_finest(2);
        forget_quiet();
        k_set_tend<<<1, 64, 0, stream_>>>(st_, fin_args(), t_end);
        if (max_steps == 0) return check("advance_uniform");
        const bool use_graph = std::getenv("HWFV1_NO_GRAPH") == nullptr;
        if (use_graph && !exec_uniform_) {
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                return fail(HWFV1_ERR_CUDA, "graph capture begin");
            launch_step_uniform();
            if (cudaStreamEndCapture(stream_, &g) != cudaSuccess) return fail(HWFV1_ERR_CUDA, "graph capture end");
            const cudaError_t e = cudaGraphInstantiate(&exec_uniform_, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                exec_uniform_ = nullptr;
                return fail(HWFV1_ERR_CUDA, "graph instantiate");
            }
        }
        for (int64_t s = 0; s < max_steps; ++s) {
            if (use_graph) {
                if (cudaGraphLaunch(exec_uniform_, stream_) != cudaSuccess) return fail(HWFV1_ERR_CUDA, "graph launch");
            } else {
                launch_step_uniform();
            }
        }
        return check("advance_uniform");
    }

    // The learned subtree skip with the network's predicted levels (net ==
    // nullptr: back to the plain step).  Every audit_K-th step, counting
    // from the first step after this call, is the exact (plain) step.
    hwfv1_status set_skipnet(SkipNet* net, int audit_K, float margin, int predict_every) override {
        if (net && (L_ < 6 || audit_K < 1 || predict_every < 1))
            return fail(HWFV1_ERR_INVALID_SPEC, "learned skip needs L >= 6, K >= 1, predict_every >= 1");
        if (!net) return skip_off();
        if (hwfv1_status r = skip_on(1, audit_K); r != HWFV1_OK) return r;
        if (skip_ != net || every_ != predict_every || margin_ != margin) {
            // the graphs hold the network, the schedule and the margin
            drop_skip_graphs();
            lstep_ = 0;
        }
        skip_ = net;
        every_ = predict_every;
        margin_ = margin;
        const uint64_t npx = 1ull << (2 * (L_ - 4));
        if (!feat_ && !alloc(&feat_, npx * 4 * sizeof(__nv_bfloat16))) return oom();
        if (!skipwork_reserve(&skw_, (int64_t)npx)) return oom();
        if (!side_ && (cudaStreamCreateWithFlags(&side_, cudaStreamNonBlocking) != cudaSuccess ||
                       cudaEventCreateWithFlags(&ev_fork_, cudaEventDisableTiming) != cudaSuccess ||
                       cudaEventCreateWithFlags(&ev_join_, cudaEventDisableTiming) != cudaSuccess))
            return fail(HWFV1_ERR_CUDA, "network stream");
        return capture_skip_graphs();
    }

    // The learned subtree skip with levels given by the caller (host,
    // row-major over level L-4), kept until the next call.
    hwfv1_status set_skip_levels(const uint8_t* levels, int audit_K) override {
        if (!levels) return skip_off();
        if (L_ < 5 || audit_K < 1) return fail(HWFV1_ERR_INVALID_SPEC, "skip levels need L >= 5, K >= 1");
        const int Ls = L_ - 4;
        const uint32_t n = 1u << (2 * Ls), S = 1u << Ls;
        std::vector<uint8_t> mort(n);
        for (uint32_t j = 0; j < S; ++j)
            for (uint32_t i = 0; i < S; ++i) {
                const uint8_t v = levels[(size_t)j * S + i];
                if (v < Ls || v > L_) return fail(HWFV1_ERR_INVALID_SPEC, "skip levels outside [L-4, L]");
                mort[morton2(i, j)] = v;
            }
        if (hwfv1_status r = skip_on(2, audit_K); r != HWFV1_OK) return r;
        skip_ = nullptr;
        every_ = 1;
        cudaMemcpyAsync(phat_, mort.data(), n, cudaMemcpyHostToDevice, stream_);
        if (hwfv1_status r = check("set_skip_levels", true); r != HWFV1_OK) return r;
        return capture_skip_graphs();
    }

    // The exact leaf-value store: subtrees whose bed is flat are stored at
    // their deepest leaf level and kept one level deeper (k_exact_levels);
    // the results are those of the plain step bit for bit.
    hwfv1_status set_leaf_store(int on) override {
        if (!on) return skipmode_ == 3 ? skip_off() : HWFV1_OK;
        if (L_ < 5) return fail(HWFV1_ERR_INVALID_SPEC, "leaf store needs L >= 5");
        if (!(spec_.eps >= 1e-30))
            return fail(HWFV1_ERR_INVALID_SPEC, "leaf store needs eps >= 1e-30 (thresholds above 0)");
        if (skipmode_ == 3) return HWFV1_OK;
        if (skipmode_) skip_off();
        const uint32_t nsub = 1u << (2 * (L_ - 4));
        if (!flat_) {
            if (!alloc(&flat_, nsub)) return oom();
            k_flat_subtrees<T><<<grid_for((uint64_t)nsub * 32), 256, 0, stream_>>>(z_ + lvl_off(L_), L_, L_ - 4, flat_);
        }
        if (hwfv1_status r = skip_on(3, 0x7FFFFFFF); r != HWFV1_OK) return r;
        skip_ = nullptr;
        every_ = 1;
        return capture_skip_graphs();
    }

    // which = 0: the predicted levels in use; 1: the storage levels
    // (host, row-major over level L-4)
    hwfv1_status get_skip_levels(int which, uint8_t* out, int64_t cap) override {
        if (L_ < 5) return fail(HWFV1_ERR_INVALID_SPEC, "skip levels need L >= 5");
        const int Ls = L_ - 4;
        const uint32_t n = 1u << (2 * Ls), S = 1u << Ls;
        if (!out || cap < (int64_t)n || (which != 0 && which != 1))
            return fail(HWFV1_ERR_INVALID_SPEC, "get_skip_levels: which 0 or 1, cap >= 4^(L-4)");
        std::vector<uint8_t> mort(n, (uint8_t)L_);
        const uint8_t* src = which == 0 ? phat_ : mlev_;
        if (src) {
            cudaMemcpyAsync(mort.data(), src, n, cudaMemcpyDeviceToHost, stream_);
            if (hwfv1_status r = check("get_skip_levels", true); r != HWFV1_OK) return r;
        }
        for (uint32_t j = 0; j < S; ++j)
            for (uint32_t i = 0; i < S; ++i) out[(size_t)j * S + i] = mort[morton2(i, j)];
        return HWFV1_OK;
    }

    hwfv1_status get_features(uint16_t* out, int64_t cap) override {
        if (L_ < 6) return fail(HWFV1_ERR_INVALID_SPEC, "features need L >= 6");
        if (cap < (int64_t)(4ull << (2 * (L_ - 4)))) return fail(HWFV1_ERR_INVALID_SPEC, "features: cap too small");
        launch_features(reinterpret_cast<__nv_bfloat16*>(out));
        return check("get_features");
    }

    hwfv1_status get_labels(uint8_t* out, int64_t cap) override {
        if (L_ < 6) return fail(HWFV1_ERR_INVALID_SPEC, "labels need L >= 6");
        if (cap < (int64_t)(1ull << (2 * (L_ - 4)))) return fail(HWFV1_ERR_INVALID_SPEC, "labels: cap too small");
        const uint32_t n = 1u << (2 * (L_ - 4));
        k_labels<<<grid_for(n), 256, 0, stream_>>>(Cb_, Cz_, L_, L_ - 4, out);
        return check("get_labels");
    }

    hwfv1_status get_fields(double* h, double* qx, double* qy) override {
        double* out[3] = {h, qx, qy};
        // with the learned skip the state may be stored above level L: its
        // finest level is formed in the other buffer, which reads it (the
        // stored state is left as it is)
        const bool other = skipmode_ != 0;
        if (other) launch_skip_finest(0);
        // a host output is formed in a staging slot and copied out on the
        // copy stream while the next field is formed (events 0-2: copy j
        // done, its slot free; 4-6: field j formed)
        bool hostp[3];
        bool any_host = false;
        for (int q = 0; q < 3; ++q) any_host |= (hostp[q] = out[q] != nullptr && on_host(out[q]));
        Staging stg{this};
        if (any_host) {
            if (hwfv1_status r = host_io_ready(); r != HWFV1_OK) return r;
            if (hwfv1_status r = stage_alloc(&stg.p); r != HWFV1_OK) return r;
        }
        double* const stage = stg.p;
        int j = 0;
        for (int q = 0; q < 3; ++q) {
            if (!out[q]) continue;
            double* dst = out[q];
            if (hostp[q]) {
                if (j >= 2) cudaStreamWaitEvent(stream_, hev_[j - 2], 0);
                dst = stage + (size_t)(j & 1) * N_;
            }
            k_morton_to_rm<T><<<grid_for(N_), 256, 0, stream_>>>(
                f_[other ? 1 : 0][q] + lvl_off(L_), f_[other ? 0 : 1][q] + lvl_off(L_), st_, dst, L_);
            if (hostp[q]) {
                cudaEventRecord(hev_[4 + j], stream_);
                cudaStreamWaitEvent(cstream_, hev_[4 + j], 0);
                if (cudaMemcpyAsync(out[q], dst, N_ * sizeof(double), cudaMemcpyDeviceToHost, cstream_) != cudaSuccess ||
                    cudaEventRecord(hev_[j], cstream_) != cudaSuccess)
                    return fail(HWFV1_ERR_CUDA, "get_fields: copy to a host field");
                ++j;
            }
        }
        if (!any_host) return check("get_fields");
        for (int k = 0; k < j; ++k) cudaStreamWaitEvent(stream_, hev_[k], 0);
        return check("get_fields", true);            // host outputs are written when the call returns
    }

    hwfv1_status set_fields(const double* h, const double* qx, const double* qy) override {
        const double* in[3] = {h, qx, qy};
        for (int q = 0; q < 3; ++q) {
            if (!in[q]) return fail(HWFV1_ERR_INVALID_SPEC, "set_fields: NULL field");
            k_rm_to_morton_cur<T><<<grid_for(N_), 256, 0, stream_>>>(
                in[q], f_[0][q] + lvl_off(L_), f_[1][q] + lvl_off(L_), st_, L_);
        }
        forget_quiet();
        stored_at_finest();
        reduce_state(/*set_dt=*/0);
        return check("set_fields");
    }

    hwfv1_status get_leaves(uint32_t* out, int64_t cap, int64_t* n) override {
        DevState s;
        if (read_state(&s) != HWFV1_OK) return HWFV1_ERR_CUDA;
        if (n) *n = s.Mall;
        if (!out) return HWFV1_OK;
        if (cap < (int64_t)s.Mall) return fail(HWFV1_ERR_INVALID_SPEC, "get_leaves: cap too small");
        {
            // the step's list is in Z-order within tiles only and leaves out
            // skipped tiles: list every leaf of the current flags into `out`
            // in Z-order (no state changes)
            // per-CTA counts, offsets and the total in the first 2 nct + 1
            // words of the handle's tile counters, below the decode list (the
            // step needs none of them across calls)
            const uint32_t nct = (ntiles_ + kTilesPerCta - 1) / kTilesPerCta;
            uint32_t* cnt = counts_;
            ensure_sig_words();
            k_trav_count<<<nct, 256, 0, stream_>>>(Sb_, cnt, nullptr, L_, kt_, ntiles_, st_, nullptr, Quiet());
            k_trav_scan<<<1, 1024, 0, stream_>>>(cnt, cnt + nct, nct, st_, cnt + 2 * nct);
            k_trav_write<<<nct, 256, 0, stream_>>>(Sb_, cnt + nct, out, L_, kt_, ntiles_, st_, nullptr);
            return check("get_leaves", true);
        }
    }

    hwfv1_status get_flags(int which, uint32_t* out, int64_t cap_words) override {
        if (cap_words < (int64_t)words_) return fail(HWFV1_ERR_INVALID_SPEC, "get_flags: cap too small");
        if (which == 1) ensure_sig_words();
        if (which == 0)
            k_or_words<<<grid_for(words_), 256, 0, stream_>>>(Tb_, Tz_, out, words_);
        else if (which == 1)
            cudaMemcpyAsync(out, Sb_, sizeof(uint32_t) * words_, cudaMemcpyDeviceToDevice, stream_);
        else
            return fail(HWFV1_ERR_INVALID_SPEC, "get_flags: which must be 0 or 1");
        return check("get_flags");
    }

    hwfv1_status get_level(int field, int level, double* out) override {
        if (field < 0 || field > 3 || level < 0 || level > L_)
            return fail(HWFV1_ERR_INVALID_SPEC, "get_level: bad field or level");
        const uint64_t n = 1ull << (2 * level);
        if (field == 3) {
            k_copy_level<T><<<grid_for(n), 256, 0, stream_>>>(z_ + lvl_off(level), nullptr, st_, out, n);
        } else if (skipmode_ && level == L_) {   // the finest level formed in the other buffer
            launch_skip_finest(0);
            k_copy_level<T><<<grid_for(n), 256, 0, stream_>>>(
                f_[1][field] + lvl_off(level), f_[0][field] + lvl_off(level), st_, out, n);
        } else {
            k_copy_level<T><<<grid_for(n), 256, 0, stream_>>>(
                f_[0][field] + lvl_off(level), f_[1][field] + lvl_off(level), st_, out, n);
        }
        return check("get_level");
    }

    hwfv1_status get_time(double* t, double* dt, int64_t* step) override {
        DevState s;
        if (read_state(&s) != HWFV1_OK) return HWFV1_ERR_CUDA;
        if (t) *t = s.t;
        if (dt) *dt = s.dt;
        if (step) *step = s.step;
        if (s.err & kErrNonFinite) return fail(HWFV1_ERR_NONFINITE, "non-finite value in the state");
        if (s.err & kErrTimeout) return fail(HWFV1_ERR_TIMEOUT, "a bounded device wait ran out");
        return HWFV1_OK;
    }

    hwfv1_status set_time(double t, double dt) override {
        DevState s;
        if (read_state(&s) != HWFV1_OK) return HWFV1_ERR_CUDA;
        s.t = t;
        s.dt = dt;
        cudaMemcpyAsync(st_, &s, sizeof s, cudaMemcpyHostToDevice, stream_);
        k_set_tend<<<1, 64, 0, stream_>>>(st_, fin_args(), s.t_end);
        return check("set_time", true);
    }

    // One plain step launched kernel by kernel with an event after every
    // launch; durations in launch order.
    // One plain step with a CUDA event after every kernel.  The step is
    // captured as a graph whose kernels are separated by event-record nodes
    // (so the times are those of kernels in a graph, without the launch
    // latency of separate stream launches); HWFV1_NO_GRAPH records the
    // events between ordinary launches.
    hwfv1_status profile_step(float* ms, const char** names, int32_t cap, int32_t* n) override {
        std::vector<std::pair<const char*, cudaEvent_t>> ev;
        cudaEvent_t e0;
        if (cudaEventCreate(&e0) != cudaSuccess) return fail(HWFV1_ERR_CUDA, "event");
        const bool use_graph = std::getenv("HWFV1_NO_GRAPH") == nullptr;
        // the step the schedule takes next (the plain step outside the skip)
        const int pkind = skipmode_ ? skip_kind(lstep_++) : kStepPlain;
        hwfv1_status r = HWFV1_OK;
        if (use_graph) {
            cudaGraph_t g = nullptr;
            cudaGraphExec_t x = nullptr;
            if (cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                cudaEventDestroy(e0);
                return fail(HWFV1_ERR_CUDA, "graph capture begin");
            }
            cudaEventRecordWithFlags(e0, stream_, cudaEventRecordExternal);
            prof_ = &ev;
            prof_external_ = true;
            launch_step(pkind);
            prof_ = nullptr;
            prof_external_ = false;
            if (cudaStreamEndCapture(stream_, &g) != cudaSuccess) r = fail(HWFV1_ERR_CUDA, "graph capture end");
            if (r == HWFV1_OK && cudaGraphInstantiate(&x, g, 0) != cudaSuccess) r = fail(HWFV1_ERR_CUDA, "graph instantiate");
            if (r == HWFV1_OK && cudaGraphLaunch(x, stream_) != cudaSuccess) r = fail(HWFV1_ERR_CUDA, "graph launch");
            if (r == HWFV1_OK) r = check("profile_step", true);
            else cudaStreamSynchronize(stream_);
            if (x) cudaGraphExecDestroy(x);
            if (g) cudaGraphDestroy(g);
        } else {
            cudaEventRecord(e0, stream_);
            prof_ = &ev;
            launch_step(pkind);
            prof_ = nullptr;
            r = check("profile_step", true);
        }
        int32_t k = 0;
        cudaEvent_t prev = e0;
        for (auto& p : ev) {
            float t = 0.f;
            if (r == HWFV1_OK && cudaEventElapsedTime(&t, prev, p.second) != cudaSuccess) r = fail(HWFV1_ERR_CUDA, "event");
            if (k < cap) {
                if (ms) ms[k] = t;
                if (names) names[k] = p.first;
            }
            ++k;
            prev = p.second;
        }
        for (auto& p : ev) cudaEventDestroy(p.second);
        cudaEventDestroy(e0);
        if (n) *n = k;
        return r;
    }

    // One plain step whose full update of the queued leaves (the pair of
    // shared-face kernels, or their one-pass form) is captured on its own and
    // replayed `reps` times between two CUDA events before the step goes on:
    // the update reads the current state and the queue and writes the next
    // state's leaf values and min/max reductions, so every replay writes the
    // same values.  *ms = the mean time of one update.
    hwfv1_status profile_update(int32_t reps, float* ms) override {
        if (reps < 1 || !ms) return fail(HWFV1_ERR_INVALID_SPEC, "profile_update: reps >= 1 and ms");
        if (hwfv1_status r = phase_guard("profile_update"); r != HWFV1_OK) return r;
        const bool onfly = onfly_flags();
        launch_encode();
        if (!onfly) launch_flag();
        launch_traverse(false, onfly);
        StepArgs<T> a = step_args();
        lk(k_fv1_dry<T>, grid_res(k_fv1_dry<T>, grid_for(N_), 256), 256, a);
        cudaGraph_t g = nullptr;
        cudaGraphExec_t x = nullptr;
        hwfv1_status r = HWFV1_OK;
        if (cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return fail(HWFV1_ERR_CUDA, "graph capture begin");
        launch_wet(a);
        if (cudaStreamEndCapture(stream_, &g) != cudaSuccess) r = fail(HWFV1_ERR_CUDA, "graph capture end");
        if (r == HWFV1_OK && cudaGraphInstantiate(&x, g, 0) != cudaSuccess) r = fail(HWFV1_ERR_CUDA, "graph instantiate");
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (r == HWFV1_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
            r = fail(HWFV1_ERR_CUDA, "event");
        if (r == HWFV1_OK) {
            cudaGraphLaunch(x, stream_);                  // once untimed
            cudaEventRecord(e0, stream_);
            for (int32_t k = 0; k < reps; ++k) cudaGraphLaunch(x, stream_);
            cudaEventRecord(e1, stream_);
            launch_decode(onfly);
            sb_valid_ = !onfly;
            r = check("profile_update", true);
            float t = 0.f;
            if (r == HWFV1_OK && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) r = fail(HWFV1_ERR_CUDA, "event");
            *ms = t / (float)reps;
        } else {
            cudaStreamSynchronize(stream_);
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (x) cudaGraphExecDestroy(x);
        if (g) cudaGraphDestroy(g);
        return r;
    }

    hwfv1_status get_counters(int64_t* steps, int64_t* lu, int64_t* au, int64_t* wu, int64_t* kps) override {
        if (kps) {
            if (!exec_ && capture(&exec_, kStepPlain) != HWFV1_OK) return HWFV1_ERR_CUDA;
            if (!exec_multi_ && !skipmode_ && std::getenv("HWFV1_NO_GRAPH") == nullptr &&
                capture(&exec_multi_, kStepPlain, kMultiSteps) != HWFV1_OK)
                return HWFV1_ERR_CUDA;
            *kps = skipmode_ ? kernels_skip_ : kernels_plain_;
        }
        DevState s;
        if (read_state(&s) != HWFV1_OK) return HWFV1_ERR_CUDA;
        if (steps) *steps = s.step;
        if (lu) *lu = (int64_t)s.leaf_updates;
        if (au) *au = (int64_t)s.act_updates;
        if (wu) *wu = (int64_t)s.wet_updates;
        return HWFV1_OK;
    }

    hwfv1_status get_stats(int64_t* M, double* smax3) override {
        DevState s;
        if (read_state(&s) != HWFV1_OK) return HWFV1_ERR_CUDA;
        if (M) *M = s.Mall;
        if (smax3)
            for (int q = 0; q < 3; ++q) smax3[q] = s.smax[q];
        return HWFV1_OK;
    }

    hwfv1_status save(void* buf, size_t cap, size_t* used) override {
        const size_t need = sizeof(SaveHeader) + 3 * N_ * sizeof(T);
        if (used) *used = need;
        if (!buf) return HWFV1_OK;
        if (cap < need) return fail(HWFV1_ERR_INVALID_SPEC, "save: buffer too small");
        // a checkpoint holds the finest state: with the learned skip every
        // subtree is brought to level L first (its storage starts again there)
        if (skipmode_) launch_skip_finest(2);
        DevState s;
        if (read_state(&s) != HWFV1_OK) return HWFV1_ERR_CUDA;
        SaveHeader hd{kSaveMagic, L_, (int32_t)(sizeof(T) * 8), s.t, s.dt, s.step};
        std::memcpy(buf, &hd, sizeof hd);
        char* p = static_cast<char*>(buf) + sizeof hd;
        for (int q = 0; q < 3; ++q)
            cudaMemcpyAsync(p + q * N_ * sizeof(T), f_[s.cur][q] + lvl_off(L_), N_ * sizeof(T),
                            cudaMemcpyDeviceToHost, stream_);
        return check("save", true);
    }

    hwfv1_status load(const void* buf, size_t n) override {
        const size_t need = sizeof(SaveHeader) + 3 * N_ * sizeof(T);
        if (!buf || n < need) return fail(HWFV1_ERR_INVALID_SPEC, "load: buffer too small");
        SaveHeader hd;
        std::memcpy(&hd, buf, sizeof hd);
        if (hd.magic != kSaveMagic || hd.L != L_ || hd.precision != (int32_t)(sizeof(T) * 8))
            return fail(HWFV1_ERR_INVALID_SPEC, "load: checkpoint of another problem");
        DevState s;
        if (read_state(&s) != HWFV1_OK) return HWFV1_ERR_CUDA;
        const char* p = static_cast<const char*>(buf) + sizeof hd;
        for (int q = 0; q < 3; ++q)
            cudaMemcpyAsync(f_[s.cur][q] + lvl_off(L_), p + q * N_ * sizeof(T), N_ * sizeof(T),
                            cudaMemcpyHostToDevice, stream_);
        s.t = hd.t;
        s.dt = hd.dt;
        s.step = hd.step;
        s.err = 0;
        cudaMemcpyAsync(st_, &s, sizeof s, cudaMemcpyHostToDevice, stream_);
        forget_quiet();
        stored_at_finest();
        reduce_state(/*set_dt=*/0);
        return check("load", true);
    }

    // Everything a batched step needs for this domain (see batch.cuh):
    // encode passes of at most enc_k levels, FV1 work of about fv1_cells
    // finest cells per thread (the block count is set by the batch).
    template <class Plan>
    void fill_plan(Plan& p, int enc_k, int /*fv1_cells*/) const {
        for (int b = 0; b < 2; ++b)
            for (int q = 0; q < 3; ++q) p.enc.f[b][q] = f_[b][q];
        p.enc.thr = thr_dyn();
        p.enc.thr4 = thr4_dyn();
        if (sizeof(T) == 8) {
            p.enc.thr4lo = st_->thr4lo;
            p.enc.thr4hi = st_->thr4hi;
        }
        p.enc.Tb = Tb_;
        p.enc.Cb = Cb_;
        p.enc.st = st_;
        p.enc.L = L_;
        p.enc.ls = L_;
        p.enc.k = enc_k;
        p.npass = 0;
        p.enc.span = 0;
        for (int ls = L_; ls > 0 && p.npass < (int)(sizeof(p.ls) / sizeof(p.ls[0]));) {
            int k = ls < enc_k ? ls : enc_k;
            // with 5 levels per pass, the first pass of a domain of L >= 8
            // stops after three levels of each 1024-cell block, as the
            // single-domain full sweep does (a shorter chain per CTA)
            if (ls == L_ && enc_k == 5 && ls >= 8) {
                k = 3;
                p.enc.span = 5;
            }
            p.ls[p.npass] = ls;
            p.kk[p.npass] = k;
            p.npass++;
            ls -= k;
        }
        p.clear_w = Tb_;
        p.clear_n = 2 * words_;
        p.flag.Tb = Tb_;
        p.flag.Cb = Cb_;
        p.flag.Sbase = Sz_;
        p.flag.Sb = Sb_;
        p.flag.L = L_;
        p.flag.predict = predict();
        p.flag.close = close();
        p.flag.st = st_;
        p.Sb = Sb_;
        p.csum = counts_;
        p.coffs = offs_;
        p.dlist = dlist_;
        p.leaves = leaves_;
        p.L = L_;
        p.kt = kt_;
        p.ntiles = ntiles_;
        p.nct = (ntiles_ + kTilesPerCta - 1) / kTilesPerCta;
        p.step = step_args();
        p.dec = decode_args();
        p.fin = fin_args();
        p.st = st_;
    }

   private:
    // ---- launch helpers -------------------------------------------------
    // blocks of 64 threads for the wet-leaf kernels: 16 per SM at most
    int wet_grid() const {
        const uint64_t g = (N_ + 63) / 64, cap = (uint64_t)nsm_ * 16;
        return (int)(g < cap ? (g < 1 ? 1 : g) : cap);
    }
    // Blocks of `threads` that one launch of kern keeps resident on the GPU.
    // A grid-stride loop over more blocks than that runs its last ones as a
    // second wave after the first, each with its full share of the work:
    // such grids are capped here.
    template <typename K>
    int resident(K kern, int threads) {
        const void* key = reinterpret_cast<const void*>(kern);
        auto it = occ_.find(key);
        if (it != occ_.end()) return it->second;
        int per = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, 0) != cudaSuccess) {
            cudaGetLastError();
            per = 0;
        }
        const int r = nsm_ * (per < 1 ? 1 : per);
        occ_[key] = r;
        return r;
    }
    template <typename K>
    int grid_res(K kern, int g, int threads) {
        const int r = resident(kern, threads);
        return g < r ? g : r;
    }
    int grid_for(uint64_t n) const {
        uint64_t g = (n + 255) / 256;
        const uint64_t cap = (uint64_t)nsm_ * 8;
        if (g > cap) g = cap;
        return g < 1 ? 1 : (int)g;
    }
    int predict() const { return (spec_.flags & HWFV1_REG_PREDICT) ? 1 : 0; }
    int close() const { return (spec_.flags & HWFV1_REG_CLOSE) ? 1 : 0; }
    const T* thr_z() const;
    const T* thr_dyn() const;
    const T* thr4_z() const;
    const T* thr4_dyn() const;
    // aux buffer: z max bits, s_max of z, bed thresholds (thr, 4 thr) per precision
    static constexpr size_t kZThrD = 16, kZThrF = kZThrD + 8 * kMaxL, kZThr4D = 256,
                            kZThr4F = kZThr4D + 8 * kMaxL, kZauxBytes = 512;

    // Passes of up to five levels from L down to 0.  With `ticket`, the
    // final one-CTA pass runs in the last CTA of the pass before it.  With
    // a.list, the first pass works on the listed tiles (k_encode_tiles).
    template <int NF>
    void encode_passes(EncodeArgs<T, NF> a, uint32_t* ticket = nullptr, int from = -1) {
        int ls = from < 0 ? L_ : from;
        bool list_reset = a.list == nullptr;
        while (ls > 0) {
            int k = ls < 5 ? ls : 5;
            a.span = 0;
            // a first pass over every one of many tiles stops after three
            // levels of each 1024-cell block: a shorter chain per CTA, and the
            // block's two top levels move to the next pass, which reads 1/64
            // of the data
            if (ls == L_ && a.zf[0] == nullptr && a.list == nullptr && NF == 3 && ls >= 8 &&
                (1u << (2 * (ls - 5))) > (uint32_t)nsm_ * 8u) {
                k = 3;
                a.span = 5;
            }
            a.ls = ls;
            a.k = k;
            const uint32_t nb = 1u << (2 * (ls - (a.span ? a.span : k)));
            const int ls2 = ls - k, k2 = ls2 < 5 ? ls2 : 5;
            if (ls == L_ && a.list != nullptr) {
                lk(k_encode_tiles<T, NF>, nsm_ * 8, 256, a);
                mark("k_encode_tiles");
            } else if (ticket && ls2 > 0 && ls2 == k2) {      // next pass is the last (one CTA)
                lk(k_encode_tail<T, NF>, nb, 256, a, ls2, k2, ticket);
                mark("k_encode_tail");
                list_reset = true;                         // its last CTA resets the list
                break;                                     // levels ls2-1 .. 0 done too
            } else {
                lk(k_encode<T, NF>, nb, 256, a);
                mark("k_encode");
            }
            ls -= k;
        }
        if (!list_reset) cudaMemsetAsync(&st_->ntodo, 0, sizeof(uint32_t), stream_);
    }

    // the first encode pass takes a tile list when quiescent tiles are
    // skipped and there are more tiles than a grid of 8 CTAs per SM
    bool tile_list() const { return quiet_on_ && ntiles_ > (uint32_t)nsm_ * 8u && L_ - kt_ > 0; }

    void launch_encode() {
        uint32_t* list = tile_list() ? work_ : nullptr;
        lk(k_clear_words, grid_for(2 * (uint64_t)words_), 256, Tb_, 2 * words_, st_,
           (const uint8_t*)tilebytes_, (const uint8_t*)(tilebytes_ + ntiles_), ntiles_, list, &st_->ndec);
        mark("k_clear_words");
        EncodeArgs<T, 3> a;
        a.list = list;
        for (int b = 0; b < 2; ++b)
            for (int q = 0; q < 3; ++q) a.f[b][q] = f_[b][q];
        a.thr = thr_dyn();
        a.thr4 = thr4_dyn();
        if (sizeof(T) == 8) {           // float pre-check of the details (float64 only)
            a.thr4lo = st_->thr4lo;
            a.thr4hi = st_->thr4hi;
        }
        a.Tb = Tb_;
        a.Cb = Cb_;
        a.st = st_;
        a.L = L_;
        if (quiet_on_) {
            a.zf[0] = tilebytes_;
            a.zf[1] = tilebytes_ + ntiles_;
        }
        encode_passes(a, &st_->enc_ticket);
    }
    void launch_flag() {
        lk(k_flag, grid_for(words_), 256, Tb_, Cb_, Sz_, Sb_, L_, predict(), close(), st_,
                                                       &st_->ndec);
        mark("k_flag");
    }
    // Where the step's traversal and decode read S: the words of k_flag, or
    // (onfly) words formed from the threshold, closure and bed flags on the
    // spot, which spares the plain step the flag kernel.
    SigSrc sig_src(bool onfly) const {
        SigSrc s;
        if (onfly) {
            s.Tb = Tb_;
            s.Cb = Cb_;
            s.Sbase = Sz_;
            s.predict = predict();
            s.close = close();
        } else {
            s.Sb = Sb_;
        }
        return s;
    }
    // the plain step forms S on the spot (the fused traversal of the full
    // sweep and the matched-flux kernels read the flag kernel's words)
    bool onfly_flags() const { return quiet_on_ && !(spec_.flags & HWFV1_FLUX_MATCH); }
    // materialise S for the readers of the words (listing, get_flags) when
    // the last step formed it on the spot
    void ensure_sig_words() {
        if (sb_valid_) return;
        lk(k_flag, grid_for(words_), 256, Tb_, Cb_, Sz_, Sb_, L_, predict(), close(),
           (const DevState*)nullptr, (uint32_t*)nullptr);
        sb_valid_ = true;
    }
    // `learned`: the flags come from the learned look-ahead, whose skipped
    // tiles need not hold the bed's static flags alone (no cached counts).
    // The four counters (ndec, Mall, M, nact) were cleared by the flag or
    // the clear kernel.
    void launch_traverse(bool learned = false, bool onfly = false) {
        const uint32_t nct = (ntiles_ + kTilesPerCta - 1) / kTilesPerCta;
        const uint32_t grid = nct < (uint32_t)nsm_ * 4u ? nct : (uint32_t)nsm_ * 4u;
        if (quiet_on_) {
            const SigSrc sg = sig_src(onfly && !learned);
            lk(k_trav_classify, (ntiles_ + 255) / 256, 256, sg, L_, kt_, ntiles_, st_, quiet(),
                                                                      learned ? nullptr : scount_, work_);
            mark("k_trav_classify");
            lk(k_trav_list, nsm_ * 8, 256, sg, dlist_, leaves_, L_, kt_, st_, work_);
            mark("k_trav_list");
        } else {
            lk(k_trav_fused, grid, 256, Sb_, dlist_, leaves_, L_, kt_, ntiles_, st_, quiet(),
                                                    learned ? nullptr : scount_);
            mark("k_trav_fused");
        }
    }
    // Launch of a kernel of the step chain with programmatic dependent launch:
    // its CTAs may be placed while the kernel ahead of it drains, and wait
    // in pdl_wait for its completion (captured into the step graph as a
    // programmatic edge).  HWFV1_NO_PDL gives ordinary launches.
    template <typename... KArgs, typename... Args>
    void lk(void (*k)(KArgs...), uint32_t grid, uint32_t block, Args... args) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(block);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = stream_;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = pdl_ ? 1 : 0;
        cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
    }
    void mark(const char* name) {
        if (!prof_) return;
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        if (prof_external_) cudaEventRecordWithFlags(e, stream_, cudaEventRecordExternal);
        else cudaEventRecord(e, stream_);
        prof_->push_back({name, e});
    }
    Quiet quiet() const {
        Quiet q;
        if (quiet_on_) {
            q.zf[0] = tilebytes_;
            q.zf[1] = tilebytes_ + ntiles_;
            q.inlet = tilebytes_ + 2 * ntiles_;
            q.act = tilebytes_ + 3 * ntiles_;
        }
        return q;
    }
    // after the stored state changed outside a step: no tile is known quiescent
    void forget_quiet() { cudaMemsetAsync(tilebytes_, 0, (size_t)ntiles_ * 2, stream_); }
    StepArgs<T> step_args() const {
        StepArgs<T> a;
        for (int b = 0; b < 2; ++b)
            for (int q = 0; q < 3; ++q) a.f[b][q] = f_[b][q];
        a.z = z_;
        a.leaves = leaves_;
        a.wet = wet_;
        a.st = st_;
        a.P = phys();
        a.lx = (T)spec_.lx;
        a.ly = (T)spec_.ly;
        a.L = L_;
        a.inflow_side = -1;
        for (int s = 0; s < 4; ++s) {
            a.bc_ref[s] = spec_.bc[s] != HWFV1_BC_TRANSMISSIVE;
            if (spec_.bc[s] == HWFV1_BC_INFLOW && spec_.inflow_n > 0 && spec_.inflow_a1 > spec_.inflow_a0)
                a.inflow_side = s;
        }
        a.a0 = spec_.inflow_a0;
        a.a1 = spec_.inflow_a1;
        a.face = face_;
        a.fcap = fcap_;
        a.mark = mark_;
        a.Sb = Sb_;
        a.fm = (spec_.flags & HWFV1_FLUX_MATCH) ? 1 : 0;
        return a;
    }
    Phys<T> phys() const {
        Phys<T> P;
        P.g = (T)spec_.g;
        P.hg = P.g * (T)0.5;                 // exact
        P.tol = (T)spec_.tol_h;
        P.nM = (T)spec_.manning_n;
        P.cfl = (T)spec_.cfl;
        P.dxL = (T)std::ldexp(spec_.lx, -L_);
        P.dyL = (T)std::ldexp(spec_.ly, -L_);
        return P;
    }
    void launch_fv1(const uint32_t* leaves = nullptr) {
        StepArgs<T> a = step_args();
        if (leaves) {
            a.leaves = leaves;
            a.fm = 0;            // every leaf on the finest level: nothing to match
        }
        lk(k_fv1_dry<T>, grid_res(k_fv1_dry<T>, grid_for(N_), 256), 256, a);
        mark("k_fv1_dry");
        launch_wet(a);
    }
    // the full update of the queued leaves (after k_fv1_dry)
    void launch_wet(const StepArgs<T>& a) {
        if (a.fm && face_) {
            // matched fluxes with shared faces: a face toward a refined
            // neighbour takes the walk over its halves in either phase
            lk(k_fv1_faces<T, true>, grid_res(k_fv1_faces<T, true>, wet_grid(), 64), 64, a);
            mark("k_fv1_faces");
            lk(k_fv1_update<T, true>, grid_res(k_fv1_update<T, true>, wet_grid(), 64), 64, a);
            mark("k_fv1_update");
        } else if (a.fm) {
            lk(k_fv1_match<T>, grid_res(k_fv1_match<T>, wet_grid(), 64), 64, a);
            mark("k_fv1_match");
        } else if (face_) {
            // 64-thread blocks: a short queue spreads over every SM's FP64 units
            // (one warp-wide FP64 instruction holds a sub-partition's unit for
            // tens of cycles, so few warps per unit means a shorter chain)
            lk(k_fv1_faces<T>, grid_res(k_fv1_faces<T>, wet_grid(), 64), 64, a);
            mark("k_fv1_faces");
            lk(k_fv1_update<T>, grid_res(k_fv1_update<T>, wet_grid(), 64), 64, a);
            mark("k_fv1_update");
        } else {
            lk(k_fv1_wet<T>, grid_res(k_fv1_wet<T>, wet_grid(), 64), 64, a);
            mark("k_fv1_wet");
        }
    }
    DecodeArgs<T> decode_args(bool onfly = false) const {
        DecodeArgs<T> a;
        for (int b = 0; b < 2; ++b)
            for (int q = 0; q < 3; ++q) a.f[b][q] = f_[b][q];
        a.z = z_;
        a.Sb = sig_src(onfly);
        a.dlist = dlist_;
        a.st = st_;
        a.tol = (T)spec_.tol_h;
        a.L = L_;
        a.kt = kt_;
        a.q = quiet();
        return a;
    }
    void launch_decode(bool onfly = false) {
        // the decode list is short once quiescent tiles are skipped: 2 CTAs per SM
        const int gd = quiet_on_ ? std::min(grid_for((uint64_t)ntiles_ * 256), nsm_ * 4)
                                 : grid_for((uint64_t)ntiles_ * 256);
        lk(k_decode_finish<T>, grid_res(k_decode_finish<T>, gd, 256), 256, decode_args(onfly), fin_args());
        mark("k_decode_finish");
    }
    void launch_step_uniform() {
        lk(k_set_uniform, 1, 32, st_, (uint32_t)N_);
        launch_fv1(uniform_leaves_);
        launch_decode();
    }
    void launch_step_all() {
        const bool onfly = onfly_flags();
        launch_encode();
        if (!onfly) launch_flag();
        launch_traverse(false, onfly);
        launch_fv1();
        launch_decode(onfly);
        sb_valid_ = !onfly;
    }
    void launch_features(__nv_bfloat16* out, cudaStream_t sm = nullptr) {
        const uint32_t n = 1u << (2 * (L_ - 4));
        const double* smax_z = reinterpret_cast<const double*>(zaux_ + 8);
        k_features<T><<<grid_for(n), 256, 0, sm ? sm : stream_>>>(
            f_[0][0], f_[1][0], f_[0][1], f_[1][1], f_[0][2], f_[1][2], z_, st_, smax_z, L_ - 4, out);
    }
    // ---- the learned subtree skip (skip.cuh) -------------------------------
    // the network's predicted levels for the next steps: features of the
    // current state's level L-4 (just encoded), three convolutions, levels
    // It runs beside the step on a second stream: forked once the step has
    // encoded (the features' level is formed) and read the levels in use,
    // joined before the decode, whose last CTA swaps the state buffers the
    // features read; the levels it writes serve the next steps.
    void fork_predict() {
        cudaEventRecord(ev_fork_, stream_);
        cudaStreamWaitEvent(side_, ev_fork_, 0);
        launch_features(feat_, side_);
        const int S = 1 << (L_ - 4);
        skipnet_forward(skip_, feat_, 1, S, S, &skw_, side_);
        k_predict<<<grid_for((uint64_t)S * S), 256, 0, side_>>>(skw_.Z3, L_ - 4, margin_, phat_);
        cudaEventRecord(ev_join_, side_);
    }
    void join_predict() { cudaStreamWaitEvent(stream_, ev_join_, 0); }
    // every subtree at level L: mode 0 into the other buffer (reading the
    // fields), 1 in place before a plain step (nothing when it will not
    // run), 2 in place unconditionally (leaving the skip, checkpoints)
    void launch_skip_finest(int mode) {
        if (!mlev_) return;
        SkipFinestArgs<T> a;
        for (int b = 0; b < 2; ++b)
            for (int q = 0; q < 3; ++q) a.f[b][q] = f_[b][q];
        a.z = z_;
        a.mlev = mlev_;
        a.flat = skipmode_ == 3 ? flat_ : nullptr;
        a.st = st_;
        a.tol = (T)spec_.tol_h;
        a.L = L_;
        a.Ls = L_ - 4;
        a.mode = mode;
        lk(k_skip_finest<T>, grid_res(k_skip_finest<T>, skip_grid(), 256), 256, a);
        mark("k_skip_finest");
    }
    int skip_grid() const {
        const uint32_t nsub = 1u << (2 * (L_ - 4));
        return grid_for((uint64_t)nsub * 64);
    }
    // one skip step; predict: the network runs (after the flags) and its
    // levels serve the following steps
    void launch_step_skip(bool predict_now) {
        const int Ls = L_ - 4;
        lk(k_clear_words, grid_for(2 * (uint64_t)words_), 256, Tb_, 2 * words_, st_, (const uint8_t*)nullptr,
           (const uint8_t*)nullptr, ntiles_, (uint32_t*)nullptr, &st_->ndec);
        mark("k_clear_words");
        const uint8_t* flat = skipmode_ == 3 ? flat_ : nullptr;
        if (flat) {
            lk(k_exact_levels, grid_for(1u << (2 * Ls)), 256, (const uint8_t*)mlev_, flat, phat_, L_, Ls,
               (const DevState*)st_);
            mark("k_exact_levels");
        }
        SkipArgs<T> a;
        for (int b = 0; b < 2; ++b)
            for (int q = 0; q < 3; ++q) a.f[b][q] = f_[b][q];
        a.flat = flat;
        a.z = z_;
        a.thr = thr_dyn();
        a.thr4 = thr4_dyn();
        if (sizeof(T) == 8) {
            a.thr4lo = st_->thr4lo;
            a.thr4hi = st_->thr4hi;
        }
        a.Tz = Tz_;
        a.Tb = Tb_;
        a.Cb = Cb_;
        a.phat = phat_;
        a.mlev = mlev_;
        a.plev = plev_;
        a.st = st_;
        a.tol = (T)spec_.tol_h;
        a.L = L_;
        a.Ls = Ls;
        lk(k_skip_encode<T>, grid_res(k_skip_encode<T>, grid_for((uint64_t)(1u << (2 * Ls)) * 32), 256), 256, a);
        mark("k_skip_encode");
        if (Ls > 0) {
            EncodeArgs<T, 3> e;
            for (int b = 0; b < 2; ++b)
                for (int q = 0; q < 3; ++q) e.f[b][q] = f_[b][q];
            e.thr = thr_dyn();
            e.thr4 = thr4_dyn();
            if (sizeof(T) == 8) {
                e.thr4lo = st_->thr4lo;
                e.thr4hi = st_->thr4hi;
            }
            e.Tb = Tb_;
            e.Cb = Cb_;
            e.st = st_;
            e.L = L_;
            encode_passes(e, &st_->enc_ticket, Ls);
        }
        lk(k_skip_flag, grid_for(words_), 256, Tb_, Cb_, Tz_, czu_, Sb_, phat_, L_, Ls, st_);
        mark("k_skip_flag");
        if (predict_now) fork_predict();
        const uint32_t nct = (ntiles_ + kTilesPerCta - 1) / kTilesPerCta;
        const uint32_t tgrid = nct < (uint32_t)nsm_ * 4u ? nct : (uint32_t)nsm_ * 4u;
        lk(k_trav_fused, tgrid, 256, Sb_, dlist_, leaves_, L_, kt_, ntiles_, st_, Quiet(),
           (const uint32_t*)nullptr);
        mark("k_trav_fused");
        StepArgs<T> sa = step_args();
        sa.own_slot = 1;
        lk(k_fv1_dry<T>, grid_res(k_fv1_dry<T>, grid_for(N_), 256), 256, sa);
        mark("k_fv1_dry");
        launch_wet(sa);
        if (predict_now) join_predict();
        SkipDecodeArgs<T> d;
        for (int b = 0; b < 2; ++b)
            for (int q = 0; q < 3; ++q) d.f[b][q] = f_[b][q];
        d.z = z_;
        d.Sb = Sb_;
        d.plev = plev_;
        d.mlev = mlev_;
        d.flat = flat;
        d.st = st_;
        d.tol = (T)spec_.tol_h;
        d.L = L_;
        d.Ls = Ls;
        lk(k_skip_decode<T>, grid_res(k_skip_decode<T>, skip_grid(), 256), 256, d, fin_args());
        mark("k_skip_decode");
        sb_valid_ = true;
    }
    // the exact audit step: every subtree at level L, no quiescence marks,
    // then the plain step (with the network after its encode when the next
    // steps take its levels)
    void launch_step_audit(bool predict_next) {
        launch_skip_finest(1);
        forget_quiet();
        const bool onfly = onfly_flags();
        launch_encode();
        if (predict_next) fork_predict();
        if (!onfly) launch_flag();
        launch_traverse(false, onfly);
        launch_fv1();
        if (predict_next) join_predict();
        launch_decode(onfly);
        sb_valid_ = !onfly;
    }
    enum { kStepPlain = 0, kStepAudit = 1, kStepAuditPredict = 2, kStepSkip = 3, kStepSkipPredict = 4 };
    // kind of the step at position `pos` (counted from the last
    // set_skipnet / set_skip_levels) in the skip mode: an audit every
    // audit_K_-th step; the network runs on the steps at multiples of every_
    // within the audit interval when a skip step follows
    int skip_kind(int64_t pos) const {
        const int64_t q = pos % audit_K_;
        const bool pred = skipmode_ == 1 && (q % every_) == 0 && q + 1 < audit_K_;
        if (q == 0) return pred ? kStepAuditPredict : kStepAudit;
        return pred ? kStepSkipPredict : kStepSkip;
    }
    void launch_step(int kind) {
        if (kind == kStepPlain) launch_step_all();
        else if (kind == kStepAudit || kind == kStepAuditPredict) launch_step_audit(kind == kStepAuditPredict);
        else launch_step_skip(kind == kStepSkipPredict);
    }
    void drop_skip_graphs() {
        for (cudaGraphExec_t& g : exec_skip_) {
            if (g) cudaGraphExecDestroy(g);
            g = nullptr;
        }
    }
    // the graphs of the kinds the schedule uses, captured now (capturing
    // runs nothing) so that the first advance does not pay for them
    hwfv1_status capture_skip_graphs() {
        if (std::getenv("HWFV1_NO_GRAPH") != nullptr) return HWFV1_OK;
        const int64_t n = audit_K_ < 64 ? audit_K_ : 64;
        for (int64_t pos = 0; pos < n; ++pos) {
            const int kind = skip_kind(pos);
            cudaGraphExec_t* g = &exec_skip_[kind - kStepAudit];
            if (!*g && capture(g, kind) != HWFV1_OK) return HWFV1_ERR_CUDA;
        }
        return HWFV1_OK;
    }
    // enter the skip mode (1 network, 2 caller's levels): buffers, the
    // static closure of the bed's flags above the subtrees, storage levels
    // from the current state
    hwfv1_status skip_on(int mode, int audit_K) {
        if (batched_) return fail(HWFV1_ERR_STATE, "a batch member is stepped by its batch (plain steps only)");
        if (spec_.flags & HWFV1_FLUX_MATCH) return fail(HWFV1_ERR_INVALID_SPEC, "learned skip with HWFV1_FLUX_MATCH");
        if (!predict() || !close())
            return fail(HWFV1_ERR_INVALID_SPEC, "learned skip needs HWFV1_REG_PREDICT and HWFV1_REG_CLOSE");
        const int Ls = L_ - 4;
        const uint32_t nsub = 1u << (2 * Ls);
        if (!phat_ && !alloc(&phat_, nsub)) return oom();
        if (!mlev_ && !alloc(&mlev_, nsub)) return oom();
        if (!plev_ && !alloc(&plev_, nsub)) return oom();
        if (!czu_) {
            if (!alloc(&czu_, (size_t)words_ * sizeof(uint32_t))) return oom();
            // closure of the bed's threshold flags of levels < Ls, on the host
            std::vector<uint32_t> tz(words_), cz(words_, 0u);
            cudaMemcpyAsync(tz.data(), Tz_, (size_t)words_ * sizeof(uint32_t), cudaMemcpyDeviceToHost, stream_);
            if (hwfv1_status r = check("skip_on", true); r != HWFV1_OK) return r;
            auto bit = [](const std::vector<uint32_t>& w, int n, uint32_t c) {
                return (w[word_off(n) + (c >> 5)] >> (c & 31u)) & 1u;
            };
            for (int n = Ls - 1; n >= 0; --n)
                for (uint32_t c = 0; c < (1u << (2 * n)); ++c) {
                    uint32_t v = bit(tz, n, c);
                    if (n + 1 < Ls)
                        for (uint32_t k = 0; k < 4; ++k) v |= bit(cz, n + 1, 4 * c + k);
                    if (v) cz[word_off(n) + (c >> 5)] |= 1u << (c & 31u);
                }
            cudaMemcpyAsync(czu_, cz.data(), (size_t)words_ * sizeof(uint32_t), cudaMemcpyHostToDevice, stream_);
        }
        if (!skipmode_) {
            cudaMemsetAsync(mlev_, L_, nsub, stream_);
            cudaMemsetAsync(phat_, L_, nsub, stream_);
        }
        // a new mode or interval restarts the schedule (the next step is an
        // audit); new levels in the same mode and interval only replace the
        // levels (the captured graphs read them on the device)
        if (skipmode_ != mode || audit_K_ != audit_K) {
            skipmode_ = mode;
            audit_K_ = audit_K;
            lstep_ = 0;
            drop_skip_graphs();
        }
        return check("skip_on", true);
    }
    hwfv1_status skip_off() {
        if (skipmode_) launch_skip_finest(2);
        skipmode_ = 0;
        skip_ = nullptr;
        drop_skip_graphs();
        forget_quiet();
        return check("skip_off", true);
    }
    // the state was replaced by finest fields
    void stored_at_finest() {
        if (mlev_) cudaMemsetAsync(mlev_, L_, 1u << (2 * (L_ - 4)), stream_);
    }
    static constexpr int kMultiSteps = 16;   // plain steps per graph in hwfv1_advance
    hwfv1_status capture(cudaGraphExec_t* out, int kind, int nsteps = 1) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return fail(HWFV1_ERR_CUDA, "graph capture begin");
        // capturing runs nothing: host state the launches update is kept
        const bool sbv = sb_valid_;
        for (int k = 0; k < nsteps; ++k) launch_step(kind);
        sb_valid_ = sbv;
        if (cudaStreamEndCapture(stream_, &g) != cudaSuccess) return fail(HWFV1_ERR_CUDA, "graph capture end");
        const int64_t nk = count_kernel_nodes(g) / nsteps;
        if (kind == kStepPlain) kernels_plain_ = nk;
        else if (kind == kStepSkipPredict || (kind == kStepSkip && every_ > 1) ||
                 (kind == kStepSkip && skipmode_ == 2))
            kernels_skip_ = nk;
        const cudaError_t e = cudaGraphInstantiate(out, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            *out = nullptr;
            return fail(HWFV1_ERR_CUDA, "graph instantiate");
        }
        return HWFV1_OK;
    }
    FinishArgs fin_args() const {
        FinishArgs a;
        a.inflow_t = it_d_;
        a.inflow_Q = iq_d_;
        a.inflow_n = it_.empty() ? 0 : (int)it_.size();
        a.L = L_;
        a.eps = spec_.eps;
        a.cfl = spec_.cfl;
        a.dt_max = spec_.dt_max;
        a.lx = spec_.lx;
        a.ly = spec_.ly;
        a.g = spec_.g;
        a.manning_n = spec_.manning_n;
        return a;
    }
    // s_max (and dt when set_dt) from the finest fields of the current buffer
    void reduce_state(int set_dt) {
        k_reset_red<<<1, 32, 0, stream_>>>(st_);
        const int g = grid_for(N_);
        k_maxabs_cur<T><<<g, 256, 0, stream_>>>(f_[0][0] + lvl_off(L_), f_[1][0] + lvl_off(L_), st_, N_, 0);
        k_maxabs_cur<T><<<g, 256, 0, stream_>>>(f_[0][1] + lvl_off(L_), f_[1][1] + lvl_off(L_), st_, N_, 1);
        k_maxabs_cur<T><<<g, 256, 0, stream_>>>(f_[0][2] + lvl_off(L_), f_[1][2] + lvl_off(L_), st_, N_, 2);
        if (set_dt) {
            k_cfl_cur<T><<<g, 256, 0, stream_>>>(f_[0][0] + lvl_off(L_), f_[1][0] + lvl_off(L_),
                                                  f_[0][1] + lvl_off(L_), f_[1][1] + lvl_off(L_),
                                                  f_[0][2] + lvl_off(L_), f_[1][2] + lvl_off(L_), st_,
                                                  N_, phys());
        }
        k_init_state<<<1, 64, 0, stream_>>>(st_, fin_args(), set_dt);
    }

    hwfv1_status read_state(DevState* s) {
        if (cudaMemcpyAsync(s, st_, sizeof *s, cudaMemcpyDeviceToHost, stream_) != cudaSuccess ||
            cudaStreamSynchronize(stream_) != cudaSuccess)
            return fail(HWFV1_ERR_CUDA, std::string("read_state: ") + cudaGetErrorString(cudaGetLastError()));
        return HWFV1_OK;
    }
    // Stream-ordered allocations from the device's default pool, which keeps
    // what handles free for the next ones (release threshold: everything),
    // so that a handle created after another one (a new run of the same
    // problem) does not map its memory again.
    static void keep_pool_memory() {
        static bool done[64] = {};
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || done[dev]) return;
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t keep = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
        done[dev] = true;
    }
    template <typename P>
    bool alloc(P** p, size_t bytes) {
        void* v = nullptr;
        keep_pool_memory();
        if (cudaMallocAsync(&v, bytes, stream_) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        allocs_.push_back(v);
        *p = static_cast<P*>(v);
        return true;
    }
    hwfv1_status oom() { return fail(HWFV1_ERR_OOM, "device allocation failed"); }
    hwfv1_status fail(hwfv1_status s, const std::string& m) {
        err = m;
        return s;
    }
    // a pointer the host reads or writes (pinned or pageable memory), as
    // opposed to device or managed memory
    static bool on_host(const void* p) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
            cudaGetLastError();
            return true;                  // unknown to CUDA: ordinary host memory
        }
        return at.type == cudaMemoryTypeUnregistered || at.type == cudaMemoryTypeHost;
    }
    hwfv1_status host_io_ready() {
        if (!cstream_ && cudaStreamCreateWithFlags(&cstream_, cudaStreamNonBlocking) != cudaSuccess)
            return fail(HWFV1_ERR_CUDA, "copy stream");
        for (cudaEvent_t& e : hev_)
            if (!e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
                return fail(HWFV1_ERR_CUDA, "copy events");
        return HWFV1_OK;
    }
    // staging for host transfers: two field slots, stream-ordered on stream_
    // and handed to the copy stream (event 8), freed by the caller on stream_
    hwfv1_status stage_alloc(double** p) {
        void* v = nullptr;
        keep_pool_memory();
        if (cudaMallocAsync(&v, 2 * N_ * sizeof(double), stream_) != cudaSuccess) {
            cudaGetLastError();
            return oom();
        }
        *p = static_cast<double*>(v);
        cudaEventRecord(hev_[8], stream_);
        cudaStreamWaitEvent(cstream_, hev_[8], 0);
        return HWFV1_OK;
    }

    hwfv1_status check(const char* what, bool sync = false) {
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess && sync) e = cudaStreamSynchronize(stream_);
        if (e != cudaSuccess) return fail(HWFV1_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
        return HWFV1_OK;
    }

    hwfv1_problem spec_;
    cudaStream_t stream_ = nullptr;
    bool own_stream_ = false;
    int nsm_ = 152;
    int L_, kt_;
    uint64_t N_, H_;
    uint32_t ntiles_, words_;
    std::vector<double> it_, iq_;
    std::vector<void*> allocs_;
    T* f_[2][3] = {};
    T* z_ = nullptr;
    uint32_t *bits_ = nullptr, *Tb_ = nullptr, *Cb_ = nullptr, *Tz_ = nullptr, *Cz_ = nullptr,
             *Sz_ = nullptr, *Sb_ = nullptr;
    uint32_t* leaves_ = nullptr;
    uint32_t* wet_ = nullptr;
    uint32_t *counts_ = nullptr, *offs_ = nullptr, *dlist_ = nullptr;
    uint8_t* tilebytes_ = nullptr;      // per tile: zf of buffer 0, zf of buffer 1, inlet, act
    bool batched_ = false;
    T* face_ = nullptr;                 // shared faces and velocities (12 x fcap_)
    std::unordered_map<const void*, int> occ_;   // resident blocks per kernel
    uint32_t fcap_ = 0;
    unsigned long long* mark_ = nullptr;   // per hierarchy cell: (epoch + 1) << 32 | queue slot
    uint32_t* scount_ = nullptr;        // per tile: leaves when it holds the bed's flags alone
    uint32_t* work_ = nullptr;          // the traversal's list of tiles to treat one warp each
    bool quiet_on_ = false;
    bool pdl_ = true;             // programmatic dependent launch in the step chain
    bool sb_valid_ = true;        // Sb_ holds the S of the last step (else formed on the spot)
    std::vector<std::pair<const char*, cudaEvent_t>>* prof_ = nullptr;   // profile_step's events
    bool prof_external_ = false;          // events recorded as graph nodes (under capture)
    DevState* st_ = nullptr;
    char* zaux_ = nullptr;
    double *it_d_ = nullptr, *iq_d_ = nullptr;
    cudaGraphExec_t exec_ = nullptr;
    cudaGraphExec_t exec_multi_ = nullptr;   // kMultiSteps plain steps
    // host field transfers (hwfv1_init, hwfv1_get_fields with host buffers):
    // the copy stream and its events, made on first use
    cudaStream_t cstream_ = nullptr;
    cudaEvent_t hev_[9] = {};
    // learned subtree skip
    int skipmode_ = 0;     // 0 plain steps, 1 levels from the network, 2 levels from the caller
    SkipNet* skip_ = nullptr;
    int audit_K_ = 10;
    int every_ = 1;        // the network runs on every every_-th step of an audit interval
    float margin_ = 0.02f;
    int64_t lstep_ = 0;    // steps since the mode was set (the audit schedule)
    SkipWork skw_;
    __nv_bfloat16* feat_ = nullptr;
    uint8_t* phat_ = nullptr;    // predicted level per subtree (Morton order over level L-4)
    uint8_t* mlev_ = nullptr;    // storage level per subtree
    uint8_t* plev_ = nullptr;    // storage level per subtree after the running step
    uint32_t* czu_ = nullptr;    // closure of the bed's flags of levels < L-4
    uint8_t* flat_ = nullptr;    // exact store: 1 where the subtree's bed is flat
    cudaStream_t side_ = nullptr;           // the network's stream beside the step
    cudaEvent_t ev_fork_ = nullptr, ev_join_ = nullptr;
    cudaGraphExec_t exec_skip_[4] = {};   // audit, audit + network, skip, skip + network
    cudaGraphExec_t exec_uniform_ = nullptr;
    uint32_t* uniform_leaves_ = nullptr;   // every finest cell as a leaf (uniform FV1)
    int64_t kernels_plain_ = 0, kernels_skip_ = 0;   // kernel nodes of the captured step graphs
};

template <>
inline const double* EngineT<double>::thr_z() const {
    return reinterpret_cast<const double*>(zaux_ + kZThrD);
}
template <>
inline const float* EngineT<float>::thr_z() const {
    return reinterpret_cast<const float*>(zaux_ + kZThrF);
}
template <>
inline const double* EngineT<double>::thr4_z() const {
    return reinterpret_cast<const double*>(zaux_ + kZThr4D);
}
template <>
inline const float* EngineT<float>::thr4_z() const {
    return reinterpret_cast<const float*>(zaux_ + kZThr4F);
}
template <>
inline const double* EngineT<double>::thr4_dyn() const {
    return st_->thr4;
}
template <>
inline const float* EngineT<float>::thr4_dyn() const {
    return st_->thr4f;
}
template <>
inline const double* EngineT<double>::thr_dyn() const {
    return st_->thr;
}
template <>
inline const float* EngineT<float>::thr_dyn() const {
    return st_->thrf;
}

}  // namespace hwfv1
