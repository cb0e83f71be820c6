// batch.cuh -- many independent HWFV1 domains (mixed L) advanced together:
// every phase of a step is one launch over all domains, each launch's flat
// grid mapped onto (domain, block) through a per-domain block-offset table,
// and the whole ensemble step captured in one CUDA graph.
#pragma once
#include <algorithm>
#include <vector>

#include "engine.cuh"

namespace hwfv1 {

constexpr int kMaxPasses = 5;

enum BatchKind {
    BK_CLEAR = 0,
    BK_ENC0,                               // encode passes 0..kMaxPasses-1
    BK_FLAG = BK_ENC0 + kMaxPasses,
    BK_TCOUNT,
    BK_TSCAN,
    BK_TWRITE,
    BK_DRY,
    BK_WET,
    BK_DEC,
    BK_FIN,
    BK_KINDS
};

// Everything one domain's step needs, resolved once on the host.
template <typename T>
struct DomainPlan {
    EncodeArgs<T, 3> enc;
    int npass;
    int ls[kMaxPasses], kk[kMaxPasses];
    uint32_t* clear_w;
    uint32_t clear_n;
    FlagArgs flag;
    const uint32_t* Sb;
    uint32_t *csum, *coffs, *dlist, *leaves;
    int L, kt;
    uint32_t ntiles, nct;
    StepArgs<T> step;
    DecodeArgs<T> dec;
    FinishArgs fin;
    DevState* st;
};

// Domain owning flat block b: the largest d with base[d] <= b (domains with
// no block for this launch have base[d] == base[d+1] and are skipped).
__device__ __forceinline__ int find_domain(const uint32_t* __restrict__ base, int D, uint32_t b) {
    int lo = 0, hi = D - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(base + mid) <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ Blk domain_blk(const uint32_t* base, int d) {
    return Blk{blockIdx.x - base[d], base[d + 1] - base[d]};
}

template <typename T>
static __global__ void __launch_bounds__(256) kb_clear(const DomainPlan<T>* P, const uint32_t* base, int D) {
    const int d = find_domain(base, D, blockIdx.x);
    clear_body(P[d].clear_w, P[d].clear_n, P[d].st, domain_blk(base, d));
}

// The bodies take their arguments from a local copy of the domain's plan:
// read through the plan's global-memory address, every field would be
// reloaded after each store the body makes (the store could alias it).

template <typename T>
static __global__ void __launch_bounds__(256) kb_encode(const DomainPlan<T>* P, const uint32_t* base, int D,
                                                        int pass) {
    const int d = find_domain(base, D, blockIdx.x);
    const EncodeArgs<T, 3> a = P[d].enc;
    encode_body<T, 3>(a, P[d].ls[pass], P[d].kk[pass], blockIdx.x - base[d]);
}

template <typename T>
static __global__ void __launch_bounds__(256) kb_flag(const DomainPlan<T>* P, const uint32_t* base, int D) {
    const int d = find_domain(base, D, blockIdx.x);
    const FlagArgs& f = P[d].flag;
    // the traversal that follows lists its decode tiles from zero
    if (blockIdx.x == base[d] && threadIdx.x == 0) {
        f.st->ndec = 0u;
        f.st->Mall = 0u;
    }
    flag_body(f.Tb, f.Cb, f.Sbase, f.Sb, f.L, f.predict, f.close, f.st, domain_blk(base, d));
}

template <typename T>
static __global__ void __launch_bounds__(256) kb_trav_count(const DomainPlan<T>* P, const uint32_t* base, int D) {
    const int d = find_domain(base, D, blockIdx.x);
    const DomainPlan<T>& p = P[d];
    trav_count_body(p.Sb, p.csum, p.dlist, p.L, p.kt, p.ntiles, p.st, domain_blk(base, d), &p.st->Mall, Quiet());
}

template <typename T>
static __global__ void __launch_bounds__(1024) kb_trav_scan(const DomainPlan<T>* P, const uint32_t* base, int D) {
    const int d = find_domain(base, D, blockIdx.x);
    const DomainPlan<T>& p = P[d];
    trav_scan_body(p.csum, p.coffs, p.nct, p.st, &p.st->M);
}

template <typename T>
static __global__ void __launch_bounds__(256) kb_trav_write(const DomainPlan<T>* P, const uint32_t* base, int D) {
    const int d = find_domain(base, D, blockIdx.x);
    const DomainPlan<T>& p = P[d];
    trav_write_body(p.Sb, p.coffs, p.leaves, p.L, p.kt, p.ntiles, p.st, domain_blk(base, d), nullptr);
}

template <typename T>
static __global__ void __launch_bounds__(256) kb_fv1_dry(const DomainPlan<T>* P, const uint32_t* base, int D) {
    const int d = find_domain(base, D, blockIdx.x);
    const StepArgs<T> a = P[d].step;
    fv1_dry_body<T>(a, domain_blk(base, d));
}

// the shared-face pair of the single-domain path (float64; float32 domains
// have no face buffer and take the one-pass update inside kb_fv1_update),
// launched, as there, in 64-thread blocks
template <typename T>
static __global__ void __launch_bounds__(64) kb_fv1_faces(const DomainPlan<T>* P, const uint32_t* base, int D) {
    const int d = find_domain(base, D, blockIdx.x);
    const StepArgs<T> a = P[d].step;
    fv1_faces_body<T>(a, domain_blk(base, d));
}

template <typename T>
static __global__ void __launch_bounds__(64) kb_fv1_update(const DomainPlan<T>* P, const uint32_t* base, int D) {
    const int d = find_domain(base, D, blockIdx.x);
    const StepArgs<T> a = P[d].step;
    fv1_update_body<T>(a, domain_blk(base, d));
}

template <typename T>
static __global__ void __launch_bounds__(256) kb_decode(const DomainPlan<T>* P, const uint32_t* base, int D) {
    const int d = find_domain(base, D, blockIdx.x);
    const DecodeArgs<T> a = P[d].dec;
    decode_body<T>(a, domain_blk(base, d));
}

template <typename T>
static __global__ void kb_finish(const DomainPlan<T>* P, int D) {
    const DomainPlan<T>& p = P[blockIdx.x];
    finish_body(p.st, p.fin);
}

template <typename T>
static __global__ void kb_set_tend(const DomainPlan<T>* P, int D, double t_end) {
    const DomainPlan<T>& p = P[blockIdx.x];
    set_tend_body(p.st, p.fin, t_end);
}

template <typename T>
class BatchT final : public Batch {
   public:
    BatchT(const hwfv1_problem* specs, int n, cudaStream_t stream) : stream_(stream) {
        specs_.assign(specs, specs + n);
    }
    ~BatchT() override {
        if (exec_) cudaGraphExecDestroy(exec_);
        if (d_plans_) cudaFree(d_plans_);
        if (d_bases_) cudaFree(d_bases_);
        for (auto* e : doms_) delete e;
        if (own_stream_) cudaStreamDestroy(stream_);
    }

    hwfv1_status init(const double* const* z, const double* const* h, const double* const* qx,
                      const double* const* qy) override {
        if (!stream_) {
            if (cudaStreamCreate(&stream_) != cudaSuccess) return fail(HWFV1_ERR_CUDA, "stream");
            own_stream_ = true;
        }
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm_, cudaDevAttrMultiProcessorCount, dev);
        const int D = (int)specs_.size();
        for (int d = 0; d < D; ++d) {
            // the batched kernels update every tile (no quiescence bookkeeping),
            // so a member never skips tiles, whichever path advances it
            hwfv1_problem sd = specs_[d];
            sd.flags |= HWFV1_FULL_SWEEP;
            auto* e = new EngineT<T>(sd, stream_, /*batched=*/true);
            doms_.push_back(e);
            const hwfv1_status s = e->init(z[d], h[d], qx[d], qy[d]);
            if (s != HWFV1_OK) return fail(s, "domain " + std::to_string(d) + ": " + e->err);
        }
        if (cudaMalloc(&d_plans_, sizeof(DomainPlan<T>) * D) != cudaSuccess ||
            cudaMalloc(&d_bases_, sizeof(uint32_t) * (D + 1) * BK_KINDS) != cudaSuccess) {
            cudaGetLastError();
            return fail(HWFV1_ERR_OOM, "batch tables");
        }
        return replan(enc_k_, fv1_cells_);
    }

    hwfv1_status advance(double t_end, int64_t max_steps) override {
        if (max_steps < 0) return fail(HWFV1_ERR_INVALID_SPEC, "max_steps < 0");
        const int D = (int)doms_.size();
        kb_set_tend<T><<<D, 64, 0, stream_>>>(d_plans_, D, t_end);
        if (!exec_) {
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                return fail(HWFV1_ERR_CUDA, "graph capture begin");
            launch_step();
            if (cudaStreamEndCapture(stream_, &g) != cudaSuccess) return fail(HWFV1_ERR_CUDA, "graph capture end");
            const cudaError_t e = cudaGraphInstantiate(&exec_, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                exec_ = nullptr;
                return fail(HWFV1_ERR_CUDA, "graph instantiate");
            }
        }
        for (int64_t s = 0; s < max_steps; ++s)
            if (cudaGraphLaunch(exec_, stream_) != cudaSuccess) return fail(HWFV1_ERR_CUDA, "graph launch");
        return check("batch advance");
    }

    // Time trial_steps ensemble steps under each candidate (levels per encode
    // pass, finest cells per FV1 thread) and keep the fastest.  Every
    // candidate computes bit-identical results; the trials advance the
    // ensemble by (candidates x trial_steps) steps.
    hwfv1_status autotune(int64_t trial_steps, int32_t* choice) override {
        if (trial_steps < 1) return fail(HWFV1_ERR_INVALID_SPEC, "trial_steps < 1");
        const int enc_c[3] = {5, 4, 3};
        const int fv1_c[4] = {8, 32, 128, 512};
        float best = 1e30f;
        int be = enc_k_, bf = fv1_cells_;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (int ek : enc_c) {
            for (int fc : fv1_c) {
                hwfv1_status s = replan(ek, fc);
                if (s != HWFV1_OK) return s;
                s = advance(HUGE_VAL, 1);           // capture + warm
                if (s != HWFV1_OK) return s;
                cudaEventRecord(e0, stream_);
                s = advance(HUGE_VAL, trial_steps);
                if (s != HWFV1_OK) return s;
                cudaEventRecord(e1, stream_);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) {
                    best = ms;
                    be = ek;
                    bf = fc;
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (choice) {
            choice[0] = be;
            choice[1] = bf;
        }
        return replan(be, bf);
    }

    Engine* member(int d) override { return (d >= 0 && d < (int)doms_.size()) ? doms_[d] : nullptr; }
    int size() const override { return (int)doms_.size(); }
    int64_t launches_per_step() const override { return launches_; }

   private:
    // Plans and block tables for a configuration (levels per encode pass,
    // finest cells per FV1 thread); drops the captured graph.
    hwfv1_status replan(int enc_k, int fv1_cells) {
        enc_k_ = enc_k;
        fv1_cells_ = fv1_cells;
        if (exec_) {
            cudaGraphExecDestroy(exec_);
            exec_ = nullptr;
        }
        const int D = (int)doms_.size();
        std::vector<DomainPlan<T>> plans(D);
        std::vector<uint32_t> nb((size_t)BK_KINDS * D, 0u);
        for (int d = 0; d < D; ++d) {
            DomainPlan<T>& p = plans[d];
            doms_[d]->fill_plan(p, enc_k, fv1_cells);
            auto set = [&](int kind, uint32_t n) { nb[(size_t)kind * D + d] = n; };
            set(BK_CLEAR, std::min<uint32_t>(64u, (p.clear_n + 255u) / 256u));
            for (int q = 0; q < kMaxPasses; ++q)
                set(BK_ENC0 + q, q < p.npass ? (1u << (2 * (p.ls[q] - ((q == 0 && p.enc.span) ? p.enc.span
                                                                                          : p.kk[q])))) : 0u);
            set(BK_FLAG, std::min<uint32_t>(64u, (bits_words(p.L) + 255u) / 256u));
            set(BK_TCOUNT, p.nct);
            set(BK_TSCAN, 1u);
            set(BK_TWRITE, p.nct);
            const uint64_t N = 1ull << (2 * p.L);
            const uint32_t fb = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(1024, N / (256ull * fv1_cells)));
            set(BK_DRY, fb);
            set(BK_WET, 4u * fb);                      // 64-thread blocks, as many threads
            set(BK_DEC, std::min<uint32_t>(p.ntiles, 64u));
            set(BK_FIN, 1u);
        }
        std::vector<uint32_t> bases((size_t)BK_KINDS * (D + 1));
        for (int k = 0; k < BK_KINDS; ++k) {
            uint32_t acc = 0;
            for (int d = 0; d < D; ++d) {
                bases[(size_t)k * (D + 1) + d] = acc;
                acc += nb[(size_t)k * D + d];
            }
            bases[(size_t)k * (D + 1) + D] = acc;
        }
        total_.assign(BK_KINDS, 0u);
        for (int k = 0; k < BK_KINDS; ++k) total_[k] = bases[(size_t)k * (D + 1) + D];
        cudaMemcpyAsync(d_plans_, plans.data(), sizeof(DomainPlan<T>) * D, cudaMemcpyHostToDevice, stream_);
        cudaMemcpyAsync(d_bases_, bases.data(), sizeof(uint32_t) * bases.size(), cudaMemcpyHostToDevice, stream_);
        launches_ = 0;
        for (int k = 0; k < BK_KINDS; ++k) launches_ += total_[k] > 0 ? 1 : 0;
        if (total_[BK_WET] > 0) launches_ += 1;        // the wet update is two kernels
        return check("batch plan", true);
    }

    const uint32_t* base(int kind) const { return d_bases_ + (size_t)kind * (doms_.size() + 1); }

    void launch_step() {
        const int D = (int)doms_.size();
        if (total_[BK_CLEAR]) kb_clear<T><<<total_[BK_CLEAR], 256, 0, stream_>>>(d_plans_, base(BK_CLEAR), D);
        for (int q = 0; q < kMaxPasses; ++q)
            if (total_[BK_ENC0 + q])
                kb_encode<T><<<total_[BK_ENC0 + q], 256, 0, stream_>>>(d_plans_, base(BK_ENC0 + q), D, q);
        kb_flag<T><<<total_[BK_FLAG], 256, 0, stream_>>>(d_plans_, base(BK_FLAG), D);
        kb_trav_count<T><<<total_[BK_TCOUNT], 256, 0, stream_>>>(d_plans_, base(BK_TCOUNT), D);
        kb_trav_scan<T><<<total_[BK_TSCAN], 1024, 0, stream_>>>(d_plans_, base(BK_TSCAN), D);
        kb_trav_write<T><<<total_[BK_TWRITE], 256, 0, stream_>>>(d_plans_, base(BK_TWRITE), D);
        kb_fv1_dry<T><<<total_[BK_DRY], 256, 0, stream_>>>(d_plans_, base(BK_DRY), D);
        kb_fv1_faces<T><<<total_[BK_WET], 64, 0, stream_>>>(d_plans_, base(BK_WET), D);
        kb_fv1_update<T><<<total_[BK_WET], 64, 0, stream_>>>(d_plans_, base(BK_WET), D);
        kb_decode<T><<<total_[BK_DEC], 256, 0, stream_>>>(d_plans_, base(BK_DEC), D);
        kb_finish<T><<<D, 64, 0, stream_>>>(d_plans_, D);
    }

    hwfv1_status fail(hwfv1_status s, const std::string& m) {
        err = m;
        return s;
    }
    hwfv1_status check(const char* what, bool sync = false) {
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess && sync) e = cudaStreamSynchronize(stream_);
        if (e != cudaSuccess) return fail(HWFV1_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
        return HWFV1_OK;
    }

    std::vector<hwfv1_problem> specs_;
    std::vector<EngineT<T>*> doms_;
    cudaStream_t stream_ = nullptr;
    bool own_stream_ = false;
    int nsm_ = 152;
    int enc_k_ = 5, fv1_cells_ = 32;
    DomainPlan<T>* d_plans_ = nullptr;
    uint32_t* d_bases_ = nullptr;
    std::vector<uint32_t> total_;
    int64_t launches_ = 0;
    cudaGraphExec_t exec_ = nullptr;
};

}  // namespace hwfv1
