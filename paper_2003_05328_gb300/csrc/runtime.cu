// runtime.cu -- the batching runtime around the per-layer kernels: a plan
// that records many layers as one CUDA graph (with an autotuner for the
// ciphertext packing and the HomConv kernel variant) and a continuous-batching
// server with HBM-budget admission.  Host C++ only; all arithmetic stays in the
// kernels of the other translation units.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <type_traits>
#include <vector>

#include "fdsc_internal.h"

namespace {

#define RT_TRY(expr)                                                                  \
    do {                                                                              \
        cudaError_t e_ = (expr);                                                      \
        if (e_ != cudaSuccess)                                                        \
            return fdsc_set_error(FDSC_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

int current_device() {
    int d = -1;
    cudaGetDevice(&d);
    return d;
}

// Device allocations freed together.
struct Arena {
    std::vector<void*> ptrs;
    int alloc(void** p, size_t bytes) {
        *p = nullptr;
        if (bytes == 0) bytes = 16;
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess)
            return fdsc_set_error(e == cudaErrorMemoryAllocation ? FDSC_ERR_OOM : FDSC_ERR_CUDA, "cudaMalloc(%zu): %s",
                                  bytes, cudaGetErrorString(e));
        ptrs.push_back(*p);
        return FDSC_OK;
    }
    void release() {
        for (void* p : ptrs) cudaFree(p);
        ptrs.clear();
    }
};

// Packing with as many blocks per slot set as fit: channels first.
void default_pack(const fdsc_params_info& I, const fdsc_layer& L, uint32_t* g_c, uint32_t* g_b) {
    const uint64_t HW = (uint64_t)L.H * L.W;
    *g_b = 1;
    if (HW > I.S) {
        *g_c = 1;
        return;
    }
    uint32_t g = (uint32_t)(I.S / HW);
    *g_c = std::max(1u, std::min(L.Ci, g));
}

// The fused online kernels take radix-8 plane lines (8 <= H, W <= 512);
// spectra spanning several ciphertexts (H W > S) included.
bool fused_ok(const DevLayer& D) { return D.logH >= 3 && D.logW >= 3 && D.logH <= 9 && D.logW <= 9; }

}  // namespace

// ====================================================================== plan
struct PlanLayer {
    fdsc_plan_layer spec;
    fdsc_layer L;
    DevLayer D;
    int variant = 0;
    bool fused = true;
    uint32_t candidates = 0;
    double tuned_us = 0;
    u64 *Phat = nullptr, *Mhat = nullptr, *ct = nullptr, *A = nullptr, *R = nullptr, *ct_out = nullptr;
    u64* Ptc = nullptr;  // the filter in the tensor-core layout (variant kTensorVariant only)
    u32 *sB = nullptr, *X = nullptr, *XB = nullptr, *SA = nullptr;
};

struct fdsc_plan {
    std::vector<PlanLayer> layers;
    Arena arena;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int device = -1;
};

namespace {

// HomConv variant number of the tensor-core kernel (homconv_tc.cu) in a plan.
constexpr int kTensorVariant = 7;
// Smallest server batch (images) whose HomConv runs on the tensor cores: from
// 4 images on, the tensor-core kernel is the faster one on the served shapes.
constexpr uint32_t kServerTensorMinImages = 4;

// The HomConv of a layer with its chosen variant.
cudaError_t plan_homconv(const DevParams& P, const PlanLayer& pl, const u64* A1, const u64* A2, cudaStream_t s) {
    if (pl.variant == kTensorVariant)
        return launch_homconv_tc(P, pl.D, pl.ct, A1, A2, pl.Ptc, pl.Mhat, pl.ct_out, s);
    return launch_homconv_v(P, pl.D, pl.ct, A1, A2, pl.Phat, pl.Mhat, pl.ct_out, pl.variant, s);
}

// Buffers of one layer for one packing (the filter plaintexts and masks
// depend on the packing).
int plan_alloc_layer(PlanLayer& pl, Arena& ar, fdsc_layout& lay) {
    const fdsc_params_info& I = pl.spec.params->info;
    int rc;
    if (pl.variant == kTensorVariant && (rc = ar.alloc((void**)&pl.Ptc, filter_tc_words(I.n, I.d, pl.D) * 8))) return rc;
    if ((rc = ar.alloc((void**)&pl.Phat, lay.filter_words * 8)) || (rc = ar.alloc((void**)&pl.Mhat, lay.mask_words * 8)) ||
        (rc = ar.alloc((void**)&pl.sB, lay.out_spectra_words * 4)) || (rc = ar.alloc((void**)&pl.ct, lay.ct_in_words * 8)) ||
        (rc = ar.alloc((void**)&pl.ct_out, lay.ct_out_words * 8)))
        return rc;
    if (pl.fused) {
        if ((rc = ar.alloc((void**)&pl.A, (u64)lay.n_in * I.n * 8)) || (rc = ar.alloc((void**)&pl.R, (u64)lay.n_in * I.n * 8)))
            return rc;
    } else {
        if ((rc = ar.alloc((void**)&pl.X, lay.in_spectra_words * 4)) || (rc = ar.alloc((void**)&pl.XB, lay.in_spectra_words * 4)) ||
            (rc = ar.alloc((void**)&pl.SA, lay.out_spectra_words * 4)))
            return rc;
    }
    return FDSC_OK;
}

int plan_setup_layer(PlanLayer& pl, cudaStream_t s) {
    const DevParams& P = pl.spec.params->dev;
    RT_TRY(launch_filter_prepare(P, pl.D, pl.spec.w, pl.spec.fh, pl.spec.fw, pl.Phat, s));
    if (pl.variant == kTensorVariant) RT_TRY(launch_filter_tc(P, pl.D, pl.Phat, pl.Ptc, s));
    RT_TRY(launch_mask_prepare(P, pl.D, pl.spec.mask_seed, nullptr, pl.spec.flood_bits, pl.Mhat, pl.sB, s));
    return FDSC_OK;
}

// The online path of one layer.  Streams st[0..3]; st[0] is the layer's main
// stream and ends joined with the others.
int plan_record_layer(PlanLayer& pl, cudaStream_t* st, cudaEvent_t* ev) {
    const DevParams& P = pl.spec.params->dev;
    const DevLayer& D = pl.D;
    const fdsc_plan_layer& sp = pl.spec;
    const u64 planes_out = (u64)D.B * D.Co;
    RT_TRY(cudaEventRecord(ev[0], st[0]));
    for (int k = 1; k < 4; k++) RT_TRY(cudaStreamWaitEvent(st[k], ev[0], 0));
    if (pl.fused) {
        RT_TRY(launch_constants(P, D, sp.t_hat, 0, sp.enc_seed, nullptr, pl.ct, st[0]));
        RT_TRY(launch_share(P, D, sp.xA, pl.A, false, st[1]));
        RT_TRY(launch_share(P, D, sp.xB, pl.R, false, st[2]));
        RT_TRY(launch_ntt2d(P, D.H, D.W, pl.sB, sp.yB, planes_out, true, st[3]));
        if (sp.pB) RT_TRY(launch_pool2x2(P, D.H, D.W, sp.yB, sp.pB, planes_out, st[3]));
        RT_TRY(cudaEventRecord(ev[1], st[1]));
        RT_TRY(cudaEventRecord(ev[2], st[2]));
        RT_TRY(cudaStreamWaitEvent(st[0], ev[1], 0));
        RT_TRY(cudaStreamWaitEvent(st[0], ev[2], 0));
        RT_TRY(plan_homconv(P, pl, pl.A, pl.R, st[0]));
        RT_TRY(launch_decrypt_share(P, D, sp.t_hat, 0, pl.ct_out, sp.yA, st[0]));
    } else {
        const u64 planes_in = (u64)D.B * D.Ci;
        RT_TRY(launch_ntt2d(P, D.H, D.W, sp.xA, pl.X, planes_in, false, st[0]));
        RT_TRY(launch_encrypt(P, D, sp.t_hat, pl.X, sp.enc_seed, pl.ct, st[0]));
        RT_TRY(launch_ntt2d(P, D.H, D.W, sp.xB, pl.XB, planes_in, false, st[1]));
        RT_TRY(launch_ntt2d(P, D.H, D.W, pl.sB, sp.yB, planes_out, true, st[3]));
        if (sp.pB) RT_TRY(launch_pool2x2(P, D.H, D.W, sp.yB, sp.pB, planes_out, st[3]));
        RT_TRY(cudaEventRecord(ev[1], st[1]));
        RT_TRY(cudaStreamWaitEvent(st[0], ev[1], 0));
        RT_TRY(launch_homrec(P, D, pl.XB, pl.ct, st[0]));
        RT_TRY(plan_homconv(P, pl, nullptr, nullptr, st[0]));
        RT_TRY(launch_decrypt(P, D, sp.t_hat, pl.ct_out, pl.SA, st[0]));
        RT_TRY(launch_ntt2d(P, D.H, D.W, pl.SA, sp.yA, planes_out, true, st[0]));
    }
    if (sp.pA) RT_TRY(launch_pool2x2(P, D.H, D.W, sp.yA, sp.pA, planes_out, st[0]));
    RT_TRY(cudaEventRecord(ev[3], st[3]));
    RT_TRY(cudaStreamWaitEvent(st[0], ev[3], 0));
    return FDSC_OK;
}

// Times one candidate packing / variant of a layer: setup, two warm runs,
// then the median of five.
int plan_time_candidate(PlanLayer& pl, cudaStream_t* st, cudaEvent_t* ev, double* us) {
    fdsc_layout lay;
    int rc = fdsc_make_layer(pl.spec.params->info, &pl.L, &pl.D, &lay);
    if (rc) return rc;
    Arena ar;
    if ((rc = plan_alloc_layer(pl, ar, lay)) || (rc = plan_setup_layer(pl, st[0]))) {
        ar.release();
        return rc;
    }
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    std::vector<float> ms;
    for (int it = 0; it < 7 && rc == FDSC_OK; it++) {
        cudaEventRecord(t0, st[0]);
        rc = plan_record_layer(pl, st, ev);
        cudaEventRecord(t1, st[0]);
        if (cudaEventSynchronize(t1) != cudaSuccess) rc = fdsc_set_error(FDSC_ERR_CUDA, "tuning run failed");
        float m = 0;
        cudaEventElapsedTime(&m, t0, t1);
        if (it >= 2) ms.push_back(m);
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    ar.release();
    if (rc) return rc;
    std::sort(ms.begin(), ms.end());
    *us = ms[ms.size() / 2] * 1e3;
    return FDSC_OK;
}

void plan_free(fdsc_plan* p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (auto s : p->streams)
        if (s) cudaStreamDestroy(s);  // never the default stream
    for (auto e : p->events)
        if (e) cudaEventDestroy(e);
    p->arena.release();
    delete p;
}

}  // namespace

extern "C" int fdsc_plan_create(const fdsc_plan_layer* layers, uint32_t count, uint32_t flags, void* stream,
                                fdsc_plan** out) {
    if (!out || !layers || count == 0) return fdsc_set_error(FDSC_ERR_ARG, "plan needs layers and an output pointer");
    *out = nullptr;
    fdsc_plan* plan = new (std::nothrow) fdsc_plan();
    if (!plan) return fdsc_set_error(FDSC_ERR_OOM, "host allocation failed");
    plan->device = current_device();
    int rc = FDSC_OK;
    auto fail = [&](int code) {
        plan_free(plan);
        return code;
    };
    plan->streams.resize(4 * (size_t)count);
    plan->events.resize(4 * (size_t)count);
    for (auto& s : plan->streams)
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
            return fail(fdsc_set_error(FDSC_ERR_CUDA, "stream creation failed"));
    for (auto& e : plan->events)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return fail(fdsc_set_error(FDSC_ERR_CUDA, "event creation failed"));
    (void)stream;  // setup and tuning run on the plan's own streams and finish before return
    // the plan's streams do not order against the caller's: let pending work
    // on the inputs (keys, weights, shares) finish first
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(fdsc_set_error(FDSC_ERR_CUDA, "device not ready"));

    plan->layers.resize(count);
    for (uint32_t i = 0; i < count; i++) {
        PlanLayer& pl = plan->layers[i];
        pl.spec = layers[i];
        const fdsc_plan_layer& sp = layers[i];
        if (!sp.params || sp.params->device != plan->device)
            return fail(fdsc_set_error(FDSC_ERR_ARG, "layer %u: params missing or on another device", i));
        if (!sp.w || !sp.t_hat || !sp.xA || !sp.xB || !sp.yA || !sp.yB)
            return fail(fdsc_set_error(FDSC_ERR_ARG, "layer %u: NULL buffer", i));
        if (((uintptr_t)sp.t_hat | (uintptr_t)sp.xA | (uintptr_t)sp.xB | (uintptr_t)sp.yA | (uintptr_t)sp.yB |
             (uintptr_t)sp.pA | (uintptr_t)sp.pB) & 15)
            return fail(fdsc_set_error(FDSC_ERR_ARG, "layer %u: buffers must be 16-byte aligned", i));
        if ((sp.pA || sp.pB) && ((sp.layer.H & 1) || (sp.layer.W & 1)))
            return fail(fdsc_set_error(FDSC_ERR_ARG, "layer %u: pooling needs even H and W", i));
        const fdsc_params_info& I = sp.params->info;
        pl.L = sp.layer;
        if (pl.L.g_c == 0 || pl.L.g_b == 0) default_pack(I, pl.L, &pl.L.g_c, &pl.L.g_b);
        fdsc_layout lay;
        if ((rc = fdsc_make_layer(I, &pl.L, &pl.D, &lay))) return fail(rc);
        if (sp.fh == 0 || sp.fw == 0 || sp.fh > pl.D.H || sp.fw > pl.D.W)
            return fail(fdsc_set_error(FDSC_ERR_ARG, "layer %u: filter does not fit the plane", i));
        pl.fused = fused_ok(pl.D);
        pl.variant = homconv_default_variant(pl.D);
        if ((flags & FDSC_PLAN_TENSOR) && homconv_tc_supported(I.n, pl.D)) pl.variant = kTensorVariant;
        cudaStream_t* st = &plan->streams[4 * (size_t)i];
        cudaEvent_t* ev = &plan->events[4 * (size_t)i];
        if ((flags & FDSC_PLAN_TUNE) && pl.fused) {
            // candidates: every split of the slot set's blocks between channels and images
            std::vector<std::pair<uint32_t, uint32_t>> packs;
            const uint32_t blocks = I.S / pl.D.HW;
            for (uint32_t gb = 1; gb <= blocks; gb *= 2) {
                const uint32_t gc = blocks / gb;
                if (gc > sp.layer.Ci * 2 || gb > sp.layer.B) continue;
                packs.push_back({std::min(gc, sp.layer.Ci), gb});
            }
            if (packs.empty()) packs.push_back({pl.L.g_c, pl.L.g_b});
            const int variants[] = {4, 10, 12, kTensorVariant};
            double best = 1e30;
            fdsc_layer bestL = pl.L;
            int bestV = pl.variant;
            for (auto pk : packs) {
                for (int v : variants) {
                    PlanLayer cand = pl;
                    cand.L.g_c = pk.first;
                    cand.L.g_b = pk.second;
                    cand.variant = v;
                    DevLayer Dt;
                    if (fdsc_make_layer(I, &cand.L, &Dt, nullptr) != FDSC_OK || Dt.T > sp.params->max_T ||
                        !fdsc_noise_ok_flood(I, Dt.T, sp.flood_bits))
                        continue;
                    if (v == kTensorVariant && !homconv_tc_supported(I.n, Dt)) continue;
                    // a variant that falls back to another one for this shape is not timed twice
                    if (v != kTensorVariant && homconv_effective_variant(Dt, v) != v) continue;
                    double us = 0;
                    if ((rc = plan_time_candidate(cand, st, ev, &us))) return fail(rc);
                    pl.candidates++;
                    if (us < best) {
                        best = us;
                        bestL = cand.L;
                        bestV = v;
                    }
                }
            }
            pl.L = bestL;
            pl.variant = bestV;
            pl.tuned_us = best;
            if ((rc = fdsc_make_layer(I, &pl.L, &pl.D, &lay))) return fail(rc);
        }
        if (pl.D.T > sp.params->max_T)
            return fail(fdsc_set_error(FDSC_ERR_NOISE, "layer %u: T = %u exceeds the params' max_T", i, pl.D.T));
        if (sp.flood_bits > FDSC_MAX_FLOOD_BITS || !fdsc_noise_ok_flood(I, pl.D.T, sp.flood_bits))
            return fail(fdsc_set_error(FDSC_ERR_NOISE, "layer %u: flooding of 2^%u breaks the noise bound", i,
                                       sp.flood_bits));
        if ((rc = plan_alloc_layer(pl, plan->arena, lay)) || (rc = plan_setup_layer(pl, st[0]))) return fail(rc);
    }
    // one eager run of every layer before recording: validates the launches and
    // lets every kernel set its shared-memory attributes outside the capture
    for (uint32_t i = 0; i < count; i++)
        if ((rc = plan_record_layer(plan->layers[i], &plan->streams[4 * (size_t)i], &plan->events[4 * (size_t)i])))
            return fail(rc);
    for (auto s : plan->streams)
        if (cudaStreamSynchronize(s) != cudaSuccess) return fail(fdsc_set_error(FDSC_ERR_CUDA, "plan setup failed"));

    // record: every layer forks from the capture stream and joins back
    cudaStream_t cap = plan->streams[0];
    cudaEvent_t fork;
    if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess)
        return fail(fdsc_set_error(FDSC_ERR_CUDA, "event creation failed"));
    plan->events.push_back(fork);
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return fail(fdsc_set_error(FDSC_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e)));
    cudaEventRecord(fork, cap);
    const bool chain = (flags & FDSC_PLAN_CHAIN) != 0;
    for (uint32_t i = 0; i < count && rc == FDSC_OK; i++) {
        cudaStream_t* st = &plan->streams[4 * (size_t)i];
        if (i > 0 && chain) {  // after the previous layer, whose main stream has joined its others
            cudaEvent_t prev;
            if (cudaEventCreateWithFlags(&prev, cudaEventDisableTiming) != cudaSuccess) {
                rc = fdsc_set_error(FDSC_ERR_CUDA, "event creation failed");
                break;
            }
            plan->events.push_back(prev);
            cudaEventRecord(prev, plan->streams[4 * (size_t)(i - 1)]);
            cudaStreamWaitEvent(st[0], prev, 0);
        } else if (i > 0) {
            cudaStreamWaitEvent(st[0], fork, 0);
        }
        rc = plan_record_layer(plan->layers[i], st, &plan->events[4 * (size_t)i]);
    }
    for (uint32_t i = 1; i < count && rc == FDSC_OK; i++) {
        cudaEvent_t done = plan->events[4 * (size_t)i + 3];
        cudaEventRecord(done, plan->streams[4 * (size_t)i]);
        cudaStreamWaitEvent(cap, done, 0);
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cap, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return fail(rc);
    }
    if (e != cudaSuccess) return fail(fdsc_set_error(FDSC_ERR_CUDA, "end capture: %s", cudaGetErrorString(e)));
    plan->graph = g;
    e = cudaGraphInstantiate(&plan->exec, g, 0);
    if (e != cudaSuccess) return fail(fdsc_set_error(FDSC_ERR_CUDA, "instantiate: %s", cudaGetErrorString(e)));
    *out = plan;
    return FDSC_OK;
}

extern "C" int fdsc_plan_launch(fdsc_plan* plan, void* stream) {
    if (!plan || !plan->exec) return fdsc_set_error(FDSC_ERR_ARG, "plan is NULL");
    if (current_device() != plan->device) return fdsc_set_error(FDSC_ERR_ARG, "plan belongs to another device");
    cudaError_t e = cudaGraphLaunch(plan->exec, (cudaStream_t)stream);
    return e == cudaSuccess ? FDSC_OK : fdsc_set_error(FDSC_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
}

extern "C" int fdsc_plan_layer_info_get(const fdsc_plan* plan, uint32_t i, fdsc_plan_layer_info* out) {
    if (!plan || !out || i >= plan->layers.size()) return fdsc_set_error(FDSC_ERR_ARG, "bad plan / layer index");
    const PlanLayer& pl = plan->layers[i];
    out->g_c = pl.L.g_c;
    out->g_b = pl.L.g_b;
    out->homconv_variant = (uint32_t)pl.variant;
    out->fused = pl.fused ? 1 : 0;
    out->candidates = pl.candidates;
    out->pad0 = 0;
    out->tuned_step_us = pl.tuned_us;
    return FDSC_OK;
}

extern "C" int fdsc_plan_destroy(fdsc_plan* plan) {
    if (plan) {
        for (auto s : plan->streams) cudaStreamSynchronize(s);
        plan_free(plan);
    }
    return FDSC_OK;
}

// ====================================================================== server
namespace {

using Clock = std::chrono::steady_clock;

struct ServerType {
    const fdsc_params* P;
    fdsc_layer L;  // B = 1
    DevLayer D1;
    fdsc_layout lay1;
    u64* Phat = nullptr;
    u64* Ptc = nullptr;  // the filter in the tensor-core layout (when the layer admits that kernel)
    const uint64_t* keys;
    uint32_t nkeys;
    uint64_t bytes_per_request;
    int variant;
};

// Host copies of one batch (request inputs into the lane's pinned staging,
// results out to the callers' buffers), split into chunks and shared by a
// few persistent threads and the calling (worker) thread.  run() returns when
// every chunk is copied and every pool thread has left the generation, so the
// chunk list can be refilled.
class CopyPool {
  public:
    struct Job {
        void* dst;
        const void* src;
        size_t bytes;
    };
    explicit CopyPool(unsigned threads) {
        for (unsigned i = 0; i < threads; i++) th_.emplace_back([this] { loop(); });
    }
    ~CopyPool() {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (auto& t : th_) t.join();
    }
    void run(const std::vector<Job>& jobs) {
        size_t total = 0;
        for (const Job& j : jobs) total += j.bytes;
        if (total <= kInline) {  // small batches: waking the pool costs more than it saves
            for (const Job& j : jobs) memcpy(j.dst, j.src, j.bytes);
            return;
        }
        chunks_.clear();
        for (const Job& j : jobs)
            for (size_t off = 0; off < j.bytes; off += kChunk)
                chunks_.push_back({static_cast<char*>(j.dst) + off, static_cast<const char*>(j.src) + off,
                                   std::min(kChunk, j.bytes - off)});
        if (chunks_.empty()) return;
        {
            std::lock_guard<std::mutex> lk(mu_);
            next_.store(0);
            left_ = th_.size();
            gen_++;
        }
        cv_.notify_all();
        work();
        std::unique_lock<std::mutex> lk(mu_);
        cv_done_.wait(lk, [&] { return left_ == 0; });
    }

  private:
    static constexpr size_t kChunk = 64 << 10, kInline = 64 << 10;
    void work() {
        for (size_t i = next_.fetch_add(1); i < chunks_.size(); i = next_.fetch_add(1))
            memcpy(chunks_[i].dst, chunks_[i].src, chunks_[i].bytes);
    }
    void loop() {
        uint64_t seen = 0;
        for (;;) {
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
                if (stop_) return;
                seen = gen_;
            }
            work();
            std::lock_guard<std::mutex> lk(mu_);
            if (--left_ == 0) cv_done_.notify_all();
        }
    }
    std::vector<std::thread> th_;
    std::vector<Job> chunks_;
    std::atomic<size_t> next_{0};
    std::mutex mu_;
    std::condition_variable cv_, cv_done_;
    uint64_t gen_ = 0;
    size_t left_ = 0;
    bool stop_ = false;
};

struct Req {
    fdsc_request r;
    uint64_t ticket;
    Clock::time_point t_submit;
};

// Request latencies in a fixed histogram: 4096 bins spaced evenly in log
// between 1 us and 100 s (each bin 0.45 % wide), so the server's memory does
// not grow with the number of requests and a percentile costs one pass over
// the bins.  A percentile reports its bin's geometric centre.
struct LatencyHist {
    static constexpr int kBins = 4096;
    static constexpr double kLo = 1.0, kHi = 1e8;
    uint64_t count[kBins] = {};
    uint64_t n = 0;
    double sum = 0, max = 0;
    void add(double us) {
        const double t = std::log(std::max(us, kLo) / kLo) / std::log(kHi / kLo);
        const int b = std::min(kBins - 1, std::max(0, (int)(t * kBins)));
        count[b]++;
        n++;
        sum += us;
        max = std::max(max, us);
    }
    double pct(double q) const {
        if (!n) return 0.0;
        const uint64_t rank = std::min<uint64_t>(n - 1, (uint64_t)(q * (double)(n - 1) + 0.5));
        uint64_t seen = 0;
        for (int b = 0; b < kBins; b++) {
            seen += count[b];
            if (seen > rank) return kLo * std::pow(kHi / kLo, (b + 0.5) / kBins);
        }
        return max;
    }
};

struct Lane {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    // the batch's independent producers run beside the lane's stream: Bob's
    // mask and output share, Alice's encryption constants, Bob's HomRec
    // plaintext; events join them before HomConv and at the batch's end
    cudaStream_t side[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t ev_seed = nullptr, ev_mask = nullptr, ev_yB = nullptr, ev_ct = nullptr, ev_R = nullptr;
    // the recorded batches: [type][G - 1], and which run HomConv on the tensor cores
    std::vector<cudaGraphExec_t> graphs;
    std::vector<char> graph_tensor;
    bool busy = false;
    std::vector<Req> batch;
    uint32_t type = 0;
    uint64_t bytes = 0;
    // device buffers sized for max_batch of the largest type
    u32 *xA = nullptr, *xB = nullptr, *yA = nullptr, *yB = nullptr, *sB = nullptr;
    u64 *ct = nullptr, *A = nullptr, *R = nullptr, *ct_out = nullptr, *M = nullptr, *keys = nullptr, *seeds = nullptr;
    // pinned staging
    u32 *h_xA = nullptr, *h_xB = nullptr, *h_yA = nullptr, *h_yB = nullptr;
    u64* h_seeds = nullptr;
};

}  // namespace

struct fdsc_server {
    fdsc_server_config cfg;
    int device = -1;
    std::vector<ServerType> types;
    std::vector<Lane> lanes;
    Arena arena;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req> pending;
    std::map<uint64_t, double> done;  // ticket -> latency (us); -1 = failed
    LatencyHist latencies;
    uint32_t lane_cap = 0;            // requests a lane's buffers hold (<= max_batch, from the budget)
    uint64_t reserved = 0;            // device bytes of the lanes' request buffers
    uint64_t next_ticket = 1, submitted = 0, completed = 0, batches = 0, batched_requests = 0;
    std::atomic<uint64_t> tensor_batches{0};  // batches whose HomConv ran on the tensor cores
    uint64_t inflight = 0, peak_inflight = 0;
    int error = FDSC_OK;
    bool started = false, stop = false;
    std::thread worker;
    std::unique_ptr<CopyPool> copies;
    // largest per-request sizes over the types (elements)
    uint64_t max_in = 0, max_out = 0, max_ct_in = 0, max_add = 0, max_ct_out = 0, max_mask = 0, max_n = 0;
};

namespace {

uint64_t request_bytes(const ServerType& t) {
    const fdsc_layout& l = t.lay1;
    const uint64_t n = t.P->info.n;
    return 8 * (l.ct_in_words + 2ull * l.n_in * n + l.ct_out_words + l.mask_words + n + 2) +
           4 * (2 * l.in_spectra_words + 3 * l.out_spectra_words);
}

// Each request's client key, gathered from its type's key pool:
// keys[b][i] = pool[idx[b]][i] (idx[b] < pool size, checked at submission).
__global__ void __launch_bounds__(256) gather_keys_kernel(const u64* __restrict__ pool, const u64* __restrict__ idx,
                                                          u32 G, u32 n, u64* __restrict__ keys) {
    const u64 total = (u64)G * n;
    for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (u64)gridDim.x * blockDim.x)
        keys[e] = pool[idx[e / n] * n + e % n];
}

// Enqueues the GPU work of a batch of G requests of type `type` on a lane,
// reading the lane's pinned staging: h_seeds = [encryption seeds][mask
// seeds][key indices] (G each), h_xA / h_xB the requests' shares; the
// results land in h_yA / h_yB.  Recorded once per (type, G) into a graph.
int record_batch(const fdsc_server* S, Lane& ln, uint32_t type, uint32_t G, bool* tensor) {
    const ServerType& t = S->types[type];
    const DevParams& P = t.P->dev;
    fdsc_layer LG = t.L;
    LG.B = G;
    LG.g_b = 1;
    DevLayer D;
    int rc = fdsc_make_layer(t.P->info, &LG, &D, nullptr);
    if (rc) return rc;
    const uint64_t in_img = t.lay1.in_spectra_words, out_img = t.lay1.out_spectra_words, n = t.P->info.n;
    cudaStream_t s = ln.stream, s_mask = ln.side[0], s_ct = ln.side[1], s_rec = ln.side[2];
    // seeds and keys first: the producers that need no share start on them
    RT_TRY(cudaMemcpyAsync(ln.seeds, ln.h_seeds, 3 * G * 8, cudaMemcpyHostToDevice, s));
    const u64 kb = ((u64)G * n + 255) / 256;
    gather_keys_kernel<<<(u32)(kb < 608 ? kb : 608), 256, 0, s>>>(t.keys, ln.seeds + 2 * G, G, (u32)n, ln.keys);
    RT_TRY(cudaGetLastError());
    RT_TRY(cudaEventRecord(ln.ev_seed, s));
    // Bob: HomShare mask, then his output share (INTT2D of s_B) and its copy out
    RT_TRY(cudaStreamWaitEvent(s_mask, ln.ev_seed, 0));
    RT_TRY(launch_mask_prepare(P, D, 0, ln.seeds + G, 0, ln.M, ln.sB, s_mask));
    RT_TRY(cudaEventRecord(ln.ev_mask, s_mask));
    RT_TRY(launch_ntt2d(P, D.H, D.W, ln.sB, ln.yB, (u64)G * D.Co, true, s_mask));
    RT_TRY(cudaMemcpyAsync(ln.h_yB, ln.yB, G * out_img * 4, cudaMemcpyDeviceToHost, s_mask));
    RT_TRY(cudaEventRecord(ln.ev_yB, s_mask));
    // Alice: encryption constants (Enc(0) of every input ciphertext)
    RT_TRY(cudaStreamWaitEvent(s_ct, ln.ev_seed, 0));
    RT_TRY(launch_constants(P, D, ln.keys, n, 0, ln.seeds, ln.ct, s_ct));
    RT_TRY(cudaEventRecord(ln.ev_ct, s_ct));
    // Bob: HomRec plaintext from his share
    RT_TRY(cudaStreamWaitEvent(s_rec, ln.ev_seed, 0));
    RT_TRY(cudaMemcpyAsync(ln.xB, ln.h_xB, G * in_img * 4, cudaMemcpyHostToDevice, s_rec));
    RT_TRY(launch_share(P, D, ln.xB, ln.R, false, s_rec));
    RT_TRY(cudaEventRecord(ln.ev_R, s_rec));
    // Alice's message on the lane's stream, then HomConv once all addends exist
    RT_TRY(cudaMemcpyAsync(ln.xA, ln.h_xA, G * in_img * 4, cudaMemcpyHostToDevice, s));
    RT_TRY(launch_share(P, D, ln.xA, ln.A, false, s));
    RT_TRY(cudaStreamWaitEvent(s, ln.ev_ct, 0));
    RT_TRY(cudaStreamWaitEvent(s, ln.ev_R, 0));
    RT_TRY(cudaStreamWaitEvent(s, ln.ev_mask, 0));
    *tensor = t.Ptc && D.GB >= kServerTensorMinImages;
    if (*tensor)
        RT_TRY(launch_homconv_tc(P, D, ln.ct, ln.A, ln.R, t.Ptc, ln.M, ln.ct_out, s));
    else
        RT_TRY(launch_homconv_v(P, D, ln.ct, ln.A, ln.R, t.Phat, ln.M, ln.ct_out, t.variant, s));
    RT_TRY(launch_decrypt_share(P, D, ln.keys, n, ln.ct_out, ln.yA, s));
    RT_TRY(cudaMemcpyAsync(ln.h_yA, ln.yA, G * out_img * 4, cudaMemcpyDeviceToHost, s));
    // the batch is done when both output shares are on the host
    RT_TRY(cudaStreamWaitEvent(s, ln.ev_yB, 0));
    return FDSC_OK;
}

// Records every (type, batch size) a lane can run into a graph, after one
// direct run per type at the smallest and largest batch (zero inputs) so
// that every kernel's attributes are set outside the capture.
int record_lane_graphs(fdsc_server* S, Lane& ln) {
    const uint32_t B = S->lane_cap;
    memset(ln.h_xA, 0, B * S->max_in * 4);
    memset(ln.h_xB, 0, B * S->max_in * 4);
    memset(ln.h_seeds, 0, 3 * (size_t)B * 8);
    bool tensor = false;
    for (uint32_t type = 0; type < S->types.size(); type++)
        for (uint32_t G : {1u, B}) {
            int rc = record_batch(S, ln, type, G, &tensor);
            if (rc) return rc;
        }
    for (cudaStream_t st : ln.side) RT_TRY(cudaStreamSynchronize(st));
    RT_TRY(cudaStreamSynchronize(ln.stream));
    ln.graphs.assign(S->types.size() * (size_t)B, nullptr);
    ln.graph_tensor.assign(ln.graphs.size(), 0);
    for (uint32_t type = 0; type < S->types.size(); type++)
        for (uint32_t G = 1; G <= B; G++) {
            RT_TRY(cudaStreamBeginCapture(ln.stream, cudaStreamCaptureModeThreadLocal));
            int rc = record_batch(S, ln, type, G, &tensor);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(ln.stream, &g);
            if (rc || e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return rc ? rc : fdsc_set_error(FDSC_ERR_CUDA, "server capture: %s", cudaGetErrorString(e));
            }
            const size_t k = (size_t)type * B + (G - 1);
            e = cudaGraphInstantiate(&ln.graphs[k], g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return fdsc_set_error(FDSC_ERR_CUDA, "server instantiate: %s", cudaGetErrorString(e));
            ln.graph_tensor[k] = tensor;
        }
    return FDSC_OK;
}

// Launches one batch on a lane (worker thread, lock NOT held): the requests'
// shares into pinned staging, then the batch's graph.
int launch_batch(fdsc_server* S, Lane& ln) {
    const ServerType& t = S->types[ln.type];
    const uint32_t G = (uint32_t)ln.batch.size();
    const uint64_t in_img = t.lay1.in_spectra_words;
    std::vector<CopyPool::Job> jobs;
    for (uint32_t b = 0; b < G; b++) {
        const fdsc_request& r = ln.batch[b].r;
        jobs.push_back({ln.h_xA + b * in_img, r.xA, in_img * 4});
        jobs.push_back({ln.h_xB + b * in_img, r.xB, in_img * 4});
        ln.h_seeds[b] = r.enc_seed;
        ln.h_seeds[G + b] = r.mask_seed;
        ln.h_seeds[2 * G + b] = r.key;
    }
    S->copies->run(jobs);
    const size_t k = (size_t)ln.type * S->lane_cap + (G - 1);
    RT_TRY(cudaGraphLaunch(ln.graphs[k], ln.stream));
    RT_TRY(cudaEventRecord(ln.done, ln.stream));
    if (ln.graph_tensor[k]) S->tensor_batches++;
    return FDSC_OK;
}

void finish_batch(fdsc_server* S, Lane& ln, bool ok) {
    const ServerType& t = S->types[ln.type];
    const uint64_t out_img = t.lay1.out_spectra_words;
    if (ok) {
        std::vector<CopyPool::Job> jobs;
        for (size_t b = 0; b < ln.batch.size(); b++) {
            const fdsc_request& r = ln.batch[b].r;
            jobs.push_back({r.yA, ln.h_yA + b * out_img, out_img * 4});
            jobs.push_back({r.yB, ln.h_yB + b * out_img, out_img * 4});
        }
        S->copies->run(jobs);
    }
    const auto now = Clock::now();
    std::lock_guard<std::mutex> lk(S->mu);
    for (auto& q : ln.batch) {
        const double us = std::chrono::duration<double, std::micro>(now - q.t_submit).count();
        S->done[q.ticket] = ok ? us : -1.0;
        if (ok) S->latencies.add(us);
        S->completed++;
    }
    S->inflight -= ln.bytes;
    ln.batch.clear();
    ln.busy = false;
    S->cv_done.notify_all();
}

// After its last batch retires the worker keeps polling for this long before it
// blocks: a wake-up through the condition variable costs tens of microseconds,
// a large part of a small request's latency (served p50 131 against 143 us).
constexpr auto kIdleSpin = std::chrono::microseconds(2000);

void worker_loop(fdsc_server* S) {
    cudaSetDevice(S->device);
    auto last_active = Clock::now();
    for (;;) {
        bool any_busy = false;
        // 1. retire finished batches
        for (auto& ln : S->lanes) {
            if (!ln.busy) continue;
            cudaError_t q = cudaEventQuery(ln.done);
            if (q == cudaErrorNotReady) {
                any_busy = true;
                continue;
            }
            if (q != cudaSuccess) {
                std::lock_guard<std::mutex> lk(S->mu);
                S->error = fdsc_set_error(FDSC_ERR_CUDA, "batch failed: %s", cudaGetErrorString(q));
            }
            finish_batch(S, ln, q == cudaSuccess);
        }
        // 2. admit: the oldest pending request picks the type; take more of that
        //    type in arrival order while the batch and the HBM budget allow
        std::unique_lock<std::mutex> lk(S->mu);
        if (S->stop && !any_busy && (S->pending.empty() || S->error)) {
            for (auto& q : S->pending) {  // never launched: report them failed
                S->done[q.ticket] = -1.0;
                S->completed++;
            }
            S->pending.clear();
            S->cv_done.notify_all();
            break;
        }
        for (auto& ln : S->lanes) {
            if (ln.busy || S->pending.empty() || S->error) continue;
            const uint32_t type = S->pending.front().r.type;
            const uint64_t per = S->types[type].bytes_per_request;
            std::vector<Req> batch;
            uint64_t bytes = 0;
            for (auto it = S->pending.begin(); it != S->pending.end() && batch.size() < S->lane_cap;) {
                if (it->r.type != type) {
                    ++it;
                    continue;
                }
                if (S->inflight + bytes + per > S->cfg.hbm_budget_bytes) break;
                batch.push_back(*it);
                bytes += per;
                it = S->pending.erase(it);
            }
            if (batch.empty()) break;  // budget full: wait for a batch to retire
            ln.batch = std::move(batch);
            ln.type = type;
            ln.bytes = bytes;
            ln.busy = true;
            S->inflight += bytes;
            S->peak_inflight = std::max(S->peak_inflight, S->inflight);
            S->batches++;
            S->batched_requests += ln.batch.size();
            lk.unlock();
            int rc = launch_batch(S, ln);
            lk.lock();
            if (rc) {
                S->error = rc;
                lk.unlock();
                for (cudaStream_t st : ln.side)
                    if (st) cudaStreamSynchronize(st);
                cudaStreamSynchronize(ln.stream);
                finish_batch(S, ln, false);
                lk.lock();
            }
            any_busy = true;
        }
        if (!any_busy && S->pending.empty() && !S->stop) {
            if (Clock::now() - last_active < kIdleSpin) {
                lk.unlock();
                std::this_thread::yield();
            } else {
                S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
            }
            continue;
        }
        last_active = Clock::now();
        lk.unlock();
        // batches in flight: poll again at once (a timed sleep would add tens of
        // microseconds to every request's latency); only yield the core
        std::this_thread::yield();
    }
}

}  // namespace

// Device bytes of a lane's request buffers for B requests of the largest type
// (each buffer 256-byte aligned inside the lane's block).
static uint64_t lane_bytes(const fdsc_server* S, uint64_t B) {
    auto al = [](uint64_t b) { return (b + 255) & ~(uint64_t)255; };
    return 2 * al(B * S->max_in * 4) + 3 * al(B * S->max_out * 4) + al(B * S->max_ct_in * 8) +
           2 * al(B * S->max_add * 8) + al(B * S->max_ct_out * 8) + al(B * S->max_mask * 8) + al(B * S->max_n * 8) +
           al(3 * B * 8);
}

extern "C" int fdsc_server_create(const fdsc_server_config* cfg, fdsc_server** out) {
    if (!cfg || !out || cfg->max_batch == 0 || cfg->lanes == 0)
        return fdsc_set_error(FDSC_ERR_ARG, "server config needs max_batch >= 1 and lanes >= 1");
    fdsc_server* S = new (std::nothrow) fdsc_server();
    if (!S) return fdsc_set_error(FDSC_ERR_OOM, "host allocation failed");
    S->cfg = *cfg;
    S->device = current_device();
    *out = S;
    return FDSC_OK;
}

extern "C" int fdsc_server_add_type(fdsc_server* S, const fdsc_params* P, const fdsc_layer* L, const int8_t* w,
                                    uint32_t fh, uint32_t fw, const uint64_t* keys, uint32_t nkeys, uint32_t* type_id) {
    if (!S || !P || !L || !w || !keys || nkeys == 0 || !type_id) return fdsc_set_error(FDSC_ERR_ARG, "NULL argument");
    if (S->started) return fdsc_set_error(FDSC_ERR_ARG, "types must be added before fdsc_server_start");
    if (P->device != S->device) return fdsc_set_error(FDSC_ERR_ARG, "params on another device");
    ServerType t;
    t.P = P;
    t.L = *L;
    t.L.B = 1;
    t.L.g_b = 1;
    if (t.L.g_c == 0) default_pack(P->info, t.L, &t.L.g_c, &t.L.g_b);
    int rc = fdsc_make_layer(P->info, &t.L, &t.D1, &t.lay1);
    if (rc) return rc;
    if (!fused_ok(t.D1) || t.D1.beta != 1)
        return fdsc_set_error(FDSC_ERR_UNSUPPORTED, "served layers need H W <= S and 8 <= H, W <= 512");
    // a batch packs one request per image group; with d > 1 slot sets the d
    // images of a group would share one ciphertext, and so one client key
    if (P->info.d != 1)
        return fdsc_set_error(FDSC_ERR_UNSUPPORTED, "served layers need one slot set per ciphertext (d = 1)");
    if (t.D1.T > P->max_T) return fdsc_set_error(FDSC_ERR_NOISE, "T = %u exceeds the params' max_T", t.D1.T);
    if (fh == 0 || fw == 0 || fh > t.D1.H || fw > t.D1.W) return fdsc_set_error(FDSC_ERR_ARG, "filter does not fit");
    t.keys = keys;
    t.nkeys = nkeys;
    t.variant = homconv_default_variant(t.D1);
    t.bytes_per_request = request_bytes(t);
    if ((rc = S->arena.alloc((void**)&t.Phat, t.lay1.filter_words * 8))) return rc;
    // batches of at least kServerTensorMinImages requests run HomConv on the tensor
    // cores when the layer admits it at the largest batch
    fdsc_layer Lmax = t.L;
    Lmax.B = std::max<uint32_t>(S->cfg.max_batch, 1);
    DevLayer Dmax;
    const bool tensor = S->cfg.max_batch >= kServerTensorMinImages &&
                        fdsc_make_layer(P->info, &Lmax, &Dmax, nullptr) == FDSC_OK &&
                        homconv_tc_supported(P->info.n, Dmax);
    if (tensor && (rc = S->arena.alloc((void**)&t.Ptc, filter_tc_words(P->info.n, P->info.d, t.D1) * 8))) return rc;
    cudaError_t e = launch_filter_prepare(P->dev, t.D1, w, fh, fw, t.Phat, 0);
    if (e == cudaSuccess && tensor) e = launch_filter_tc(P->dev, t.D1, t.Phat, t.Ptc, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fdsc_set_error(FDSC_ERR_CUDA, "filter_prepare: %s", cudaGetErrorString(e));
    const uint64_t n = P->info.n;
    S->max_in = std::max<uint64_t>(S->max_in, t.lay1.in_spectra_words);
    S->max_out = std::max<uint64_t>(S->max_out, t.lay1.out_spectra_words);
    S->max_ct_in = std::max<uint64_t>(S->max_ct_in, t.lay1.ct_in_words);
    S->max_add = std::max<uint64_t>(S->max_add, (uint64_t)t.lay1.n_in * n);
    S->max_ct_out = std::max<uint64_t>(S->max_ct_out, t.lay1.ct_out_words);
    S->max_mask = std::max<uint64_t>(S->max_mask, t.lay1.mask_words);
    S->max_n = std::max<uint64_t>(S->max_n, n);
    *type_id = (uint32_t)S->types.size();
    S->types.push_back(t);
    return FDSC_OK;
}

extern "C" int fdsc_server_start(fdsc_server* S) {
    if (!S || S->types.empty()) return fdsc_set_error(FDSC_ERR_ARG, "server needs at least one type");
    if (S->started) return FDSC_OK;
    // The lanes' request buffers are what requests in flight occupy, so the
    // budget sizes them: every lane holds the same number of requests of the
    // largest type, as many as max_batch and the budget's share allow; when
    // not even one fits per lane, fewer lanes are made (FDSC_ERR_BUDGET if
    // not one request fits at all).  One device block per lane.
    const uint64_t per = lane_bytes(S, 1);
    uint64_t nl = S->cfg.lanes, cap = std::min<uint64_t>(S->cfg.max_batch, S->cfg.hbm_budget_bytes / (nl * per));
    if (cap == 0) {
        nl = std::min<uint64_t>(nl, S->cfg.hbm_budget_bytes / per);
        cap = 1;
    }
    if (nl == 0)
        return fdsc_set_error(FDSC_ERR_BUDGET, "the budget of %llu bytes holds no request (%llu bytes each)",
                              (unsigned long long)S->cfg.hbm_budget_bytes, (unsigned long long)per);
    S->lane_cap = (uint32_t)cap;
    const uint64_t B = cap;
    S->lanes.resize(nl);
    for (auto& ln : S->lanes) {
        int rc;
        unsigned char* blk = nullptr;
        const uint64_t bytes = lane_bytes(S, B);
        if ((rc = S->arena.alloc((void**)&blk, bytes))) return rc;
        S->reserved += bytes;
        uint64_t off = 0;
        auto carve = [&](auto** p, uint64_t b) {
            *p = reinterpret_cast<std::remove_reference_t<decltype(**p)>*>(blk + off);
            off += (b + 255) & ~(uint64_t)255;
        };
        carve(&ln.xA, B * S->max_in * 4);
        carve(&ln.xB, B * S->max_in * 4);
        carve(&ln.yA, B * S->max_out * 4);
        carve(&ln.yB, B * S->max_out * 4);
        carve(&ln.sB, B * S->max_out * 4);
        carve(&ln.ct, B * S->max_ct_in * 8);
        carve(&ln.A, B * S->max_add * 8);
        carve(&ln.R, B * S->max_add * 8);
        carve(&ln.ct_out, B * S->max_ct_out * 8);
        carve(&ln.M, B * S->max_mask * 8);
        carve(&ln.keys, B * S->max_n * 8);
        carve(&ln.seeds, 3 * B * 8);
        if (cudaStreamCreateWithFlags(&ln.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&ln.side[0], cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&ln.side[1], cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&ln.side[2], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ln.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ln.ev_seed, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ln.ev_mask, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ln.ev_yB, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ln.ev_ct, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ln.ev_R, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost((void**)&ln.h_xA, B * S->max_in * 4) != cudaSuccess ||
            cudaMallocHost((void**)&ln.h_xB, B * S->max_in * 4) != cudaSuccess ||
            cudaMallocHost((void**)&ln.h_yA, B * S->max_out * 4) != cudaSuccess ||
            cudaMallocHost((void**)&ln.h_yB, B * S->max_out * 4) != cudaSuccess ||
            cudaMallocHost((void**)&ln.h_seeds, 3 * B * 8) != cudaSuccess)
            return fdsc_set_error(FDSC_ERR_CUDA, "lane setup failed");
        if ((rc = record_lane_graphs(S, ln))) return rc;
    }
    // host copies: a quarter of the host's threads (2 to 8) besides the worker
    const unsigned hw = std::thread::hardware_concurrency();
    S->copies.reset(new CopyPool(std::min(8u, std::max(2u, hw / 4))));
    S->started = true;
    S->worker = std::thread(worker_loop, S);
    return FDSC_OK;
}

extern "C" int fdsc_server_submit(fdsc_server* S, const fdsc_request* r, uint64_t* ticket) {
    if (!S || !r || !ticket) return fdsc_set_error(FDSC_ERR_ARG, "NULL argument");
    if (!S->started) return fdsc_set_error(FDSC_ERR_ARG, "server not started");
    if (r->type >= S->types.size()) return fdsc_set_error(FDSC_ERR_ARG, "unknown request type %u", r->type);
    const ServerType& t = S->types[r->type];
    if (r->key >= t.nkeys) return fdsc_set_error(FDSC_ERR_ARG, "key %u outside the pool of %u", r->key, t.nkeys);
    if (!r->xA || !r->xB || !r->yA || !r->yB) return fdsc_set_error(FDSC_ERR_ARG, "NULL request buffer");
    if (t.bytes_per_request > S->cfg.hbm_budget_bytes)
        return fdsc_set_error(FDSC_ERR_BUDGET, "request needs %llu bytes, budget %llu",
                              (unsigned long long)t.bytes_per_request, (unsigned long long)S->cfg.hbm_budget_bytes);
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->error) return fdsc_set_error(S->error, "server failed earlier");
    Req q{*r, S->next_ticket++, Clock::now()};
    *ticket = q.ticket;
    S->pending.push_back(q);
    S->submitted++;
    S->cv_work.notify_one();
    return FDSC_OK;
}

extern "C" int fdsc_server_wait(fdsc_server* S, uint64_t ticket, uint32_t timeout_ms, double* latency_us) {
    if (!S) return fdsc_set_error(FDSC_ERR_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(S->mu);
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
    for (;;) {
        auto it = S->done.find(ticket);
        if (it != S->done.end()) {
            const double us = it->second;
            S->done.erase(it);
            if (us < 0) return fdsc_set_error(FDSC_ERR_CUDA, "request %llu failed", (unsigned long long)ticket);
            if (latency_us) *latency_us = us;
            return FDSC_OK;
        }
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && S->done.find(ticket) == S->done.end())
            return fdsc_set_error(FDSC_ERR_TIMEOUT, "request %llu not done within %u ms", (unsigned long long)ticket,
                                  timeout_ms);
    }
}

extern "C" int fdsc_server_stats_get(fdsc_server* S, fdsc_server_stats* out) {
    if (!S || !out) return fdsc_set_error(FDSC_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    const LatencyHist& h = S->latencies;
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->batches = S->batches;
    out->tensor_batches = S->tensor_batches.load();
    out->peak_inflight_bytes = S->peak_inflight;
    out->mean_batch = S->batches ? (double)S->batched_requests / S->batches : 0.0;
    out->p50_us = h.pct(0.50);
    out->p99_us = h.pct(0.99);
    out->mean_us = h.n ? h.sum / (double)h.n : 0.0;
    out->max_us = h.max;
    out->lanes = (uint32_t)S->lanes.size();
    out->lane_capacity = S->lane_cap;
    out->reserved_bytes = S->reserved;
    return S->error;
}

extern "C" int fdsc_server_destroy(fdsc_server* S) {
    if (!S) return FDSC_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    S->copies.reset();
    for (auto& ln : S->lanes) {
        for (cudaStream_t st : ln.side)
            if (st) {
                cudaStreamSynchronize(st);
                cudaStreamDestroy(st);
            }
        if (ln.stream) {
            cudaStreamSynchronize(ln.stream);
            cudaStreamDestroy(ln.stream);
        }
        for (cudaEvent_t ev : {ln.done, ln.ev_seed, ln.ev_mask, ln.ev_yB, ln.ev_ct, ln.ev_R})
            if (ev) cudaEventDestroy(ev);
        for (cudaGraphExec_t g : ln.graphs)
            if (g) cudaGraphExecDestroy(g);
        cudaFreeHost(ln.h_xA);
        cudaFreeHost(ln.h_xB);
        cudaFreeHost(ln.h_yA);
        cudaFreeHost(ln.h_yB);
        cudaFreeHost(ln.h_seeds);
    }
    S->arena.release();
    delete S;
    return FDSC_OK;
}
