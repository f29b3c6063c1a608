// Tile tuning, the autotuner, and batched stepping of many independent
// contexts in one CUDA graph (include/ib.h).
//
// Batch: the steps of all contexts are captured as parallel branches of one
// graph (fork from a private capture stream, one branch stream per context,
// join back), optionally several steps per branch.  One graph launch then
// advances every instance; kernels of different instances run concurrently
// and fill the SMs that a small grid leaves idle.  The graph is recaptured
// lazily when a member context's captured work went stale (new structure or
// tuning).
//
// Autotuner: coordinate descent over the compiled FFT tile variants and the
// grid of the persistent marker kernels, timing graph-launched steps with
// CUDA events; the state is saved in a device snapshot first and restored
// after every trial, so tuning leaves the simulation where it was.
#include <algorithm>
#include <cstdio>
#include <string>
#include <vector>

#include "ib_internal.cuh"

using namespace ibgb;

struct ib_batch {
    std::vector<ib_ctx *> ctx;
    std::vector<uint64_t> version;
    std::vector<cudaStream_t> branch;
    std::vector<cudaEvent_t> join;
    cudaStream_t cap = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t fork = nullptr;
    cudaGraphExec_t graph = nullptr;
    int steps_per_launch = 1;
    int device = 0;
};

namespace {

ib_status err(ib_status st, const std::string &msg) { return set_error(st, msg.c_str()); }

ib_status cuda_err(const char *what, cudaError_t e)
{
    return err(IB_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CKB(call)                                            \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_err(#call, e_);   \
    } while (0)

// Compiled tile variants of the y and z passes, and of the x forward pass
// (FP32: rows of 4, rows of 8, and rows of 4 marching along z with staged
// planes); the x inverse pass takes rows of 8 for x variant 1, else 4.
int n_variants(const ib_ctx *c) { return c->fp64 ? 1 : 2; }
int n_variants_x(const ib_ctx *c) { return c->fp64 ? 1 : 3; }

bool valid_tuning(const ib_ctx *c, const ib_tuning &t)
{
    const int nv = n_variants(c);
    return t.fft_x >= 0 && t.fft_x < n_variants_x(c) && t.fft_y >= 0 && t.fft_y < nv && t.fft_z >= 0 &&
           t.fft_z < nv && t.marker_blocks >= 0;
}

void apply(ib_ctx *c, const ib_tuning &t)
{
    c->fft_tune.x = t.fft_x;
    c->fft_tune.y = t.fft_y;
    c->fft_tune.z = t.fft_z;
    c->marker_blocks = t.marker_blocks;
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    ++c->version;
}

ib_tuning current(const ib_ctx *c)
{
    ib_tuning t{};
    t.fft_x = c->fft_tune.x;
    t.fft_y = c->fft_tune.y;
    t.fft_z = c->fft_tune.z;
    t.marker_blocks = c->marker_blocks;
    return t;
}

// Candidate values per coordinate: FFT variants, then marker-kernel grids
// (0 = every SM at full occupancy, then 2, 1, 1/2 and 1/4 blocks per SM).
std::vector<std::vector<int32_t>> candidates(const ib_ctx *c)
{
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    std::vector<int32_t> v, vx;
    for (int i = 0; i < n_variants(c); ++i) v.push_back(i);
    for (int i = 0; i < n_variants_x(c); ++i) vx.push_back(i);
    return {vx, v, v, {0, 2 * nsm, nsm, std::max(1, nsm / 2), std::max(1, nsm / 4)}};
}

int32_t &coord(ib_tuning &t, int k)
{
    return k == 0 ? t.fft_x : (k == 1 ? t.fft_y : (k == 2 ? t.fft_z : t.marker_blocks));
}

// Coordinate descent: time(t) returns ms (negative on failure).
template <class Time> ib_status descend(ib_tuning &best, const std::vector<std::vector<int32_t>> &cand, Time time)
{
    double best_ms = time(best);
    if (best_ms < 0) return IB_ERR_CUDA;
    for (int k = 0; k < 4; ++k)
        for (int32_t v : cand[k]) {
            if (v == coord(best, k)) continue;
            ib_tuning t = best;
            coord(t, k) = v;
            const double ms = time(t);
            if (ms < 0) return IB_ERR_CUDA;
            if (ms < best_ms) {
                best_ms = ms;
                best = t;
            }
        }
    return IB_OK;
}

ib_status capture_batch(ib_batch *b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    for (ib_ctx *c : b->ctx) CKB(cudaStreamSynchronize(c->stream));
    CKB(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed));
    cudaEventRecord(b->fork, b->cap);
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        cudaStreamWaitEvent(b->branch[i], b->fork, 0);
        for (int k = 0; k < b->steps_per_launch; ++k) enqueue_step_on(b->ctx[i], b->branch[i]);
        cudaEventRecord(b->join[i], b->branch[i]);
        cudaStreamWaitEvent(b->cap, b->join[i], 0);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    if (e != cudaSuccess) return cuda_err("batch capture", e);
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->graph = nullptr;
        return cuda_err("batch graph instantiate", e);
    }
    for (size_t i = 0; i < b->ctx.size(); ++i) b->version[i] = b->ctx[i]->version;
    return IB_OK;
}

bool stale(const ib_batch *b)
{
    if (!b->graph) return true;
    for (size_t i = 0; i < b->ctx.size(); ++i)
        if (b->version[i] != b->ctx[i]->version) return true;
    return false;
}

// Device snapshots of every member (to restore the state after tuning).
struct Saved {
    std::vector<void *> buf;
    ~Saved()
    {
        for (void *p : buf)
            if (p) cudaFree(p);
    }
};

ib_status save_all(const std::vector<ib_ctx *> &cs, Saved &sv)
{
    for (ib_ctx *c : cs) {
        void *p = nullptr;
        const int64_t bytes = ib_snapshot_bytes(c);
        if (cudaMalloc(&p, (size_t)bytes) != cudaSuccess) {
            cudaGetLastError();
            return err(IB_ERR_NOMEM, "autotune: no memory for a state snapshot");
        }
        sv.buf.push_back(p);
        ib_status st = ib_snapshot_save(c, p);
        if (st != IB_OK) return st;
    }
    return IB_OK;
}

void restore_all(const std::vector<ib_ctx *> &cs, const Saved &sv)
{
    for (size_t i = 0; i < cs.size(); ++i) ib_snapshot_load(cs[i], sv.buf[i]);
}

}  // namespace

extern "C" {

ib_status ib_set_tuning(ib_ctx *c, const ib_tuning *t)
{
    if (!c || !t) return err(IB_ERR_ARG, "ib_set_tuning: null argument");
    if (!valid_tuning(c, *t))
        return err(IB_ERR_ARG, c->fp64 ? "ib_set_tuning: FP64 contexts have one FFT variant (0)"
                                       : "ib_set_tuning: FFT variants are 0 or 1, marker_blocks >= 0");
    CKB(cudaStreamSynchronize(c->stream));
    apply(c, *t);
    return IB_OK;
}

ib_status ib_get_tuning(const ib_ctx *c, ib_tuning *t)
{
    if (!c || !t) return err(IB_ERR_ARG, "ib_get_tuning: null argument");
    *t = current(c);
    return IB_OK;
}

ib_status ib_autotune(ib_ctx *c, int32_t reps, ib_tuning *best_out)
{
    if (!c) return err(IB_ERR_ARG, "ib_autotune: null context");
    if (!c->have_structure) return err(IB_ERR_STATE, "ib_autotune: call ib_set_structure first");
    if (reps < 1) return err(IB_ERR_ARG, "ib_autotune: reps must be >= 1");
    CKB(cudaStreamSynchronize(c->stream));
    std::vector<ib_ctx *> one{c};
    Saved sv;
    ib_status st = save_all(one, sv);
    if (st != IB_OK) return st;
    cudaEvent_t e0, e1;
    CKB(cudaEventCreate(&e0));
    CKB(cudaEventCreate(&e1));
    auto time = [&](const ib_tuning &t) -> double {
        apply(c, t);
        restore_all(one, sv);
        if (ib_step(c, 2) != IB_OK) return -1;      // captures the graph, warms up
        cudaEventRecord(e0, c->stream);
        if (ib_step(c, reps) != IB_OK) return -1;
        cudaEventRecord(e1, c->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) return -1;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms / reps;
    };
    ib_tuning best = current(c);
    st = descend(best, candidates(c), time);
    apply(c, best);
    restore_all(one, sv);
    cudaStreamSynchronize(c->stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != IB_OK) return err(st, "ib_autotune: a trial step failed");
    if (best_out) *best_out = best;
    return IB_OK;
}

ib_status ib_batch_create(ib_ctx *const *ctxs, int32_t n, int32_t steps_per_launch, void *stream, ib_batch **out)
{
    if (!ctxs || !out || n < 1) return err(IB_ERR_ARG, "ib_batch_create: need n >= 1 contexts and an output");
    if (steps_per_launch < 1) return err(IB_ERR_ARG, "ib_batch_create: steps_per_launch must be >= 1");
    *out = nullptr;
    for (int32_t i = 0; i < n; ++i) {
        if (!ctxs[i]) return err(IB_ERR_ARG, "ib_batch_create: null context");
        if (!ctxs[i]->have_structure) return err(IB_ERR_STATE, "ib_batch_create: a context has no structure");
        if (ctxs[i]->device != ctxs[0]->device) return err(IB_ERR_ARG, "ib_batch_create: contexts on different devices");
        for (int32_t j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return err(IB_ERR_ARG, "ib_batch_create: a context appears twice");
    }
    ib_batch *b = new ib_batch();
    b->ctx.assign(ctxs, ctxs + n);
    b->version.assign(n, 0);
    b->steps_per_launch = steps_per_launch;
    b->stream = (cudaStream_t)stream;
    b->device = ctxs[0]->device;
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int32_t i = 0; i < n && e == cudaSuccess; ++i) {
        cudaStream_t s = nullptr;
        cudaEvent_t ev = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        b->branch.push_back(s);
        b->join.push_back(ev);
    }
    if (e != cudaSuccess) {
        ib_batch_destroy(b);
        return cuda_err("ib_batch_create", e);
    }
    *out = b;
    return IB_OK;
}

ib_status ib_batch_step(ib_batch *b, int64_t nsteps)
{
    if (!b) return err(IB_ERR_ARG, "ib_batch_step: null batch");
    if (nsteps < 0 || nsteps % b->steps_per_launch)
        return err(IB_ERR_ARG, "ib_batch_step: nsteps must be a non-negative multiple of steps_per_launch");
    if (nsteps == 0) return IB_OK;
    if (stale(b)) {
        ib_status st = capture_batch(b);
        if (st != IB_OK) return st;
    }
    for (int64_t i = 0; i < nsteps / b->steps_per_launch; ++i) CKB(cudaGraphLaunch(b->graph, b->stream));
    return IB_OK;
}

ib_status ib_batch_autotune(ib_batch *b, int32_t reps)
{
    if (!b) return err(IB_ERR_ARG, "ib_batch_autotune: null batch");
    if (reps < 1) return err(IB_ERR_ARG, "ib_batch_autotune: reps must be >= 1");
    for (ib_ctx *c : b->ctx) CKB(cudaStreamSynchronize(c->stream));
    CKB(cudaStreamSynchronize(b->stream));
    Saved sv;
    ib_status st = save_all(b->ctx, sv);
    if (st != IB_OK) return st;
    for (ib_ctx *c : b->ctx) CKB(cudaStreamSynchronize(c->stream));
    bool all_fp32 = true;
    for (ib_ctx *c : b->ctx) all_fp32 = all_fp32 && !c->fp64;
    cudaEvent_t e0, e1;
    CKB(cudaEventCreate(&e0));
    CKB(cudaEventCreate(&e1));
    auto time = [&](const ib_tuning &t) -> double {
        for (ib_ctx *c : b->ctx) apply(c, t);
        restore_all(b->ctx, sv);
        for (ib_ctx *c : b->ctx) cudaStreamSynchronize(c->stream);
        if (ib_batch_step(b, b->steps_per_launch) != IB_OK) return -1;   // recaptures, warms up
        cudaEventRecord(e0, b->stream);
        if (ib_batch_step(b, (int64_t)reps * b->steps_per_launch) != IB_OK) return -1;
        cudaEventRecord(e1, b->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) return -1;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms / reps;
    };
    ib_tuning best = current(b->ctx[0]);
    std::vector<std::vector<int32_t>> cand = candidates(b->ctx[0]);
    if (!all_fp32) cand[0] = cand[1] = cand[2] = {0};
    st = descend(best, cand, time);
    for (ib_ctx *c : b->ctx) apply(c, best);
    restore_all(b->ctx, sv);
    for (ib_ctx *c : b->ctx) cudaStreamSynchronize(c->stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != IB_OK) return err(st, "ib_batch_autotune: a trial failed");
    return IB_OK;
}

ib_status ib_batch_sync(ib_batch *b)
{
    if (!b) return err(IB_ERR_ARG, "ib_batch_sync: null batch");
    CKB(cudaStreamSynchronize(b->stream));
    for (ib_ctx *c : b->ctx) {
        ib_status st = ib_sync(c);
        if (st != IB_OK) return st;
    }
    return IB_OK;
}

ib_status ib_batch_destroy(ib_batch *b)
{
    if (!b) return IB_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (cudaStream_t s : b->branch)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->join)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return IB_OK;
}

}  // extern "C"
