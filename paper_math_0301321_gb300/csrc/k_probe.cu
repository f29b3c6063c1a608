// Marker probe: the normal displacement eta_i = (X_i - X0_i) . dir_i of
// chosen markers (the membrane's centre line, Section 5: the paper studies
// the travelling wave through the centre line's normal displacement and its
// envelope over time), recorded on the device every `every` steps into a
// ring of records, with the running envelope max |eta_i|.  The recording
// kernel is part of the captured step, so a run of many steps needs no host
// involvement; ib_read_probe drains the ring.
#include <algorithm>
#include <string>
#include <vector>

#include "ib_internal.cuh"

using namespace ibgb;

namespace ibgb {

// One block: every thread reads the step counter before any thread updates it.
template <class T>
__global__ void __launch_bounds__(1024)
    k_probe(int n, const int32_t *__restrict__ idx, const double *__restrict__ dir, const T *__restrict__ d,
            const T *__restrict__ dlo, int m,
            const double *__restrict__ d_time, int every, int cap, double *__restrict__ ring, double *__restrict__ times,
            double *__restrict__ env, long long *ctl)
{
    PDL_ENTRY();
    const long long k = ctl[0] + 1;            // this step's number since ib_set_probe
    const long long r = ctl[1];
    const bool rec = (k % every) == 0;
    if (rec) {
        const long long slot = r % cap;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int l = idx[i];
            double dd[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) dd[c] = (double)d[c * m + l] + (dlo ? (double)dlo[c * m + l] : 0.0);
            const double eta = dd[0] * dir[i] + dd[1] * dir[n + i] + dd[2] * dir[2 * n + i];
            ring[slot * n + i] = eta;
            env[i] = fmax(env[i], fabs(eta));
        }
        if (threadIdx.x == 0) times[slot] = d_time[0];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ctl[0] = k;
        if (rec) ctl[1] = r + 1;
    }
}

void launch_probe(ib_ctx *c, cudaStream_t s)
{
    if (c->probe_n <= 0) return;
    const int nt = std::min(1024, (c->probe_n + 31) / 32 * 32);
    if (c->fp64)
        launch_pdl(k_probe<double>, dim3(1), dim3(nt), 0, s, c->probe_n, c->probe_idx, c->probe_dir,
                   (const double *)c->mk.d, (const double *)nullptr, (int)c->mk.m, c->d_time, c->probe_every, c->probe_cap, c->probe_ring,
                   c->probe_t, c->probe_env, c->probe_ctl);
    else
        launch_pdl(k_probe<float>, dim3(1), dim3(nt), 0, s, c->probe_n, c->probe_idx, c->probe_dir,
                   (const float *)c->mk.d, (const float *)c->mk.d + 3 * c->mk.m, (int)c->mk.m, c->d_time, c->probe_every, c->probe_cap, c->probe_ring,
                   c->probe_t, c->probe_env, c->probe_ctl);
}

template <class P> static void pfree(P *&p)
{
    if (p) cudaFree((void *)p);
    p = nullptr;
}

void free_probe(ib_ctx *c)
{
    pfree(c->probe_idx);
    pfree(c->probe_dir);
    pfree(c->probe_ring);
    pfree(c->probe_t);
    pfree(c->probe_env);
    pfree(c->probe_ctl);
    c->probe_n = c->probe_every = c->probe_cap = 0;
    c->probe_read = 0;
}

}  // namespace ibgb

namespace {

ib_status perr(ib_status st, const std::string &m) { return set_error(st, m.c_str()); }

#define CKP(call)                                                                                 \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return perr(IB_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <class P> ib_status palloc(P *&p, size_t bytes)
{
    if (cudaMalloc((void **)&p, bytes ? bytes : 16) != cudaSuccess) {
        cudaGetLastError();
        return perr(IB_ERR_NOMEM, "ib_set_probe: device allocation failed");
    }
    return IB_OK;
}

}  // namespace

extern "C" {

ib_status ib_set_probe(ib_ctx *c, int32_t n, const int32_t *markers, const double *dir, int32_t every, int32_t capacity)
{
    if (!c) return perr(IB_ERR_ARG, "ib_set_probe: null context");
    if (!c->have_structure) return perr(IB_ERR_STATE, "ib_set_probe: call ib_set_structure first");
    if (n < 0 || (n > 0 && (!markers || !dir || every < 1 || capacity < 1)))
        return perr(IB_ERR_ARG, "ib_set_probe: need markers, dir, every >= 1 and capacity >= 1");
    const int64_t m = c->mk.m;
    for (int32_t i = 0; i < n; ++i)
        if (markers[i] < 0 || markers[i] >= m) return perr(IB_ERR_ARG, "ib_set_probe: marker id out of range");
    CKP(cudaStreamSynchronize(c->stream));
    free_probe(c);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    ++c->version;
    if (n == 0) return IB_OK;
    // caller ids -> internal numbering
    std::vector<int32_t> qmap(m), inv(m), idx(n);
    CKP(cudaMemcpy(qmap.data(), c->mk.qmap, 4 * (size_t)m, cudaMemcpyDeviceToHost));
    for (int64_t l = 0; l < m; ++l) inv[qmap[l]] = (int32_t)l;
    for (int32_t i = 0; i < n; ++i) idx[i] = inv[markers[i]];
    ib_status st;
    if ((st = palloc(c->probe_idx, 4 * (size_t)n)) != IB_OK) return st;
    if ((st = palloc(c->probe_dir, 8 * 3 * (size_t)n)) != IB_OK) return st;
    if ((st = palloc(c->probe_ring, 8 * (size_t)n * capacity)) != IB_OK) return st;
    if ((st = palloc(c->probe_t, 8 * (size_t)capacity)) != IB_OK) return st;
    if ((st = palloc(c->probe_env, 8 * (size_t)n)) != IB_OK) return st;
    if ((st = palloc(c->probe_ctl, 2 * sizeof(long long))) != IB_OK) return st;
    CKP(cudaMemcpy(c->probe_idx, idx.data(), 4 * (size_t)n, cudaMemcpyHostToDevice));
    CKP(cudaMemcpy(c->probe_dir, dir, 8 * 3 * (size_t)n, cudaMemcpyHostToDevice));
    CKP(cudaMemset(c->probe_env, 0, 8 * (size_t)n));
    CKP(cudaMemset(c->probe_ctl, 0, 2 * sizeof(long long)));
    c->probe_n = n;
    c->probe_every = every;
    c->probe_cap = capacity;
    c->probe_read = 0;
    return IB_OK;
}

ib_status ib_read_probe(ib_ctx *c, double *eta, double *times, double *envelope, int64_t *count)
{
    if (!c || !count) return perr(IB_ERR_ARG, "ib_read_probe: null argument");
    *count = 0;
    if (c->probe_n <= 0) return perr(IB_ERR_STATE, "ib_read_probe: no probe set");
    CKP(cudaStreamSynchronize(c->stream));
    long long ctl[2];
    CKP(cudaMemcpy(ctl, c->probe_ctl, sizeof ctl, cudaMemcpyDeviceToHost));
    const long long fresh = ctl[1] - c->probe_read;
    const long long k = std::min<long long>(fresh, c->probe_cap);
    const int n = c->probe_n;
    if (k > 0 && (eta || times)) {
        std::vector<double> ring((size_t)c->probe_cap * n), tt(c->probe_cap);
        CKP(cudaMemcpy(ring.data(), c->probe_ring, 8 * ring.size(), cudaMemcpyDeviceToHost));
        CKP(cudaMemcpy(tt.data(), c->probe_t, 8 * tt.size(), cudaMemcpyDeviceToHost));
        for (long long j = 0; j < k; ++j) {
            const long long slot = (ctl[1] - k + j) % c->probe_cap;
            if (eta) std::copy(ring.begin() + slot * n, ring.begin() + (slot + 1) * n, eta + j * n);
            if (times) times[j] = tt[slot];
        }
    }
    if (envelope) CKP(cudaMemcpy(envelope, c->probe_env, 8 * (size_t)n, cudaMemcpyDeviceToHost));
    c->probe_read = ctl[1];
    *count = fresh;
    return IB_OK;
}

}  // extern "C"
