// C ABI of the immersed-boundary step (include/ib.h): contexts, structure
// preprocessing, state transfer, the captured step graph and the stand-alone
// spread / interp / fluid-solve / bin-sort calls.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "fft_core.cuh"
#include "ib_internal.cuh"

namespace ibgb {
template <class T>
void fluid_impl(ib_ctx *c, const void *u_n, const void *F, void *u_np1, void *p, bool use_touched, int mode,
                cudaStream_t s, cudaEvent_t *ev);

bool fft_length_supported(int n) { return n == 32 || n == 64 || n == 96 || n == 128 || n == 256; }

void launch_fluid_mode(ib_ctx *c, const void *u_n, const void *F, void *u_np1, void *p, bool use_touched, int mode,
                       cudaStream_t s, cudaEvent_t *ev)
{
    if (c->fp64) fluid_impl<double>(c, u_n, F, u_np1, p, use_touched, mode, s, ev);
    else fluid_impl<float>(c, u_n, F, u_np1, p, use_touched, mode, s, ev);
}

void launch_fluid(ib_ctx *c, const void *u_n, const void *F, void *u_np1, void *p, bool use_touched, bool step_mode,
                  cudaStream_t s, cudaEvent_t *ev)
{
    launch_fluid_mode(c, u_n, F, u_np1, p, use_touched, step_mode ? FLUID_STEP : FLUID_PLAIN, s, ev);
}
}  // namespace ibgb

using namespace ibgb;

namespace {

thread_local std::string g_err;

ib_status fail(ib_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CK(call)                                                                                    \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return fail(IB_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));    \
    } while (0)

#define CKM(ptr, bytes)                                                                             \
    do {                                                                                            \
        cudaError_t e_ = cudaMalloc((void **)&(ptr), (bytes) > 0 ? (bytes) : 16);                   \
        if (e_ != cudaSuccess) {                                                                    \
            cudaGetLastError();                                                                     \
            return fail(IB_ERR_NOMEM, "cudaMalloc(%zu bytes): %s", (size_t)(bytes), cudaGetErrorString(e_)); \
        }                                                                                           \
    } while (0)

template <class P> void dfree(P *&p)
{
    if (p) cudaFree((void *)p);
    p = nullptr;
}

bool on_device(const ib_ctx *c) { return (c->desc.flags & IB_PTR_DEVICE) != 0; }

// host -> device (or device -> device) copy of a caller buffer
cudaError_t copy_in(const ib_ctx *c, void *dst, const void *src, size_t bytes)
{
    return cudaMemcpyAsync(dst, src, bytes, on_device(c) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           c->stream);
}

cudaError_t copy_out(const ib_ctx *c, void *dst, const void *src, size_t bytes)
{
    return cudaMemcpyAsync(dst, src, bytes, on_device(c) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           c->stream);
}

ib_status check_status(ib_ctx *c)
{
    int st = 0;
    CK(cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st) {
        CK(cudaMemset(c->d_status, 0, sizeof(int)));
        const char *vel = "non-finite marker velocity";
        const char *pos = "marker position non-finite or more than 2^30 cells from the origin";
        if ((st & DEV_NONFINITE) && (st & DEV_RANGE)) return fail(IB_ERR_NONFINITE, "%s; %s", pos, vel);
        if (st & DEV_NONFINITE) return fail(IB_ERR_NONFINITE, "%s", vel);
        if (st & DEV_RANGE) return fail(IB_ERR_NONFINITE, "%s", pos);
        if (st & DEV_TIMEOUT) return fail(IB_ERR_TIMEOUT, "a bounded wait for an asynchronous copy ran out");
        return fail(IB_ERR_STATE, "device error flags 0x%x", st);
    }
    return IB_OK;
}

void drop_graph(ib_ctx *c)
{
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    ++c->version;
}

void free_markers(ib_ctx *c)
{
    auto &mk = c->mk;
    dfree(mk.X0);
    dfree(mk.qmap);
    dfree(mk.qinv);
    dfree(mk.cell0);
    dfree(mk.r0);
    dfree(mk.d);
    dfree(mk.sp_off);
    dfree(mk.sp_j);
    dfree(mk.sp_k);
    dfree(mk.sp_L0);
    dfree(mk.sp_e0);
    dfree(mk.sp_c0);
    dfree(mk.tk);
    dfree(mk.mf_dir);
    dfree(mk.bslot);
    dfree(mk.bn);
    dfree(mk.bc);
    dfree(mk.key);
    dfree(mk.key_alt);
    dfree(mk.key_s);
    dfree(mk.perm_alt);
    dfree(mk.perm);
    dfree(mk.hist);
    dfree(mk.rfrac);
    dfree(mk.rec);
    dfree(mk.f);
    dfree(mk.U);
    dfree(mk.Us);
    dfree(mk.Xtmp);
    dfree(mk.lamD);
    dfree(mk.lamDo);
    dfree(mk.rec2);
    dfree(mk.lf_s);
    dfree(mk.lX_s);
    dfree(mk.lf);
    dfree(mk.lX);
    dfree(mk.bunit);
    dfree(mk.bseg);
    dfree(mk.gterm);
    dfree(mk.seg_off);
    dfree(mk.seg_slot);
    dfree(mk.gseg);
    mk = MarkerArrays{};
    free_probe(c);
    dfree(c->forcing.rows);
    c->forcing = Forcing{};
    c->have_structure = false;
}

// Marker arrays in the caller's numbering <-> internal numbering (q[internal]
// = caller's id); index i runs over 3*m entries [c][marker].
// d = X - X0 (FP64 difference, rounded to the context's real type)
// FP32 contexts keep the displacement as a pair of floats, d = hi + lo
// (lo = the rounding error of hi, |lo| <= ulp(hi)/2): lo is the second half of
// the same array, at d + 3m; FP64 contexts pass lo = null.
template <class T> __device__ __forceinline__ void put_disp(T *d, T *lo, long long i, double v)
{
    const T hi = (T)v;
    d[i] = hi;
    if (lo) lo[i] = (T)(v - (double)hi);
}

template <class T> __device__ __forceinline__ double get_disp(const T *d, const T *lo, long long i)
{
    return lo ? (double)d[i] + (double)lo[i] : (double)d[i];
}

// The transfer kernels run over the caller's order: thread i of block row c
// handles entry [c][i] of the caller's array (coalesced, also when it is
// host memory read in place) and internal marker qinv[i].
// d = X - X0 (FP64 difference)
template <class T>
__global__ void k_set_disp(int m, const int32_t *qinv, const double *X, const double *X0, T *d, T *lo)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const long long c = blockIdx.y, l = c * m + qinv[i];
    put_disp(d, lo, l, X[c * m + i] - X0[l]);
}

// X = X0 + d
template <class T>
__global__ void k_get_pos(int m, const int32_t *qinv, const double *X0, const T *d, const T *lo, double *X)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const long long c = blockIdx.y, l = c * m + qinv[i];
    X[c * m + i] = X0[l] + get_disp(d, lo, l);
}

// d = D
// The last sort from the context's state in the caller's numbering:
// key[i] = key of caller marker i, perm[j] = caller id at sorted position j,
// internal[j] = caller id of internal marker j.
__global__ void k_bin_order_out(int m, const int32_t *qmap, const int32_t *qinv, const int32_t *ikey,
                                const int32_t *iperm, int32_t *key, int32_t *perm, int32_t *internal)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= m) return;
    if (key) key[l] = ikey[qinv[l]];
    if (perm) perm[l] = qmap[iperm[l]];
    if (internal) internal[l] = qmap[l];
}

// Mean velocity of a field u [3][G] in FP64 (FP32 contexts' zero-wavenumber
// mode): 1024 blocks of fixed strided sums, then one block over their
// partials in index order (deterministic).
template <class T> __global__ void k_mean_part(const T *u, long long G, double *part)
{
    __shared__ double red[3][8];
    const int tid = threadIdx.x;
    for (int c = 0; c < 3; ++c) {
        double v = 0.0;
        for (long long i = (long long)blockIdx.x * blockDim.x + tid; i < G; i += (long long)gridDim.x * blockDim.x)
            v += (double)u[c * G + i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0) red[c][tid >> 5] = v;
    }
    __syncthreads();
    if (tid < 3) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += red[tid][w];
        part[tid * gridDim.x + blockIdx.x] = v;
    }
}

__global__ void k_mean_final(const double *part, int nb, long long G, double *mean)
{
    __shared__ double red[3][8];
    const int tid = threadIdx.x;
    for (int c = 0; c < 3; ++c) {
        double v = 0.0;
        for (int i = tid; i < nb; i += blockDim.x) v += part[c * nb + i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0) red[c][tid >> 5] = v;
    }
    __syncthreads();
    if (tid < 3) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += red[tid][w];
        mean[tid] = v / (double)G;
    }
}

template <class T> __global__ void k_set_d(int m, const int32_t *qinv, const double *D, T *d, T *lo)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const long long c = blockIdx.y, l = c * m + qinv[i];
    put_disp(d, lo, l, D[c * m + i]);
}

// D = d
template <class T> __global__ void k_get_d(int m, const int32_t *qinv, const T *d, const T *lo, double *D)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const long long c = blockIdx.y, l = c * m + qinv[i];
    D[c * m + i] = get_disp(d, lo, l);
}

dim3 transfer_grid(int64_t m) { return dim3((unsigned)((m + 255) / 256), 3); }

// Device address of a caller's host buffer that kernels may read or write in
// place (page-locked or registered memory), or null when the buffer has to be
// staged through device memory.
void *host_alias(const void *p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return (a.type == cudaMemoryTypeHost && a.devicePointer) ? a.devicePointer : nullptr;
}

template <class T> std::vector<T> conv(const std::vector<double> &v)
{
    return std::vector<T>(v.begin(), v.end());
}

template <class T> ib_status upload(void *&dst, const std::vector<double> &v)
{
    std::vector<T> t = conv<T>(v);
    CKM(dst, sizeof(T) * t.size());
    if (!t.empty()) CK(cudaMemcpy(dst, t.data(), sizeof(T) * t.size(), cudaMemcpyHostToDevice));
    return IB_OK;
}

template <class I> ib_status upload_i(I *&dst, const std::vector<I> &v)
{
    CKM(dst, sizeof(I) * v.size());
    if (!v.empty()) CK(cudaMemcpy(dst, v.data(), sizeof(I) * v.size(), cudaMemcpyHostToDevice));
    return IB_OK;
}

template <class P> ib_status ensure(P *&p, size_t bytes)
{
    if (!p) CKM(p, bytes);
    return IB_OK;
}

// Device time-advance parameters [dt, body amplitude, body omega, marker
// amplitude, marker omega] (synchronous).
ib_status upload_tparams(ib_ctx *c)
{
    const double tp[5] = {c->desc.dt, c->forcing.mag, c->forcing.omega, c->forcing.mamp, c->forcing.momega};
    CK(cudaMemcpy(c->d_tparams, tp, sizeof tp, cudaMemcpyHostToDevice));
    return IB_OK;
}

// Host staging of the device time state at time t.
void stage_time(ib_ctx *c, double t)
{
    c->t_pair[0] = t;
    c->t_pair[1] = c->forcing.mag * std::cos(c->forcing.omega * t);
    c->t_pair[2] = c->forcing.mamp * std::cos(c->forcing.momega * t);
    c->t_pair[3] = 0.0;
}

// c_{i-1}, c_i, c_{i+1} of every bending slot for stiffnesses b [n_seg]:
// b_seg dw / ds^3, the same product as the force law's definition
std::vector<double> bend_coefficients(const MarkerArrays &mk, const double *b)
{
    const int64_t nb = mk.nb;
    std::vector<double> bc(3 * std::max<int64_t>(nb, 1), 0.0);
    for (int64_t i = 0; i < 3 * nb; ++i) {
        const int32_t sg = mk.h_bseg3[i];
        if (sg < 0) continue;
        const double ds = mk.h_bds3[i];
        bc[i] = b[sg] * mk.h_bdw3[i] / (ds * ds * ds);
    }
    return bc;
}

// one forward step enqueued on stream s (captured into the step graph); ev
// (nullable): IB_NSTAGES + 1 events bracketing the stages
void enqueue_step(ib_ctx *c, cudaStream_t s, cudaEvent_t *ev = nullptr)
{
    if (ev) cudaEventRecord(ev[0], s);
    launch_keys_state(c, s);
    if (ev) cudaEventRecord(ev[1], s);
    launch_sort(c, s);
    launch_bin_plan(c, s);
    if (ev) cudaEventRecord(ev[2], s);
    launch_records(c, 1, nullptr, s);
    if (ev) cudaEventRecord(ev[3], s);
    launch_spread(c, c->F, false, s);
    if (ev) cudaEventRecord(ev[4], s);
    launch_fluid(c, c->u, c->F, c->u, nullptr, true, true, s, ev ? ev + 5 : nullptr);
    if (ev) cudaEventRecord(ev[9], s);
    launch_interp(c, c->u, c->mk.d, true, s);
    launch_probe(c, s);
    if (ev) cudaEventRecord(ev[10], s);
}

const char *const kStageNames[IB_NSTAGES] = {"keys",       "sort",       "records",   "spread",    "fft_x_fwd",
                                             "fft_y_fwd", "fft_z_proj", "fft_y_inv", "fft_x_inv", "interp"};

}  // namespace

namespace ibgb {
void enqueue_step_on(ib_ctx *c, cudaStream_t s) { enqueue_step(c, s); }

ib_status set_error(ib_status st, const char *msg)
{
    g_err = msg;
    return st;
}
}  // namespace ibgb

extern "C" {

const char *ib_last_error(void) { return g_err.c_str(); }

ib_status ib_create(const ib_grid_desc *desc, ib_ctx **out)
{
    if (!desc || !out) return fail(IB_ERR_ARG, "ib_create: null argument");
    *out = nullptr;
    for (int j = 0; j < 3; ++j)
        if (!fft_length_supported(desc->n[j]))
            return fail(IB_ERR_UNSUPPORTED, "grid size n[%d] = %d not in {32, 64, 96, 128, 256}", j, desc->n[j]);
    if (!(desc->h > 0) || !(desc->rho > 0) || !(desc->mu >= 0) || !(desc->dt > 0))
        return fail(IB_ERR_ARG, "ib_create: need h, rho, dt > 0 and mu >= 0");
    if (desc->prec != IB_FP32 && desc->prec != IB_FP64 && desc->prec != IB_FP32_TCFFT)
        return fail(IB_ERR_ARG, "ib_create: bad precision");
    int dev = 0;
    CK(cudaGetDevice(&dev));
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, dev));
    if (prop.major != 10 || prop.minor != 3)
        return fail(IB_ERR_CUDA, "device %d is sm_%d%d; this library is built for sm_103a only", dev, prop.major,
                    prop.minor);

    ib_ctx *c = new (std::nothrow) ib_ctx();
    if (!c) return fail(IB_ERR_NOMEM, "host allocation failed");
    c->desc = *desc;
    c->device = dev;
    c->fp64 = desc->prec == IB_FP64;
    c->tc_fft = desc->prec == IB_FP32_TCFFT;
    c->elt = c->fp64 ? 8 : 4;
    c->stream = (cudaStream_t)desc->stream;
    auto &g = c->dim;
    g.nx = desc->n[0];
    g.ny = desc->n[1];
    g.nz = desc->n[2];
    g.ntx = g.nx / TILE;
    g.nty = g.ny / TILE;
    g.ntz = g.nz / TILE;
    g.ntiles = g.ntx * g.nty * g.ntz;
    g.G = (long long)g.nx * g.ny * g.nz;
    const size_t fld = (size_t)c->elt * 3 * g.G;
    const size_t cpx = 2 * (size_t)c->elt;
    const int ntiles = g.ntx * g.nty * g.ntz;
    ib_status st = IB_OK;
    auto bail = [&](ib_status s) {
        ib_destroy(c);
        return s;
    };
#define TRY(x)                         \
    do {                               \
        st = (x);                      \
        if (st != IB_OK) return bail(st); \
    } while (0)
    auto alloc = [&](void *&p, size_t bytes) -> ib_status {
        CKM(p, bytes);
        return IB_OK;
    };
    TRY(alloc(c->u, fld));
    TRY(alloc(c->F, fld));
    if (cudaMemset(c->u, 0, fld) != cudaSuccess) return bail(fail(IB_ERR_CUDA, "cudaMemset failed"));
    TRY(alloc(c->spec, cpx * 4 * g.nz * g.ny * (g.nx / 2)));
    TRY(alloc(c->nyq, cpx * 4 * g.nz * g.ny));
    void *tmp = nullptr;
    TRY(alloc(tmp, ntiles));
    c->touched = (uint8_t *)tmp;
    tmp = nullptr;
    TRY(alloc(tmp, sizeof(int) * ntiles));
    c->tile_list = (int *)tmp;
    tmp = nullptr;
    TRY(alloc(tmp, sizeof(int) * 2));
    c->tile_count = (int *)tmp;
    c->tile_next = (int *)tmp + 1;
    tmp = nullptr;
    TRY(alloc(tmp, sizeof(int32_t) * (ntiles + 1)));
    c->bin_start = (int32_t *)tmp;
    tmp = nullptr;
    TRY(alloc(tmp, sizeof(int32_t) * (ntiles + 1)));
    c->item_start = (int32_t *)tmp;
    tmp = nullptr;
    TRY(alloc(tmp, sizeof(int) * 4));
    c->item_ctl = (int *)tmp;
    tmp = nullptr;
    TRY(alloc(tmp, sizeof(int2) * (ntiles / 1024 + 2)));
    c->bscan_tmp_plan = (int2 *)tmp;
    tmp = nullptr;
    if (cudaMemset(c->bin_start, 0, sizeof(int32_t) * (ntiles + 1)) != cudaSuccess ||
        cudaMemset(c->item_start, 0, sizeof(int32_t) * (ntiles + 1)) != cudaSuccess ||
        cudaMemset(c->item_ctl, 0, sizeof(int) * 4) != cudaSuccess)
        return bail(fail(IB_ERR_CUDA, "cudaMemset failed"));
    TRY(alloc(tmp, 8 * sizeof(double)));
    c->d_time = (double *)tmp;
    tmp = nullptr;
    if (!c->fp64) {
        // FP64 mean mode: per-block sums of the x pass (at least 4 rows per
        // block), also the partials of the state-mean reduction (1024 blocks)
        const long long nqp = 3LL * std::max<long long>((long long)c->dim.ny * c->dim.nz / 4, 1024);
        TRY(alloc(tmp, nqp * sizeof(double)));
        c->qpart = (double *)tmp;
        tmp = nullptr;
    }
    TRY(alloc(tmp, 5 * sizeof(double)));
    c->d_tparams = (double *)tmp;
    tmp = nullptr;
    TRY(alloc(tmp, sizeof(int)));
    c->d_status = (int *)tmp;
    if (cudaMemset(c->d_time, 0, 8 * sizeof(double)) != cudaSuccess ||
        cudaMemset(c->d_status, 0, sizeof(int)) != cudaSuccess || upload_tparams(c) != IB_OK)
        return bail(fail(IB_ERR_CUDA, "cudaMemset failed"));
    // FFT twiddles W_n^j = exp(-2 pi i j/n) and the per-axis symbols
    for (int a = 0; a < 3; ++a) {
        const int n = desc->n[a];
        std::vector<double> tw(2 * n), ss(n), sa(n);
        for (int j = 0; j < n; ++j) {
            const CD w = ct_unit(-j, n);
            tw[2 * j] = w.re;
            tw[2 * j + 1] = w.im;
            ss[j] = (2 * j) % n == 0 ? 0.0 : ct_unit(j, n).im / desc->h;
            const double sn = ct_unit(j, 2 * n).im;   // sin(pi j / n)
            sa[j] = 4.0 * desc->mu / (desc->h * desc->h) * sn * sn;
        }
        if (c->fp64) {
            TRY(upload<double>(c->tw[a], tw));
            TRY(upload<double>(c->sym_s[a], ss));
            TRY(upload<double>(c->sym_a[a], sa));
        } else {
            TRY(upload<float>(c->tw[a], tw));
            TRY(upload<float>(c->sym_s[a], ss));
            TRY(upload<float>(c->sym_a[a], sa));
        }
    }
    if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(IB_ERR_CUDA, "cudaStreamCreate failed"));
#undef TRY
    *out = c;
    return IB_OK;
}

ib_status ib_destroy(ib_ctx *c)
{
    if (!c) return IB_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    drop_graph(c);
    free_markers(c);
    dfree(c->u);
    dfree(c->F);
    dfree(c->ubuf);
    dfree(c->Fbuf);
    dfree(c->p);
    dfree(c->touched);
    dfree(c->tile_list);
    dfree(c->tile_count);
    dfree(c->spec);
    dfree(c->nyq);
    for (int a = 0; a < 3; ++a) {
        dfree(c->tw[a]);
        dfree(c->sym_s[a]);
        dfree(c->sym_a[a]);
    }
    dfree(c->bin_start);
    dfree(c->item_start);
    dfree(c->item_ctl);
    dfree(c->bscan_tmp_plan);
    dfree(c->items);
    dfree(c->partial);
    dfree(c->bscan_tmp);
    dfree(c->d_time);
    dfree(c->qpart);
    dfree(c->d_tparams);
    dfree(c->d_status);
    dfree(c->adj_u1);
    dfree(c->adj_lw);
    if (c->cap) cudaStreamDestroy(c->cap);
    delete c;
    return IB_OK;
}

ib_status ib_info(const ib_ctx *c, int64_t *m, int64_t *G, int32_t *prec)
{
    if (!c) return fail(IB_ERR_ARG, "ib_info: null context");
    if (m) *m = c->mk.m;
    if (G) *G = c->dim.G;
    if (prec) *prec = c->desc.prec;
    return IB_OK;
}

ib_status ib_set_structure(ib_ctx *c, const ib_structure_desc *s)
{
    if (!c || !s) return fail(IB_ERR_ARG, "ib_set_structure: null argument");
    const int64_t m = s->m;
    // marker kernels index [3][m] arrays as c*m + l in 32-bit arithmetic
    if (m < 0 || m > (int64_t)INT32_MAX / 3)
        return fail(IB_ERR_ARG, "ib_set_structure: marker count %lld (at most %d)", (long long)m, INT32_MAX / 3);
    if (m > 0 && !s->X0) return fail(IB_ERR_ARG, "ib_set_structure: X0 is null");
    if (s->n_spring < 0 || s->n_tether < 0 || s->n_sheet < 0 || s->n_seg < 0)
        return fail(IB_ERR_ARG, "ib_set_structure: negative count");
    for (int64_t e = 0; e < s->n_spring; ++e) {
        const int32_t i = s->spring_ij[2 * e], j = s->spring_ij[2 * e + 1];
        if (i < 0 || i >= m || j < 0 || j >= m || i == j)
            return fail(IB_ERR_ARG, "spring %lld joins invalid markers (%d, %d)", (long long)e, i, j);
    }
    for (int64_t e = 0; e < s->n_tether; ++e)
        if (s->tether_i[e] < 0 || s->tether_i[e] >= m)
            return fail(IB_ERR_ARG, "tether %lld on invalid marker %d", (long long)e, s->tether_i[e]);
    if (s->n_mforce < 0 || (s->n_mforce > 0 && (!s->mforce_i || !s->mforce_dir)))
        return fail(IB_ERR_ARG, "ib_set_structure: bad external marker force arrays");
    {
        std::vector<char> seen(s->n_mforce > 0 ? m : 0, 0);
        for (int64_t j = 0; j < s->n_mforce; ++j) {
            const int32_t i = s->mforce_i[j];
            if (i < 0 || i >= m || seen[i])
                return fail(IB_ERR_ARG, "external force %lld on invalid or repeated marker %d", (long long)j, i);
            seen[i] = 1;
        }
    }
    std::vector<int32_t> bslot(m, -1);
    int64_t nb = 0;
    for (int q = 0; q < s->n_sheet; ++q) {
        const ib_sheet &sh = s->sheets[q];
        if (sh.n1 < 1 || sh.n2 < 1 || sh.first < 0 || sh.first + (int64_t)sh.n1 * sh.n2 > m || !(sh.ds > 0))
            return fail(IB_ERR_ARG, "sheet %d out of range", q);
        for (int32_t i = 0; i < sh.n1; ++i) {
            if (sh.seg_of_row[i] < 0 || sh.seg_of_row[i] >= s->n_seg)
                return fail(IB_ERR_ARG, "sheet %d row %d: segment %d out of range", q, i, sh.seg_of_row[i]);
            for (int32_t a = 0; a < sh.n2; ++a) {
                const int64_t l = sh.first + (int64_t)i * sh.n2 + a;
                if (bslot[l] >= 0) return fail(IB_ERR_ARG, "marker %lld is in more than one sheet", (long long)l);
                bslot[l] = (int32_t)nb++;
            }
        }
    }
    cudaStreamSynchronize(c->stream);
    drop_graph(c);
    free_markers(c);
    auto &mk = c->mk;
    mk.m = m;
    const double h = c->desc.h, inv_h = 1.0 / h;
    const size_t R = c->elt;
    // positions
    std::vector<double> X0(s->X0, s->X0 + 3 * m);
    // Internal numbering: markers ordered by their initial cell (tile-major
    // key, ties by id).  The step sorts markers by tile and keeps id order
    // within a tile, so with this numbering the markers of one cell stay
    // adjacent while displacements are small.  qmap[internal] = caller's id.
    std::vector<int32_t> qmap(m), inv(m);
    {
        std::vector<int64_t> key0(m);
        const auto &g = c->dim;
        for (int64_t l = 0; l < m; ++l) {
            int b[3];
            for (int cc = 0; cc < 3; ++cc) {
                const int n = cc == 0 ? g.nx : (cc == 1 ? g.ny : g.nz);
                long long v = (long long)std::floor(X0[cc * m + l] * inv_h) % n;
                b[cc] = (int)(v < 0 ? v + n : v);
            }
            key0[l] = tile_key(g, b[0], b[1], b[2]);
        }
        for (int64_t l = 0; l < m; ++l) qmap[l] = (int32_t)l;
        std::stable_sort(qmap.begin(), qmap.end(), [&](int32_t a, int32_t b) { return key0[a] < key0[b]; });
        for (int64_t l = 0; l < m; ++l) inv[qmap[l]] = (int32_t)l;
    }
    {
        ib_status st0 = upload_i(mk.qmap, qmap);
        if (st0 != IB_OK) return st0;
        st0 = upload_i(mk.qinv, inv);
        if (st0 != IB_OK) return st0;
        std::vector<double> X0i(3 * m);
        for (int cc = 0; cc < 3; ++cc)
            for (int64_t l = 0; l < m; ++l) X0i[cc * m + l] = X0[cc * m + qmap[l]];
        if (upload_i(mk.X0, X0i) != IB_OK) return IB_ERR_NOMEM;
    }
    if (!c->fp64) {
        std::vector<int32_t> cell(3 * m);
        std::vector<double> r0(3 * m);
        for (int cc = 0; cc < 3; ++cc)
            for (int64_t l = 0; l < m; ++l) {
                const double sv = X0[cc * m + qmap[l]] * inv_h;
                const double fl = std::floor(sv);
                cell[cc * m + l] = (int32_t)fl;
                r0[cc * m + l] = sv - fl;
            }
        ib_status st = upload_i(mk.cell0, cell);
        if (st != IB_OK) return st;
        if ((st = upload<float>(mk.r0, r0)) != IB_OK) return st;
    }
    // FP32 contexts: hi [3][m] then lo [3][m]
    const size_t dbytes = R * 3 * m * (c->fp64 ? 1 : 2);
    CKM(mk.d, dbytes);
    CK(cudaMemset(mk.d, 0, dbytes));
    // springs: CSR rows per marker, each link in both end rows
    std::vector<int32_t> off(m + 1, 0);
    for (int64_t e = 0; e < s->n_spring; ++e) {
        off[inv[s->spring_ij[2 * e]] + 1]++;
        off[inv[s->spring_ij[2 * e + 1]] + 1]++;
    }
    for (int64_t i = 0; i < m; ++i) off[i + 1] += off[i];
    const int64_t nnz = off[m];
    std::vector<int32_t> sj(nnz), fill(off.begin(), off.end() - 1);
    std::vector<double> sk(nnz), sL0(nnz), se0(3 * nnz), sc0(nnz);
    for (int64_t e = 0; e < s->n_spring; ++e) {
        const int32_t i = s->spring_ij[2 * e], j = s->spring_ij[2 * e + 1];
        double e0[3], n2 = 0;
        for (int cc = 0; cc < 3; ++cc) {
            e0[cc] = X0[cc * m + j] - X0[cc * m + i];
            n2 += e0[cc] * e0[cc];
        }
        const double L0 = s->spring_L0[e];
        const int32_t ends[2] = {inv[i], inv[j]}, others[2] = {inv[j], inv[i]};
        for (int side = 0; side < 2; ++side) {
            const int32_t at = fill[ends[side]]++;
            sj[at] = others[side];
            sk[at] = s->spring_k[e];
            sL0[at] = L0;
            for (int cc = 0; cc < 3; ++cc) se0[cc * nnz + at] = side == 0 ? e0[cc] : -e0[cc];
            sc0[at] = n2 - L0 * L0;
        }
    }
    mk.nnz = nnz;
    ib_status st;
    if ((st = upload_i(mk.sp_off, off)) != IB_OK) return st;
    if ((st = upload_i(mk.sp_j, sj)) != IB_OK) return st;
    auto upT = [&](void *&dst, const std::vector<double> &v) {
        return c->fp64 ? upload<double>(dst, v) : upload<float>(dst, v);
    };
    if ((st = upT(mk.sp_k, sk)) != IB_OK) return st;
    if ((st = upT(mk.sp_L0, sL0)) != IB_OK) return st;
    if ((st = upT(mk.sp_e0, se0)) != IB_OK) return st;
    if ((st = upT(mk.sp_c0, sc0)) != IB_OK) return st;
    // tethers (stiffness summed per marker)
    std::vector<double> tk(m, 0.0);
    for (int64_t e = 0; e < s->n_tether; ++e) tk[inv[s->tether_i[e]]] += s->tether_k[e];
    if ((st = upT(mk.tk, tk)) != IB_OK) return st;
    // external marker force directions, zero on unforced markers
    if (s->n_mforce > 0 && s->mforce_amp != 0.0) {
        std::vector<double> dir(3 * m, 0.0);
        for (int64_t j = 0; j < s->n_mforce; ++j)
            for (int cc = 0; cc < 3; ++cc) dir[cc * m + inv[s->mforce_i[j]]] = s->mforce_dir[cc * s->n_mforce + j];
        if ((st = upT(mk.mf_dir, dir)) != IB_OK) return st;
    }
    // bending: per sheet marker, the 5 line neighbours and c_{i-1}, c_i, c_{i+1}
    // (c_row = b_seg(row) dw_row / ds^3 on interior rows, else no term); the
    // segment, dw and ds of each term are kept to rebuild c when b changes
    mk.nb = nb;
    mk.n_seg = s->n_seg;
    std::vector<int32_t> bn(5 * std::max<int64_t>(nb, 1), -1);
    mk.h_bseg3.assign(3 * std::max<int64_t>(nb, 1), -1);
    mk.h_bdw3.assign(3 * std::max<int64_t>(nb, 1), 0.0);
    mk.h_bds3.assign(3 * std::max<int64_t>(nb, 1), 1.0);
    for (int q = 0; q < s->n_sheet; ++q) {
        const ib_sheet &sh = s->sheets[q];
        for (int32_t i = 0; i < sh.n1; ++i)
            for (int32_t a = 0; a < sh.n2; ++a) {
                const int64_t l = sh.first + (int64_t)i * sh.n2 + a;
                const int32_t slot = bslot[l];
                for (int o = -2; o <= 2; ++o) {
                    const int32_t r = i + o;
                    bn[(o + 2) * nb + slot] =
                        (r >= 0 && r < sh.n1) ? inv[sh.first + (int64_t)r * sh.n2 + a] : -1;
                }
                for (int o = -1; o <= 1; ++o) {
                    const int32_t row = i + o;
                    if (row < 1 || row > sh.n1 - 2) continue;
                    mk.h_bseg3[(o + 1) * nb + slot] = sh.seg_of_row[row];
                    mk.h_bdw3[(o + 1) * nb + slot] = sh.dw[row];
                    mk.h_bds3[(o + 1) * nb + slot] = sh.ds;
                }
            }
    }
    if (nb > 0) {
        std::vector<int32_t> bslot_i(m);
        for (int64_t l = 0; l < m; ++l) bslot_i[l] = bslot[qmap[l]];
        if ((st = upload_i(mk.bslot, bslot_i)) != IB_OK) return st;
        if ((st = upload_i(mk.bn, bn)) != IB_OK) return st;
        std::vector<double> bc = bend_coefficients(mk, s->bend_b);
        if ((st = upT(mk.bc, bc)) != IB_OK) return st;
        // stiffness gradient: unit coefficients and segments of the terms
        // centred at rows i-1, i, i+1 of every slot, and the slots of each
        // segment (by its centred term) in slot order
        std::vector<double> bunit(3 * nb, 0.0);
        std::vector<int32_t> bseg(3 * nb, -1), soff(s->n_seg + 1, 0);
        for (int64_t q = 0; q < 3 * nb; ++q) {
            const int32_t sg = mk.h_bseg3[q];
            if (sg < 0) continue;
            const double ds = mk.h_bds3[q];
            bunit[q] = mk.h_bdw3[q] / (ds * ds * ds);
            bseg[q] = sg;
        }
        for (int64_t q = 0; q < nb; ++q)
            if (bseg[nb + q] >= 0) soff[bseg[nb + q] + 1]++;
        for (int32_t g = 0; g < s->n_seg; ++g) soff[g + 1] += soff[g];
        std::vector<int32_t> sslot(std::max<int32_t>(soff[s->n_seg], 1)), sfill(soff.begin(), soff.end() - 1);
        for (int64_t q = 0; q < nb; ++q)
            if (bseg[nb + q] >= 0) sslot[sfill[bseg[nb + q]]++] = (int32_t)q;
        if ((st = upload_i(mk.bunit, bunit)) != IB_OK) return st;
        if ((st = upload_i(mk.bseg, bseg)) != IB_OK) return st;
        if ((st = upload_i(mk.seg_off, soff)) != IB_OK) return st;
        if ((st = upload_i(mk.seg_slot, sslot)) != IB_OK) return st;
    }
    // forcing: per grid row, the x-range of cells in the region
    if (s->n_mforce > 0 && s->mforce_amp != 0.0) {
        c->forcing.mamp = s->mforce_amp;
        c->forcing.momega = s->mforce_omega;
    }
    const ib_forcing &fo = s->forcing;
    if (fo.amp != 0.0) {
        const auto &g = c->dim;
        std::vector<int2> rows((size_t)g.nz * g.ny, make_int2(1, 0));
        for (int k = 0; k < g.nz; ++k)
            for (int j = 0; j < g.ny; ++j) {
                int lo = -1, hi = -2;
                for (int i = 0; i < g.nx; ++i) {
                    const double d0 = h * (double)i - fo.center[0];
                    const double d1 = h * (double)j - fo.center[1];
                    const double d2 = h * (double)k - fo.center[2];
                    const double along = d0 * fo.direction[0] + d1 * fo.direction[1] + d2 * fo.direction[2];
                    const double perp2 = d0 * d0 + d1 * d1 + d2 * d2 - along * along;
                    if (std::fabs(along) <= fo.half_len && perp2 <= fo.radius * fo.radius) {
                        if (lo < 0) lo = i;
                        else if (hi != i - 1) return fail(IB_ERR_UNSUPPORTED, "forcing region not convex along x");
                        hi = i;
                    }
                }
                if (lo >= 0) rows[(size_t)k * g.ny + j] = make_int2(lo, hi);
            }
        if ((st = upload_i(c->forcing.rows, rows)) != IB_OK) return st;
        c->forcing.active = 1;
        for (int a = 0; a < 3; ++a) c->forcing.dir[a] = fo.direction[a];
        c->forcing.mag = c->desc.rho * fo.amp * fo.omega;
        c->forcing.omega = fo.omega;
    }
    {
        // keep the device's forcing factor consistent with the current time
        double tt = 0;
        CK(cudaMemcpy(&tt, c->d_time, sizeof(double), cudaMemcpyDeviceToHost));
        stage_time(c, tt);
        CK(cudaMemcpy(c->d_time, c->t_pair, sizeof c->t_pair, cudaMemcpyHostToDevice));
        ib_status st2 = upload_tparams(c);
        if (st2 != IB_OK) return st2;
    }
    // work space
    const int64_t nchunks = (m + RS_CHUNK - 1) / RS_CHUNK;
    mk.hist_len = 256 * std::max<int64_t>(nchunks, 1) + 1;
    CKM(mk.key, 4 * m);
    CKM(mk.key_alt, 4 * m);
    CKM(mk.key_s, 4 * m);
    CKM(mk.perm_alt, 4 * m);
    CKM(mk.perm, 4 * m);
    CKM(mk.hist, 4 * mk.hist_len);
    CKM(mk.rfrac, R * 3 * m);
    CKM(mk.rec, (c->fp64 ? sizeof(Record<double>) : sizeof(Record<float>)) * m);
    CKM(mk.f, R * 3 * m);
    CKM(mk.U, R * 3 * m);
    CKM(mk.Us, R * 3 * m);
    CKM(mk.Xtmp, 8 * 3 * m);
    dfree(c->items);
    dfree(c->partial);
    c->max_items = spread_max_items(c->dim, m);
    CKM(c->items, sizeof(int2) * c->max_items);
    CKM(c->partial, (size_t)R * (3 * PAD3 + 3) * c->max_items);
    const int64_t need = mk.hist_len / SCAN_TILE + 4;
    if (need > c->bscan_tmp_len) {
        dfree(c->bscan_tmp);
        CKM(c->bscan_tmp, 4 * need);
        c->bscan_tmp_len = need;
    }
    c->have_structure = true;
    return IB_OK;
}

ib_status ib_set_state(ib_ctx *c, const void *u, const double *X, double t)
{
    if (!c) return fail(IB_ERR_ARG, "ib_set_state: null context");
    if (X && !c->have_structure) return fail(IB_ERR_STATE, "ib_set_state: no structure");
    if (u) CK(copy_in(c, c->u, u, (size_t)c->elt * 3 * c->dim.G));
    const long long n = 3 * c->mk.m;
    if (X && n > 0) {
        const double *Xd = X;
        if (!on_device(c) && !(Xd = static_cast<const double *>(host_alias(X)))) {
            CK(cudaMemcpyAsync(c->mk.Xtmp, X, 8 * n, cudaMemcpyHostToDevice, c->stream));
            Xd = c->mk.Xtmp;
        }
        const int mm = (int)c->mk.m;
        if (c->fp64)
            k_set_disp<double><<<transfer_grid(mm), 256, 0, c->stream>>>(mm, c->mk.qinv, Xd, c->mk.X0, (double *)c->mk.d,
                                                                         nullptr);
        else
            k_set_disp<float><<<transfer_grid(mm), 256, 0, c->stream>>>(mm, c->mk.qinv, Xd, c->mk.X0, (float *)c->mk.d,
                                                                        (float *)c->mk.d + 3LL * mm);
        CK(cudaGetLastError());
    }
    c->t = t;
    stage_time(c, t);
    CK(cudaMemcpyAsync(c->d_time, c->t_pair, sizeof c->t_pair, cudaMemcpyHostToDevice, c->stream));
    if (u && c->qpart) {
        // the FP64 mean velocity that FP32 steps carry starts from this field
        k_mean_part<float><<<1024, 256, 0, c->stream>>>((const float *)c->u, c->dim.G, c->qpart);
        k_mean_final<<<1, 256, 0, c->stream>>>(c->qpart, 1024, c->dim.G, c->d_time + 4);
        CK(cudaGetLastError());
    }
    CK(cudaStreamSynchronize(c->stream));
    return IB_OK;
}

ib_status ib_get_state(ib_ctx *c, void *u, double *X, double *t)
{
    if (!c) return fail(IB_ERR_ARG, "ib_get_state: null context");
    if (u) CK(copy_out(c, u, c->u, (size_t)c->elt * 3 * c->dim.G));
    const long long n = 3 * c->mk.m;
    if (X && n > 0) {
        double *Xd = X;
        const bool staged = !on_device(c) && !(Xd = static_cast<double *>(host_alias(X)));
        if (staged) Xd = c->mk.Xtmp;
        const int mm = (int)c->mk.m;
        if (c->fp64)
            k_get_pos<double><<<transfer_grid(mm), 256, 0, c->stream>>>(mm, c->mk.qinv, c->mk.X0, (const double *)c->mk.d,
                                                                        nullptr, Xd);
        else
            k_get_pos<float><<<transfer_grid(mm), 256, 0, c->stream>>>(mm, c->mk.qinv, c->mk.X0, (const float *)c->mk.d,
                                                                       (const float *)c->mk.d + 3LL * mm, Xd);
        CK(cudaGetLastError());
        if (staged) CK(cudaMemcpyAsync(X, Xd, 8 * n, cudaMemcpyDeviceToHost, c->stream));
    }
    double tt = 0;
    CK(cudaMemcpyAsync(&tt, c->d_time, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->t = tt;
    if (t) *t = tt;
    return check_status(c);
}

ib_status ib_set_displacement(ib_ctx *c, const double *D)
{
    if (!c) return fail(IB_ERR_ARG, "ib_set_displacement: null context");
    if (!c->have_structure) return fail(IB_ERR_STATE, "ib_set_displacement: no structure");
    const long long n = 3 * c->mk.m;
    if (n == 0) return IB_OK;
    if (!D) return fail(IB_ERR_ARG, "ib_set_displacement: null D");
    const double *Dd = D;
    if (!on_device(c) && !(Dd = static_cast<const double *>(host_alias(D)))) {
        CK(cudaMemcpyAsync(c->mk.Xtmp, D, 8 * n, cudaMemcpyHostToDevice, c->stream));
        Dd = c->mk.Xtmp;
    }
    const int mm = (int)c->mk.m;
    if (c->fp64) k_set_d<double><<<transfer_grid(mm), 256, 0, c->stream>>>(mm, c->mk.qinv, Dd, (double *)c->mk.d, nullptr);
    else
        k_set_d<float><<<transfer_grid(mm), 256, 0, c->stream>>>(mm, c->mk.qinv, Dd, (float *)c->mk.d,
                                                                 (float *)c->mk.d + 3LL * mm);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->stream));
    return IB_OK;
}

ib_status ib_get_displacement(ib_ctx *c, double *D)
{
    if (!c) return fail(IB_ERR_ARG, "ib_get_displacement: null context");
    const long long n = 3 * c->mk.m;
    if (n > 0 && !D) return fail(IB_ERR_ARG, "ib_get_displacement: null D");
    if (n > 0) {
        double *Dd = D;
        const bool staged = !on_device(c) && !(Dd = static_cast<double *>(host_alias(D)));
        if (staged) Dd = c->mk.Xtmp;
        const int mm = (int)c->mk.m;
        if (c->fp64)
            k_get_d<double><<<transfer_grid(mm), 256, 0, c->stream>>>(mm, c->mk.qinv, (const double *)c->mk.d, nullptr, Dd);
        else
            k_get_d<float><<<transfer_grid(mm), 256, 0, c->stream>>>(mm, c->mk.qinv, (const float *)c->mk.d,
                                                                     (const float *)c->mk.d + 3LL * mm, Dd);
        CK(cudaGetLastError());
        if (staged) CK(cudaMemcpyAsync(D, Dd, 8 * n, cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    return check_status(c);
}

ib_status ib_step(ib_ctx *c, int64_t nsteps)
{
    if (!c) return fail(IB_ERR_ARG, "ib_step: null context");
    if (!c->have_structure) return fail(IB_ERR_STATE, "ib_step: call ib_set_structure first");
    if (nsteps < 0) return fail(IB_ERR_ARG, "ib_step: negative step count");
    if (nsteps == 0) return IB_OK;
    if (!c->graph) {
        // set kernel attributes outside the capture, then capture one step
        CK(cudaStreamSynchronize(c->stream));
        CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeRelaxed));
        enqueue_step(c, c->cap);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->cap, &g);
        if (e != cudaSuccess) return fail(IB_ERR_CUDA, "step capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&c->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            c->graph = nullptr;
            return fail(IB_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
        }
    }
    for (int64_t i = 0; i < nsteps; ++i) CK(cudaGraphLaunch(c->graph, c->stream));
    c->sort_from_state = true;
    return IB_OK;
}

ib_status ib_get_mean_velocity(ib_ctx *c, double *mean)
{
    if (!c || !mean) return fail(IB_ERR_ARG, "ib_get_mean_velocity: null argument");
    double *dm = c->d_time + 4;
    if (!c->qpart) {
        // FP64 contexts: the mean of the field itself, in a fixed order
        double *part = nullptr;
        CKM(part, 3 * 1024 * sizeof(double));
        k_mean_part<double><<<1024, 256, 0, c->stream>>>((const double *)c->u, c->dim.G, part);
        k_mean_final<<<1, 256, 0, c->stream>>>(part, 1024, c->dim.G, c->d_time + 4);
        cudaError_t e = cudaGetLastError();
        cudaStreamSynchronize(c->stream);
        cudaFree(part);
        if (e != cudaSuccess) return fail(IB_ERR_CUDA, "ib_get_mean_velocity: %s", cudaGetErrorString(e));
    }
    CK(cudaMemcpyAsync(mean, dm, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return IB_OK;
}

ib_status ib_get_bin_order(ib_ctx *c, int32_t *key, int32_t *perm, int32_t *internal)
{
    if (!c) return fail(IB_ERR_ARG, "ib_get_bin_order: null context");
    if (!c->have_structure) return fail(IB_ERR_STATE, "ib_get_bin_order: call ib_set_structure first");
    if (!c->sort_from_state)
        return fail(IB_ERR_STATE, "ib_get_bin_order: no sort from the context's state since the last explicit-position call");
    const int64_t m = c->mk.m;
    if (m == 0) return IB_OK;
    int32_t *tmp = nullptr;
    const bool dev = on_device(c);
    int32_t *out[3] = {key, perm, internal};
    if (!dev) {
        // stage through the context's position buffer (3m doubles = 6m int32)
        tmp = reinterpret_cast<int32_t *>(c->mk.Xtmp);
        for (int i = 0; i < 3; ++i) out[i] = (i == 0 ? key : i == 1 ? perm : internal) ? tmp + i * m : nullptr;
    }
    k_bin_order_out<<<(unsigned)((m + 255) / 256), 256, 0, c->stream>>>((int)m, c->mk.qmap, c->mk.qinv, c->mk.key,
                                                                        c->mk.perm, out[0], out[1], out[2]);
    CK(cudaGetLastError());
    if (!dev) {
        int32_t *dst[3] = {key, perm, internal};
        for (int i = 0; i < 3; ++i)
            if (dst[i]) CK(cudaMemcpyAsync(dst[i], tmp + i * m, 4 * m, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return IB_OK;
}

ib_status ib_spread(ib_ctx *c, const double *X, const void *f, void *F)
{
    if (!c || !X || !f || !F) return fail(IB_ERR_ARG, "ib_spread: null argument");
    if (!c->have_structure) return fail(IB_ERR_STATE, "ib_spread: call ib_set_structure first");
    const int64_t m = c->mk.m;
    const size_t fb = (size_t)c->elt * 3 * c->dim.G;
    const double *Xd = X;
    const void *fd = f;
    void *Fd = F;
    if (!on_device(c)) {
        ib_status st = ensure(c->Fbuf, fb);
        if (st != IB_OK) return st;
        if (m > 0) {
            CK(cudaMemcpyAsync(c->mk.Xtmp, X, 8 * 3 * m, cudaMemcpyHostToDevice, c->stream));
            CK(cudaMemcpyAsync(c->mk.f, f, (size_t)c->elt * 3 * m, cudaMemcpyHostToDevice, c->stream));
        }
        Xd = c->mk.Xtmp;
        fd = c->mk.f;
        Fd = c->Fbuf;
    }
    launch_keys_X(c, Xd, c->stream);
    launch_sort(c, c->stream);
    launch_bin_plan(c, c->stream);
    launch_records(c, 2, fd, c->stream);
    launch_spread(c, Fd, true, c->stream);
    CK(cudaGetLastError());
    if (!on_device(c)) {
        CK(cudaMemcpyAsync(F, Fd, fb, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return IB_OK;
}

ib_status ib_interp(ib_ctx *c, const double *X, const void *u, void *U)
{
    if (!c || !X || !u || !U) return fail(IB_ERR_ARG, "ib_interp: null argument");
    if (!c->have_structure) return fail(IB_ERR_STATE, "ib_interp: call ib_set_structure first");
    const int64_t m = c->mk.m;
    const size_t fb = (size_t)c->elt * 3 * c->dim.G;
    const double *Xd = X;
    const void *ud = u;
    void *Ud = U;
    if (!on_device(c)) {
        ib_status st = ensure(c->ubuf, fb);
        if (st != IB_OK) return st;
        if (m > 0) CK(cudaMemcpyAsync(c->mk.Xtmp, X, 8 * 3 * m, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(c->ubuf, u, fb, cudaMemcpyHostToDevice, c->stream));
        Xd = c->mk.Xtmp;
        ud = c->ubuf;
        Ud = c->mk.U;
    }
    launch_keys_X(c, Xd, c->stream);
    launch_sort(c, c->stream);
    launch_bin_plan(c, c->stream);
    launch_records(c, 0, nullptr, c->stream);
    launch_interp(c, ud, Ud, false, c->stream);
    CK(cudaGetLastError());
    if (!on_device(c)) {
        if (m > 0) CK(cudaMemcpyAsync(U, Ud, (size_t)c->elt * 3 * m, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return IB_OK;
}

ib_status ib_fluid_solve(ib_ctx *c, const void *u_n, const void *F, void *u_np1, void *p)
{
    if (!c || !u_n || !F || !u_np1) return fail(IB_ERR_ARG, "ib_fluid_solve: null argument");
    const size_t fb = (size_t)c->elt * 3 * c->dim.G;
    const void *ud = u_n, *Fd = F;
    void *od = u_np1, *pd = p;
    if (!on_device(c)) {
        ib_status st;
        if ((st = ensure(c->ubuf, fb)) != IB_OK) return st;
        if ((st = ensure(c->Fbuf, fb)) != IB_OK) return st;
        if (p && (st = ensure(c->p, fb / 3)) != IB_OK) return st;
        CK(cudaMemcpyAsync(c->ubuf, u_n, fb, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(c->Fbuf, F, fb, cudaMemcpyHostToDevice, c->stream));
        ud = c->ubuf;
        Fd = c->Fbuf;
        od = c->ubuf;
        pd = p ? c->p : nullptr;
    }
    launch_fluid(c, ud, Fd, od, pd, false, false, c->stream);
    CK(cudaGetLastError());
    if (!on_device(c)) {
        CK(cudaMemcpyAsync(u_np1, od, fb, cudaMemcpyDeviceToHost, c->stream));
        if (p) CK(cudaMemcpyAsync(p, pd, fb / 3, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return IB_OK;
}

ib_status ib_bin_sort(ib_ctx *c, const double *X, int32_t *key, int32_t *perm)
{
    if (!c || !X) return fail(IB_ERR_ARG, "ib_bin_sort: null argument");
    if (!c->have_structure) return fail(IB_ERR_STATE, "ib_bin_sort: call ib_set_structure first");
    const int64_t m = c->mk.m;
    const double *Xd = X;
    if (!on_device(c)) {
        if (m > 0) CK(cudaMemcpyAsync(c->mk.Xtmp, X, 8 * 3 * m, cudaMemcpyHostToDevice, c->stream));
        Xd = c->mk.Xtmp;
    }
    launch_keys_X(c, Xd, c->stream);
    launch_sort(c, c->stream);
    CK(cudaGetLastError());
    if (m > 0) {
        if (key) CK(copy_out(c, key, c->mk.key, 4 * m));
        if (perm) CK(copy_out(c, perm, c->mk.perm, 4 * m));
    }
    if (!on_device(c)) CK(cudaStreamSynchronize(c->stream));
    return IB_OK;
}

ib_status ib_adjoint_step(ib_ctx *c, const void *u_np1, const void *lam_u, const double *lam_D, void *lam_u_out,
                          double *lam_D_out, double *grad_b)
{
    if (!c) return fail(IB_ERR_ARG, "ib_adjoint_step: null context");
    if (!c->have_structure) return fail(IB_ERR_STATE, "ib_adjoint_step: call ib_set_structure first");
    if (!lam_u || !lam_u_out) return fail(IB_ERR_ARG, "ib_adjoint_step: null lam_u or lam_u_out");
    auto &mk = c->mk;
    const int64_t m = mk.m;
    if (m > 0 && (!lam_D || !lam_D_out)) return fail(IB_ERR_ARG, "ib_adjoint_step: null lam_D or lam_D_out");
    const size_t R = c->elt;
    const size_t fb = R * 3 * (size_t)c->dim.G;
    ib_status st;
    if ((st = ensure(c->adj_u1, fb)) != IB_OK) return st;
    if ((st = ensure(c->adj_lw, fb)) != IB_OK) return st;
    if (m > 0) {
        const size_t recb = c->fp64 ? sizeof(Record<double>) : sizeof(Record<float>);
        if ((st = ensure(mk.lamD, R * 3 * m)) != IB_OK) return st;
        if ((st = ensure(mk.lamDo, R * 3 * m)) != IB_OK) return st;
        if ((st = ensure(mk.rec2, recb * m)) != IB_OK) return st;
        if ((st = ensure(mk.lf_s, R * 3 * m)) != IB_OK) return st;
        if ((st = ensure(mk.lX_s, R * 3 * m)) != IB_OK) return st;
        if ((st = ensure(mk.lf, R * 3 * m)) != IB_OK) return st;
        if ((st = ensure(mk.lX, R * 3 * m)) != IB_OK) return st;
        if (mk.nb > 0 && (st = ensure(mk.gterm, 8 * mk.nb)) != IB_OK) return st;
    }
    if (mk.n_seg > 0) {
        if ((st = ensure(mk.gseg, 8 * (size_t)mk.n_seg)) != IB_OK) return st;
        CK(cudaMemsetAsync(mk.gseg, 0, 8 * (size_t)mk.n_seg, c->stream));
    }
    cudaStream_t s = c->stream;
    const bool dev = on_device(c);
    // caller inputs on the device
    const void *lu = lam_u;
    const void *u1 = u_np1;
    if (!dev) {
        if ((st = ensure(c->ubuf, fb)) != IB_OK) return st;
        CK(cudaMemcpyAsync(c->ubuf, lam_u, fb, cudaMemcpyHostToDevice, s));
        lu = c->ubuf;
        if (u_np1) {
            CK(cudaMemcpyAsync(c->adj_u1, u_np1, fb, cudaMemcpyHostToDevice, s));
            u1 = c->adj_u1;
        }
    }
    if (m > 0) {
        const double *Dd = lam_D;
        if (!dev) {
            CK(cudaMemcpyAsync(mk.Xtmp, lam_D, 8 * 3 * m, cudaMemcpyHostToDevice, s));
            Dd = mk.Xtmp;
        }
        if (c->fp64) k_set_d<double><<<transfer_grid(m), 256, 0, s>>>((int)m, mk.qinv, Dd, (double *)mk.lamD, nullptr);
        else k_set_d<float><<<transfer_grid(m), 256, 0, s>>>((int)m, mk.qinv, Dd, (float *)mk.lamD, nullptr);
    }
    // forward pieces about the current state: bins, weights, forces f^n
    launch_keys_state(c, s);
    launch_sort(c, s);
    launch_bin_plan(c, s);
    launch_records(c, 1, nullptr, s);
    if (!u1) {
        // u^{n+1} as the step computes it (body force at the current time,
        // which is not advanced)
        launch_spread(c, c->F, false, s);
        launch_fluid_mode(c, c->u, c->F, c->adj_u1, nullptr, true, FLUID_REPLAY, s);
        u1 = c->adj_u1;
    }
    // lam_u' + I^T lam_U: spread of h^3 dt lam_D, then the solve with w given
    const double h = c->desc.h;
    launch_records(c, 2, mk.lamD, s, mk.rec2, h * h * h * c->desc.dt);
    launch_spread(c, c->F, false, s, mk.rec2);
    launch_fluid_mode(c, lu, c->F, c->adj_lw, nullptr, true, FLUID_DIRECT, s);
    // grid output
    if (!dev && (st = ensure(c->Fbuf, fb)) != IB_OK) return st;
    void *luo = dev ? lam_u_out : c->Fbuf;
    launch_adv_adjoint(c, c->adj_lw, luo, s);
    // marker outputs
    if (m > 0) {
        launch_adj_markers(c, u1, c->adj_lw, s);
        double *Do = dev ? lam_D_out : mk.Xtmp;
        if (c->fp64) k_get_d<double><<<transfer_grid(m), 256, 0, s>>>((int)m, mk.qinv, (const double *)mk.lamDo, nullptr, Do);
        else k_get_d<float><<<transfer_grid(m), 256, 0, s>>>((int)m, mk.qinv, (const float *)mk.lamDo, nullptr, Do);
        if (!dev) CK(cudaMemcpyAsync(lam_D_out, Do, 8 * 3 * m, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaGetLastError());
    if (grad_b && mk.n_seg > 0) {
        if (dev) {
            launch_grad_accumulate(c, grad_b, s);
        } else {
            std::vector<double> g(mk.n_seg);
            CK(cudaMemcpyAsync(g.data(), mk.gseg, 8 * (size_t)mk.n_seg, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            for (int32_t i = 0; i < mk.n_seg; ++i) grad_b[i] += g[i];
        }
    }
    if (!dev) {
        CK(cudaMemcpyAsync(lam_u_out, luo, fb, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    CK(cudaGetLastError());
    return IB_OK;
}

int64_t ib_snapshot_bytes(const ib_ctx *c)
{
    if (!c) return -1;
    const int64_t fb = (int64_t)c->elt * 3 * c->dim.G, db = (int64_t)c->elt * 3 * c->mk.m * (c->fp64 ? 1 : 2);
    return fb + ((db + 15) / 16) * 16 + 64;
}

// snapshot layout: u [3][G] | d [3][m] internal numbering (padded to 16 bytes)
// | the device time state and the FP64 mean velocity, 8 doubles
ib_status ib_snapshot_save(ib_ctx *c, void *buf)
{
    if (!c || !buf) return fail(IB_ERR_ARG, "ib_snapshot_save: null argument");
    const size_t fb = (size_t)c->elt * 3 * c->dim.G, db = (size_t)c->elt * 3 * c->mk.m * (c->fp64 ? 1 : 2);
    char *b = static_cast<char *>(buf);
    CK(cudaMemcpyAsync(b, c->u, fb, cudaMemcpyDeviceToDevice, c->stream));
    if (db) CK(cudaMemcpyAsync(b + fb, c->mk.d, db, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(b + fb + (db + 15) / 16 * 16, c->d_time, 64, cudaMemcpyDeviceToDevice, c->stream));
    return IB_OK;
}

ib_status ib_snapshot_load(ib_ctx *c, const void *buf)
{
    if (!c || !buf) return fail(IB_ERR_ARG, "ib_snapshot_load: null argument");
    const size_t fb = (size_t)c->elt * 3 * c->dim.G, db = (size_t)c->elt * 3 * c->mk.m * (c->fp64 ? 1 : 2);
    const char *b = static_cast<const char *>(buf);
    CK(cudaMemcpyAsync(c->u, b, fb, cudaMemcpyDeviceToDevice, c->stream));
    if (db) CK(cudaMemcpyAsync(c->mk.d, b + fb, db, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_time, b + fb + (db + 15) / 16 * 16, 64, cudaMemcpyDeviceToDevice, c->stream));
    return IB_OK;
}

ib_status ib_set_bend_stiffness(ib_ctx *c, const double *bend_b)
{
    if (!c) return fail(IB_ERR_ARG, "ib_set_bend_stiffness: null context");
    if (!c->have_structure) return fail(IB_ERR_STATE, "ib_set_bend_stiffness: call ib_set_structure first");
    auto &mk = c->mk;
    if (mk.n_seg > 0 && !bend_b) return fail(IB_ERR_ARG, "ib_set_bend_stiffness: null bend_b");
    if (mk.nb == 0) return IB_OK;
    std::vector<double> b(mk.n_seg);
    if (on_device(c)) CK(cudaMemcpy(b.data(), bend_b, 8 * (size_t)mk.n_seg, cudaMemcpyDeviceToHost));
    else std::copy(bend_b, bend_b + mk.n_seg, b.begin());
    for (int32_t i = 0; i < mk.n_seg; ++i)
        if (!std::isfinite(b[i])) return fail(IB_ERR_ARG, "ib_set_bend_stiffness: bend_b[%d] is not finite", i);
    const std::vector<double> bc = bend_coefficients(mk, b.data());
    CK(cudaStreamSynchronize(c->stream));
    if (c->fp64) {
        CK(cudaMemcpy(mk.bc, bc.data(), 8 * 3 * (size_t)mk.nb, cudaMemcpyHostToDevice));
    } else {
        std::vector<float> bf(bc.begin(), bc.begin() + 3 * mk.nb);
        CK(cudaMemcpy(mk.bc, bf.data(), 4 * 3 * (size_t)mk.nb, cudaMemcpyHostToDevice));
    }
    return IB_OK;
}

const char *ib_stage_name(int32_t i) { return (i >= 0 && i < IB_NSTAGES) ? kStageNames[i] : ""; }

ib_status ib_profile(ib_ctx *c, int64_t nsteps, double *stage_ms, int64_t *active_tiles)
{
    if (!c || !stage_ms) return fail(IB_ERR_ARG, "ib_profile: null argument");
    if (!c->have_structure) return fail(IB_ERR_STATE, "ib_profile: call ib_set_structure first");
    if (nsteps < 1) return fail(IB_ERR_ARG, "ib_profile: need at least one step");
    cudaEvent_t ev[IB_NSTAGES + 1];
    for (auto &e : ev) CK(cudaEventCreate(&e));
    std::vector<double> acc(IB_NSTAGES, 0.0);
    ib_status st = IB_OK;
    for (int64_t n = 0; n < nsteps && st == IB_OK; ++n) {
        enqueue_step(c, c->stream, ev);
        cudaError_t e = cudaEventSynchronize(ev[IB_NSTAGES]);
        if (e != cudaSuccess) {
            st = fail(IB_ERR_CUDA, "ib_profile: %s", cudaGetErrorString(e));
            break;
        }
        for (int i = 0; i < IB_NSTAGES; ++i) {
            float ms = 0;
            cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
            acc[i] += ms;
        }
    }
    for (auto &e : ev) cudaEventDestroy(e);
    if (st != IB_OK) return st;
    for (int i = 0; i < IB_NSTAGES; ++i) stage_ms[i] = acc[i] / (double)nsteps;
    if (active_tiles) {
        int cnt = 0;
        CK(cudaMemcpy(&cnt, c->tile_count, sizeof(int), cudaMemcpyDeviceToHost));
        *active_tiles = cnt;
    }
    return check_status(c);
}

ib_status ib_sync(ib_ctx *c)
{
    if (!c) return fail(IB_ERR_ARG, "ib_sync: null context");
    CK(cudaStreamSynchronize(c->stream));
    return check_status(c);
}

ib_status ib_check_bounded_wait(ib_ctx *c, int32_t polls)
{
    if (!c) return fail(IB_ERR_ARG, "ib_check_bounded_wait: null context");
    if (polls < 1 || polls > (1 << 20))
        return fail(IB_ERR_ARG, "ib_check_bounded_wait: polls %d (1 .. 2^20)", (int)polls);
    launch_wait_check(c->d_status, polls, c->stream);
    CK(cudaGetLastError());
    return IB_OK;
}

}  // extern "C"
