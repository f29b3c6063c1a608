// Marker-side kernels of the IB step:
//  - bin keys: the cell floor(X/h) of each marker and its fractional offset;
//  - a stable LSD radix sort of marker ids by tile (the cell key's high bits)
//    -> marker order used by spreading and interpolation (bit-exact,
//    deterministic; within a tile markers keep their id order);
//  - bucket starts: exclusive scan of per-bucket counts (a bucket is TILE
//    consecutive cells along x of one grid row);
//  - records: per sorted marker, the 4-point delta weights along x, y, z
//    (Section 3.2, definition of delta_h) and the marker force (step 1);
//  - interpolation of u at the markers (Eq. discreteX) and the position update.
#include <cstdio>

#include "ib_internal.cuh"
#include "marker_forces.cuh"

namespace ibgb {



__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }
__device__ __forceinline__ int modi(int v, int n)
{
    int r = v % n;
    return r < 0 ? r + n : r;
}

// ---------------------------------------------------------------------------
// keys
// ---------------------------------------------------------------------------
// One count per tile, aggregated over the lanes of a warp that share it.
__device__ __forceinline__ void count_tile(int key, int32_t *tile_count)
{
    const int tile = key / (TILE * TILE * TILE);
    const unsigned peers = __match_any_sync(__activemask(), tile);
    if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&tile_count[tile], __popc(peers));
}

// FP64 state: s = (X0 + d) * (1/h), one rounded add and one rounded multiply
// (as the oracle forms floor(X / h) from X = X0 + D).
// FP32 state: t = r0 + d_hi/h in single precision gives the offset from the
// reference cell cell0; floor(t) is the cell unless t lies within the single
// precision error bound of a cell face, where the cell is decided from
// s = (X0 + (d_hi + d_lo)) * (1/h) in FP64 exactly as above.  So both
// precisions take the FP64 decision, and the key equals the oracle's for the
// positions X0 + D the context holds.  A non-finite offset or one beyond
// 2^30 cells sets DEV_RANGE in *status (the cell is then meaningless).
template <class T>
__global__ void k_keys_state(int m, GridDims g, const int32_t *__restrict__ cell0, const T *__restrict__ r0,
                             const double *__restrict__ X0, const T *__restrict__ d, double inv_h, T inv_h_t,
                             int32_t *__restrict__ key, T *__restrict__ rfrac, int32_t *__restrict__ tile_count,
                             int *__restrict__ status)
{
    PDL_ENTRY();
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = l < m;
    const int n[3] = {g.nx, g.ny, g.nz};
    int b[3] = {0, 0, 0};
    T r[3] = {0, 0, 0};
    bool bad = false;
    if constexpr (sizeof(T) == 4) {
        // single precision offset from the reference cell; a lane whose offset
        // lies within the error bound of a face takes the FP64 decision below
        unsigned near = 0;
        if (valid) {
            float rr[3], dd[3];
            int cc0[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                rr[c] = r0[c * m + l];
                dd[c] = d[c * m + l];
                cc0[c] = cell0[c * m + l];
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float dh = __fmul_rn(dd[c], inv_h_t);   // 1/h rounded to FP32 on the host
                const float t = __fadd_rn(rr[c], dh);
                const float fl = floorf(t);
                const float fr = t - fl;
                // |t - (s - cell0)| <= 2^-25 (r0) + 3 * 2^-24 (|d_hi/h| + |t|) + FP64 rounding
                const float eps = 9.5367431640625e-7f * (2.0f + fabsf(t) + fabsf(dh));   // 2^-20 (...)
                if (!(fabsf(t) < 1073741824.0f)) {
                    bad = true;
                } else if (fr < eps || fr > 1.0f - eps) {
                    near |= 1u << c;
                } else {
                    b[c] = cc0[c] + (int)fl;
                    r[c] = fr;
                }
            }
        }
        // a warp-uniform branch: the FP64 work runs only in warps that need it
        if (__any_sync(0xffffffffu, near != 0) && near) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (!(near >> c & 1)) continue;
                const double D = __dadd_rn((double)d[c * m + l], (double)d[(3 + c) * m + l]);   // exact
                const double s = __dmul_rn(__dadd_rn(X0[c * m + l], D), inv_h);
                const double fs = floor(s);
                b[c] = (int)fs;
                r[c] = (float)(s - fs);
            }
        }
    } else {
        if (valid) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double s = __dmul_rn(__dadd_rn(X0[c * m + l], (double)d[c * m + l]), inv_h);
                if (!(fabs(s) < 1073741824.0)) {
                    bad = true;
                } else {
                    const double fl = floor(s);
                    b[c] = (int)fl;
                    r[c] = (T)(s - fl);
                }
            }
        }
    }
    if (!valid) return;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        b[c] = modi(b[c], n[c]);
        rfrac[c * m + l] = r[c];
    }
    if (bad) atomicOr(status, DEV_RANGE);
    const int k = tile_key(g, b[0], b[1], b[2]);
    key[l] = k;
    count_tile(k, tile_count);
}

// Explicit FP64 positions: s = X * (1/h) (one rounded multiply, as the
// oracle), base cell floor(s), fraction s - floor(s).
template <class T>
__global__ void k_keys_X(int m, GridDims g, const double *__restrict__ X, double inv_h, int32_t *__restrict__ key,
                         T *__restrict__ rfrac, int32_t *__restrict__ tile_count, int *__restrict__ status)
{
    PDL_ENTRY();
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= m) return;
    const int n[3] = {g.nx, g.ny, g.nz};
    int b[3];
    bool bad = false;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double s = __dmul_rn(X[c * m + l], inv_h);
        if (!(fabs(s) < 1073741824.0)) {
            bad = true;
            b[c] = 0;
            rfrac[c * m + l] = (T)0;
            continue;
        }
        const double fl = floor(s);
        b[c] = modi((int)fl, n[c]);
        rfrac[c * m + l] = (T)(s - fl);
    }
    if (bad) atomicOr(status, DEV_RANGE);
    const int k = tile_key(g, b[0], b[1], b[2]);
    key[l] = k;
    count_tile(k, tile_count);
}

// ---------------------------------------------------------------------------
// exclusive scan (per-block sums, then each block adds its predecessors' sums), in place, a[len] = total
// ---------------------------------------------------------------------------
constexpr int SC_THREADS = 512;
constexpr int SC_PER = 8;
constexpr int SC_TILE = SC_THREADS * SC_PER;
static_assert(SC_TILE == SCAN_TILE, "scan work space sized by SCAN_TILE");

__device__ __forceinline__ int block_excl_scan(int v, int *warp_sums, int *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) warp_sums[lane] = s;
    }
    __syncthreads();
    const int before = warp ? warp_sums[warp - 1] : 0;
    if (total) *total = warp_sums[nw - 1];
    const int r = before + x - v;
    __syncthreads();
    return r;
}

__global__ void k_scan_reduce(const int32_t *__restrict__ a, long long len, int32_t *__restrict__ part)
{
    PDL_ENTRY();
    __shared__ int ws[32];
    const long long base = (long long)blockIdx.x * SC_TILE;
    int s = 0;
    for (int i = threadIdx.x; i < SC_TILE; i += SC_THREADS) {
        const long long idx = base + i;
        if (idx < len) s += a[idx];
    }
    int tot;
    block_excl_scan(s, ws, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// Block b adds the sums of blocks 0 .. b-1 (a short reduction over part,
// done by every block instead of a separate scan launch); the last block
// also writes the total after the array.
__global__ void k_scan_apply(int32_t *__restrict__ a, long long len, const int32_t *__restrict__ part, int nblk)
{
    PDL_ENTRY();
    __shared__ int ws[32];
    int pre = 0;
    for (int i = threadIdx.x; i < (int)blockIdx.x; i += SC_THREADS) pre += part[i];
    int before;
    block_excl_scan(pre, ws, &before);
    const long long base = (long long)blockIdx.x * SC_TILE + (long long)threadIdx.x * SC_PER;
    int v[SC_PER];
    int s = 0;
#pragma unroll
    for (int j = 0; j < SC_PER; ++j) {
        v[j] = base + j < len ? a[base + j] : 0;
        s += v[j];
    }
    int total;
    int run = block_excl_scan(s, ws, &total) + before;
#pragma unroll
    for (int j = 0; j < SC_PER; ++j) {
        if (base + j < len) a[base + j] = run;
        run += v[j];
    }
    if (blockIdx.x == nblk - 1 && threadIdx.x == 0) a[len] = before + total;
}

static void scan_exclusive(int32_t *a, long long len, int32_t *tmp, cudaStream_t s)
{
    const int nblk = (int)((len + SC_TILE - 1) / SC_TILE);
    launch_pdl(k_scan_reduce, dim3(nblk), dim3(SC_THREADS), 0, s, a, len, tmp);
    launch_pdl(k_scan_apply, dim3(nblk), dim3(SC_THREADS), 0, s, a, len, tmp, nblk);
}

// ---------------------------------------------------------------------------
// stable LSD radix sort, 8-bit digits
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(RS_THREADS)
    k_radix_hist(const int32_t *__restrict__ keys, int m, int shift, int nchunks, int32_t *__restrict__ hist)
{
    PDL_ENTRY();
    __shared__ int cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int base = blockIdx.x * RS_CHUNK;
    for (int i = threadIdx.x; i < RS_CHUNK; i += RS_THREADS) {
        const int p = base + i;
        // one shared-memory atomic per distinct digit of the warp (neighbouring
        // markers often share a digit)
        const int dg = p < m ? (keys[p] >> shift) & 255 : 256;
        const unsigned peers = __match_any_sync(0xffffffffu, dg);
        if (dg < 256 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&cnt[dg], __popc(peers));
    }
    __syncthreads();
    hist[threadIdx.x * nchunks + blockIdx.x] = cnt[threadIdx.x];
}

// Chunk keys are ranked in order, 256 at a time: within a warp by a
// bit-wise ballot match on the digit, across warps by a per-digit prefix, so
// equal digits keep their input order.
__global__ void __launch_bounds__(RS_THREADS)
    k_radix_scatter(const int32_t *__restrict__ kin, const int32_t *__restrict__ vin, int m, int shift, int nchunks,
                    const int32_t *__restrict__ hscan, int32_t *__restrict__ kout, int32_t *__restrict__ vout)
{
    PDL_ENTRY();
    __shared__ int offs[256];
    __shared__ int wcnt[RS_THREADS / 32][256];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    offs[tid] = hscan[tid * nchunks + blockIdx.x];
    const int base = blockIdx.x * RS_CHUNK;
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        const int p = base + r * RS_THREADS + tid;
        const bool valid = p < m;
        const int k = valid ? kin[p] : 0;
        const int v = valid ? (vin ? vin[p] : p) : 0;
        const int dg = (k >> shift) & 255;
        unsigned peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const unsigned bb = __ballot_sync(0xffffffffu, (dg >> b) & 1);
            peers &= ((dg >> b) & 1) ? bb : ~bb;
        }
        for (int j = tid; j < (RS_THREADS / 32) * 256; j += RS_THREADS) (&wcnt[0][0])[j] = 0;
        __syncthreads();
        const int rank = __popc(peers & lt);
        if (valid && rank == 0) wcnt[warp][dg] = __popc(peers);
        __syncthreads();
        {
            int run = offs[tid];
#pragma unroll
            for (int w = 0; w < RS_THREADS / 32; ++w) {
                const int cc = wcnt[w][tid];
                wcnt[w][tid] = run;
                run += cc;
            }
            offs[tid] = run;
        }
        __syncthreads();
        if (valid) {
            const int pos = wcnt[warp][dg] + rank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
    }
}


// ---------------------------------------------------------------------------
// records: weights + forces
// ---------------------------------------------------------------------------
// phi at the four stencil nodes b-1, b, b+1, b+2 of a coordinate with
// fractional offset r = s - b in [0, 1).  With q = sqrt(1 + 4 r (1 - r)):
//   phi(r+1) = (3 - 2r - q)/8, phi(r) = (3 - 2r + q)/8,
//   phi(1-r) = (1 + 2r + q)/8, phi(2-r) = (1 + 2r - q)/8
// (the inner branch of phi at r and 1-r shares the root q; the outer
// branch is 1/2 minus the inner one).
template <class T> __device__ __forceinline__ void stencil_weights(T r, T *w)
{
    const T q = sqrt((T)1 + (T)4 * r * ((T)1 - r));
    const T e = (T)0.125;
    w[0] = ((T)3 - (T)2 * r - q) * e;
    w[1] = ((T)3 - (T)2 * r + q) * e;
    w[2] = ((T)1 + (T)2 * r + q) * e;
    w[3] = ((T)1 + (T)2 * r - q) * e;
}

// Force on marker l from the displacement field d (X = X0 + d):
//  spring (l, j): e = e0 + (d_j - d_l), r = |e|, r - L0 = (|e0|^2 - L0^2 + dd.(2 e0 + dd))/(r + L0)
//  tether: -k d_l
//  bending: -(c_{i-1} Dd_{i-1} - 2 c_i Dd_i + c_{i+1} Dd_{i+1}), Dd_x the second
//  difference of d along the line at row x (equal to v_x - v0_x);
//  external (oval window load): amp cos(omega t) dir_l, amp cos(omega t) from
//  the device time state.
template <class T> __device__ __forceinline__ void marker_force(const ForceArgs<T> &a, int l, T *f)
{
    const int m = a.m;
    const T dl[3] = {a.d[l], a.d[m + l], a.d[2 * m + l]};
    f[0] = f[1] = f[2] = 0;
    const T kt = a.tk[l];
    if (kt != (T)0) {
        f[0] -= kt * dl[0];
        f[1] -= kt * dl[1];
        f[2] -= kt * dl[2];
    }
    const int e1 = a.sp_off[l + 1];
    for (int e = a.sp_off[l]; e < e1; ++e) {
        const int j = a.sp_j[e];
        const T dd[3] = {a.d[j] - dl[0], a.d[m + j] - dl[1], a.d[2 * m + j] - dl[2]};
        const T e0[3] = {a.sp_e0[e], a.sp_e0[a.nnz + e], a.sp_e0[2 * a.nnz + e]};
        const T ee[3] = {e0[0] + dd[0], e0[1] + dd[1], e0[2] + dd[2]};
        const T r = sqrt(ee[0] * ee[0] + ee[1] * ee[1] + ee[2] * ee[2]);
        const T num = a.sp_c0[e] + (dd[0] * ((T)2 * e0[0] + dd[0]) + dd[1] * ((T)2 * e0[1] + dd[1]) +
                                    dd[2] * ((T)2 * e0[2] + dd[2]));
        const T fac = a.sp_k[e] * (num / (r + a.sp_L0[e])) / r;
        f[0] += fac * ee[0];
        f[1] += fac * ee[1];
        f[2] += fac * ee[2];
    }
    const int slot = a.bslot ? a.bslot[l] : -1;
    if (slot >= 0) {
        int nbr[5];
        T cc[3];
#pragma unroll
        for (int q = 0; q < 5; ++q) nbr[q] = a.bn[q * a.nb + slot];
#pragma unroll
        for (int q = 0; q < 3; ++q) cc[q] = a.bc[q * a.nb + slot];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            // second differences of d = hi + lo: the hi parts of neighbouring
            // markers are close, so their second difference is nearly exact and
            // the lo parts carry what hi cannot hold
            T dv[5], dl[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                dv[q] = nbr[q] >= 0 ? a.d[c * m + nbr[q]] : (T)0;
                dl[q] = (nbr[q] >= 0 && a.dlo) ? a.dlo[c * m + nbr[q]] : (T)0;
            }
            T g = 0;
            if (cc[0] != (T)0) g += cc[0] * ((dv[0] - (T)2 * dv[1] + dv[2]) + (dl[0] - (T)2 * dl[1] + dl[2]));
            if (cc[1] != (T)0) g -= (T)2 * cc[1] * ((dv[1] - (T)2 * dv[2] + dv[3]) + (dl[1] - (T)2 * dl[2] + dl[3]));
            if (cc[2] != (T)0) g += cc[2] * ((dv[2] - (T)2 * dv[3] + dv[4]) + (dl[2] - (T)2 * dl[3] + dl[4]));
            f[c] -= g;
        }
    }
    if (a.mf_dir) {
        const T amp = (T)a.d_time[2];
#pragma unroll
        for (int c = 0; c < 3; ++c) f[c] += amp * a.mf_dir[c * m + l];
    }
}

template <class T>
__device__ __forceinline__ void records_body(int m, const int32_t *__restrict__ perm, const T *__restrict__ rfrac,
                                             const ForceArgs<T> &fa, int mode, const T *__restrict__ fext, T fscale,
                                             Record<T> *__restrict__ rec)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= m) return;
    const int l = perm[p];
    Record<T> R;
#pragma unroll
    for (int c = 0; c < 3; ++c) stencil_weights<T>(rfrac[c * m + l], R.w[c]);
    if (mode == 2) {
        R.f[0] = fscale * fext[l];
        R.f[1] = fscale * fext[m + l];
        R.f[2] = fscale * fext[2 * m + l];
    } else if (mode == 1) {
        marker_force<T>(fa, l, R.f);
    } else {
        R.f[0] = R.f[1] = R.f[2] = 0;
    }
    R.pad = 0;
    rec[p] = R;
}

// FP32 (k_records): registers capped for 12 resident blocks of 128 threads
// per SM — the kernel waits on chains of dependent gathers, and more resident
// warps hide them better than the few values spilled to L1.  FP64
// (k_records_f64): the compiler's own register choice.
__global__ void __launch_bounds__(128, 12)
    k_records(int m, const int32_t *__restrict__ perm, const float *__restrict__ rfrac, ForceArgs<float> fa, int mode,
              const float *__restrict__ fext, float fscale, Record<float> *__restrict__ rec)
{
    PDL_ENTRY();
    records_body<float>(m, perm, rfrac, fa, mode, fext, fscale, rec);
}

__global__ void __launch_bounds__(128)
    k_records_f64(int m, const int32_t *__restrict__ perm, const double *__restrict__ rfrac, ForceArgs<double> fa,
                  int mode, const double *__restrict__ fext, double fscale, Record<double> *__restrict__ rec)
{
    PDL_ENTRY();
    records_body<double>(m, perm, rfrac, fa, mode, fext, fscale, rec);
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static int key_bits(long long G)
{
    int b = 1;
    while ((1LL << b) < G) ++b;
    return b;
}

// The sort orders markers by tile (the key without its low 9 cell bits);
// the full keys travel along.
constexpr int TILE_SHIFT = 9;   // log2(TILE^3)

int sort_passes(long long G)
{
    const int bits = key_bits(G) - TILE_SHIFT;
    return bits <= 0 ? 1 : (bits + 7) / 8;
}

void launch_keys_state(ib_ctx *c, cudaStream_t s)
{
    auto &mk = c->mk;
    const int m = (int)mk.m;
    c->sort_from_state = true;
    cudaMemsetAsync(c->bin_start, 0, sizeof(int32_t) * (c->dim.ntiles + 1), s);
    if (m == 0) return;
    const int nb = (m + 255) / 256;
    if (c->fp64)
        launch_pdl(k_keys_state<double>, dim3(nb), dim3(256), 0, s, m, c->dim, mk.cell0, nullptr, mk.X0,
                   (const double *)mk.d, 1.0 / c->desc.h, 1.0 / c->desc.h, mk.key, (double *)mk.rfrac, c->bin_start,
                   c->d_status);
    else
        launch_pdl(k_keys_state<float>, dim3(nb), dim3(256), 0, s, m, c->dim, mk.cell0, (const float *)mk.r0, mk.X0,
                   (const float *)mk.d, 1.0 / c->desc.h, (float)(1.0 / c->desc.h), mk.key, (float *)mk.rfrac,
                   c->bin_start, c->d_status);
}

void launch_keys_X(ib_ctx *c, const double *X, cudaStream_t s)
{
    auto &mk = c->mk;
    const int m = (int)mk.m;
    c->sort_from_state = false;
    cudaMemsetAsync(c->bin_start, 0, sizeof(int32_t) * (c->dim.ntiles + 1), s);
    if (m == 0) return;
    const int nb = (m + 255) / 256;
    if (c->fp64)
        launch_pdl(k_keys_X<double>, dim3(nb), dim3(256), 0, s, m, c->dim, X, 1.0 / c->desc.h, mk.key, (double *)mk.rfrac, c->bin_start, c->d_status);
    else
        launch_pdl(k_keys_X<float>, dim3(nb), dim3(256), 0, s, m, c->dim, X, 1.0 / c->desc.h, mk.key, (float *)mk.rfrac, c->bin_start, c->d_status);
}

void launch_sort(ib_ctx *c, cudaStream_t s)
{
    auto &mk = c->mk;
    const int m = (int)mk.m;
    if (m == 0) return;
    const int nchunks = (m + RS_CHUNK - 1) / RS_CHUNK;
    const int np = sort_passes(c->dim.G);
    int32_t *kb[2] = {mk.key_alt, mk.key_s};
    int32_t *vb[2] = {mk.perm_alt, mk.perm};
    // pass i writes buffer (np - 1 - i) % 2 so that the last pass lands in key_s / perm
    const int32_t *kin = mk.key;
    const int32_t *vin = nullptr;
    for (int i = 0; i < np; ++i) {
        const int ob = (np - 1 - i) % 2 == 0 ? 1 : 0;
        launch_pdl(k_radix_hist, dim3(nchunks), dim3(RS_THREADS), 0, s, kin, m, TILE_SHIFT + 8 * i, nchunks, mk.hist);
        scan_exclusive(mk.hist, 256LL * nchunks, c->bscan_tmp, s);
        launch_pdl(k_radix_scatter, dim3(nchunks), dim3(RS_THREADS), 0, s, kin, vin, m, TILE_SHIFT + 8 * i, nchunks, mk.hist, kb[ob],
                                                       vb[ob]);
        kin = kb[ob];
        vin = vb[ob];
    }
}

// Bin planning in two passes over the tiles (P tiles per block): per-block
// sums of the marker counts and of the chunk counts ceil(count/CHUNK); then
// (each block adding the sums of the blocks before it) bin_start /
// item_start and the spreading work items (tile, chunk) of every tile.
// ctl[0] = item count,
// ctl[1] = ctl[2] = 0 (work counters of the interpolation kernel and of the
// reverse step's marker gather).
constexpr int BP_THREADS = 256;
constexpr int BP_PER = 4;
constexpr int BP_TILES = BP_THREADS * BP_PER;

__global__ void __launch_bounds__(BP_THREADS) k_bin_sums(int ntiles, const int32_t *__restrict__ cnt, int2 *part)
{
    PDL_ENTRY();
    __shared__ int ws[32];
    int sm = 0, si = 0;
    for (int j = 0; j < BP_PER; ++j) {
        const int t = blockIdx.x * BP_TILES + threadIdx.x * BP_PER + j;
        const int c = t < ntiles ? cnt[t] : 0;
        sm += c;
        si += (c + CHUNK - 1) / CHUNK;
    }
    int tm, ti;
    block_excl_scan(sm, ws, &tm);
    block_excl_scan(si, ws, &ti);
    if (threadIdx.x == 0) part[blockIdx.x] = make_int2(tm, ti);
}

__global__ void __launch_bounds__(BP_THREADS)
    k_bin_fill(int ntiles, int nblk, const int2 *__restrict__ part, int32_t *__restrict__ bin_start,
               int32_t *__restrict__ item_start, int2 *__restrict__ items, int *__restrict__ ctl)
{
    PDL_ENTRY();
    __shared__ int ws[32];
    // sums of the blocks before this one (each block reduces part itself)
    int pm0 = 0, pi0 = 0;
    for (int i = threadIdx.x; i < (int)blockIdx.x; i += BP_THREADS) {
        pm0 += part[i].x;
        pi0 += part[i].y;
    }
    int bm, bi;
    block_excl_scan(pm0, ws, &bm);
    block_excl_scan(pi0, ws, &bi);
    int c[BP_PER];
    int sm = 0, si = 0;
    const int t0 = blockIdx.x * BP_TILES + threadIdx.x * BP_PER;
    for (int j = 0; j < BP_PER; ++j) {
        c[j] = t0 + j < ntiles ? bin_start[t0 + j] : 0;
        sm += c[j];
        si += (c[j] + CHUNK - 1) / CHUNK;
    }
    int tm, ti;
    int pm = bm + block_excl_scan(sm, ws, &tm);
    int pi = bi + block_excl_scan(si, ws, &ti);
    if ((int)blockIdx.x == nblk - 1 && threadIdx.x == 0) {
        bin_start[ntiles] = bm + tm;
        item_start[ntiles] = bi + ti;
        ctl[0] = bi + ti;
        ctl[1] = 0;
        ctl[2] = 0;
    }
    for (int j = 0; j < BP_PER; ++j) {
        if (t0 + j >= ntiles) break;
        bin_start[t0 + j] = pm;
        item_start[t0 + j] = pi;
        const int nch = (c[j] + CHUNK - 1) / CHUNK;
        for (int q = 0; q < nch; ++q) items[pi + q] = make_int2(t0 + j, q);
        pm += c[j];
        pi += nch;
    }
}

void launch_bin_plan(ib_ctx *c, cudaStream_t s)
{
    const int nt = c->dim.ntiles;
    const int nblk = (nt + BP_TILES - 1) / BP_TILES;
    int2 *part = reinterpret_cast<int2 *>(c->bscan_tmp_plan);
    launch_pdl(k_bin_sums, dim3(nblk), dim3(BP_THREADS), 0, s, nt, c->bin_start, part);
    launch_pdl(k_bin_fill, dim3(nblk), dim3(BP_THREADS), 0, s, nt, nblk, part, c->bin_start, c->item_start, c->items,
               c->item_ctl);
}

void radix_sort_raw(const int32_t *key, int m, long long G, int32_t *kbuf0, int32_t *kbuf1, int32_t *vbuf0,
                    int32_t *vout, int32_t *hist, int32_t *scan_tmp, cudaStream_t s)
{
    if (m <= 0) return;
    const int nchunks = (m + RS_CHUNK - 1) / RS_CHUNK;
    const int np = sort_passes(G);
    int32_t *kb[2] = {kbuf0, kbuf1};
    int32_t *vb[2] = {vbuf0, vout};
    const int32_t *kin = key;
    const int32_t *vin = nullptr;
    for (int i = 0; i < np; ++i) {
        const int ob = (np - 1 - i) % 2 == 0 ? 1 : 0;
        launch_pdl(k_radix_hist, dim3(nchunks), dim3(RS_THREADS), 0, s, kin, m, TILE_SHIFT + 8 * i, nchunks, hist);
        scan_exclusive(hist, 256LL * nchunks, scan_tmp, s);
        launch_pdl(k_radix_scatter, dim3(nchunks), dim3(RS_THREADS), 0, s, kin, vin, m, TILE_SHIFT + 8 * i, nchunks, hist, kb[ob], vb[ob]);
        kin = kb[ob];
        vin = vb[ob];
    }
}

void launch_records(ib_ctx *c, int mode, const void *f, cudaStream_t s, void *rec, double fscale)
{
    auto &mk = c->mk;
    const int m = (int)mk.m;
    if (m == 0) return;
    if (!rec) rec = mk.rec;
    const int nb = (m + 127) / 128;
    if (c->fp64)
        launch_pdl(k_records_f64, dim3(nb), dim3(128), 0, s, m, mk.perm, (const double *)mk.rfrac, force_args<double>(c), mode,
                                             (const double *)f, fscale, (Record<double> *)rec);
    else
        launch_pdl(k_records, dim3(nb), dim3(128), 0, s, m, mk.perm, (const float *)mk.rfrac, force_args<float>(c), mode,
                                            (const float *)f, (float)fscale, (Record<float> *)rec);
}


}  // namespace ibgb
