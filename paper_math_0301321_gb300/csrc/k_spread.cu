// Force spreading, Eq. (discreteF): F(x) = sum_l f_l delta_h(x - X_l).
//
// Atomic-free and deterministic.  The grid is cut into TILE^3 tiles; one
// block owns a tile and gathers every marker whose 4-point stencil reaches
// it, i.e. whose base cell b = floor(X/h) lies in [lo-2, lo+TILE]^3.  Markers
// were counting-sorted by cell, and the cells of one grid row are bucketed by
// TILE along x, so the candidates of a tile are 11 x 11 rows x 3 buckets of
// contiguous sorted positions.  Each warp takes a fixed contiguous share of
// the candidates, stages their records in shared memory 32 at a time, sums
// runs of markers in the same cell in registers (lane = 2 stencil nodes) and
// adds each run to its own private copy of the tile; the copies are summed
// in fixed order at the end.  The sum order depends only on the sorted
// marker order, so the result is bitwise reproducible.
//
// The tile the spreading region of some marker reaches were flagged when the
// keys were computed; a compacted list of them feeds a persistent grid.
#include "ib_internal.cuh"

namespace ibgb {

constexpr int SP_WARPS = 8;
constexpr int SP_THREADS = SP_WARPS * 32;
constexpr int SP_ZS = TILE * TILE + 4;      // padded z-plane stride (bank-conflict free)
constexpr int SP_CS = TILE * SP_ZS;         // one component of a tile copy
constexpr int SP_PRIV = 3 * SP_CS;          // one warp's copy
constexpr int SP_REG = TILE + 3;            // candidate base cells per axis: lo-2 .. lo+TILE
constexpr int SP_NR = SP_REG * SP_REG * 3;  // (row, bucket) ranges per tile

template <class T> static size_t spread_smem() { return sizeof(T) * SP_WARPS * SP_PRIV + sizeof(Record<T>) * SP_WARPS * 32; }

// single block: list of flagged tiles in index order, count in *count
__global__ void __launch_bounds__(1024) k_tile_list(const uint8_t *__restrict__ on, int ntiles, int *list, int *count,
                                                    int *next)
{
    __shared__ int ws[32];
    __shared__ int carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    constexpr int PER = 32;
    for (int base = 0; base < ntiles; base += 1024 * PER) {
        const int t0 = base + tid * PER;
        int cnt = 0;
        for (int j = 0; j < PER; ++j) cnt += (t0 + j < ntiles && on[t0 + j]) ? 1 : 0;
        int x = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) ws[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int s = ws[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            ws[lane] = s;
        }
        __syncthreads();
        int pos = carry + (warp ? ws[warp - 1] : 0) + x - cnt;
        for (int j = 0; j < PER; ++j)
            if (t0 + j < ntiles && on[t0 + j]) list[pos++] = t0 + j;
        __syncthreads();
        if (tid == 0) carry += ws[31];
        __syncthreads();
    }
    if (tid == 0) {
        *count = carry;
        *next = 0;
    }
}

template <class T>
__global__ void __launch_bounds__(SP_THREADS)
    k_spread(GridDims g, const int32_t *__restrict__ bstart, const int32_t *__restrict__ skey,
             const Record<T> *__restrict__ rec, T *__restrict__ F, const int *__restrict__ tile_list,
             const int *__restrict__ tile_count, int *tile_next, T inv_h3)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *priv = reinterpret_cast<T *>(smem_raw);
    Record<T> *stage = reinterpret_cast<Record<T> *>(priv + SP_WARPS * SP_PRIV);
    __shared__ int r_start[SP_NR];
    __shared__ int r_pref[SP_NR + 1];
    __shared__ int4 r_meta[SP_NR];   // row base key, dx offset, packed (dy+2, dz+2)
    __shared__ int s_tile;
    __shared__ int ws[32];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int kx = lane & 3, ky = (lane >> 2) & 3, kz0 = lane >> 4;
    const int ntile_active = *tile_count;
    T *P = priv + warp * SP_PRIV;
    Record<T> *st = stage + warp * 32;

    for (;;) {
        if (tid == 0) s_tile = atomicAdd(tile_next, 1);
        __syncthreads();
        const int ti = s_tile;
        if (ti >= ntile_active) break;
        const int tile = tile_list[ti];
        const int tx = tile % g.ntx, ty = (tile / g.ntx) % g.nty, tz = tile / (g.ntx * g.nty);

        // candidate ranges: rows (dz, dy) of the region, buckets tx-1, tx, tx+1
        int len2[2] = {0, 0};
        for (int q = 0; q < 2; ++q) {
            const int r = tid * 2 + q;
            if (r < SP_NR) {
                const int bi = r % 3, row = r / 3, dyi = row % SP_REG, dzi = row / SP_REG;
                int y = ty * TILE + dyi - 2, z = tz * TILE + dzi - 2;
                y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
                z = z < 0 ? z + nz : (z >= nz ? z - nz : z);
                int xb = tx + bi - 1, adj = 0;
                if (xb < 0) {
                    xb += g.nbx;
                    adj = -nx;
                } else if (xb >= g.nbx) {
                    xb -= g.nbx;
                    adj = nx;
                }
                const long long bucket = ((long long)z * ny + y) * g.nbx + xb;
                const int s0 = bstart[bucket], s1 = bstart[bucket + 1];
                r_start[r] = s0;
                len2[q] = s1 - s0;
                r_meta[r] = make_int4((z * ny + y) * nx, -tx * TILE + adj, dyi | (dzi << 8), 0);
            }
        }
        {
            // exclusive scan of the range lengths (2 per thread)
            const int v = len2[0] + len2[1];
            int x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) ws[warp] = x;
            __syncthreads();
            if (warp == 0) {
                int s = lane < SP_WARPS ? ws[lane] : 0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, s, o);
                    if (lane >= o) s += y;
                }
                if (lane < SP_WARPS) ws[lane] = s;
            }
            __syncthreads();
            const int ex = (warp ? ws[warp - 1] : 0) + x - v;
            if (tid * 2 < SP_NR) r_pref[tid * 2] = ex;
            if (tid * 2 + 1 < SP_NR) r_pref[tid * 2 + 1] = ex + len2[0];
            if (tid == 0) r_pref[SP_NR] = ws[SP_WARPS - 1];
        }
        for (int i = tid; i < SP_WARPS * SP_PRIV; i += SP_THREADS) priv[i] = (T)0;
        __syncthreads();
        const int total = r_pref[SP_NR];

        // this warp's share of the candidates
        const int v0 = (int)((long long)total * warp / SP_WARPS);
        const int v1 = (int)((long long)total * (warp + 1) / SP_WARPS);
        int cur_key = -1, cdx = 0, cdy = 0, cdz = 0;
        T a0x = 0, a0y = 0, a0z = 0, a1x = 0, a1y = 0, a1z = 0;
        auto flush = [&]() {
            if (cur_key < 0) return;
            const int xr = cdx + kx - 1, yr = cdy + ky - 1, z0 = cdz + kz0 - 1, z1 = z0 + 2;
            if ((unsigned)xr < (unsigned)TILE && (unsigned)yr < (unsigned)TILE) {
                if ((unsigned)z0 < (unsigned)TILE) {
                    const int o = z0 * SP_ZS + yr * TILE + xr;
                    P[o] += a0x;
                    P[SP_CS + o] += a0y;
                    P[2 * SP_CS + o] += a0z;
                }
                if ((unsigned)z1 < (unsigned)TILE) {
                    const int o = z1 * SP_ZS + yr * TILE + xr;
                    P[o] += a1x;
                    P[SP_CS + o] += a1y;
                    P[2 * SP_CS + o] += a1z;
                }
            }
            __syncwarp();
        };
        for (int vb = v0; vb < v1; vb += 32) {
            const int v = vb + lane;
            int key = -1, coords = 0;
            bool inreg = false;
            int p = 0;
            if (v < v1) {
                int lo = 0, hi = SP_NR;   // largest r with r_pref[r] <= v
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (r_pref[mid] <= v) lo = mid;
                    else hi = mid;
                }
                const int r = lo;
                p = r_start[r] + (v - r_pref[r]);
                key = skey[p];
                const int4 mt = r_meta[r];
                const int dx = key - mt.x + mt.y;
                inreg = dx >= -2 && dx <= TILE;
                coords = (dx + 2) | ((mt.z & 255) << 8) | ((mt.z >> 8) << 16);
            }
            if (inreg) st[lane] = rec[p];
            unsigned msk = __ballot_sync(0xffffffffu, inreg);
            __syncwarp();
            while (msk) {
                const int j = __ffs(msk) - 1;
                msk &= msk - 1;
                const int kj = __shfl_sync(0xffffffffu, key, j);
                const int cj = __shfl_sync(0xffffffffu, coords, j);
                if (kj != cur_key) {
                    flush();
                    cur_key = kj;
                    cdx = (cj & 255) - 2;
                    cdy = ((cj >> 8) & 255) - 2;
                    cdz = ((cj >> 16) & 255) - 2;
                    a0x = a0y = a0z = a1x = a1y = a1z = (T)0;
                }
                const T *R = reinterpret_cast<const T *>(st + j);
                const T wxy = R[kx] * R[4 + ky];
                const T w0 = wxy * R[8 + kz0], w1 = wxy * R[10 + kz0];
                const T fx = R[12], fy = R[13], fz = R[14];
                a0x += w0 * fx;
                a0y += w0 * fy;
                a0z += w0 * fz;
                a1x += w1 * fx;
                a1y += w1 * fy;
                a1z += w1 * fz;
            }
            __syncwarp();
        }
        flush();
        __syncthreads();

        // sum the private copies in fixed order and store the tile
        for (int idx = tid; idx < 3 * TILE * TILE * TILE; idx += SP_THREADS) {
            const int c = idx / (TILE * TILE * TILE), cell = idx - c * (TILE * TILE * TILE);
            const int z = cell / (TILE * TILE), y = (cell / TILE) % TILE, x = cell % TILE;
            const int o = c * SP_CS + z * SP_ZS + y * TILE + x;
            T s = 0;
#pragma unroll
            for (int w = 0; w < SP_WARPS; ++w) s += priv[w * SP_PRIV + o];
            F[c * g.G + ((long long)(tz * TILE + z) * ny + ty * TILE + y) * nx + tx * TILE + x] = s * inv_h3;
        }
        __syncthreads();
    }
}

template <class T> static void spread_impl(ib_ctx *c, void *F, bool dense, cudaStream_t s)
{
    const int ntiles = c->dim.ntx * c->dim.nty * c->dim.ntz;
    if (dense) cudaMemsetAsync(F, 0, sizeof(T) * 3 * (size_t)c->dim.G, s);
    k_tile_list<<<1, 1024, 0, s>>>(c->touched, ntiles, c->tile_list, c->tile_count, c->tile_next);
    if (c->mk.m == 0) return;
    const size_t smem = spread_smem<T>();
    static bool attr_set[2] = {false, false};
    if (!attr_set[sizeof(T) == 8]) {
        cudaFuncSetAttribute(k_spread<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr_set[sizeof(T) == 8] = true;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spread<T>, SP_THREADS, smem);
    if (per_sm < 1) per_sm = 1;
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    const double h = c->desc.h;
    k_spread<T><<<nsm * per_sm, SP_THREADS, smem, s>>>(c->dim, c->bcount, c->mk.key_s, (const Record<T> *)c->mk.rec,
                                                       (T *)F, c->tile_list, c->tile_count, c->tile_next,
                                                       (T)(1.0 / (h * h * h)));
}

void launch_spread(ib_ctx *c, void *F, bool dense, cudaStream_t s)
{
    if (c->fp64) spread_impl<double>(c, F, dense, s);
    else spread_impl<float>(c, F, dense, s);
}

}  // namespace ibgb
