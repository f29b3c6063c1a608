// Force spreading, Eq. (discreteF): F(x) = sum_l f_l delta_h(x - X_l).
//
// Atomic-free and deterministic, each marker handled once.
//  1. Scatter.  Markers are sorted by tile-major cell key, so the markers of
//     one TILE^3 bin are contiguous and those of one cell adjacent.  A bin is
//     cut into work items of at most CHUNK markers.  One warp takes an item:
//     it stages 32 records at a time in shared memory, sums each run of
//     same-cell markers in registers (lane = 2 of the 64 stencil nodes) and
//     adds the run into its private PAD^3 box (the bin's cells plus the
//     stencil reach: one cell below, two above), then writes the box out as
//     the item's partial.
//  2. Gather.  One block per touched tile sums, for each of its cells, the
//     partials of every item of every neighbouring bin whose box covers the
//     cell, bins in (z, y, x) order and items in order, and stores F.
// The sum order depends only on the sorted marker order, so results are
// bitwise reproducible.
#include "ib_internal.cuh"

namespace ibgb {

constexpr int SC_WARPS = 4;                  // warps per scatter block (independent)
constexpr int PSTRIDE = 3 * PAD3 + 3;        // floats per partial box (3 components, padded to 16 B)

int64_t spread_max_items(const GridDims &g, int64_t m) { return (int64_t)g.ntiles + (m + CHUNK - 1) / CHUNK; }

template <class T> static size_t scatter_smem() { return SC_WARPS * (sizeof(T) * PSTRIDE + 32 * sizeof(Record<T>)); }

// tiles whose cells some bin's box covers: a neighbour bin (or itself) is non-empty
__global__ void k_bin_touched(GridDims g, const int32_t *__restrict__ bin_start, uint8_t *__restrict__ touched)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.ntiles) return;
    const int tx = t % g.ntx, ty = (t / g.ntx) % g.nty, tz = t / (g.ntx * g.nty);
    uint8_t on = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int bx = (tx + dx + g.ntx) % g.ntx, by = (ty + dy + g.nty) % g.nty,
                          bz = (tz + dz + g.ntz) % g.ntz;
                const int b = (bz * g.nty + by) * g.ntx + bx;
                on |= bin_start[b + 1] > bin_start[b];
            }
    touched[t] = on;
}

// single block: list of flagged tiles in index order, count in *count
__global__ void __launch_bounds__(1024) k_tile_list(const uint8_t *__restrict__ on, int ntiles, int *list, int *count)
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
    if (tid == 0) *count = carry;
}

// Scatter: one work item per warp at a time, items taken from a counter.
template <class T>
__global__ void __launch_bounds__(SC_WARPS * 32)
    k_bin_scatter(const int32_t *__restrict__ bin_start, const int32_t *__restrict__ skey,
                  const Record<T> *__restrict__ rec, const int2 *__restrict__ items, int *ctl, T *__restrict__ partial)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T *P = reinterpret_cast<T *>(smem_raw) + warp * PSTRIDE;
    Record<T> *st = reinterpret_cast<Record<T> *>(reinterpret_cast<T *>(smem_raw) + SC_WARPS * PSTRIDE) + warp * 32;
    const int kx = lane & 3, ky = (lane >> 2) & 3, kz0 = lane >> 4;
    const int nitems = ctl[0];
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(&ctl[1], 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= nitems) break;
        const int2 item = items[it];
        const int s0 = bin_start[item.x] + item.y * CHUNK;
        const int s1 = min(s0 + CHUNK, bin_start[item.x + 1]);
        for (int i = lane; i < PSTRIDE; i += 32) P[i] = (T)0;
        __syncwarp();

        int cur = -1, lx = 0, ly = 0, lz = 0;
        T a0x = 0, a0y = 0, a0z = 0, a1x = 0, a1y = 0, a1z = 0;
        // add the current run into the box: node (kx, ky, kz) of cell (lx, ly, lz)
        // sits at box coordinate (lx + kx, ly + ky, lz + kz)
        auto flush = [&]() {
            if (cur < 0) return;
            const int o = ((lz + kz0) * PAD + ly + ky) * PAD + lx + kx;
            P[o] += a0x;
            P[PAD3 + o] += a0y;
            P[2 * PAD3 + o] += a0z;
            P[o + 2 * PAD * PAD] += a1x;
            P[PAD3 + o + 2 * PAD * PAD] += a1y;
            P[2 * PAD3 + o + 2 * PAD * PAD] += a1z;
            __syncwarp();
        };
        for (int b = s0; b < s1; b += 32) {
            const int cnt = min(32, s1 - b);
            // stage the batch's records (contiguous, coalesced) and keys
            {
                const float4 *src = reinterpret_cast<const float4 *>(rec + b);
                float4 *dst = reinterpret_cast<float4 *>(st);
                constexpr int V = sizeof(Record<T>) / 16;
                for (int i = lane; i < cnt * V; i += 32) dst[i] = src[i];
            }
            const int key = lane < cnt ? skey[b + lane] : -1;
            __syncwarp();
            for (int j = 0; j < cnt; ++j) {
                const int kj = __shfl_sync(0xffffffffu, key, j);
                if (kj != cur) {
                    flush();
                    cur = kj;
                    const int l = kj % (TILE * TILE * TILE);
                    lx = l % TILE;
                    ly = (l / TILE) % TILE;
                    lz = l / (TILE * TILE);
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
        T *dst = partial + (long long)it * PSTRIDE;
        for (int i = lane; i < PSTRIDE; i += 32) dst[i] = P[i];
        __syncwarp();
    }
}

// Gather: one block per touched tile; thread = cell (x fastest), all components.
template <class T>
__global__ void __launch_bounds__(256)
    k_bin_gather(GridDims g, const int *__restrict__ tile_list, const int *__restrict__ tile_count,
                 const int32_t *__restrict__ item_start, const T *__restrict__ partial, T *__restrict__ F, T inv_h3)
{
    const int ti = blockIdx.x;
    if (ti >= *tile_count) return;
    const int t = tile_list[ti];
    const int tx = t % g.ntx, ty = (t / g.ntx) % g.nty, tz = t / (g.ntx * g.nty);
    for (int cell = threadIdx.x; cell < TILE * TILE * TILE; cell += blockDim.x) {
        const int x = cell % TILE, y = (cell / TILE) % TILE, z = cell / (TILE * TILE);
        T s0 = 0, s1 = 0, s2 = 0;
        // bin t+d covers this cell at box coordinate l - TILE*d + 1 when it lies in [0, PAD)
        for (int dz = -1; dz <= 1; ++dz) {
            const int pz = z - TILE * dz + 1;
            if (pz < 0 || pz >= PAD) continue;
            for (int dy = -1; dy <= 1; ++dy) {
                const int py = y - TILE * dy + 1;
                if (py < 0 || py >= PAD) continue;
                for (int dx = -1; dx <= 1; ++dx) {
                    const int px = x - TILE * dx + 1;
                    if (px < 0 || px >= PAD) continue;
                    const int bx = (tx + dx + g.ntx) % g.ntx, by = (ty + dy + g.nty) % g.nty,
                              bz = (tz + dz + g.ntz) % g.ntz;
                    const int b = (bz * g.nty + by) * g.ntx + bx;
                    const int o = (pz * PAD + py) * PAD + px;
                    const int i1 = item_start[b + 1];
                    for (int i = item_start[b]; i < i1; ++i) {
                        const T *Pi = partial + (long long)i * PSTRIDE;
                        s0 += Pi[o];
                        s1 += Pi[PAD3 + o];
                        s2 += Pi[2 * PAD3 + o];
                    }
                }
            }
        }
        const long long q = ((long long)(tz * TILE + z) * g.ny + ty * TILE + y) * g.nx + tx * TILE + x;
        F[q] = s0 * inv_h3;
        F[g.G + q] = s1 * inv_h3;
        F[2 * g.G + q] = s2 * inv_h3;
    }
}

template <class T> static void spread_impl(ib_ctx *c, void *F, bool dense, cudaStream_t s)
{
    const auto &g = c->dim;
    if (dense) cudaMemsetAsync(F, 0, sizeof(T) * 3 * (size_t)g.G, s);
    k_bin_touched<<<(g.ntiles + 255) / 256, 256, 0, s>>>(g, c->bin_start, c->touched);
    k_tile_list<<<1, 1024, 0, s>>>(c->touched, g.ntiles, c->tile_list, c->tile_count);
    if (c->mk.m == 0) return;
    const size_t smem = scatter_smem<T>();
    cudaFuncSetAttribute(k_bin_scatter<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bin_scatter<T>, SC_WARPS * 32, smem);
    if (per_sm < 1) per_sm = 1;
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    k_bin_scatter<T><<<nsm * per_sm, SC_WARPS * 32, smem, s>>>(c->bin_start, c->mk.key_s,
                                                               (const Record<T> *)c->mk.rec, c->items, c->item_ctl,
                                                               (T *)c->partial);
    const double h = c->desc.h;
    k_bin_gather<T><<<g.ntiles, 256, 0, s>>>(g, c->tile_list, c->tile_count, c->item_start, (const T *)c->partial,
                                             (T *)F, (T)(1.0 / (h * h * h)));
}

void launch_spread(ib_ctx *c, void *F, bool dense, cudaStream_t s)
{
    if (c->fp64) spread_impl<double>(c, F, dense, s);
    else spread_impl<float>(c, F, dense, s);
}

}  // namespace ibgb
