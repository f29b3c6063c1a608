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

// Tiles whose cells some bin's box covers (a neighbour bin or the tile's own
// bin is non-empty): flag them and append them to list (warp-aggregated
// atomics; *count must be 0 on entry).  The list's order varies from run to
// run, but each tile's sums do not depend on it.
__global__ void k_bin_touched(GridDims g, const int32_t *__restrict__ bin_start, uint8_t *__restrict__ touched,
                              int *__restrict__ list, int *__restrict__ count)
{
    PDL_ENTRY();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    uint8_t on = 0;
    if (t < g.ntiles) {
        const int tx = t % g.ntx, ty = (t / g.ntx) % g.nty, tz = t / (g.ntx * g.nty);
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
    const unsigned mask = __ballot_sync(0xffffffffu, on != 0);
    if (mask) {
        const int lane = threadIdx.x & 31;
        int base = 0;
        if (lane == 0) base = atomicAdd(count, __popc(mask));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (on) list[base + __popc(mask & ((1u << lane) - 1))] = t;
    }
}

// Scatter: one work item per warp at a time, items taken from a counter.
template <class T>
__global__ void __launch_bounds__(SC_WARPS * 32)
    k_bin_scatter(const int32_t *__restrict__ bin_start, const int32_t *__restrict__ skey,
                  const Record<T> *__restrict__ rec, const int2 *__restrict__ items, const int *__restrict__ ctl,
                  int *__restrict__ work, T *__restrict__ partial)
{
    PDL_ENTRY();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T *P = reinterpret_cast<T *>(smem_raw) + warp * PSTRIDE;
    Record<T> *st = reinterpret_cast<Record<T> *>(reinterpret_cast<T *>(smem_raw) + SC_WARPS * PSTRIDE) + warp * 32;
    const int kx = lane & 3, ky = (lane >> 2) & 3, kz0 = lane >> 4;
    const int nitems = ctl[0];
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(work, 1);
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
        constexpr int V = sizeof(Record<T>) / 16;   // float4 per record
        // batch b's records are loaded into registers (lane i: float4 i, i+32, ...)
        // one batch ahead and stored to shared memory when the batch starts
        float4 pre[V];
        int prekey = -1;
        auto fetch = [&](int b) {
            const int cnt = min(32, s1 - b);
            const float4 *src = reinterpret_cast<const float4 *>(rec + b);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const int i = lane + 32 * v;
                if (i < cnt * V) pre[v] = src[i];
            }
            prekey = lane < cnt ? skey[b + lane] : -1;
        };
        if (s0 < s1) fetch(s0);
        for (int b = s0; b < s1; b += 32) {
            const int cnt = min(32, s1 - b);
            {
                float4 *dst = reinterpret_cast<float4 *>(st);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const int i = lane + 32 * v;
                    if (i < cnt * V) dst[i] = pre[v];
                }
            }
            const int key = prekey;
            if (b + 32 < s1) fetch(b + 32);
            // order the batch by cell (ties keep lane order): bitonic sort of
            // (local cell << 5 | lane) across the warp; empty lanes sort last.
            // Markers keep their cell order within a bin while they stay in
            // the cells they were numbered in, so a batch that is already in
            // order (checked with one ballot) skips the network: same result.
            int sk = lane < cnt ? (((key & (TILE * TILE * TILE - 1)) << 5) | lane) : 0x7fffffff;
            const bool desc = sk < __shfl_up_sync(0xffffffffu, sk, 1) && lane > 0;
            if (__any_sync(0xffffffffu, desc)) {
#pragma unroll
                for (int size = 2; size <= 32; size <<= 1)
#pragma unroll
                    for (int stride = size >> 1; stride > 0; stride >>= 1) {
                        const int other = __shfl_xor_sync(0xffffffffu, sk, stride);
                        const bool up = (lane & size) == 0;
                        const bool lower = (lane & stride) == 0;
                        const int mn = min(sk, other), mx = max(sk, other);
                        sk = (lower == up) ? mn : mx;
                    }
            }
            const int slot = sk & 31;                       // staged record of the lane's marker
            const int cellk = sk >> 5;                      // its local cell
            const int prevc = __shfl_up_sync(0xffffffffu, cellk, 1);
            // lanes that start a run of equal cells within the sorted batch
            unsigned starts = __ballot_sync(0xffffffffu, lane < cnt && (lane == 0 || cellk != prevc));
            __syncwarp();
            while (starts) {
                const int j0 = __ffs(starts) - 1;
                starts &= starts - 1;
                const int j1 = starts ? __ffs(starts) - 1 : cnt;
                const int kj = __shfl_sync(0xffffffffu, cellk, j0);
                if (kj != cur) {
                    flush();
                    cur = kj;
                    lx = kj & (TILE - 1);
                    ly = (kj >> 3) & (TILE - 1);
                    lz = kj >> 6;
                    a0x = a0y = a0z = a1x = a1y = a1z = (T)0;
                }
                // markers j0 .. j1-1 (in sorted order) share the cell
#pragma unroll 4
                for (int j = j0; j < j1; ++j) {
                    const int r = __shfl_sync(0xffffffffu, slot, j);
                    const T *R = reinterpret_cast<const T *>(st + r);
                    T fr[4];
                    ld4(R + 12, fr);   // f and pad
                    const T wxy = R[kx] * R[4 + ky];
                    const T w0 = wxy * R[8 + kz0], w1 = wxy * R[10 + kz0];
                    const T fx = fr[0], fy = fr[1], fz = fr[2];
                    a0x += w0 * fx;
                    a0y += w0 * fy;
                    a0z += w0 * fz;
                    a1x += w1 * fx;
                    a1y += w1 * fy;
                    a1z += w1 * fz;
                }
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
// Along one axis, cell l of tile t lies in the box of bin t (box coordinate
// l + 1), of bin t-1 when l <= 1 (coordinate l + TILE + 1) and of bin t+1
// when l = TILE-1 (coordinate 0): coordinate l + 1 - TILE d for bin offset
// d, so a covering bin (dz, dy, dx) shifts the cell's own-box offset by
// -TILE (dz PAD^2 + dy PAD + dx).  A cell's class (lo, mid, hi along each
// axis) fixes its covering offsets; the block lists, per class, the
// non-empty covering bins in increasing (z, y, x) order with their item
// ranges and shifts, and each cell sums the partials of its class's bins in
// that order, each bin's items in order.
constexpr int GA_THREADS = 256;

template <class T>
__global__ void __launch_bounds__(GA_THREADS)
    k_bin_gather(GridDims g, const int *__restrict__ tile_list, const int *__restrict__ tile_count,
                 const int32_t *__restrict__ item_start, const T *__restrict__ partial, T *__restrict__ F, T inv_h3)
{
    static_assert(TILE == 8, "cell classes assume 8-cell tiles");
    PDL_ENTRY();
    __shared__ int2 irange[27];   // item range of neighbour bin (dz, dy, dx) + 1
    __shared__ int4 ent[27][8];   // per class: (first item, end item, offset shift, 0)
    __shared__ int nent[27];
    const int ti = blockIdx.x;
    if (ti >= *tile_count) return;
    const int t = tile_list[ti];
    const int tx = t % g.ntx, ty = (t / g.ntx) % g.nty, tz = t / (g.ntx * g.nty);
    const int tid = threadIdx.x;
    if (tid < 27) {
        const int dz = tid / 9 - 1, dy = (tid / 3) % 3 - 1, dx = tid % 3 - 1;
        const int bx = (tx + dx + g.ntx) % g.ntx, by = (ty + dy + g.nty) % g.nty, bz = (tz + dz + g.ntz) % g.ntz;
        const int b = (bz * g.nty + by) * g.ntx + bx;
        irange[tid] = make_int2(item_start[b], item_start[b + 1]);
    }
    __syncthreads();
    if (tid < 27) {
        // class (cz, cy, cx): 0 = cells 0, 1 (offsets -1, 0), 1 = cells 2 .. 6
        // (offset 0), 2 = cell 7 (offsets 0, +1)
        const int cz = tid / 9, cy = (tid / 3) % 3, cx = tid % 3;
        int n = 0;
        for (int dz = cz == 0 ? -1 : 0; dz <= (cz == 2 ? 1 : 0); ++dz)
            for (int dy = cy == 0 ? -1 : 0; dy <= (cy == 2 ? 1 : 0); ++dy)
                for (int dx = cx == 0 ? -1 : 0; dx <= (cx == 2 ? 1 : 0); ++dx) {
                    const int2 ir = irange[(dz + 1) * 9 + (dy + 1) * 3 + dx + 1];
                    if (ir.y > ir.x) ent[tid][n++] = make_int4(ir.x, ir.y, -TILE * ((dz * PAD + dy) * PAD + dx), 0);
                }
        nent[tid] = n;
    }
    __syncthreads();
    for (int cell = tid; cell < TILE * TILE * TILE; cell += GA_THREADS) {
        const int x = cell & (TILE - 1), y = (cell >> 3) & (TILE - 1), z = cell >> 6;
        const int cls = (z <= 1 ? 0 : (z == TILE - 1 ? 2 : 1)) * 9 + (y <= 1 ? 0 : (y == TILE - 1 ? 2 : 1)) * 3 +
                        (x <= 1 ? 0 : (x == TILE - 1 ? 2 : 1));
        const int o0 = ((z + 1) * PAD + y + 1) * PAD + x + 1;   // own-box offset
        const int n = nent[cls];
        T s0 = 0, s1 = 0, s2 = 0;
        for (int e = 0; e < n; ++e) {
            const int4 en = ent[cls][e];
            const T *Pe = partial + o0 + en.z;
#pragma unroll 4
            for (int i = en.x; i < en.y; ++i) {
                const T *Pi = Pe + (long long)i * PSTRIDE;
                s0 += Pi[0];
                s1 += Pi[PAD3];
                s2 += Pi[2 * PAD3];
            }
        }
        const long long q = ((long long)(tz * TILE + z) * g.ny + ty * TILE + y) * g.nx + tx * TILE + x;
        F[q] = s0 * inv_h3;
        F[g.G + q] = s1 * inv_h3;
        F[2 * g.G + q] = s2 * inv_h3;
    }
}

// Interpolation, Eq. (discreteX): U_l = sum_x u(x) delta_h(x - X_l) h^3.
// Persistent blocks take work items (bin chunks): the bin's PAD^3 box of u is
// staged in shared memory, then one thread per marker reads the marker's key
// and stencil weights from global memory and sums its 64 nodes x 3
// components from the box, (ky, kz) pairs then kx.
constexpr int IP_THREADS = 256;

template <class T>
__global__ void __launch_bounds__(IP_THREADS)
    k_bin_interp(GridDims g, const int32_t *__restrict__ bin_start, const int32_t *__restrict__ skey,
                 const Record<T> *__restrict__ rec, const int2 *__restrict__ items,
                 int *__restrict__ ctl, const T *__restrict__ u, T *__restrict__ out, T dt, int step_mode,
                 int *status)
{
    PDL_ENTRY();
    __shared__ T box[3 * PAD3];
    __shared__ int next_item;
    const int tid = threadIdx.x;
    const int nitems = ctl[0];
    const int m = g.nmark;
    constexpr int NW = IP_THREADS / 32;                  // warps
    constexpr int PPW = (3 * PAD + NW - 1) / NW;         // box planes per warp
    constexpr int PSLOT = (PAD * PAD + 31) / 32;         // plane elements per lane
    const int warp = tid >> 5, lane = tid & 31;
    int spx[PSLOT], spy[PSLOT];
#pragma unroll
    for (int j = 0; j < PSLOT; ++j) {
        const int e = min(lane + 32 * j, PAD * PAD - 1);
        spy[j] = e / PAD;
        spx[j] = e - spy[j] * PAD;
    }
    for (;;) {
        // items are taken from the counter ctl[1] (zeroed by the bin plan and
        // by the move kernel that follows)
        __syncthreads();
        if (tid == 0) next_item = atomicAdd(&ctl[1], 1);
        __syncthreads();
        const int it = next_item;
        if (it >= nitems) break;
        const int2 item = items[it];
        const int t = item.x;
        const int tx = t % g.ntx, ty = (t / g.ntx) % g.nty, tz = t / (g.ntx * g.nty);
        const int ox = tx * TILE - 1, oy = ty * TILE - 1, oz = tz * TILE - 1;
        const int s0 = bin_start[t] + item.y * CHUNK;
        const int s1 = min(s0 + CHUNK, bin_start[t + 1]);
        {
            // the box as 3*PAD planes (c, pz) of PAD*PAD values: warp w stages
            // planes w, w + NW, ...; lane slot j holds plane element
            // lane + 32 j, whose wrapped grid row/column offset is formed once
            // per item
            int roff[PSLOT];
#pragma unroll
            for (int j = 0; j < PSLOT; ++j) {
                int x = ox + spx[j], y = oy + spy[j];
                x = x < 0 ? x + g.nx : (x >= g.nx ? x - g.nx : x);
                y = y < 0 ? y + g.ny : (y >= g.ny ? y - g.ny : y);
                roff[j] = y * g.nx + x;
            }
            T v[PPW][PSLOT];
#pragma unroll
            for (int i = 0; i < PPW; ++i) {
                const int pl = warp + i * NW;
                if (pl < 3 * PAD) {
                    const int c = pl / PAD, pz = pl - c * PAD;
                    int z = oz + pz;
                    z = z < 0 ? z + g.nz : (z >= g.nz ? z - g.nz : z);
                    const T *base = u + c * g.G + (long long)z * g.ny * g.nx;
#pragma unroll
                    for (int j = 0; j < PSLOT; ++j)
                        if (lane + 32 * j < PAD * PAD) v[i][j] = __ldg(base + roff[j]);
                }
            }
#pragma unroll
            for (int i = 0; i < PPW; ++i) {
                const int pl = warp + i * NW;
                if (pl < 3 * PAD) {
#pragma unroll
                    for (int j = 0; j < PSLOT; ++j)
                        if (lane + 32 * j < PAD * PAD) box[pl * PAD * PAD + lane + 32 * j] = v[i][j];
                }
            }
        }
        __syncthreads();   // the box is staged
        // the thread's markers s0 + tid, s0 + tid + IP_THREADS, ...
        for (int p = s0 + tid; p < s1; p += IP_THREADS) {
            const int key = skey[p];
            T wx[4], wy[4], wz[4];
            const T *R = reinterpret_cast<const T *>(rec + p);
            ld4(R, wx);
            ld4(R + 4, wy);
            ld4(R + 8, wz);
            const int l = key & (TILE * TILE * TILE - 1);   // keys are >= 0
            const int lx = l & (TILE - 1), ly = (l >> 3) & (TILE - 1), lz = l >> 6;
            T acc[3] = {0, 0, 0};
            // (ky, kz) pairs i: ky = i % 4, kz = i / 4; then kx
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int ky = i & 3, kz = i >> 2;
                const T wyz = wy[ky] * wz[kz];
                const int o = ((lz + kz) * PAD + ly + ky) * PAD + lx;
#pragma unroll
                for (int kx = 0; kx < 4; ++kx) {
                    const T w = wx[kx] * wyz;
#pragma unroll
                    for (int c = 0; c < 3; ++c) acc[c] += box[c * PAD3 + o + kx] * w;
                }
            }
            // by sorted position; the move kernel applies it per marker
            bool bad = false;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (!isfinite(acc[c])) bad = true;
                out[(long long)c * m + p] = acc[c];
            }
            if (bad) atomicOr(status, DEV_NONFINITE);
        }
    }
}

// U (sorted order) -> marker order: step mode d[perm[p]] += dt * U[p], else
// Uout[perm[p]] = U[p].  With lo (FP32 contexts) the displacement is the pair
// hi + lo and the increment is added exactly (two-sum), then renormalised so
// that |lo| <= ulp(hi)/2: increments below hi's precision accumulate in lo.
template <class T>
__global__ void k_move(int m, const int32_t *__restrict__ perm, const T *__restrict__ Us, T *__restrict__ out,
                       T *__restrict__ lo, T dt, int step_mode, int *__restrict__ ctl)
{
    PDL_ENTRY();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0) ctl[1] = 0;   // the interpolation's work counter, for its next launch
    if (p >= m) return;
    const int id = perm[p];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const long long i = (long long)c * m + id;
        const T v = Us[(long long)c * m + p];
        if (!step_mode) {
            out[i] = v;
        } else if (!lo) {
            out[i] += dt * v;
        } else {
            const T a = out[i], b = dt * v;
            const T s = a + b;
            const T bb = s - a;
            const T e = (a - (s - bb)) + (b - bb) + lo[i];
            const T hi = s + e;
            out[i] = hi;
            lo[i] = e - (hi - s);
        }
    }
}

template <class T> static void interp_impl(ib_ctx *c, const void *u, void *U, bool step_mode, cudaStream_t s)
{
    if (c->mk.m == 0) return;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bin_interp<T>, IP_THREADS, 0);
    if (per_sm > 8) per_sm = 8;
    if (per_sm < 1) per_sm = 1;
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    GridDims g = c->dim;
    g.nmark = (int)c->mk.m;
    T *Us = (T *)c->mk.Us;
    launch_pdl(k_bin_interp<T>, dim3(persistent_grid(c, nsm * per_sm)), dim3(IP_THREADS), 0, s, g, c->bin_start,
               c->mk.key_s, (const Record<T> *)c->mk.rec, c->items, c->item_ctl, (const T *)u, Us,
               (T)c->desc.dt, step_mode ? 1 : 0, c->d_status);
    const int m = (int)c->mk.m;
    T *lo = (step_mode && !c->fp64) ? (T *)c->mk.d + 3LL * m : nullptr;   // U is mk.d in step mode
    launch_pdl(k_move<T>, dim3((m + 255) / 256), dim3(256), 0, s, m, c->mk.perm, Us, (T *)U, lo, (T)c->desc.dt,
               step_mode ? 1 : 0, c->item_ctl);
}

void launch_interp(ib_ctx *c, const void *u, void *U, bool step_mode, cudaStream_t s)
{
    if (c->fp64) interp_impl<double>(c, u, U, step_mode, s);
    else interp_impl<float>(c, u, U, step_mode, s);
}

template <class T> static void spread_impl(ib_ctx *c, void *F, bool dense, cudaStream_t s, const void *rec)
{
    const auto &g = c->dim;
    if (dense) cudaMemsetAsync(F, 0, sizeof(T) * 3 * (size_t)g.G, s);
    // zero the touched-tile count and the scatter's work counter (adjacent)
    cudaMemsetAsync(c->tile_count, 0, 2 * sizeof(int), s);
    launch_pdl(k_bin_touched, dim3((g.ntiles + 255) / 256), dim3(256), 0, s, g, c->bin_start, c->touched, c->tile_list, c->tile_count);
    if (c->mk.m == 0) return;
    const size_t smem = scatter_smem<T>();
    cudaFuncSetAttribute(k_bin_scatter<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bin_scatter<T>, SC_WARPS * 32, smem);
    if (per_sm < 1) per_sm = 1;
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    launch_pdl(k_bin_scatter<T>, dim3(persistent_grid(c, nsm * per_sm)), dim3(SC_WARPS * 32), smem, s, c->bin_start, c->mk.key_s,
                                                               (const Record<T> *)(rec ? rec : c->mk.rec), c->items,
                                                               c->item_ctl, c->tile_next, (T *)c->partial);
    const double h = c->desc.h;
    launch_pdl(k_bin_gather<T>, dim3(g.ntiles), dim3(GA_THREADS), 0, s, g, c->tile_list, c->tile_count, c->item_start,
               (const T *)c->partial, (T *)F, (T)(1.0 / (h * h * h)));
}

void launch_spread(ib_ctx *c, void *F, bool dense, cudaStream_t s, const void *rec)
{
    if (c->fp64) spread_impl<double>(c, F, dense, s, rec);
    else spread_impl<float>(c, F, dense, s, rec);
}

}  // namespace ibgb
