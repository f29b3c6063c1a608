// x forward pass with staged planes (FP32): the right-hand side of Eq.
// (discreteNS1) and the real-to-complex x FFT, as k_xfwd computes them, for
// a block that marches along z.
//
// Block (blockIdx.x, blockIdx.y): rows y0 .. y0+RY-1 (y0 = blockIdx.x * RY)
// of planes z0 .. z0+ZB-1 (z0 = blockIdx.y * ZB).  A ring of XP_SLOTS plane
// slots in shared memory holds u at rows y0-1 .. y0+RY (wrapped in y) of the
// planes z-1, z, z+1 that plane z's right-hand side reads; once that is
// formed, one warp refills the slot of plane z-1 with plane z+2, a bulk
// asynchronous copy per row and component (cp.async.bulk, completing on the
// slot's mbarrier), which lands while the block runs plane z's FFT and
// stores.  Every u value a block uses then comes from shared
// memory at offsets fixed at compile time (the x, y and z neighbours of a
// thread's column are constant offsets from three slot pointers); F is read
// from global memory on touched tiles only.  The point formula (rhs_point)
// and the FFT, mean-mode partials and stores (xfwd_finish) are the ones
// k_xfwd uses, so both give the same values.
#pragma once

#include "async_copy.cuh"

namespace ibgb {

constexpr int XP_SLOTS = 3;   // planes z-1, z, z+1; after plane z's right-hand side the slot of z-1 takes z+2

template <int N, int RY> struct XPipe {
    static constexpr int ROWS = RY + 2;                  // rows y0-1 .. y0+RY
    static constexpr int SLOT = 3 * ROWS * N;            // floats per plane slot
    static constexpr int NTH = xfwd_threads<float, N, RY>();
    static constexpr size_t bytes()
    {
        return sizeof(float) * XP_SLOTS * SLOT + sizeof(float2) * (N + 3 * RY / 2 * RowAcc<N>::LEN) +
               sizeof(uint64_t) * XP_SLOTS;
    }
};

template <int N, int RY, int ZB, bool ADV>
__global__ void __launch_bounds__(XPipe<N, RY>::NTH, 3) k_xfwd_pipe(FluidArgs<float> a)
{
    PDL_ENTRY();
    using P = XPipe<N, RY>;
    static_assert(RY == 4, "one 4-row group per block (mean-mode partials)");
    constexpr int ROWS = P::ROWS, SLOT = P::SLOT, LEN = RowAcc<N>::LEN;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *slots = reinterpret_cast<float *>(smem_raw);
    float2 *tw = reinterpret_cast<float2 *>(slots + XP_SLOTS * SLOT);
    float2 *lines = tw + N;
    uint64_t *bar = reinterpret_cast<uint64_t *>(lines + 3 * RY / 2 * LEN);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int *status = a.status;
    const int ny = a.ny, nz = a.nz;
    const long long G = a.G;
    const int plane = N * ny;
    const int y0 = blockIdx.x * RY, z0 = blockIdx.y * ZB;

    if (tid < XP_SLOTS) mbar_init(&bar[tid], 1);
    if (tid == 0) mbar_init_fence();
    for (int i = tid; i < N; i += P::NTH) tw[i] = a.tw[i];
    __syncthreads();

    // plane j of the block's sequence (plane z0 - 1 + j) into slot j % XP_SLOTS:
    // lane 0 arms the barrier with the byte count, lanes 0 .. 3*ROWS-1 issue
    // one row each (warp 0)
    auto issue = [&](int j) {
        const int s = j % XP_SLOTS;
        int pz = z0 - 1 + j;
        pz = pz < 0 ? pz + nz : (pz >= nz ? pz - nz : pz);
        if (lane == 0) mbar_arrive_expect_tx(&bar[s], (uint32_t)(sizeof(float) * SLOT));
        __syncwarp();
        if (lane < 3 * ROWS) {
            const int c = lane / ROWS, r = lane - c * ROWS;
            int y = y0 - 1 + r;
            y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
            bulk_copy_g2s(slots + s * SLOT + (c * ROWS + r) * N, a.u + c * G + (long long)pz * plane + (long long)y * N,
                          (uint32_t)(sizeof(float) * N), &bar[s]);
        }
    };
    static_assert(3 * (RY + 2) <= 32, "one row per lane of warp 0");
    int issued = 0;   // planes issued so far (kept by warp 0)
    if (warp == 0) {
        fence_proxy_async_smem();
        issue(0);
        issue(1);
        issue(2);
        issued = 3;
    }
    float gl = 0.0f;
    if (a.frows && (threadIdx.x & 31) == 0) gl = (float)a.d_time[1];   // one conversion per warp
    const int wl = P::NTH - (int)(threadIdx.x & ~31u);                  // threads in this warp
    const float gcos = __shfl_sync(wl >= 32 ? 0xffffffffu : (1u << wl) - 1u, gl, 0);
    const int x = tid;
    const int xm = x == 0 ? N - 1 : x - 1, xp = x == N - 1 ? 0 : x + 1;
    bool ok = true;

    for (int k = 0; k < ZB; ++k) {
        const int z = z0 + k;
        // plane z + 1 (sequence index k + 2) was issued after the previous
        // step's right-hand side (the prologue for k = 0, 1)
        for (int j = (k == 0 ? 0 : k + 2); j <= k + 2; ++j)
            ok = ok && mbar_wait_bounded(&bar[j % XP_SLOTS], (uint32_t)((j / XP_SLOTS) & 1), status);
        if (!__syncthreads_and(ok)) break;   // a copy never landed: give up this block (flag set)

        float qacc[RY / 4][3] = {};
        if (tid < N) {
            const float *Sz = slots + ((k + 1) % XP_SLOTS) * SLOT;    // plane z
            const float *Sm = slots + (k % XP_SLOTS) * SLOT;          // plane z - 1
            const float *Sp = slots + ((k + 2) % XP_SLOTS) * SLOT;    // plane z + 1
            const bool fon =
                !a.touched || a.touched[((z / TILE) * a.nty + y0 / TILE) * a.ntx + x / TILE] != 0;
            const float *Fz = a.F + (long long)z * plane + (long long)y0 * N + x;
#pragma unroll 1
            for (int r = 0; r < RY; ++r) {
                float uc[3], dm[3][3], dp[3][3], f[3], w[3], q[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int o = (c * ROWS + r + 1) * N;   // row y0 + r of component c
                    uc[c] = Sz[o + x];
                    dm[c][0] = Sz[o + xm];
                    dp[c][0] = Sz[o + xp];
                    dm[c][1] = Sz[o - N + x];
                    dp[c][1] = Sz[o + N + x];
                    dm[c][2] = Sm[o + x];
                    dp[c][2] = Sp[o + x];
                    f[c] = 0.0f;
                    if (fon) f[c] = __ldg(Fz + c * G + r * N);
                }
                const int2 fr = a.frows ? a.frows[z * ny + y0 + r] : make_int2(1, 0);
                rhs_point<float, ADV>(a, uc, dm, dp, f, x >= fr.x && x <= fr.y, gcos, w, q);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    qacc[0][c] += q[c];   // RY = 4: one group of rows
                    float *el = reinterpret_cast<float *>(lines + (c * (RY / 2) + (r >> 1)) * LEN + RowAcc<N>()(x));
                    el[r & 1] = w[c];
                }
            }
        }
        __syncthreads();   // every read of plane z - 1 is done: its slot takes plane z + 2
        if (warp == 0 && k + 3 < ZB + 2) {
            fence_proxy_async_smem();
            issue(k + 3);
            issued = k + 4;
        }
        xfwd_finish<float, N, RY>(a, lines, tw, qacc, z, y0, tid);
        __syncthreads();   // the lines are free again
    }
    if (!ok && warp == 0) {
        // let copies still in flight land before the block's shared memory
        // is released (bounded as well)
        for (int j = 0; j < issued; ++j)
            mbar_wait_bounded(&bar[j % XP_SLOTS], (uint32_t)((j / XP_SLOTS) & 1), status, 1 << 16);
    }
}

}  // namespace ibgb
