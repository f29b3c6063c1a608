// y pass of the fluid solve (Section 3.2, step 3: the FFT that diagonalises
// Eqs. discreteNS1-2) as DFT matrix products on the tensor cores, for
// IB_FP32_TCFFT contexts with ny = 256.
//
// A y line of length 256 = 16 x 16 is transformed in two radix-16 stages,
//   Y[j2][k1] = W256^(j2 k1) sum_j1 W16^(j1 k1) x[j2 + 16 j1],
//   X[k1 + 16 k2] = sum_j2 W16^(j2 k2) Y[j2][k1],
// (W_n = exp(-2 pi i / n) forward, its conjugate inverse), each stage one
// real product D = A B^T with M = 128 rows (16 line positions x 8 columns
// of a tile), K = 32 (real and imaginary parts of the 16 inputs) and N = 32
// (real and imaginary parts of the 16 outputs): B is the real form of the
// 16-point DFT matrix, [[Re W, -Im W], [Im W, Re W]].  The operands are FP32
// values split into two BF16 parts, a = a_hi + a_lo with a_lo = bf16(a -
// a_hi), and D = A_hi B_hi + A_hi B_lo + A_lo B_hi is accumulated in FP32 in
// tensor memory by tcgen05.mma (the A_lo B_lo term, 2^-16 of the others, is
// left out).  The twiddle W256^(j2 k1) is applied in FP32 between the stages.
//
// Block: 128 threads (one accumulator row each), one 8-column tile of one
// (component, z) plane of the half spectrum at a time; tiles strided over
// the grid.  The kx = nx/2 plane's lines take the CUDA-core y pass.
#include <cuda_bf16.h>

#include "fft_core.cuh"
#include "tcgen05.cuh"

namespace ibgb {

namespace {

constexpr int TC_N = 256;                // line length
constexpr int TC_R = 16;                 // radix of both stages
constexpr int TC_LW = 8;                 // columns per tile
constexpr int TC_M = TC_R * TC_LW;       // accumulator rows (128)
constexpr int TC_K = 2 * TC_R;           // 32
constexpr uint32_t TC_LBO = 128;         // core matrices along K
constexpr uint32_t TC_SBO = 4 * 128;     // core matrices along M / N (K = 32: 4 core matrices per row group)
constexpr int TC_A_BYTES = TC_M / 8 * TC_SBO;     // 8 KB per A part
constexpr int TC_B_BYTES = TC_K / 8 * TC_SBO;     // 2 KB per B part

struct TcSmem {
    alignas(128) unsigned char ah[TC_A_BYTES];
    alignas(128) unsigned char al[TC_A_BYTES];
    alignas(128) unsigned char bh[TC_B_BYTES];
    alignas(128) unsigned char bl[TC_B_BYTES];
    float2 tw[TC_N];                     // W256^j in the pass's direction
    uint64_t bar;
    uint32_t taddr;
};

// byte offset of element (row, k) in a K-major, no-swizzle operand
__device__ __forceinline__ int op_off(int row, int k)
{
    return (row >> 3) * TC_SBO + (k >> 3) * TC_LBO + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16 &h, __nv_bfloat16 &l)
{
    h = __float2bfloat16_rn(v);
    l = __float2bfloat16_rn(v - __bfloat162float(h));
}

// 8 values of row `row` of A at columns k0 .. k0+7, hi and lo, as one
// 16-byte store each
__device__ __forceinline__ void store_chunk(TcSmem &S, int row, int k0, const float (&v)[8])
{
    __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) split_bf16(v[e], h[e], l[e]);
    const int o = op_off(row, k0);
    *reinterpret_cast<uint4 *>(S.ah + o) = *reinterpret_cast<const uint4 *>(h);
    *reinterpret_cast<uint4 *>(S.al + o) = *reinterpret_cast<const uint4 *>(l);
}

}  // namespace

// DIR = -1 forward, +1 inverse.  spec: [ncomp][nz][256][nxh] complex.
template <int DIR>
__global__ void __launch_bounds__(TC_M, 6) k_ytc(float2 *spec, int nxh, int ntiles, const float2 *twg, int *status)
{
    PDL_ENTRY();
    __shared__ TcSmem S;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) tmem_alloc(&S.taddr, 32);
    if (tid == 0) {
        mbar_init(&S.bar, 1);
        mbar_init_fence();
    }
    for (int i = tid; i < TC_N; i += TC_M) {
        const float2 w = twg[i];   // W256^i, forward
        S.tw[i] = make_float2(w.x, DIR > 0 ? -w.y : w.y);
    }
    __syncthreads();
    // B: rows n = k1 (real part of output k1) and 16 + k1 (imaginary part),
    // columns k = j1 (real part of input j1) and 16 + j1 (imaginary part)
    for (int e = tid; e < TC_K * TC_K; e += TC_M) {
        const int n = e / TC_K, k = e - n * TC_K;
        const int k1 = n & (TC_R - 1), j1 = k & (TC_R - 1);
        const float2 w = S.tw[(TC_R * j1 * k1) & (TC_N - 1)];   // W16^(j1 k1) = W256^(16 j1 k1)
        float b;
        if (n < TC_R) b = k < TC_R ? w.x : -w.y;
        else b = k < TC_R ? w.y : w.x;
        __nv_bfloat16 h, l;
        split_bf16(b, h, l);
        const int o = op_off(n, k);
        *reinterpret_cast<__nv_bfloat16 *>(S.bh + o) = h;
        *reinterpret_cast<__nv_bfloat16 *>(S.bl + o) = l;
    }
    fence_proxy_async_smem();
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t taddr = S.taddr;
    const uint32_t trow = taddr + ((uint32_t)(32 * warp) << 16);   // this warp's 32 accumulator rows
    constexpr uint32_t idesc = umma_idesc_bf16(TC_M, TC_K);
    const uint64_t dah = umma_desc(S.ah, TC_LBO, TC_SBO), dal = umma_desc(S.al, TC_LBO, TC_SBO);
    const uint64_t dbh = umma_desc(S.bh, TC_LBO, TC_SBO), dbl = umma_desc(S.bl, TC_LBO, TC_SBO);
    // K = 32 in two MMAs of K = 16: the second starts two core matrices on
    // (256 bytes, 16 in the descriptor's address units)
    auto mma3 = [&]() {
        if (tid == 0) {
            tc_fence_after_sync();
#pragma unroll
            for (int kb = 0; kb < 2; ++kb) {
                const uint64_t off = (uint64_t)(kb * 2 * TC_LBO) >> 4;
                umma_bf16(taddr, dah + off, dbh + off, idesc, kb > 0);
                umma_bf16(taddr, dah + off, dbl + off, idesc, true);
                umma_bf16(taddr, dal + off, dbh + off, idesc, true);
            }
            umma_commit(&S.bar);
        }
    };
    const int nkb = nxh / TC_LW;
    uint32_t phase = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int kb = tile % nkb, zc = tile / nkb;
        float2 *base = spec + (long long)zc * TC_N * nxh + kb * TC_LW;
        // stage 1: row m = (j2, l) holds x[j2 + 16 j1][l], j1 = 0..15
        {
            // inputs j1 = 8h .. 8h+7: real parts to columns 8h .., imaginary
            // parts to columns 16 + 8h ..
            const int j2 = tid >> 3, l = tid & 7;
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                float re[8], im[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const float2 v = base[(long long)(j2 + TC_R * (8 * hh + e)) * nxh + l];
                    re[e] = v.x;
                    im[e] = v.y;
                }
                store_chunk(S, tid, 8 * hh, re);
                store_chunk(S, tid, TC_R + 8 * hh, im);
            }
        }
        fence_proxy_async_smem();
        tc_fence_before_sync();
        __syncthreads();
        mma3();
        ok = mbar_wait_bounded(&S.bar, phase, status);
        phase ^= 1;
        tc_fence_after_sync();
        if (!__syncthreads_and(ok)) break;
        // twiddle, then stage 2's rows m' = (k1, l): element (k1*8 + l, j2) / (.., 16 + j2)
        {
            float v[32];
            tmem_ld32(trow, v);
            const int j2 = tid >> 3, l = tid & 7;
#pragma unroll
            for (int k1 = 0; k1 < TC_R; ++k1) {
                const float2 w = S.tw[j2 * k1];
                const float yr = v[k1] * w.x - v[TC_R + k1] * w.y;
                const float yi = v[k1] * w.y + v[TC_R + k1] * w.x;
                __nv_bfloat16 h, lo;
                const int row = k1 * TC_LW + l;
                split_bf16(yr, h, lo);
                *reinterpret_cast<__nv_bfloat16 *>(S.ah + op_off(row, j2)) = h;
                *reinterpret_cast<__nv_bfloat16 *>(S.al + op_off(row, j2)) = lo;
                split_bf16(yi, h, lo);
                *reinterpret_cast<__nv_bfloat16 *>(S.ah + op_off(row, TC_R + j2)) = h;
                *reinterpret_cast<__nv_bfloat16 *>(S.al + op_off(row, TC_R + j2)) = lo;
            }
        }
        fence_proxy_async_smem();
        tc_fence_before_sync();
        __syncthreads();
        mma3();
        ok = mbar_wait_bounded(&S.bar, phase, status);
        phase ^= 1;
        tc_fence_after_sync();
        if (!__syncthreads_and(ok)) break;
        // row m' = (k1, l) holds X[k1 + 16 k2][l], k2 = 0..15
        {
            float v[32];
            tmem_ld32(trow, v);
            const int k1 = tid >> 3, l = tid & 7;
#pragma unroll
            for (int k2 = 0; k2 < TC_R; ++k2) base[(long long)(k1 + TC_R * k2) * nxh + l] = make_float2(v[k2], v[TC_R + k2]);
        }
        tc_fence_before_sync();
        __syncthreads();   // every accumulator row is read: the next tile's MMAs may overwrite them
    }
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, 32);
}

// The main tiles of a y pass on the tensor cores (ny = 256); returns false
// when the shape is not supported (the caller takes the CUDA-core pass).
bool launch_ytc(float2 *spec, int nxh, int nz, int ncomp, const float2 *tw, int dir, int *status, int nsm,
                cudaStream_t s)
{
    if (nxh % TC_LW != 0) return false;
    const int ntiles = ncomp * nz * (nxh / TC_LW);
    const int grid = ntiles < 8 * nsm ? ntiles : 8 * nsm;
    if (dir < 0) launch_pdl(k_ytc<-1>, dim3(grid), dim3(TC_M), 0, s, spec, nxh, ntiles, tw, status);
    else launch_pdl(k_ytc<+1>, dim3(grid), dim3(TC_M), 0, s, spec, nxh, ntiles, tw, status);
    return true;
}

}  // namespace ibgb
