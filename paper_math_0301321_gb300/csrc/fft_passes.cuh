// Fluid solve of Eqs. (discreteNS1)-(discreteNS2) by FFT (Section 3.2, step 3).
//
// The system is linear with constant coefficients on a periodic grid:
//   (rho/dt) u' - mu sum_k D+_k D-_k u' + D0 p = w,   D0 . u' = 0,
//   w = rho u/dt - rho sum_k u_k D+-_k u + F   (upwind advection, explicit).
// Per Fourier mode, D0 -> i s (s_j = sin(2 pi k_j/n_j)/h) and
// sum D+D- -> -(4/h^2) sum sin^2(pi k_j/n_j), so
//   u'^ = (w^ - s (s.w^)/|s|^2) / a,   p^ = -i (s.w^)/|s|^2,
//   a = rho/dt + (4 mu/h^2) sum_j sin^2(pi k_j/n_j),
// and modes with s = 0 (k_j in {0, n_j/2} for all j) are not projected.
//
// Five passes over HBM, each a batched line FFT in shared memory:
//   x-fwd  : w (upwind RHS and body force fused) -> real-to-complex along x
//            (two real rows packed as one complex line); the half spectrum
//            kx < nx/2 is stored [c][z][y][kx], the kx = nx/2 plane apart;
//   y-fwd  : complex FFT along y on column tiles;
//   z-proj : FFT along z, projection + Helmholtz factor + 1/G scaling and the
//            inverse FFT along z, all three components in one tile;
//   y-inv  : inverse FFT along y;
//   x-inv  : complex-to-real along x (two rows per complex line) -> u'.
#pragma once
#include <cstdio>

#include "fft_core.cuh"

namespace ibgb {

template <class T> struct FluidArgs {
    int nx, ny, nz;
    long long G;
    const T *u;              // [3][G]
    const T *F;              // [3][G]
    const uint8_t *touched;  // [ntiles] or null (F dense)
    int ntx, nty;
    T rho_dt, rho_h;            // rho/dt (1 for a given w), rho/h
    int advect;
    const int2 *frows;       // [nz*ny] forced x-range per row, or null
    T fdir0, fdir1, fdir2;      // body-force direction (rounded to T once, on the host)
    const double *d_time;    // [t, rho*amp*omega*cos(omega t)]
    cplx_t<T> *spec;         // [ncomp][nz][ny][nx/2]
    cplx_t<T> *nyq;          // [ncomp][nz][ny]
    const cplx_t<T> *tw;     // forward twiddles W_nx^j
    double *qpart;           // [3][nz][ny/4] sums of w - rho_dt u per 4-row group (FP32 step), or null
    int *status;             // device error flags (bounded waits)
};

template <class T> __device__ __forceinline__ T ld(const T *p) { return __ldg(p); }

// ---------------------------------------------------------------------------
// x forward: RHS + real-to-complex.  Block: RY rows (y0 .. y0+RY-1) at one z,
// all three components -> 3*RY/2 complex lines (row pairs of one component).
// ---------------------------------------------------------------------------
template <class T, int N, int RY> __host__ __device__ constexpr int xfwd_threads()
{
    return 3 * RY / 2 * tpl<N>() > N ? 3 * RY / 2 * tpl<N>() : N;
}

// The right-hand side at one grid point: w = rho_dt u - rho A(u) + F (+ the
// body force) and q = w - rho_dt u, from the point's velocity uc, its
// neighbours dm (-e_d) and dp (+e_d) per component c and axis d, and its
// force f.  A is the upwind term of Eq. (discreteNS1):
//   h A_c = sum_d u_d (u_c - u_c(-e_d)) for u_d > 0, u_d (u_c(+e_d) - u_c) otherwise,
// written as |u_d| (u_c - u_c(-s e_d)) with s the sign of u_d (the same
// product exactly: both factors only change sign), so only the upwind
// neighbour is needed (with u_d = 0 the product is zero either way).  Every
// x-pass kernel forms the right-hand side here, so every tile variant gives
// the same values.
template <class T, bool ADV>
__device__ __forceinline__ void rhs_point(const FluidArgs<T> &a, const T (&uc)[3], const T (&dm)[3][3],
                                          const T (&dp)[3][3], const T (&f)[3], bool forced, T gcos, T (&w)[3],
                                          T (&q)[3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) q[c] = f[c];
    if constexpr (ADV) {
        T A[3] = {0, 0, 0};
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const T ud = uc[d];
                const T nb = ud > (T)0 ? dm[c][d] : dp[c][d];
                A[c] += fabs(ud) * (uc[c] - nb);
            }
#pragma unroll
        for (int c = 0; c < 3; ++c) q[c] -= a.rho_h * A[c];
    }
    if (forced) {
        q[0] += gcos * a.fdir0;
        q[1] += gcos * a.fdir1;
        q[2] += gcos * a.fdir2;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) w[c] = a.rho_dt * uc[c] + q[c];
}

// Right-hand side of Eq. (discreteNS1) moved to known terms,
//   w = rho_dt u - rho A(u) + F (+ the body force),
// at column x of rows y0 .. y0+RB-1 of plane z (A the upwind term).  u at rows
// y0-1 .. y0+RB is kept in registers, so the y neighbours cost nothing; of
// the x and z neighbours only the upwind one is loaded (the sign of the
// point's u_x or u_z picks the address; L1 hits for x).  Row y0+ry is stored packed for the real-to-complex
// x FFT: line (c*cpairs + pbase + ry/2) of stride lstride, element x, real
// part for even ry, imaginary part for odd ry.
template <class T, int N, int RB, bool ADV>
__device__ __forceinline__ void rhs_column(const FluidArgs<T> &a, int z, int y0, int x, T gcos, cplx_t<T> *lines,
                                           int lstride, int cpairs, int pbase, T (&qacc)[(RB + 3) / 4][3])
{
    const int ny = a.ny, nz = a.nz;
    const int G = (int)a.G;
    const int plane = N * ny;
    {
        const int xm = x == 0 ? N - 1 : x - 1, xp = x == N - 1 ? 0 : x + 1;
        const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
        const T *U0 = a.u;
        // the block's rows lie in one tile row (RB divides TILE, y0 % RB == 0):
        // one touched-tile test serves all of them
        static_assert(TILE % RB == 0, "rows of one RHS call must share a tile");
        const bool fon = !a.touched || a.touched[((z / TILE) * a.nty + y0 / TILE) * a.ntx + x / TILE] != 0;
        T col[3][RB + 2];
#pragma unroll
        for (int r = 0; r < RB + 2; ++r) {
            int y = y0 - 1 + r;
            y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
#pragma unroll
            for (int c = 0; c < 3; ++c) col[c][r] = ld(U0 + c * G + z * plane + y * N + x);
        }
        // the loads of row ry + 1 are issued before the arithmetic of row ry
        struct RowIn {
            T nb[3][2];   // upwind x and z neighbours
            T f[3];
        };
        auto load_row = [&](int ry, RowIn &in) {
            const int y = y0 + ry;
            const int row = z * plane + y * N;
            const int ox = row + (col[0][ry + 1] > (T)0 ? xm : xp);
            const int oz = (col[2][ry + 1] > (T)0 ? zm : zp) * plane + y * N + x;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const T *Uc = U0 + c * G;
                if constexpr (ADV) {
                    in.nb[c][0] = ld(Uc + ox);
                    in.nb[c][1] = ld(Uc + oz);
                }
                // predicated: F is read on touched tiles only
                in.f[c] = (T)0;
                if (fon) in.f[c] = ld(a.F + c * G + row + x);
            }
        };
        auto row_rhs = [&](int ry, const RowIn &in) {
            T uc[3], dm[3][3], dp[3][3], w[3], q[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                // x and z: the upwind neighbour on both sides (rhs_point picks it)
                uc[c] = col[c][ry + 1];
                dm[c][0] = dp[c][0] = in.nb[c][0];
                dm[c][1] = col[c][ry];
                dp[c][1] = col[c][ry + 2];
                dm[c][2] = dp[c][2] = in.nb[c][1];
            }
            // forced x-range of the row (empty when unforced; a small table, L1 hits)
            const int2 fr = a.frows ? a.frows[z * ny + y0 + ry] : make_int2(1, 0);
            rhs_point<T, ADV>(a, uc, dm, dp, in.f, x >= fr.x && x <= fr.y, gcos, w, q);
#pragma unroll
            for (int c = 0; c < 3; ++c) qacc[ry / 4][c] += q[c];   // per group of 4 rows: the same sums whatever RB
            const int pr = ry >> 1;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                T *el = reinterpret_cast<T *>(lines + (c * cpairs + pbase + pr) * lstride + RowAcc<N>()(x));
                el[ry & 1] = w[c];
            }
        };
        static_assert(RB % 2 == 0, "rows are processed in pairs");
        RowIn ina, inb;
        load_row(0, ina);
#pragma unroll
        for (int ry = 0; ry < RB; ry += 2) {
            load_row(ry + 1, inb);
            row_rhs(ry, ina);
            if (ry + 2 < RB) load_row(ry + 2, ina);
            row_rhs(ry + 1, inb);
        }
    }
}

// FP32 at N >= 128: registers capped for about 1024 resident threads per SM
template <class T, int N, int RY> constexpr int xfwd_min_blocks()
{
    return (sizeof(T) == 4 && N >= 128) ? 1024 / xfwd_threads<T, N, RY>() : 1;
}

// The x pass after the right-hand side of rows y0 .. y0+RY-1 of plane z
// is in `lines` (all threads of the block call it): the mean-mode column
// sums, the real-to-complex FFT of the row pairs, the mean-mode partials of
// the plane's 4-row groups and the half spectrum's stores.  qacc: thread
// tid < N's sums of q over each group of 4 rows.
//
// Mean mode (FP32 step): each column's sums go to shared memory; after the
// FFT the columns are summed in FP32 in a fixed order, one value per (4-row
// group, plane) written to qpart: the same sums for every row-tile variant,
// so every variant gives the same step (the plane sums are added in FP64 by
// the z pass).
template <class T, int N, int RY>
__device__ __forceinline__ void xfwd_finish(const FluidArgs<T> &a, cplx_t<T> *lines, const cplx_t<T> *tw,
                                            const T (&qacc)[RY / 4][3], int z, int y0, int tid)
{
    using C = cplx_t<T>;
    constexpr int LPC = 3 * RY / 2;
    constexpr int TPL = tpl<N>();
    constexpr int LEN = RowAcc<N>::LEN;
    constexpr int NH = N / 2;
    constexpr int QG = RY / 4;
    constexpr int nth = xfwd_threads<T, N, RY>();
    const int ny = a.ny, nz = a.nz;
    __shared__ T qcol[QG][3][N];
    const bool want_q = a.qpart != nullptr;
    if (want_q && tid < N) {
#pragma unroll
        for (int g4 = 0; g4 < QG; ++g4)
#pragma unroll
            for (int c = 0; c < 3; ++c) qcol[g4][c][tid] = qacc[g4][c];
    }
    __syncthreads();
    {
        const int line = tid / TPL, tl = tid - line * TPL;
        fft_line<N, -1, T>(lines + (line < LPC ? line : 0) * LEN, RowAcc<N>(), tl, line < LPC, tw);
    }
    if (want_q) {
        // (fft_line ends with a barrier, so every column sum is visible.)  The
        // block's whole warps take the (4-row group, component) sums in turn:
        // lane i adds columns i*N/32 .. (i+1)*N/32 - 1 in order, a fixed
        // shuffle tree adds the lanes, lane 0 writes the sum (no barrier: the
        // other warps go on to the stores)
        static_assert(N % 32 == 0, "whole groups of 32 columns");
        constexpr int PL = N / 32;
        constexpr int NWW = nth / 32;   // whole warps
        static_assert(NWW >= 1, "one whole warp");
        const int warp = tid >> 5, lane = tid & 31;
        if (warp < NWW) {
            for (int grp = warp; grp < 3 * QG; grp += NWW) {
                const int g4 = grp / 3, c = grp - g4 * 3;
                T v = 0;
#pragma unroll
                for (int i = 0; i < PL; ++i) v += qcol[g4][c][lane * PL + i];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) {
                    // partial index: (4-row group, plane), the same for every variant
                    const long long nq = (long long)(ny / 4) * nz;
                    a.qpart[c * nq + (long long)z * (ny / 4) + y0 / 4 + g4] = (double)v;
                }
            }
        }
    }
    // Z = FFT(a + i b): A[k] = (Z[k] + conj Z[N-k])/2, B[k] = (Z[k] - conj Z[N-k])/(2i).
    // kx < N/2 go to the half spectrum (NH consecutive entries per row), kx = N/2
    // to the separate plane.
    auto unpack = [&](int line, int k, C &xa, C &xb) {
        const C *L = lines + line * LEN;
        const C zk = L[RowAcc<N>()(k)];
        const C zm = L[RowAcc<N>()(k == 0 ? 0 : N - k)];
        xa = C{(zk.x + zm.x) * (T)0.5, (zk.y - zm.y) * (T)0.5};
        xb = C{(zk.y + zm.y) * (T)0.5, (zm.x - zk.x) * (T)0.5};
    };
    constexpr int LG = nth / NH;   // lines taken at a time
    if constexpr (nth % NH == 0 && LPC % LG == 0) {
        // thread = (k, line group): its k and its smem offsets are fixed
        const int k = tid % NH, lg = tid / NH;
        const long long cst = (long long)nz * ny * NH;
        C *base = a.spec + ((long long)z * ny + y0) * NH + k;
#pragma unroll
        for (int i = 0; i < LPC / LG; ++i) {
            const int line = lg + LG * i;
            C xa, xb;
            unpack(line, k, xa, xb);
            const int c = line / (RY / 2), pr = line - c * (RY / 2);
            C *dst = base + c * cst + 2 * pr * NH;
            dst[0] = xa;
            dst[NH] = xb;
        }
    } else {
        for (int idx = tid; idx < LPC * NH; idx += nth) {
            const int line = idx / NH, k = idx - line * NH;
            C xa, xb;
            unpack(line, k, xa, xb);
            const int c = line / (RY / 2), pr = line - c * (RY / 2);
            C *dst = a.spec + (((long long)c * nz + z) * ny + y0 + 2 * pr) * NH + k;
            dst[0] = xa;
            dst[NH] = xb;
        }
    }
    if (tid < LPC) {
        const int line = tid;
        C xa, xb;
        unpack(line, NH, xa, xb);
        const int c = line / (RY / 2), pr = line - c * (RY / 2);
        C *dst = a.nyq + ((long long)c * nz + z) * ny + y0 + 2 * pr;
        dst[0] = xa;
        dst[1] = xb;
    }
}

template <class T, int N, int RY>
__global__ void __launch_bounds__(xfwd_threads<T, N, RY>(), (xfwd_min_blocks<T, N, RY>())) k_xfwd(FluidArgs<T> a)
{
    PDL_ENTRY();
    using C = cplx_t<T>;
    constexpr int LEN = RowAcc<N>::LEN;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tw = reinterpret_cast<C *>(smem_raw);
    C *lines = tw + N;
    const int tid = threadIdx.x;
    constexpr int nth = xfwd_threads<T, N, RY>();
    const int z = blockIdx.y, y0 = blockIdx.x * RY;

    for (int i = tid; i < N; i += nth) tw[i] = a.tw[i];

    // d_time[1] holds rho*amp*omega*cos(omega t) for the current time; one
    // lane per warp converts it (the FP64 pipe is slow) and shares it
    T gl = (T)0;
    if (a.frows && (tid & 31) == 0) gl = (T)a.d_time[1];
    const int wl = nth - (tid & ~31);   // threads in this warp (the block's last warp may be partial)
    const T gcos = __shfl_sync(wl >= 32 ? 0xffffffffu : (1u << wl) - 1u, gl, 0);

    // Thread x owns column x of the block's rows, taken 4 rows at a time (the
    // registers of one 4-row group; more rows per block only widen the FFT).
    static_assert(RY % 4 == 0, "rows in groups of 4");
    T qacc[RY / 4][3] = {};
    if (tid < N) {
#pragma unroll
        for (int g = 0; g < RY / 4; ++g) {
            T(&qg)[1][3] = *reinterpret_cast<T(*)[1][3]>(&qacc[g]);
            if (a.advect) rhs_column<T, N, 4, true>(a, z, y0 + 4 * g, tid, gcos, lines, LEN, RY / 2, 2 * g, qg);
            else rhs_column<T, N, 4, false>(a, z, y0 + 4 * g, tid, gcos, lines, LEN, RY / 2, 2 * g, qg);
        }
    }
    xfwd_finish<T, N, RY>(a, lines, tw, qacc, z, y0, tid);
}

}  // namespace ibgb

#include "fft_xfwd_pipe.cuh"

namespace ibgb {

// ---------------------------------------------------------------------------
// x inverse: complex-to-real.  Line (c, pair) holds Z = A + i B with A, B the
// Hermitian spectra of rows ya, ya+1; the inverse FFT gives row ya in the
// real part and row ya+1 in the imaginary part.
// ---------------------------------------------------------------------------
template <class T, int N, int RY>
__global__ void __launch_bounds__(3 * RY / 2 * tpl<N>())
    k_xinv(const cplx_t<T> *spec, const cplx_t<T> *nyq, int ncomp, int ny, int nz, T *out, const cplx_t<T> *twg,
           double *d_time, const double *tp)
{
    PDL_ENTRY();
    using C = cplx_t<T>;
    constexpr int TPL = tpl<N>();
    constexpr int LEN = RowAcc<N>::LEN;
    constexpr int NH = N / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tw = reinterpret_cast<C *>(smem_raw);
    C *lines = tw + N;
    const int lpc = ncomp * RY / 2;
    constexpr int nth = 3 * RY / 2 * TPL;
    const int tid = threadIdx.x;
    const int z = blockIdx.y, y0 = blockIdx.x * RY;
    const long long G = (long long)N * ny * nz;
    // thread = (line, q): line tid / TPL, elements q + TPL j of it (every
    // per-thread offset below is formed once; RowAcc(q + TPL j) = RowAcc(q) +
    // j * STR because TPL is a multiple of the pad period R2)
    constexpr int R2 = Plan<N>::R2;
    static_assert(TPL % R2 == 0, "pad period divides the threads per line");
    constexpr int STR = TPL + TPL / R2;
    const int line = tid / TPL, q = tid - line * TPL;
    const bool act = line < lpc;
    const int c = line / (RY / 2), pr = line - c * (RY / 2);
    C *L = lines + line * LEN;

    for (int i = tid; i < N; i += nth) tw[i] = twg[i];
    if (act) {
        // Z[k] = A[k] + i B[k] for k <= N/2 and Z[N-k] = conj A[k] + i conj B[k];
        // the imaginary parts of A, B at k = 0 and N/2 are dropped (real rows)
        constexpr int KJ = NH / TPL;
        static_assert(KJ * TPL == NH, "whole k groups");
        const C *src = spec + (((long long)c * nz + z) * ny + y0 + 2 * pr) * NH + q;
        C va[KJ], vb[KJ];
#pragma unroll
        for (int j = 0; j < KJ; ++j) {
            va[j] = src[TPL * j];
            vb[j] = src[TPL * j + NH];
        }
        const int lk = RowAcc<N>()(q);                       // RowAcc(k), k = q + TPL j
        const int lm = q == 0 ? 0 : RowAcc<N>()(TPL - q);    // RowAcc(N - k) = lm + (jm - j) STR
        const int jm = q == 0 ? N / TPL : N / TPL - 1;
#pragma unroll
        for (int j = 0; j < KJ; ++j) {
            const C xa = va[j], xb = vb[j];
            if (q == 0 && j == 0) {
                L[0] = C{xa.x, xb.x};
            } else {
                L[lk + j * STR] = C{xa.x - xb.y, xa.y + xb.x};
                L[lm + (jm - j) * STR] = C{xa.x + xb.y, xb.x - xa.y};
            }
        }
        if (q == 0) {
            const C *sn = nyq + ((long long)c * nz + z) * ny + y0 + 2 * pr;
            L[RowAcc<N>()(NH)] = C{sn[0].x, sn[1].x};
        }
    }
    __syncthreads();
    fft_line<N, +1, T>(L, RowAcc<N>(), q, act, tw);
    if (act) {
        T *dst = out + c * G + ((long long)z * ny + y0 + 2 * pr) * N + q;
        const int lk = RowAcc<N>()(q);
#pragma unroll
        for (int j = 0; j < N / TPL; ++j) {
            const C v = L[lk + j * STR];
            dst[TPL * j] = v.x;
            dst[TPL * j + N] = v.y;
        }
    }
    if (d_time && blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) {
        // tp = [dt, body amplitude, body omega, marker amplitude, marker omega]
        const double t = d_time[0] + tp[0];
        d_time[0] = t;
        d_time[1] = tp[1] * cos(tp[2] * t);
        d_time[2] = tp[3] * cos(tp[4] * t);
    }
}

// ---------------------------------------------------------------------------
// y pass, one launch for both parts of the spectrum.  Blocks [0, nmain): a
// column tile of LW consecutive kx of one (component, z) plane, element
// (line l, y) at base[y*nxh + l].  Blocks from nmain on: LW lines of the
// kx = nx/2 plane, contiguous rows nyq[c][z][:] (these few blocks run in
// the main tiles' tail instead of in a launch of their own).
// ---------------------------------------------------------------------------
template <class T, int N, int LW> __host__ __device__ constexpr size_t ypass_smem()
{
    return sizeof(cplx_t<T>) * (N + (N * LW > LW * RowAcc<N>::LEN ? N * LW : LW * RowAcc<N>::LEN));
}

template <class T, int N, int DIR, int LW>
__global__ void __launch_bounds__(LW * tpl<N>())
    k_ypass(cplx_t<T> *spec, cplx_t<T> *nyq, int nxh, int nz, int nmain, int nlines, const cplx_t<T> *twg)
{
    PDL_ENTRY();
    using C = cplx_t<T>;
    constexpr int TPL = tpl<N>();
    constexpr int LEN = RowAcc<N>::LEN;
    constexpr int nth = LW * TPL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tw = reinterpret_cast<C *>(smem_raw);
    C *work = tw + N;
    const int tid = threadIdx.x;
    for (int i = tid; i < N; i += nth) tw[i] = twg[i];
    if ((int)blockIdx.x < nmain) {
        const int nkb = nxh / LW;
        const int kb = blockIdx.x % nkb, zc = blockIdx.x / nkb;   // zc = c * nz + z
        C *base = spec + ((long long)zc * N) * nxh + kb * LW;
        {
            constexpr int PER = N * LW / nth;
            static_assert(PER * nth == N * LW, "tile must divide evenly");
            C v[PER];
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                const int idx = tid + j * nth;
                const int y = idx / LW, l = idx - y * LW;
                v[j] = base[(long long)y * nxh + l];
            }
#pragma unroll
            for (int j = 0; j < PER; ++j) work[tid + j * nth] = v[j];
        }
        __syncthreads();
        {
            const int l = tid % LW, tl = tid / LW;
            fft_line<N, DIR, T>(work + l, ColAcc<LW>(), tl, true, tw);
        }
        for (int idx = tid; idx < N * LW; idx += nth) {
            const int y = idx / LW, l = idx - y * LW;
            base[(long long)y * nxh + l] = work[idx];
        }
    } else {
        const int l0 = (blockIdx.x - nmain) * LW;
        for (int idx = tid; idx < LW * N; idx += nth) {
            const int l = idx / N, y = idx - l * N;
            if (l0 + l < nlines) work[l * LEN + RowAcc<N>()(y)] = nyq[(long long)(l0 + l) * N + y];
        }
        __syncthreads();
        {
            const int l = tid / TPL, tl = tid - l * TPL;
            fft_line<N, DIR, T>(work + l * LEN, RowAcc<N>(), tl, l0 + l < nlines, tw);
        }
        for (int idx = tid; idx < LW * N; idx += nth) {
            const int l = idx / N, y = idx - l * N;
            if (l0 + l < nlines) nyq[(long long)(l0 + l) * N + y] = work[l * LEN + RowAcc<N>()(y)];
        }
    }
}

// ---------------------------------------------------------------------------
// z pass with the projection.  LW lines (consecutive kx, or consecutive ky
// on the kx = nx/2 plane) x 3 components; element (c, l, kz) at
// base + c*cstride + kz*pitch + l.  Mode (kx, ky) of line l is
// (kx0 + l*dkx, ky0 + l*dky).  want_p: also write p^ to component 3.
// ---------------------------------------------------------------------------
// Padding (complex elements) between the components of the z pass's tile.
constexpr int ZCPAD = 8;

template <class T> struct ZArgs {
    cplx_t<T> *spec;
    cplx_t<T> *nyq;
    int nxh, ny, nz;
    long long cstride_main, cstride_nyq;
    const T *sx, *sy, *sz;      // sin(2 pi k/n)/h tables
    const T *ax, *ay, *az;      // (4 mu/h^2) sin^2(pi k/n) tables
    T rho_dt, scale;            // rho/dt, 1/G
    const cplx_t<T> *tw;        // W_nz^j
    int want_p;
    // FP64 mean mode (FP32 step): mean_mode 1 sets the k = 0 mode to
    // umean + dt_rho_G * sum(qpart) and stores that in umean, 2 the same
    // without storing (a recomputed step), 0 leaves the mode to the FFT
    int mean_mode;
    const double *qpart;        // [3][nq] per-block sums of w - rho_dt u (x pass)
    int nq;
    double *umean;              // [3] mean velocity of the state, FP64
    double dt_rho_G;            // dt / (rho G)
};

// Blocks [0, nmain) take the main spectrum's column tiles, the rest the
// kx = nx/2 plane's (one launch; the few plane blocks fill the main tail).
template <class T, int N, int LW>
__global__ void __launch_bounds__(3 * LW * tpl<N>()) k_zproj(ZArgs<T> a, int nmain)
{
    PDL_ENTRY();
    using C = cplx_t<T>;
    constexpr int TPL = tpl<N>();
    constexpr int nth = 3 * LW * TPL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tw = reinterpret_cast<C *>(smem_raw);
    T *zs = reinterpret_cast<T *>(tw + N);   // [N] sin(2 pi kz/nz)/h
    T *za = zs + N;                          // [N] (4 mu/h^2) sin^2(pi kz/nz)
    // [ncomp][N][LW], components ZCPAD complex apart so that a warp's three
    // components fall on different bank halves
    C *tile = reinterpret_cast<C *>(za + N + (N & 1));
    constexpr int CST = N * LW + ZCPAD;
    const int tid = threadIdx.x;
    C *base;
    long long pitch, cstride;
    int kx0, dkx, ky0, dky;
    if ((int)blockIdx.x < nmain) {
        const int nkb = a.nxh / LW;
        const int kb = blockIdx.x % nkb, ky = blockIdx.x / nkb;
        base = a.spec + (long long)ky * a.nxh + kb * LW;
        pitch = (long long)a.ny * a.nxh;
        cstride = a.cstride_main;
        kx0 = kb * LW;
        dkx = 1;
        ky0 = ky;
        dky = 0;
    } else {
        const int kyb = blockIdx.x - nmain;
        base = a.nyq + kyb * LW;
        pitch = a.ny;
        cstride = a.cstride_nyq;
        kx0 = a.nxh;
        dkx = 0;
        ky0 = kyb * LW;
        dky = 1;
    }
    for (int i = tid; i < N; i += nth) {
        tw[i] = a.tw[i];
        zs[i] = a.sz[i];
        za[i] = a.az[i];
    }
    // the zero-wavenumber mode (line 0 of block 0): its new value in FP64
    __shared__ double zmean[3];
    const bool mean_blk = a.mean_mode != 0 && blockIdx.x == 0;
    if (mean_blk) {
        // two warps take part whatever the tile variant (every variant has at
        // least 64 threads), so the FP64 sum has the same order in all
        constexpr int NWF = 2;
        static_assert(nth >= NWF * 32, "two whole warps");
        __shared__ double zred[3][NWF];
        if (tid < NWF * 32) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                double v = 0.0;
                for (int i = tid; i < a.nq; i += NWF * 32) v += a.qpart[(long long)c * a.nq + i];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if ((tid & 31) == 0) zred[c][tid >> 5] = v;
            }
        }
        __syncthreads();
        if (tid < 3) {
            double q = 0.0;
            for (int w = 0; w < NWF; ++w) q += zred[tid][w];
            const double un = a.umean[tid] + a.dt_rho_G * q;
            zmean[tid] = un;
            if (a.mean_mode == 1) a.umean[tid] = un;
        }
    }
    // thread = (line (c, l), tl): the first FFT stage's inputs, rows tl + R2 j
    // of column l of component c, go from global memory straight to registers
    constexpr int R1 = Plan<N>::R1, R2 = Plan<N>::R2;
    const int zline = tid % (3 * LW), ztl = tid / (3 * LW);
    const int zc = zline / LW, zl = zline - zc * LW;
    const int zp = (int)pitch;   // rows of a component fit in int offsets
    C vin[R1];
    if (ztl < R2) {
        const C *src = base + zc * cstride + ztl * zp + zl;
#pragma unroll
        for (int j = 0; j < R1; ++j) vin[j] = src[R2 * j * zp];
    }
    __syncthreads();   // the twiddle and wavenumber tables are staged
    fft_line_from<N, -1, T>(tile + zc * CST + zl, ColAcc<LW>(), ztl, true, tw, vin);
    {
        // nth is a multiple of LW, so a thread's column l (and its kx, ky) is fixed
        static_assert((3 * LW * TPL) % LW == 0, "columns per thread");
        const int l = tid % LW;
        const int kx = kx0 + l * dkx, ky = ky0 + l * dky;
        const T s0 = a.sx[kx], s1 = a.sy[ky];
        const T a01 = a.rho_dt + a.ax[kx] + a.ay[ky];
        for (int idx = tid; idx < N * LW; idx += nth) {
            const int kz = idx / LW;
            const T s2 = zs[kz];
            const T aa = a01 + za[kz];
            C w0 = tile[0 * CST + idx], w1 = tile[1 * CST + idx], w2 = tile[2 * CST + idx];
            const T ss = s0 * s0 + s1 * s1 + s2 * s2;
            T f;
            C pp{0, 0};
            if (ss > (T)0) {
                // one division serves 1/|s|^2 and 1/a(k): r = 1/(a |s|^2)
                const T r = (T)1 / (aa * ss);
                f = a.scale * ss * r;
                const C sw{s0 * w0.x + s1 * w1.x + s2 * w2.x, s0 * w0.y + s1 * w1.y + s2 * w2.y};
                const T inv = aa * r;
                w0.x -= s0 * sw.x * inv;
                w0.y -= s0 * sw.y * inv;
                w1.x -= s1 * sw.x * inv;
                w1.y -= s1 * sw.y * inv;
                w2.x -= s2 * sw.x * inv;
                w2.y -= s2 * sw.y * inv;
                // p^ = -i (s.w^)/|s|^2, scaled
                pp = C{sw.y * inv * a.scale, -sw.x * inv * a.scale};
            } else {
                f = a.scale / aa;
            }
            if (mean_blk && idx == 0) {
                // mode (0, 0, 0): mean velocity, carried in FP64 (1/G applied)
                w0 = C{(T)zmean[0], (T)0};
                w1 = C{(T)zmean[1], (T)0};
                w2 = C{(T)zmean[2], (T)0};
                f = (T)1;
            }
            tile[0 * CST + idx] = C{w0.x * f, w0.y * f};
            tile[1 * CST + idx] = C{w1.x * f, w1.y * f};
            tile[2 * CST + idx] = C{w2.x * f, w2.y * f};
            if (a.want_p) tile[3 * CST + idx] = pp;
        }
    }
    __syncthreads();
    const int ncomp = a.want_p ? 4 : 3;
    {
        // inverse z: up to 4*LW lines on 3*LW*TPL threads, two rounds when p
        // is wanted; the last stage's outputs, rows tl + R1 k2, go straight
        // to global memory
        for (int round = 0; round < (a.want_p ? 2 : 1); ++round) {
            const int line = tid % (3 * LW) + round * 3 * LW, tl = tid / (3 * LW);
            const int c = line / LW, l = line - c * LW;
            const bool act = line < ncomp * LW;
            C *dst = base + (act ? c : 0) * cstride + tl * zp + l;
            fft_line_to<N, +1, T>(tile + (act ? c : 0) * CST + l % LW, ColAcc<LW>(), tl, act, tw,
                                  [&](int k2, const C &v) { dst[R1 * k2 * zp] = v; });
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

template <class K> static void set_smem(K kernel, size_t bytes)
{
    if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Tile shapes of the passes: rows per block of the x passes, columns per
// block of the y and z passes.  FP32 contexts choose among the compiled
// variants at run time (FftTune, set by ib_set_tuning / ib_autotune); FP64
// contexts have one variant.
template <class T> struct Variants;
template <> struct Variants<float> {
    static constexpr int RY[2] = {4, 8}, YLW[2] = {16, 8}, ZLW[2] = {8, 4};
};
template <> struct Variants<double> {
    static constexpr int RY[1] = {8}, YLW[1] = {8}, ZLW[1] = {4};
};

template <class T, int N, int RY> static void run_xfwd(const FluidArgs<T> &a, cudaStream_t s)
{
    constexpr int nth = xfwd_threads<T, N, RY>();
    const size_t smem = sizeof(cplx_t<T>) * (N + 3 * RY / 2 * RowAcc<N>::LEN);
    set_smem(k_xfwd<T, N, RY>, smem);
    launch_pdl(k_xfwd<T, N, RY>, dim3(a.ny / RY, a.nz), dim3(nth), smem, s, a);
}

// FP32 staged x pass: RY = 4 rows per block, ZB = 16 planes per block
template <int N> static void run_xfwd_pipe(const FluidArgs<float> &a, cudaStream_t s)
{
    constexpr int RY = 4, ZB = 16;
    const size_t smem = XPipe<N, RY>::bytes();
    const dim3 grid(a.ny / RY, a.nz / ZB);
    if (a.advect) {
        set_smem(k_xfwd_pipe<N, RY, ZB, true>, smem);
        launch_pdl(k_xfwd_pipe<N, RY, ZB, true>, grid, dim3(XPipe<N, RY>::NTH), smem, s, a);
    } else {
        set_smem(k_xfwd_pipe<N, RY, ZB, false>, smem);
        launch_pdl(k_xfwd_pipe<N, RY, ZB, false>, grid, dim3(XPipe<N, RY>::NTH), smem, s, a);
    }
}

template <class T, int N, int RY>
static void run_xinv(const cplx_t<T> *spec, const cplx_t<T> *nyq, int ncomp, int ny, int nz, T *out,
                     const cplx_t<T> *tw, double *d_time, const double *tp, cudaStream_t s)
{
    constexpr int nth = 3 * RY / 2 * tpl<N>();
    const size_t smem = sizeof(cplx_t<T>) * (N + 3 * RY / 2 * RowAcc<N>::LEN);
    set_smem(k_xinv<T, N, RY>, smem);
    launch_pdl(k_xinv<T, N, RY>, dim3(ny / RY, nz), dim3(nth), smem, s, spec, nyq, ncomp, ny, nz, out, tw, d_time,
               tp);
}

template <class T, int N, int DIR, int LW>
static void run_y(cplx_t<T> *spec, cplx_t<T> *nyq, int nxh, int nz, int ncomp, const cplx_t<T> *tw, cudaStream_t s)
{
    const size_t smem = ypass_smem<T, N, LW>();
    set_smem(k_ypass<T, N, DIR, LW>, smem);
    const int nmain = nxh / LW * nz * ncomp, nlines = ncomp * nz;
    launch_pdl(k_ypass<T, N, DIR, LW>, dim3(nmain + (nlines + LW - 1) / LW), dim3(LW * tpl<N>()), smem, s, spec, nyq, nxh,
               nz, nmain, nlines, tw);
}

// only the kx = nx/2 plane's lines of a y pass (the main tiles run elsewhere)
template <class T, int N, int DIR, int LW>
static void run_y_nyq(cplx_t<T> *spec, cplx_t<T> *nyq, int nxh, int nz, int ncomp, const cplx_t<T> *tw, cudaStream_t s)
{
    const size_t smem = ypass_smem<T, N, LW>();
    set_smem(k_ypass<T, N, DIR, LW>, smem);
    const int nlines = ncomp * nz;
    launch_pdl(k_ypass<T, N, DIR, LW>, dim3((nlines + LW - 1) / LW), dim3(LW * tpl<N>()), smem, s, spec, nyq, nxh,
               nz, 0, nlines, tw);
}

template <class T, int N, int LW> static void run_z(const ZArgs<T> &a, cudaStream_t s)
{
    const size_t smem = sizeof(cplx_t<T>) * (N + (a.want_p ? 4 : 3) * (N * LW + ZCPAD)) + sizeof(T) * (2 * N + 2);
    set_smem(k_zproj<T, N, LW>, sizeof(cplx_t<T>) * (N + 4 * (N * LW + ZCPAD)) + sizeof(T) * (2 * N + 2));
    const int nmain = a.nxh / LW * a.ny;
    launch_pdl(k_zproj<T, N, LW>, dim3(nmain + (a.ny + LW - 1) / LW), dim3(3 * LW * tpl<N>()), smem, s, a, nmain);
}

#define IB_DISPATCH_N(n, FN, ...)                       \
    switch (n) {                                        \
    case 32: FN<32>(__VA_ARGS__); break;                \
    case 64: FN<64>(__VA_ARGS__); break;                \
    case 96: FN<96>(__VA_ARGS__); break;                \
    case 128: FN<128>(__VA_ARGS__); break;              \
    case 256: FN<256>(__VA_ARGS__); break;              \
    default: break;                                     \
    }

// The passes of one line length N with the tile variant chosen at run time
// (index into Variants<T>; out-of-range indices take variant 0).  Explicitly
// instantiated per (T, N) in their own translation units.
template <class T, int N> struct FftN {
    static void xfwd(const FluidArgs<T> &a, int v, cudaStream_t s)
    {
        if constexpr (sizeof(T) == 4) {
            // variant 1: rows of 8; variant 2: rows of 4 marching along z
            // with planes staged by bulk asynchronous copies; else rows of 4
            if (v == 1) return run_xfwd<T, N, Variants<T>::RY[1]>(a, s);
            if (v == 2) return run_xfwd_pipe<N>(a, s);
        }
        run_xfwd<T, N, Variants<T>::RY[0]>(a, s);
    }
    static void y(cplx_t<T> *sp, cplx_t<T> *nq, int nxh, int nz, int nc, const cplx_t<T> *tw, int dir, int v,
                  cudaStream_t s)
    {
        if constexpr (sizeof(T) == 4) {
            if (v == 1) {
                if (dir < 0) return run_y<T, N, -1, Variants<T>::YLW[1]>(sp, nq, nxh, nz, nc, tw, s);
                return run_y<T, N, +1, Variants<T>::YLW[1]>(sp, nq, nxh, nz, nc, tw, s);
            }
        }
        if (dir < 0) return run_y<T, N, -1, Variants<T>::YLW[0]>(sp, nq, nxh, nz, nc, tw, s);
        run_y<T, N, +1, Variants<T>::YLW[0]>(sp, nq, nxh, nz, nc, tw, s);
    }
    static void z(const ZArgs<T> &a, int v, cudaStream_t s)
    {
        if constexpr (sizeof(T) == 4) {
            if (v == 1) return run_z<T, N, Variants<T>::ZLW[1]>(a, s);
        }
        run_z<T, N, Variants<T>::ZLW[0]>(a, s);
    }
    static void xinv(const cplx_t<T> *sp, const cplx_t<T> *nq, int nc, int ny, int nz, T *out, const cplx_t<T> *tw,
                     double *dtm, const double *tp, int v, cudaStream_t s)
    {
        if constexpr (sizeof(T) == 4) {
            if (v == 1) return run_xinv<T, N, Variants<T>::RY[1]>(sp, nq, nc, ny, nz, out, tw, dtm, tp, s);
        }
        run_xinv<T, N, Variants<T>::RY[0]>(sp, nq, nc, ny, nz, out, tw, dtm, tp, s);
    }
};

template <class T> struct Passes {
    template <int N> static void xfwd(const FluidArgs<T> &a, int v, cudaStream_t s) { FftN<T, N>::xfwd(a, v, s); }
    template <int N>
    static void yfwd(cplx_t<T> *sp, cplx_t<T> *nq, int nxh, int nz, int nc, const cplx_t<T> *tw, int v,
                     cudaStream_t s)
    {
        FftN<T, N>::y(sp, nq, nxh, nz, nc, tw, -1, v, s);
    }
    template <int N>
    static void yinv(cplx_t<T> *sp, cplx_t<T> *nq, int nxh, int nz, int nc, const cplx_t<T> *tw, int v,
                     cudaStream_t s)
    {
        FftN<T, N>::y(sp, nq, nxh, nz, nc, tw, +1, v, s);
    }
    template <int N> static void z(const ZArgs<T> &a, int v, cudaStream_t s) { FftN<T, N>::z(a, v, s); }
    template <int N>
    static void xinv(const cplx_t<T> *sp, const cplx_t<T> *nq, int nc, int ny, int nz, T *out, const cplx_t<T> *tw,
                     double *dtm, const double *tp, int v, cudaStream_t s)
    {
        FftN<T, N>::xinv(sp, nq, nc, ny, nz, out, tw, dtm, tp, v, s);
    }
};

#define IB_FFT_EXTERN(T)                     \
    extern template struct FftN<T, 32>;      \
    extern template struct FftN<T, 64>;      \
    extern template struct FftN<T, 96>;      \
    extern template struct FftN<T, 128>;     \
    extern template struct FftN<T, 256>;

template <class T>
void fluid_impl(ib_ctx *c, const void *u_n, const void *F, void *u_np1, void *p, bool use_touched,
                       int mode, cudaStream_t s, cudaEvent_t *ev)
{
    using C = cplx_t<T>;
    const int nx = c->dim.nx, ny = c->dim.ny, nz = c->dim.nz, nxh = nx / 2;
    const long long G = c->dim.G;
    C *spec = static_cast<C *>(c->spec);
    C *nyq = static_cast<C *>(c->nyq);

    FluidArgs<T> a{};
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.G = G;
    a.u = static_cast<const T *>(u_n);
    a.F = static_cast<const T *>(F);
    a.touched = use_touched ? c->touched : nullptr;
    a.ntx = c->dim.ntx;
    a.nty = c->dim.nty;
    const bool direct = mode == FLUID_DIRECT;
    const bool body = mode == FLUID_STEP || mode == FLUID_REPLAY;
    a.rho_dt = direct ? (T)1 : (T)(c->desc.rho / c->desc.dt);
    a.rho_h = (T)(c->desc.rho / c->desc.h);
    a.advect = (direct || (c->desc.flags & IB_NO_ADVECTION)) ? 0 : 1;
    a.frows = (body && c->forcing.active) ? c->forcing.rows : nullptr;
    a.fdir0 = (T)c->forcing.dir[0];
    a.fdir1 = (T)c->forcing.dir[1];
    a.fdir2 = (T)c->forcing.dir[2];
    a.d_time = c->d_time;
    a.spec = spec;
    a.nyq = nyq;
    a.tw = static_cast<const C *>(c->tw[0]);
    const FftTune &tv = c->fft_tune;
    // FP32 steps carry the zero-wavenumber mode in FP64 (the state's mean
    // velocity in d_time[4..6]); other solves leave it to the FFT
    const int mean_mode = (sizeof(T) == 4 && c->qpart) ? (mode == FLUID_STEP ? 1 : mode == FLUID_REPLAY ? 2 : 0) : 0;
    a.qpart = mean_mode ? c->qpart : nullptr;
    a.status = c->d_status;
    IB_DISPATCH_N(nx, Passes<T>::template xfwd, a, tv.x, s);
    if (ev) cudaEventRecord(ev[0], s);

    const int ncomp = p ? 4 : 3;
    // IB_FP32_TCFFT: main tiles of the y passes on the tensor cores (ny = 256)
    auto y_tc = [&](int dir, int nc) -> bool {
        if constexpr (sizeof(T) == 4) {
            if (!c->tc_fft || ny != 256) return false;
            int nsm = 0;
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
            if (!launch_ytc(reinterpret_cast<float2 *>(spec), nxh, nz, nc, static_cast<const float2 *>(c->tw[1]), dir,
                            c->d_status, nsm, s))
                return false;
            if (dir < 0) run_y_nyq<float, 256, -1, 8>(spec, nyq, nxh, nz, nc, static_cast<const C *>(c->tw[1]), s);
            else run_y_nyq<float, 256, +1, 8>(spec, nyq, nxh, nz, nc, static_cast<const C *>(c->tw[1]), s);
            return true;
        }
        return false;
    };
    if (!y_tc(-1, 3))
        IB_DISPATCH_N(ny, Passes<T>::template yfwd, spec, nyq, nxh, nz, 3, static_cast<const C *>(c->tw[1]), tv.y, s);
    if (ev) cudaEventRecord(ev[1], s);

    ZArgs<T> z{};
    z.spec = spec;
    z.nyq = nyq;
    z.nxh = nxh;
    z.ny = ny;
    z.nz = nz;
    z.cstride_main = (long long)nz * ny * nxh;
    z.cstride_nyq = (long long)nz * ny;
    z.sx = static_cast<const T *>(c->sym_s[0]);
    z.sy = static_cast<const T *>(c->sym_s[1]);
    z.sz = static_cast<const T *>(c->sym_s[2]);
    z.ax = static_cast<const T *>(c->sym_a[0]);
    z.ay = static_cast<const T *>(c->sym_a[1]);
    z.az = static_cast<const T *>(c->sym_a[2]);
    z.rho_dt = (T)(c->desc.rho / c->desc.dt);
    z.scale = (T)(1.0 / (double)G);
    z.tw = static_cast<const C *>(c->tw[2]);
    z.want_p = p ? 1 : 0;
    z.mean_mode = mean_mode;
    z.qpart = c->qpart;
    z.nq = (ny / 4) * nz;
    z.umean = c->d_time + 4;
    z.dt_rho_G = c->desc.dt / (c->desc.rho * (double)G);
    IB_DISPATCH_N(nz, Passes<T>::template z, z, tv.z, s);
    if (ev) cudaEventRecord(ev[2], s);

    if (!y_tc(+1, ncomp))
        IB_DISPATCH_N(ny, Passes<T>::template yinv, spec, nyq, nxh, nz, ncomp, static_cast<const C *>(c->tw[1]), tv.y,
                      s);
    if (ev) cudaEventRecord(ev[3], s);
    IB_DISPATCH_N(nx, Passes<T>::template xinv, spec, nyq, 3, ny, nz, static_cast<T *>(u_np1),
                  static_cast<const C *>(c->tw[0]), mode == FLUID_STEP ? c->d_time : nullptr, c->d_tparams, tv.x, s);
    if (p) {
        const long long off_main = 3LL * nz * ny * nxh, off_nyq = 3LL * nz * ny;
        IB_DISPATCH_N(nx, Passes<T>::template xinv, spec + off_main, nyq + off_nyq, 1, ny, nz, static_cast<T *>(p),
                      static_cast<const C *>(c->tw[0]), nullptr, nullptr, tv.x, s);
    }
}

}  // namespace ibgb
