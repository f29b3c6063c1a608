// Register-level small DFTs and a two-stage shared-memory line FFT.
//
// Used by the fluid solve of Eqs. (discreteNS1)-(discreteNS2): the system
// has constant coefficients on a periodic grid, so each Fourier mode
// decouples.  All transforms compute X[k] = sum_j x[j] exp(DIR 2 pi i jk/N)
// (DIR = -1 forward, +1 inverse, unscaled).
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "ib_internal.cuh"

namespace ibgb {

// ---------------------------------------------------------------------------
// Compile-time unit roots.  cos/sin of 2 pi m / n from a Taylor series on an
// argument reduced to [0, pi/4] by exact quadrant and octant reflections.
// ---------------------------------------------------------------------------
struct CD {
    double re, im;
};

constexpr double kPi = 3.14159265358979323846264338327950288;

__host__ __device__ constexpr double ct_sin_small(double x)
{
    double term = x, sum = x;
    for (int k = 1; k < 14; ++k) {
        term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
        sum += term;
    }
    return sum;
}

__host__ __device__ constexpr double ct_cos_small(double x)
{
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 14; ++k) {
        term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
        sum += term;
    }
    return sum;
}

// exp(+2 pi i m / n)
__host__ __device__ constexpr CD ct_unit(long long m, long long n)
{
    m %= n;
    if (m < 0) m += n;
    long long q = (4 * m) / n;          // quadrant
    long long r = 4 * m - q * n;        // angle in quadrant = (pi/2) r / n, r in [0, n)
    double c = 0.0, s = 0.0;
    if (2 * r <= n) {
        double x = (kPi / 2.0) * (double)r / (double)n;
        c = ct_cos_small(x);
        s = ct_sin_small(x);
    } else {
        double x = (kPi / 2.0) * (double)(n - r) / (double)n;
        c = ct_sin_small(x);
        s = ct_cos_small(x);
    }
    if (r == 0) {
        c = 1.0;
        s = 0.0;
    }
    switch (q) {
    case 0: return CD{c, s};
    case 1: return CD{-s, c};
    case 2: return CD{-c, -s};
    default: return CD{s, -c};
    }
}

// ---------------------------------------------------------------------------
// complex helpers (float2 / double2)
// ---------------------------------------------------------------------------
template <class C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <class C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <class C> __device__ __forceinline__ C cmul(C a, C b)
{
    return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <class C> __device__ __forceinline__ C cconj(C a) { return C{a.x, -a.y}; }
// multiply by DIR * i
template <int DIR, class C> __device__ __forceinline__ C cmul_i(C a)
{
    if constexpr (DIR > 0) return C{-a.y, a.x};
    else return C{a.y, -a.x};
}

template <int B, int E, class F> __device__ __forceinline__ void static_for(F &&f)
{
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

// v *= exp(DIR 2 pi i M / N), exact for the trivial angles
template <int M, int N, int DIR, class T> __device__ __forceinline__ void twmul(cplx_t<T> &v)
{
    constexpr int mm = ((M % N) + N) % N;
    if constexpr (mm == 0) {
        return;
    } else if constexpr (2 * mm == N) {
        v.x = -v.x;
        v.y = -v.y;
    } else if constexpr (4 * mm == N) {
        v = cmul_i<DIR>(v);
    } else if constexpr (4 * mm == 3 * N) {
        v = cmul_i<-DIR>(v);
    } else {
        constexpr CD w = ct_unit(mm, N);
        constexpr T c = (T)w.re;
        constexpr T s = (T)(DIR * w.im);
        T x = v.x * c - v.y * s;
        T y = v.x * s + v.y * c;
        v.x = x;
        v.y = y;
    }
}

// ---------------------------------------------------------------------------
// In-register DFT of length N in natural order.
// ---------------------------------------------------------------------------
template <int N, int DIR, class T> struct DFT;

template <int DIR, class T> struct DFT<1, DIR, T> {
    static __device__ __forceinline__ void run(cplx_t<T> *) {}
};

template <int DIR, class T> struct DFT<2, DIR, T> {
    static __device__ __forceinline__ void run(cplx_t<T> *v)
    {
        cplx_t<T> a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <int DIR, class T> struct DFT<3, DIR, T> {
    static __device__ __forceinline__ void run(cplx_t<T> *v)
    {
        // W = exp(DIR 2 pi i / 3) = -1/2 + DIR i sqrt(3)/2
        constexpr T h3 = (T)0.86602540378443864676372317075294;
        cplx_t<T> a = v[0], b = v[1], c = v[2];
        cplx_t<T> s = cadd(b, c), d = csub(b, c);
        cplx_t<T> m{a.x - (T)0.5 * s.x, a.y - (T)0.5 * s.y};
        cplx_t<T> r = cmul_i<DIR>(d);
        r.x *= h3;
        r.y *= h3;
        v[0] = cadd(a, s);
        v[1] = cadd(m, r);
        v[2] = csub(m, r);
    }
};

template <int DIR, class T> struct DFT<4, DIR, T> {
    static __device__ __forceinline__ void run(cplx_t<T> *v)
    {
        cplx_t<T> a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
        cplx_t<T> c = cadd(v[1], v[3]), d = cmul_i<DIR>(csub(v[1], v[3]));
        v[0] = cadd(a, c);
        v[2] = csub(a, c);
        v[1] = cadd(b, d);
        v[3] = csub(b, d);
    }
};

// N = P * Q, decimation in time: input j = j1 + P j2, output k = k1 + Q k2.
template <int N, int DIR, class T> struct DFT {
    static constexpr int P = (N % 4 == 0) ? 4 : ((N % 2 == 0) ? 2 : 3);
    static constexpr int Q = N / P;
    static_assert(P * Q == N && Q > 1, "unsupported DFT length");
    static __device__ __forceinline__ void run(cplx_t<T> *v)
    {
        cplx_t<T> y[P][Q];
        static_for<0, P>([&](auto j1_) {
            constexpr int j1 = decltype(j1_)::value;
            cplx_t<T> t[Q];
            static_for<0, Q>([&](auto j2_) {
                constexpr int j2 = decltype(j2_)::value;
                t[j2] = v[j1 + P * j2];
            });
            DFT<Q, DIR, T>::run(t);
            static_for<0, Q>([&](auto k1_) {
                constexpr int k1 = decltype(k1_)::value;
                twmul<j1 * k1, N, DIR, T>(t[k1]);
                y[j1][k1] = t[k1];
            });
        });
        static_for<0, Q>([&](auto k1_) {
            constexpr int k1 = decltype(k1_)::value;
            cplx_t<T> t[P];
            static_for<0, P>([&](auto j1_) {
                constexpr int j1 = decltype(j1_)::value;
                t[j1] = y[j1][k1];
            });
            DFT<P, DIR, T>::run(t);
            static_for<0, P>([&](auto k2_) {
                constexpr int k2 = decltype(k2_)::value;
                v[k1 + Q * k2] = t[k2];
            });
        });
    }
};

// ---------------------------------------------------------------------------
// Two-stage line FFT of length N = R1 * R2 in shared memory.
//   stage A: R2 threads, thread t: R1-point DFT of x[t + R2 j], times W_N^{t k1},
//            written back in place;
//   stage B: R1 threads, thread k1: R2-point DFT of the block [R2 k1, R2 k1 + R2),
//            output X[k1 + R1 k2].
// ---------------------------------------------------------------------------
template <int N> struct Plan;
template <> struct Plan<32> { static constexpr int R1 = 8, R2 = 4; };
template <> struct Plan<48> { static constexpr int R1 = 8, R2 = 6; };
template <> struct Plan<64> { static constexpr int R1 = 8, R2 = 8; };
template <> struct Plan<96> { static constexpr int R1 = 8, R2 = 12; };
template <> struct Plan<128> { static constexpr int R1 = 16, R2 = 8; };
template <> struct Plan<192> { static constexpr int R1 = 16, R2 = 12; };
template <> struct Plan<256> { static constexpr int R1 = 16, R2 = 16; };

template <int N> __host__ __device__ constexpr int tpl() { return Plan<N>::R1 > Plan<N>::R2 ? Plan<N>::R1 : Plan<N>::R2; }

// Element addressing: a line stored contiguously with one pad slot after
// every R2 elements (conflict-free for both stages) ...
template <int N> struct RowAcc {
    static constexpr int R2 = Plan<N>::R2;
    static constexpr int LEN = N + N / R2;
    __device__ __forceinline__ int operator()(int i) const { return i + i / R2; }
};
// ... or lines interleaved, element i of line l at i*LW + l.
template <int LW> struct ColAcc {
    __device__ __forceinline__ int operator()(int i) const { return i * LW; }
};

// Stage A of a line FFT on a thread's R1 inputs v[j] = x[tl + R2 j]
// (tl < R2): the R1-point DFT and the twiddles W_N^(tl k1), written back in
// place to elements tl + R2 k1.
template <int N, int DIR, class T, class Acc>
__device__ __forceinline__ void fft_stage_a(cplx_t<T> *line, Acc acc, int tl, const cplx_t<T> *tw,
                                            cplx_t<T> (&v)[Plan<N>::R1])
{
    constexpr int R1 = Plan<N>::R1, R2 = Plan<N>::R2;
    using C = cplx_t<T>;
    DFT<R1, DIR, T>::run(v);
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1) {
        C w = tw[tl * k1];
        if (DIR > 0) w.y = -w.y;
        v[k1] = cmul(v[k1], w);
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) line[acc(tl + R2 * k1)] = v[k1];
}

// All threads of the block must call this (it synchronises).  `line` points
// at element 0 of this thread's line (ignored when active == false); tl is
// the thread's index within its line's group; tw holds W_N^j (forward) in
// shared memory.
template <int N, int DIR, class T, class Acc>
__device__ __forceinline__ void fft_line(cplx_t<T> *line, Acc acc, int tl, bool active, const cplx_t<T> *tw)
{
    constexpr int R1 = Plan<N>::R1, R2 = Plan<N>::R2;
    using C = cplx_t<T>;
    if (active && tl < R2) {
        C v[R1];
#pragma unroll
        for (int j = 0; j < R1; ++j) v[j] = line[acc(tl + R2 * j)];
        fft_stage_a<N, DIR, T>(line, acc, tl, tw, v);
    }
    __syncthreads();
    C v[R2];
    if (active && tl < R1) {
#pragma unroll
        for (int t = 0; t < R2; ++t) v[t] = line[acc(R2 * tl + t)];
        DFT<R2, DIR, T>::run(v);
    }
    __syncthreads();
    if (active && tl < R1) {
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) line[acc(tl + R1 * k2)] = v[k2];
    }
    __syncthreads();
}

// fft_line whose input the caller has already loaded into registers:
// v[j] = x[tl + R2 j] for threads with tl < R2 (the caller loads them from
// global memory, so the line is never staged in shared memory).
template <int N, int DIR, class T, class Acc>
__device__ __forceinline__ void fft_line_from(cplx_t<T> *line, Acc acc, int tl, bool active, const cplx_t<T> *tw,
                                              cplx_t<T> (&vin)[Plan<N>::R1])
{
    constexpr int R1 = Plan<N>::R1, R2 = Plan<N>::R2;
    using C = cplx_t<T>;
    if (active && tl < R2) fft_stage_a<N, DIR, T>(line, acc, tl, tw, vin);
    __syncthreads();
    C v[R2];
    if (active && tl < R1) {
#pragma unroll
        for (int t = 0; t < R2; ++t) v[t] = line[acc(R2 * tl + t)];
        DFT<R2, DIR, T>::run(v);
    }
    __syncthreads();
    if (active && tl < R1) {
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) line[acc(tl + R1 * k2)] = v[k2];
    }
    __syncthreads();
}

// fft_line whose output goes to out(k2, X[tl + R1 k2]) (threads with
// tl < R1) instead of back to the line; the line is left as stage A wrote it.
template <int N, int DIR, class T, class Acc, class Out>
__device__ __forceinline__ void fft_line_to(cplx_t<T> *line, Acc acc, int tl, bool active, const cplx_t<T> *tw,
                                            Out out)
{
    constexpr int R1 = Plan<N>::R1, R2 = Plan<N>::R2;
    using C = cplx_t<T>;
    if (active && tl < R2) {
        C v[R1];
#pragma unroll
        for (int j = 0; j < R1; ++j) v[j] = line[acc(tl + R2 * j)];
        fft_stage_a<N, DIR, T>(line, acc, tl, tw, v);
    }
    __syncthreads();
    if (active && tl < R1) {
        C v[R2];
#pragma unroll
        for (int t = 0; t < R2; ++t) v[t] = line[acc(R2 * tl + t)];
        DFT<R2, DIR, T>::run(v);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) out(k2, v[k2]);
    }
}

// fft_line with both: input in registers (as fft_line_from) and output to
// out(k2, X[tl + R1 k2]) (as fft_line_to); shared memory holds only the
// transpose between the two stages.
template <int N, int DIR, class T, class Acc, class Out>
__device__ __forceinline__ void fft_line_from_to(cplx_t<T> *line, Acc acc, int tl, bool active, const cplx_t<T> *tw,
                                                 cplx_t<T> (&vin)[Plan<N>::R1], Out out)
{
    constexpr int R1 = Plan<N>::R1, R2 = Plan<N>::R2;
    using C = cplx_t<T>;
    if (active && tl < R2) fft_stage_a<N, DIR, T>(line, acc, tl, tw, vin);
    __syncthreads();
    if (active && tl < R1) {
        C v[R2];
#pragma unroll
        for (int t = 0; t < R2; ++t) v[t] = line[acc(R2 * tl + t)];
        DFT<R2, DIR, T>::run(v);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) out(k2, v[k2]);
    }
}

}  // namespace ibgb
