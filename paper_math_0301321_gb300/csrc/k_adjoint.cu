// Reverse (adjoint) time step: the transpose of the linearised step of
// Section 3.2 (steps 1-4), about the state (u^n, X^n = X0 + d^n).
//
// Forward:  f = f(d; b)                      (springs, tethers, bending)
//           F = S(X) f + body(t)             (Eq. discreteF)
//           w = rho u/dt - rho A(u) + F      (Eq. discreteNS1, upwind A)
//           u' = L w                         (Eqs. discreteNS1-2, FFT solve)
//           d' = d + dt I(X) u'              (Eq. discreteX)
// Reverse, given lam_u' = dJ/du', lam_d' = dJ/dd':
//           lam_U = dt lam_d'
//           lam_w = L (lam_u' + I(X)^T lam_U)          L is real symmetric
//           lam_u = rho lam_w/dt - rho (dA/du)^T lam_w
//           lam_f = S(X)^T lam_w = h^-3 I(X) lam_w
//           lam_X = [dI(X)u'/dX]^T lam_U + [dS(X)f/dX]^T lam_w
//           lam_d = lam_d' + lam_X + (df/dd) lam_f,  dJ/db_s = lam_f . df/db_s
// I(X)^T lam_U is the spread of h^3 lam_U and L runs through the forward FFT
// passes with w given directly; this file holds the remaining kernels: the
// transposed upwind stencil, the reverse marker gather (both interpolation
// transposes in one pass), the elastic Hessian product and the stiffness
// gradient.
#include "ib_internal.cuh"
#include "marker_forces.cuh"

namespace ibgb {

// ---------------------------------------------------------------------------
// lam_u = rho_dt lw - rho (dA/du)^T lw, as a gather per node q:
//  (dA/du)^T lw at (q, j) =
//     sum_i lw_i(q) D_j u_i(q)                       u_j(q) as the coefficient
//   + lw_j(q) sum_k |u_k(q)| / h                       u_j(q) differenced at q
//   - sum_k [u_k(q+e_k)]^+ lw_j(q+e_k) / h             ... as the backward neighbour
//   + sum_k [u_k(q-e_k)]^- lw_j(q-e_k) / h             ... as the forward neighbour
// with D_j the upwind difference the forward term takes at q (backward for
// u_j > 0, forward for u_j < 0, none for u_j = 0).
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256)
    k_adv_adjoint(GridDims g, const T *__restrict__ u, const T *__restrict__ lw, T *__restrict__ out, T rho_dt,
                  T rho, T inv_h, int advect)
{
    PDL_ENTRY();
    // one thread per node of plane z = blockIdx.y; 32-bit index arithmetic
    // (3 G fits in int for every supported grid)
    const int nxy = g.nx * g.ny;
    const int idx = blockIdx.x * 256 + threadIdx.x;
    if (idx >= nxy) return;
    const int z = blockIdx.y;
    const int q = z * nxy + idx;
    const int G = (int)g.G;
    T L[3], res[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        L[c] = __ldg(lw + c * G + q);
        res[c] = rho_dt * L[c];
    }
    if (advect) {
        const int y = idx / g.nx, x = idx - y * g.nx;
        const int sx = 1, sy = g.nx, sz = nxy;
        // linear offsets of the -e_k and +e_k neighbours (periodic)
        const int om[3] = {x == 0 ? (g.nx - 1) * sx : -sx, y == 0 ? (g.ny - 1) * sy : -sy,
                           z == 0 ? (g.nz - 1) * sz : -sz};
        const int op[3] = {x == g.nx - 1 ? -(g.nx - 1) * sx : sx, y == g.ny - 1 ? -(g.ny - 1) * sy : sy,
                           z == g.nz - 1 ? -(g.nz - 1) * sz : sz};
        T uq[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) uq[c] = __ldg(u + c * G + q);
        T acc[3] = {0, 0, 0};
        // the upwind neighbour of direction j: one address chosen by the sign
        // of u_j, its difference negated (exactly) when it lies on the + side
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const bool pos = uq[j] > (T)0;
            if (pos || uq[j] < (T)0) {
                const int n = q + (pos ? om[j] : op[j]);
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const T dq = (uq[i] - __ldg(u + i * G + n)) * inv_h;
                    acc[j] += L[i] * (pos ? dq : -dq);
                }
            }
        }
        const T sa = (fabs(uq[0]) + fabs(uq[1]) + fabs(uq[2])) * inv_h;
#pragma unroll
        for (int j = 0; j < 3; ++j) acc[j] += L[j] * sa;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int np = q + op[k], nm = q + om[k];
            const T up = __ldg(u + k * G + np);
            if (up > (T)0) {
#pragma unroll
                for (int j = 0; j < 3; ++j) acc[j] -= (up * inv_h) * __ldg(lw + j * G + np);
            }
            const T um = __ldg(u + k * G + nm);
            if (um < (T)0) {
#pragma unroll
                for (int j = 0; j < 3; ++j) acc[j] += (um * inv_h) * __ldg(lw + j * G + nm);
            }
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) res[j] -= rho * acc[j];
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) out[j * G + q] = res[j];
}

// ---------------------------------------------------------------------------
// Reverse marker gather.  Per work item (tile, chunk) the padded boxes of lw
// and u1 are staged in shared memory; one thread per sorted marker p reads
// its records and fractional offsets from global memory and sums its 64
// stencil nodes ((ky, kz) pairs, then kx):
//   lf_s[p] = h^-3 sum_x lw(x) W(x)
//   lX_s[p] = (1/h) sum_x [lamU . u1(x) + h^-3 f . lw(x)] grad_r W(x)
// W = wx wy wz the stencil weights, grad_r their derivatives in the
// fractional offsets r: with q = sqrt(1 + 4r(1-r)) and q' = (2 - 4r)/q,
//   dw = ((-2 - q'), (-2 + q'), (2 + q'), (2 - q')) / 8
// (the derivative of phi's two branches at distances 1+r, r, 1-r, 2-r).
// ---------------------------------------------------------------------------
constexpr int AI_THREADS = 256;

template <class T> constexpr size_t adj_interp_smem() { return sizeof(T) * 6 * PAD3; }

template <class T> __device__ __forceinline__ void stencil_dweights(T r, T *dw)
{
    const T q = sqrt((T)1 + (T)4 * r * ((T)1 - r));
    const T qp = ((T)2 - (T)4 * r) / q;
    const T e = (T)0.125;
    dw[0] = (-(T)2 - qp) * e;
    dw[1] = (-(T)2 + qp) * e;
    dw[2] = ((T)2 + qp) * e;
    dw[3] = ((T)2 - qp) * e;
}

template <class T>
__global__ void __launch_bounds__(AI_THREADS)
    k_adj_interp(GridDims g, const int32_t *__restrict__ bin_start, const int32_t *__restrict__ skey,
                 const int32_t *__restrict__ perm, const T *__restrict__ rfrac, const Record<T> *__restrict__ rec,
                 const Record<T> *__restrict__ rec2, const int2 *__restrict__ items, int *__restrict__ ctl,
                 const T *__restrict__ u1, const T *__restrict__ lw, T inv_h3, T inv_h, T *__restrict__ lf_s,
                 T *__restrict__ lX_s)
{
    PDL_ENTRY();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *boxW = reinterpret_cast<T *>(smem_raw);
    T *boxU = boxW + 3 * PAD3;

    const int tid = threadIdx.x;
    const int nitems = ctl[0];
    const int m = g.nmark;
    // box planes (c, pz) of PAD*PAD values: warp w stages planes w, w + NW, ...;
    // lane slot j holds plane element lane + 32 j
    constexpr int NW = AI_THREADS / 32;
    constexpr int PSLOT = (PAD * PAD + 31) / 32;
    const int warp = tid >> 5, lane = tid & 31;
    int spx[PSLOT], spy[PSLOT];
#pragma unroll
    for (int j = 0; j < PSLOT; ++j) {
        const int e = min(lane + 32 * j, PAD * PAD - 1);
        spy[j] = e / PAD;
        spx[j] = e - spy[j] * PAD;
    }
    __shared__ int next_item;
    for (;;) {
        // items are taken from the counter ctl[2] (zeroed by the bin plan and
        // by the gather's move kernel)
        __syncthreads();
        if (tid == 0) next_item = atomicAdd(&ctl[2], 1);
        __syncthreads();
        const int it = next_item;
        if (it >= nitems) break;
        const int2 item = items[it];
        const int t = item.x;
        const int tx = t % g.ntx, ty = (t / g.ntx) % g.nty, tz = t / (g.ntx * g.nty);
        const int ox = tx * TILE - 1, oy = ty * TILE - 1, oz = tz * TILE - 1;
        int roff[PSLOT];
#pragma unroll
        for (int j = 0; j < PSLOT; ++j) {
            int x = ox + spx[j], y = oy + spy[j];
            x = x < 0 ? x + g.nx : (x >= g.nx ? x - g.nx : x);
            y = y < 0 ? y + g.ny : (y >= g.ny ? y - g.ny : y);
            roff[j] = y * g.nx + x;
        }
        for (int pl = warp; pl < 3 * PAD; pl += NW) {
            const int c = pl / PAD, pz = pl - c * PAD;
            int z = oz + pz;
            z = z < 0 ? z + g.nz : (z >= g.nz ? z - g.nz : z);
            const long long base = c * g.G + (long long)z * g.ny * g.nx;
            T vw[PSLOT], vu[PSLOT];
#pragma unroll
            for (int j = 0; j < PSLOT; ++j) {
                if (lane + 32 * j < PAD * PAD) {
                    vw[j] = __ldg(lw + base + roff[j]);
                    vu[j] = __ldg(u1 + base + roff[j]);
                }
            }
#pragma unroll
            for (int j = 0; j < PSLOT; ++j) {
                if (lane + 32 * j < PAD * PAD) {
                    boxW[pl * PAD * PAD + lane + 32 * j] = vw[j];
                    boxU[pl * PAD * PAD + lane + 32 * j] = vu[j];
                }
            }
        }
        const int s0 = bin_start[t] + item.y * CHUNK;
        const int s1 = min(s0 + CHUNK, bin_start[t + 1]);
        __syncthreads();   // the boxes are staged
        for (int p = s0 + tid; p < s1; p += AI_THREADS) {
            const int l = skey[p] & (TILE * TILE * TILE - 1);   // keys are >= 0
            const int lx = l & (TILE - 1), ly = (l >> 3) & (TILE - 1), lz = l >> 6;
            const int id = perm[p];
            const T *R = reinterpret_cast<const T *>(rec + p);
            const T *R2 = reinterpret_cast<const T *>(rec2 + p);
            T wx[4], wy[4], wz[4], dx[4], dy[4], dz[4];
            ld4(R, wx);
            ld4(R + 4, wy);
            ld4(R + 8, wz);
            stencil_dweights<T>(rfrac[id], dx);
            stencil_dweights<T>(rfrac[(long long)m + id], dy);
            stencil_dweights<T>(rfrac[2LL * m + id], dz);
            // R2.f = h^3 dt lam_d = h^3 lam_U
            const T lU[3] = {R2[12] * inv_h3, R2[13] * inv_h3, R2[14] * inv_h3};
            const T fh[3] = {R[12] * inv_h3, R[13] * inv_h3, R[14] * inv_h3};
            T af[3] = {0, 0, 0}, ag[3] = {0, 0, 0};
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int ky = i & 3, kz = i >> 2;
                const T wyz = wy[ky] * wz[kz], dyz = dy[ky] * wz[kz], wdz = wy[ky] * dz[kz];
                const int o = ((lz + kz) * PAD + ly + ky) * PAD + lx;
#pragma unroll
                for (int kx = 0; kx < 4; ++kx) {
                    T vw[3], vu[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        vw[c] = boxW[c * PAD3 + o + kx];
                        vu[c] = boxU[c * PAD3 + o + kx];
                    }
                    const T W = wx[kx] * wyz;
#pragma unroll
                    for (int c = 0; c < 3; ++c) af[c] += vw[c] * W;
                    const T sv = (lU[0] * vu[0] + lU[1] * vu[1] + lU[2] * vu[2]) +
                                 (fh[0] * vw[0] + fh[1] * vw[1] + fh[2] * vw[2]);
                    ag[0] += sv * (dx[kx] * wyz);
                    ag[1] += sv * (wx[kx] * dyz);
                    ag[2] += sv * (wx[kx] * wdz);
                }
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                lf_s[(long long)c * m + p] = af[c] * inv_h3;
                lX_s[(long long)c * m + p] = ag[c] * inv_h;
            }
        }
    }
}

// sorted position -> marker: lf[perm[p]] = lf_s[p], lX[perm[p]] = lX_s[p]
template <class T>
__global__ void k_adj_move(int m, const int32_t *__restrict__ perm, const T *__restrict__ lf_s,
                           const T *__restrict__ lX_s, T *__restrict__ lf, T *__restrict__ lX, int *__restrict__ ctl)
{
    PDL_ENTRY();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0) ctl[2] = 0;   // the marker gather's work counter, for its next launch
    if (p >= m) return;
    const int id = perm[p];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        lf[(long long)c * m + id] = lf_s[(long long)c * m + p];
        lX[(long long)c * m + id] = lX_s[(long long)c * m + p];
    }
}

// ---------------------------------------------------------------------------
// Per marker l: lamDo = lamD + lX + (df/dd) lf, where (df/dd) is the
// (symmetric) Jacobian of the forces of step 1:
//  spring (l, j), e = e0 + d_j - d_l, r = |e|:
//     K = k [(1 - L0/r) I + L0 e e^T / r^3],  contribution K (lf_j - lf_l)
//     (1 - L0/r = (r - L0)/r is formed as in the forward force, from
//     |e0|^2 - L0^2 + dd.(2 e0 + dd), so it keeps its relative precision);
//  tether: -k lf_l;
//  bending: linear in d, so the bending force evaluated at lf.
// Each marker with a bending term centred on it also writes, in FP64, its
// share of the stiffness derivative of its segment s.  The derivative is
//   dJ/db_s = sum_{i in s} C_i . (-lf_{i-1} + 2 lf_i - lf_{i+1}),
//   C_i = unit_i dev_i   (dev the second difference of d along the line),
// summed by parts over the segment's rows a..b, so that the second
// difference falls on C (exact to FP64 from the compensated displacement)
// instead of on lf (a smooth field whose second difference would cancel
// most of its digits):
//   share_j = lf_j . (2 C_j - [j+1 in s] C_{j+1} - [j-1 in s] C_{j-1})
//             - [j = a] C_a . lf_{a-1} - [j = b] C_b . lf_{b+1}.
template <class T>
__global__ void __launch_bounds__(256)
    k_adj_markers(ForceArgs<T> a, const T *__restrict__ lf, const T *__restrict__ lX, const T *__restrict__ lamD,
                  T *__restrict__ lamDo, const double *__restrict__ bunit, const int32_t *__restrict__ bseg,
                  double *__restrict__ gterm)
{
    PDL_ENTRY();
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = a.m;
    if (l >= m) return;
    const T dl[3] = {a.d[l], a.d[m + l], a.d[2 * m + l]};
    const T ll[3] = {lf[l], lf[m + l], lf[2 * m + l]};
    T out[3] = {0, 0, 0};
    const T kt = a.tk[l];
    if (kt != (T)0) {
#pragma unroll
        for (int c = 0; c < 3; ++c) out[c] -= kt * ll[c];
    }
    const int e1 = a.sp_off[l + 1];
    for (int e = a.sp_off[l]; e < e1; ++e) {
        const int j = a.sp_j[e];
        const T dd[3] = {a.d[j] - dl[0], a.d[m + j] - dl[1], a.d[2 * m + j] - dl[2]};
        const T e0[3] = {a.sp_e0[e], a.sp_e0[a.nnz + e], a.sp_e0[2 * a.nnz + e]};
        const T ee[3] = {e0[0] + dd[0], e0[1] + dd[1], e0[2] + dd[2]};
        const T r2 = ee[0] * ee[0] + ee[1] * ee[1] + ee[2] * ee[2];
        const T r = sqrt(r2);
        const T num = a.sp_c0[e] + (dd[0] * ((T)2 * e0[0] + dd[0]) + dd[1] * ((T)2 * e0[1] + dd[1]) +
                                    dd[2] * ((T)2 * e0[2] + dd[2]));
        const T k = a.sp_k[e], L0 = a.sp_L0[e];
        const T f1 = k * (num / (r + L0)) / r;
        const T f2 = k * L0 / (r2 * r);
        const T dv[3] = {lf[j] - ll[0], lf[m + j] - ll[1], lf[2 * m + j] - ll[2]};
        const T ed = ee[0] * dv[0] + ee[1] * dv[1] + ee[2] * dv[2];
#pragma unroll
        for (int c = 0; c < 3; ++c) out[c] += f1 * dv[c] + (f2 * ed) * ee[c];
    }
    const int slot = a.bslot ? a.bslot[l] : -1;
    if (slot >= 0) {
        int nbr[5];
        T cc[3];
#pragma unroll
        for (int q = 0; q < 5; ++q) nbr[q] = a.bn[q * a.nb + slot];
#pragma unroll
        for (int q = 0; q < 3; ++q) cc[q] = a.bc[q * a.nb + slot];
        const int nb = (int)a.nb;
        const int sgo = bseg[nb + slot];                 // segment of the term centred here
        const bool in_m = sgo >= 0 && bseg[slot] == sgo, in_p = sgo >= 0 && bseg[2 * nb + slot] == sgo;
        double gacc = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            T lv[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) lv[q] = nbr[q] >= 0 ? lf[c * m + nbr[q]] : (T)0;
            T g = 0;
            if (cc[0] != (T)0) g += cc[0] * (lv[0] - (T)2 * lv[1] + lv[2]);
            if (cc[1] != (T)0) g -= (T)2 * cc[1] * (lv[1] - (T)2 * lv[2] + lv[3]);
            if (cc[2] != (T)0) g += cc[2] * (lv[2] - (T)2 * lv[3] + lv[4]);
            out[c] -= g;
            if (sgo >= 0) {
                // C at rows i-1, i, i+1 (those of this segment), FP64 from d = hi + lo
                auto disp = [&](int q) -> double {
                    return (double)a.d[c * m + nbr[q]] + (a.dlo ? (double)a.dlo[c * m + nbr[q]] : 0.0);
                };
                const double d1 = disp(1), d2 = disp(2), d3 = disp(3);
                const double C0 = bunit[nb + slot] * (d3 - 2.0 * d2 + d1);
                const double Cm = in_m ? bunit[slot] * (d2 - 2.0 * d1 + disp(0)) : 0.0;
                const double Cp = in_p ? bunit[2 * nb + slot] * (disp(4) - 2.0 * d3 + d2) : 0.0;
                gacc += (double)lv[2] * (2.0 * C0 - Cm - Cp);
                if (!in_m) gacc -= C0 * (double)lv[1];
                if (!in_p) gacc -= C0 * (double)lv[3];
            }
        }
        gterm[slot] = gacc;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) lamDo[c * m + l] = lamD[c * m + l] + lX[c * m + l] + out[c];
}

// One block per segment: the segment's terms in slot order, strided over the
// threads, then a fixed tree: the same sum on every run (FP64).
constexpr int SEG_THREADS = 256;

__global__ void __launch_bounds__(SEG_THREADS)
    k_seg_reduce(const int32_t *__restrict__ seg_off, const int32_t *__restrict__ seg_slot,
                 const double *__restrict__ gterm, double *__restrict__ gseg)
{
    PDL_ENTRY();
    __shared__ double part[SEG_THREADS];
    const int s = blockIdx.x;
    double acc = 0.0;
    for (int i = seg_off[s] + threadIdx.x; i < seg_off[s + 1]; i += SEG_THREADS) acc += gterm[seg_slot[i]];
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int w = SEG_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) gseg[s] = part[0];
}

__global__ void k_add_f64(int n, const double *__restrict__ src, double *__restrict__ dst)
{
    PDL_ENTRY();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] += src[i];
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <class T> static void adv_adjoint_impl(ib_ctx *c, const void *lw, void *out, cudaStream_t s)
{
    const int advect = (c->desc.flags & IB_NO_ADVECTION) ? 0 : 1;
    launch_pdl(k_adv_adjoint<T>, dim3((unsigned)((c->dim.nx * c->dim.ny + 255) / 256), c->dim.nz), dim3(256), 0, s,
        c->dim, (const T *)c->u, (const T *)lw, (T *)out, (T)(c->desc.rho / c->desc.dt), (T)c->desc.rho,
        (T)(1.0 / c->desc.h), advect);
}

void launch_adv_adjoint(ib_ctx *c, const void *lw, void *lam_u_out, cudaStream_t s)
{
    if (c->fp64) adv_adjoint_impl<double>(c, lw, lam_u_out, s);
    else adv_adjoint_impl<float>(c, lw, lam_u_out, s);
}

template <class T> static void adj_markers_impl(ib_ctx *c, const void *u1, const void *lw, cudaStream_t s)
{
    auto &mk = c->mk;
    const int m = (int)mk.m;
    if (m == 0) return;
    const double h = c->desc.h;
    GridDims g = c->dim;
    g.nmark = m;
    const size_t smem = adj_interp_smem<T>();
    cudaFuncSetAttribute(k_adj_interp<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adj_interp<T>, AI_THREADS, smem);
    if (per_sm > 8) per_sm = 8;
    if (per_sm < 1) per_sm = 1;
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    launch_pdl(k_adj_interp<T>, dim3(persistent_grid(c, nsm * per_sm)), dim3(AI_THREADS), smem, s, 
        g, c->bin_start, mk.key_s, mk.perm, (const T *)mk.rfrac, (const Record<T> *)mk.rec,
        (const Record<T> *)mk.rec2, c->items, c->item_ctl, (const T *)u1, (const T *)lw, (T)(1.0 / (h * h * h)),
        (T)(1.0 / h), (T *)mk.lf_s, (T *)mk.lX_s);
    const int nb = (m + 255) / 256;
    launch_pdl(k_adj_move<T>, dim3(nb), dim3(256), 0, s, m, mk.perm, (const T *)mk.lf_s, (const T *)mk.lX_s, (T *)mk.lf, (T *)mk.lX,
               c->item_ctl);
    launch_pdl(k_adj_markers<T>, dim3(nb), dim3(256), 0, s, force_args<T>(c), (const T *)mk.lf, (const T *)mk.lX, (const T *)mk.lamD,
                                        (T *)mk.lamDo, mk.bunit, mk.bseg, mk.gterm);
    if (mk.n_seg > 0 && mk.nb > 0)
        launch_pdl(k_seg_reduce, dim3(mk.n_seg), dim3(SEG_THREADS), 0, s, mk.seg_off, mk.seg_slot, mk.gterm, mk.gseg);
}

void launch_adj_markers(ib_ctx *c, const void *u1, const void *lw, cudaStream_t s)
{
    if (c->fp64) adj_markers_impl<double>(c, u1, lw, s);
    else adj_markers_impl<float>(c, u1, lw, s);
}

void launch_grad_accumulate(ib_ctx *c, double *grad_b, cudaStream_t s)
{
    const int n = c->mk.n_seg;
    if (n > 0) launch_pdl(k_add_f64, dim3((n + 255) / 256), dim3(256), 0, s, n, c->mk.gseg, grad_b);
}

}  // namespace ibgb
