/*
 * Plain FP64 CPU oracle for the first-order immersed-boundary (IB) time step
 * of Givelberg & Bunn, "A Comprehensive Three-Dimensional Model of the
 * Cochlea", Section 3.2 ("The Numerical Method").
 *
 * TEST INFRASTRUCTURE: only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  The CUDA library never
 * links, calls or reads it, and it shares no code with it.
 *
 * Every function is a direct, unblocked transcription of the definitions it
 * cites: nested loops, no fusion, no reordering.  Compiled with
 * -ffp-contract=off so that no multiply-add is fused behind the reader's back.
 *
 * Grid layout: a field component is [z][y][x] with x fastest; a vector field
 * is [c][z][y][x].  Marker arrays are [c][m].  Lattice node (i, j, k) sits at
 * x = h (i, j, k) (Eq. discreteX's summation lattice).
 *
 * Readings of the paper where it is silent:
 *  - upwind difference with u_k = 0 contributes zero (Eq. discreteNS1 lists
 *    only u_k > 0 and u_k < 0);
 *  - modes where every sin(2 pi k_j / n_j) vanishes receive no projection and
 *    zero pressure (the null space of D0 on an even periodic grid);
 *  - markers carry force f(q) dq directly (per-marker force, dyn);
 *  - the shell bending force (deferred by the paper to Givelberg's thesis,
 *    which is not available) is a discrete beam law on the length-wise
 *    lattice lines, measured from the rest shape:
 *      E = sum_lines sum_i 1/2 c_i |v_i - v0_i|^2,  v_i = X_{i+1} - 2 X_i + X_{i-1},
 *      c_i = b_seg(i) dw_i / ds^3;
 *  - positions are never wrapped, only grid indices are;
 *  - positions are carried as X = X0 + D (reference plus displacement, both
 *    FP64) so that nanometre displacements keep full precision.
 *
 * Parity status: every function here is pinned by the CPU tests (closed
 * forms, brute force, a dense direct solve, invariants).  The nonlinear
 * upwind advection term is pinned by hand-computed values on a small grid
 * and, on random fields of both signs, by identities whose right-hand sides
 * come from periodic shifts alone: A(u) + A(-u) is the central difference
 * sum_d u_d (u(+e_d) - u(-e_d)) / h, A(u) - A(-u) is
 * sum_d |u_d| (2u - u(+e_d) - u(-e_d)) / h, and A(2u) = 4 A(u).  The reverse time step
 * (or_adjoint_step and its parts, at the end of this file) is pinned by the
 * moment identities of phi' and by central finite differences of the forward
 * functions above, one and two steps deep.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

typedef struct {
    int64_t first;
    int32_t n1, n2;
    double ds;
    const double *dw;          /* [n1] */
    const int32_t *seg_of_row; /* [n1] */
} or_sheet;

typedef struct {
    double center[3];
    double direction[3];
    double radius;
    double half_len;
    double amp;
    double omega;
} or_forcing;

typedef struct {
    int64_t m;
    const double *X0;          /* [3][m] */
    int64_t n_spring;
    const int32_t *spring_ij;  /* [n_spring][2] */
    const double *spring_k;
    const double *spring_L0;
    int64_t n_tether;
    const int32_t *tether_i;
    const double *tether_k;
    int32_t n_sheet;
    const or_sheet *sheets;
    int32_t n_seg;
    const double *bend_b;
    or_forcing forcing;
    /* external marker force: amp cos(omega t) dir_j on marker mforce_i[j]
     * (the oval window's stapes load, Section 4) */
    int64_t n_mforce;
    const int32_t *mforce_i;
    const double *mforce_dir;  /* [3][n_mforce] */
    double mforce_amp, mforce_omega;
} or_structure;

typedef struct {
    int32_t n[3];
    double h, rho, mu, dt;
    int32_t no_advection;      /* 1: drop the advection term (Stokes) */
} or_grid;

static int64_t grid_size(const or_grid *g) { return (int64_t)g->n[0] * g->n[1] * g->n[2]; }

static int64_t wrap(int64_t i, int64_t n) { return ((i % n) + n) % n; }

static int64_t node(const or_grid *g, int64_t i, int64_t j, int64_t k)
{
    return (wrap(k, g->n[2]) * g->n[1] + wrap(j, g->n[1])) * g->n[0] + wrap(i, g->n[0]);
}

/* ------------------------------------------------------------------------
 * The 4-point delta kernel phi (Section 3.2, definition of delta_h).
 * ------------------------------------------------------------------------ */
double or_phi(double r)
{
    double a = fabs(r);
    if (a <= 1.0)
        return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
    if (a <= 2.0)
        return 0.5 - or_phi(2.0 - a);
    return 0.0;
}

/* Stencil of one coordinate: first node i0 = floor(x/h) - 1 and the four
 * weights phi(x/h - (i0 + a)), a = 0..3 (nodes outside [i0, i0+3] have
 * |x/h - i| >= 2 and weight 0).  x/h is one FP64 multiply by 1/h. */
static void stencil(double x, double inv_h, int64_t *i0, double w[4])
{
    double s = x * inv_h;
    int64_t b = (int64_t)floor(s);
    *i0 = b - 1;
    for (int a = 0; a < 4; a++)
        w[a] = or_phi(s - (double)(*i0 + a));
}

/* ------------------------------------------------------------------------
 * Eq. (discreteF): F(x) = sum_l f_l delta_h(x - X_l), delta_h = h^-3 phi phi phi.
 * F is overwritten.  X, f: [3][m]; F: [3][G].
 * ------------------------------------------------------------------------ */
void or_spread(const or_grid *g, int64_t m, const double *X, const double *f, double *F)
{
    int64_t G = grid_size(g);
    double inv_h = 1.0 / g->h;
    double inv_h3 = 1.0 / (g->h * g->h * g->h);
    memset(F, 0, sizeof(double) * 3 * G);
    for (int64_t l = 0; l < m; l++) {
        int64_t i0[3];
        double w[3][4];
        for (int c = 0; c < 3; c++)
            stencil(X[c * m + l], inv_h, &i0[c], w[c]);
        for (int c3 = 0; c3 < 4; c3++)
            for (int c2 = 0; c2 < 4; c2++)
                for (int c1 = 0; c1 < 4; c1++) {
                    double d = w[0][c1] * w[1][c2] * w[2][c3] * inv_h3;
                    int64_t q = node(g, i0[0] + c1, i0[1] + c2, i0[2] + c3);
                    for (int c = 0; c < 3; c++)
                        F[c * G + q] += f[c * m + l] * d;
                }
    }
}

/* ------------------------------------------------------------------------
 * Eq. (discreteX), velocity part: U_l = sum_x u(x) delta_h(x - X_l) h^3.
 * u: [3][G]; U: [3][m] (overwritten).
 * ------------------------------------------------------------------------ */
void or_interp(const or_grid *g, int64_t m, const double *X, const double *u, double *U)
{
    int64_t G = grid_size(g);
    double inv_h = 1.0 / g->h;
    for (int64_t l = 0; l < m; l++) {
        int64_t i0[3];
        double w[3][4];
        double acc[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c < 3; c++)
            stencil(X[c * m + l], inv_h, &i0[c], w[c]);
        for (int c3 = 0; c3 < 4; c3++)
            for (int c2 = 0; c2 < 4; c2++)
                for (int c1 = 0; c1 < 4; c1++) {
                    double d = w[0][c1] * w[1][c2] * w[2][c3];
                    int64_t q = node(g, i0[0] + c1, i0[1] + c2, i0[2] + c3);
                    for (int c = 0; c < 3; c++)
                        acc[c] += u[c * G + q] * d;
                }
        for (int c = 0; c < 3; c++)
            U[c * m + l] = acc[c];
    }
}

/* ------------------------------------------------------------------------
 * Markers sorted into grid cells: the key of cell (i, j, k) = floor(X/h)
 * (indices wrapped) enumerates cells tile by tile, 8^3-cell tiles in
 * (z, y, x) order and cells within a tile in (z, y, x) order:
 *   key = ((k/8 * nty + j/8) * ntx + i/8) * 512 + ((k%8) * 8 + j%8) * 8 + i%8,
 * with nt = ceil(n/8); perm = marker ids sorted stably by tile (key / 512),
 * i.e. by (tile, id).
 * ------------------------------------------------------------------------ */
typedef struct { int64_t key; int64_t id; } kv;   /* key: the tile of the marker's cell */

static int kv_cmp(const void *a, const void *b)
{
    const kv *p = a, *q = b;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    return p->id < q->id ? -1 : (p->id > q->id);
}

void or_bin_sort(const or_grid *g, int64_t m, const double *X, int32_t *key, int32_t *perm)
{
    double inv_h = 1.0 / g->h;
    kv *a = malloc(sizeof(kv) * (m > 0 ? m : 1));
    for (int64_t l = 0; l < m; l++) {
        int64_t b[3];
        for (int c = 0; c < 3; c++)
            b[c] = (int64_t)floor(X[c * m + l] * inv_h);
        int64_t i = wrap(b[0], g->n[0]), j = wrap(b[1], g->n[1]), k = wrap(b[2], g->n[2]);
        int64_t ntx = (g->n[0] + 7) / 8, nty = (g->n[1] + 7) / 8;
        int64_t cell_key = ((k / 8 * nty + j / 8) * ntx + i / 8) * 512 + ((k % 8) * 8 + j % 8) * 8 + i % 8;
        a[l].key = cell_key / 512;
        a[l].id = l;
        key[l] = (int32_t)cell_key;
    }
    qsort(a, m, sizeof(kv), kv_cmp);
    for (int64_t l = 0; l < m; l++)
        perm[l] = (int32_t)a[l].id;
    free(a);
}

/* ------------------------------------------------------------------------
 * Marker positions are carried as X = X0 + D: the structure's reference
 * position X0 plus a displacement D, both FP64, so that the nanometre
 * displacements of the model (Section 2.1) keep full precision instead of
 * being rounded against centimetre coordinates.
 *
 * Marker forces f (per marker, dyn), in fixed order: springs, tethers,
 * membrane bending.  Springs (Peskin's fiber links): e = X_j - X_i,
 * r = |e|, f_i += k (r - L0) e / r, f_j -= the same.  Tethers:
 * f_i += -k (X_i - X0_i).  Bending: see the header.  Every difference of
 * positions is formed as (X0 difference) + (D difference), which equals the
 * position difference in exact arithmetic.
 * ------------------------------------------------------------------------ */
static double pos_diff(const or_structure *s, const double *D, int c, int64_t j, int64_t i)
{
    int64_t m = s->m;
    return (s->X0[c * m + j] - s->X0[c * m + i]) + (D[c * m + j] - D[c * m + i]);
}

/* v_i - v0_i = (X_{i+1} - 2 X_i + X_{i-1}) - (X0_{i+1} - 2 X0_i + X0_{i-1}) */
static double bend_dev(const or_structure *s, const double *D, int c, int64_t im, int64_t i0, int64_t ip)
{
    int64_t m = s->m;
    return D[c * m + ip] - 2.0 * D[c * m + i0] + D[c * m + im];
}

void or_forces(const or_structure *s, const double *D, double *f)
{
    int64_t m = s->m;
    memset(f, 0, sizeof(double) * 3 * m);
    for (int64_t e = 0; e < s->n_spring; e++) {
        int64_t i = s->spring_ij[2 * e], j = s->spring_ij[2 * e + 1];
        double d[3], r2 = 0.0;
        for (int c = 0; c < 3; c++) {
            d[c] = pos_diff(s, D, c, j, i);
            r2 += d[c] * d[c];
        }
        double r = sqrt(r2);
        double t = s->spring_k[e] * (r - s->spring_L0[e]) / r;
        for (int c = 0; c < 3; c++) {
            f[c * m + i] += t * d[c];
            f[c * m + j] -= t * d[c];
        }
    }
    for (int64_t e = 0; e < s->n_tether; e++) {
        int64_t i = s->tether_i[e];
        for (int c = 0; c < 3; c++)
            f[c * m + i] += -s->tether_k[e] * D[c * m + i];
    }
    for (int q = 0; q < s->n_sheet; q++) {
        const or_sheet *sh = &s->sheets[q];
        for (int32_t a = 0; a < sh->n2; a++)
            for (int32_t i = 1; i + 1 < sh->n1; i++) {
                int64_t im = sh->first + (int64_t)(i - 1) * sh->n2 + a;
                int64_t i0 = sh->first + (int64_t)i * sh->n2 + a;
                int64_t ip = sh->first + (int64_t)(i + 1) * sh->n2 + a;
                double cb = s->bend_b[sh->seg_of_row[i]] * sh->dw[i] / (sh->ds * sh->ds * sh->ds);
                for (int c = 0; c < 3; c++) {
                    double gv = cb * bend_dev(s, D, c, im, i0, ip);
                    f[c * m + im] -= gv;
                    f[c * m + i0] += 2.0 * gv;
                    f[c * m + ip] -= gv;
                }
            }
    }
}

/* External marker force at time t, added to f: a force field orthogonal to
 * the oval window whose magnitude varies sinusoidally with the input tone
 * (Section 4): f_i += amp cos(omega t) dir_j for i = mforce_i[j]. */
void or_marker_forcing(const or_structure *s, double t, double *f)
{
    if (s->n_mforce == 0 || s->mforce_amp == 0.0) return;
    int64_t m = s->m;
    double a = s->mforce_amp * cos(s->mforce_omega * t);
    for (int64_t j = 0; j < s->n_mforce; j++) {
        int64_t i = s->mforce_i[j];
        for (int c = 0; c < 3; c++) f[c * m + i] += a * s->mforce_dir[c * s->n_mforce + j];
    }
}

/* Elastic energy whose negative gradient is or_forces (springs
 * 1/2 k (r - L0)^2, tethers 1/2 k |X - X0|^2, bending as in the header). */
double or_energy(const or_structure *s, const double *D)
{
    int64_t m = s->m;
    double E = 0.0;
    for (int64_t e = 0; e < s->n_spring; e++) {
        int64_t i = s->spring_ij[2 * e], j = s->spring_ij[2 * e + 1];
        double r2 = 0.0;
        for (int c = 0; c < 3; c++) {
            double d = pos_diff(s, D, c, j, i);
            r2 += d * d;
        }
        double x = sqrt(r2) - s->spring_L0[e];
        E += 0.5 * s->spring_k[e] * x * x;
    }
    for (int64_t e = 0; e < s->n_tether; e++) {
        int64_t i = s->tether_i[e];
        for (int c = 0; c < 3; c++) {
            double d = D[c * m + i];
            E += 0.5 * s->tether_k[e] * d * d;
        }
    }
    for (int q = 0; q < s->n_sheet; q++) {
        const or_sheet *sh = &s->sheets[q];
        for (int32_t a = 0; a < sh->n2; a++)
            for (int32_t i = 1; i + 1 < sh->n1; i++) {
                int64_t im = sh->first + (int64_t)(i - 1) * sh->n2 + a;
                int64_t i0 = sh->first + (int64_t)i * sh->n2 + a;
                int64_t ip = sh->first + (int64_t)(i + 1) * sh->n2 + a;
                double cb = s->bend_b[sh->seg_of_row[i]] * sh->dw[i] / (sh->ds * sh->ds * sh->ds);
                for (int c = 0; c < 3; c++) {
                    double dv = bend_dev(s, D, c, im, i0, ip);
                    E += 0.5 * cb * dv * dv;
                }
            }
    }
    return E;
}

/* ------------------------------------------------------------------------
 * Body force G(x, t): rho * amp * omega * cos(omega t) * direction on the
 * nodes x = h (i, j, k) with |(x - C).dir| <= half_len and
 * |x - C|^2 - ((x - C).dir)^2 <= radius^2.  Added to F.
 * ------------------------------------------------------------------------ */
void or_body_force(const or_grid *g, const or_forcing *fo, double rho, double t, double *F)
{
    if (fo->amp == 0.0) return;
    int64_t G = grid_size(g);
    double mag = rho * fo->amp * fo->omega * cos(fo->omega * t);
    for (int64_t k = 0; k < g->n[2]; k++)
        for (int64_t j = 0; j < g->n[1]; j++)
            for (int64_t i = 0; i < g->n[0]; i++) {
                double d0 = g->h * (double)i - fo->center[0];
                double d1 = g->h * (double)j - fo->center[1];
                double d2 = g->h * (double)k - fo->center[2];
                double along = d0 * fo->direction[0] + d1 * fo->direction[1] + d2 * fo->direction[2];
                double perp2 = d0 * d0 + d1 * d1 + d2 * d2 - along * along;
                if (fabs(along) <= fo->half_len && perp2 <= fo->radius * fo->radius) {
                    int64_t q = (k * g->n[1] + j) * g->n[0] + i;
                    for (int c = 0; c < 3; c++)
                        F[c * G + q] += mag * fo->direction[c];
                }
            }
}

/* ------------------------------------------------------------------------
 * Upwind advection term of Eq. (discreteNS1): A_i = sum_k u_k D_k^(+-) u_i,
 * D_k^- for u_k > 0, D_k^+ for u_k < 0, zero for u_k = 0.  u, A: [3][G].
 * ------------------------------------------------------------------------ */
void or_advection(const or_grid *g, const double *u, double *A)
{
    int64_t G = grid_size(g);
    double h = g->h;
    for (int64_t k = 0; k < g->n[2]; k++)
        for (int64_t j = 0; j < g->n[1]; j++)
            for (int64_t i = 0; i < g->n[0]; i++) {
                int64_t q = node(g, i, j, k);
                int64_t minus[3] = {node(g, i - 1, j, k), node(g, i, j - 1, k), node(g, i, j, k - 1)};
                int64_t plus[3] = {node(g, i + 1, j, k), node(g, i, j + 1, k), node(g, i, j, k + 1)};
                for (int c = 0; c < 3; c++) {
                    double acc = 0.0;
                    for (int d = 0; d < 3; d++) {
                        double uk = u[d * G + q];
                        double diff;
                        if (uk > 0.0)
                            diff = (u[c * G + q] - u[c * G + minus[d]]) / h;   /* D_k^- */
                        else if (uk < 0.0)
                            diff = (u[c * G + plus[d]] - u[c * G + q]) / h;    /* D_k^+ */
                        else
                            diff = 0.0;
                        acc += uk * diff;
                    }
                    A[c * G + q] = acc;
                }
            }
}

/* Right-hand side of Eq. (discreteNS1) moved to known terms:
 * w = rho u / dt - rho A(u) + F.  All [3][G]. */
void or_rhs(const or_grid *g, const double *u, const double *F, double *w)
{
    int64_t G = grid_size(g);
    double *A = calloc(3 * G, sizeof(double));
    if (!g->no_advection)
        or_advection(g, u, A);
    for (int64_t q = 0; q < 3 * G; q++)
        w[q] = g->rho * u[q] / g->dt - g->rho * A[q] + F[q];
    free(A);
}

/* ------------------------------------------------------------------------
 * Discrete Fourier transform, mixed radix, decimation in time:
 *   X[k] = sum_j x[j] exp(sign 2 pi i j k / n).
 * The length splits as n = p q with p its smallest prime factor; the q-point
 * sub-transforms of the p interleaved subsequences combine by a direct
 * p-point sum with twiddles exp(sign 2 pi i r (k + q s) / n).
 * W[t] = exp(sign 2 pi i t / Wn) with n dividing Wn; scratch holds 2n.
 * ------------------------------------------------------------------------ */
static int smallest_factor(int n)
{
    for (int p = 2; p * p <= n; p++)
        if (n % p == 0) return p;
    return n;
}

static void dft_rec(const cplx *in, int64_t istride, cplx *out, int n, const cplx *W, int Wn, cplx *scratch)
{
    if (n == 1) {
        out[0] = in[0];
        return;
    }
    int p = smallest_factor(n), q = n / p;
    for (int r = 0; r < p; r++)
        dft_rec(in + r * istride, istride * p, out + r * q, q, W, Wn, scratch + n);
    cplx *tmp = scratch;
    int step = Wn / n;
    for (int k = 0; k < q; k++)
        for (int s = 0; s < p; s++) {
            cplx acc = 0.0;
            for (int r = 0; r < p; r++) {
                int t = (r * (k + q * s)) % n;
                acc += W[t * step] * out[r * q + k];
            }
            tmp[k + q * s] = acc;
        }
    memcpy(out, tmp, sizeof(cplx) * n);
}

static cplx *twiddles(int n, int sign)
{
    cplx *W = malloc(sizeof(cplx) * n);
    for (int t = 0; t < n; t++) {
        double a = 2.0 * M_PI * (double)t / (double)n;
        W[t] = cos(a) + (double)sign * sin(a) * I;
    }
    return W;
}

/* 1-D transform of every line of a [nz][ny][nx] complex array along axis
 * ``axis`` (0 = x, 1 = y, 2 = z).  sign = -1 forward, +1 inverse (unscaled). */
static void dft_axis(const or_grid *g, cplx *a, int axis, int sign)
{
    int n = g->n[axis];
    int64_t stride = axis == 0 ? 1 : (axis == 1 ? g->n[0] : (int64_t)g->n[0] * g->n[1]);
    int64_t G = grid_size(g);
    cplx *W = twiddles(n, sign);
    cplx *line = malloc(sizeof(cplx) * n), *res = malloc(sizeof(cplx) * n);
    cplx *scratch = malloc(sizeof(cplx) * 4 * n);
    for (int64_t base = 0; base < G; base++) {
        /* a line starts at every index whose coordinate along ``axis`` is 0 */
        int64_t coord = (base / stride) % n;
        if (coord != 0) continue;
        for (int t = 0; t < n; t++) line[t] = a[base + t * stride];
        dft_rec(line, 1, res, n, W, n, scratch);
        for (int t = 0; t < n; t++) a[base + t * stride] = res[t];
    }
    free(W);
    free(line);
    free(res);
    free(scratch);
}

/* Complex 3-D DFT in place (unscaled).  a: [nz][ny][nx]. */
void or_dft3(const or_grid *g, double *re, double *im, int sign)
{
    int64_t G = grid_size(g);
    cplx *a = malloc(sizeof(cplx) * G);
    for (int64_t q = 0; q < G; q++) a[q] = re[q] + im[q] * I;
    for (int axis = 0; axis < 3; axis++) dft_axis(g, a, axis, sign);
    for (int64_t q = 0; q < G; q++) {
        re[q] = creal(a[q]);
        im[q] = cimag(a[q]);
    }
    free(a);
}

/* 1-D transform of one contiguous line of length n (for the DFT pins). */
void or_dft1(int n, double *re, double *im, int sign)
{
    cplx *W = twiddles(n, sign);
    cplx *line = malloc(sizeof(cplx) * n), *res = malloc(sizeof(cplx) * n);
    cplx *scratch = malloc(sizeof(cplx) * 4 * n);
    for (int t = 0; t < n; t++) line[t] = re[t] + im[t] * I;
    dft_rec(line, 1, res, n, W, n, scratch);
    for (int t = 0; t < n; t++) {
        re[t] = creal(res[t]);
        im[t] = cimag(res[t]);
    }
    free(W);
    free(line);
    free(res);
    free(scratch);
}

/* ------------------------------------------------------------------------
 * Solve Eqs. (discreteNS1)-(discreteNS2) for u' and p given the known terms
 * w (see or_rhs):
 *   (rho/dt) u' - mu sum_k D_k^+ D_k^- u' + D0 p = w,   D0 . u' = 0.
 * Per Fourier mode k: D0 -> i s, s_j = sin(2 pi k_j / n_j) / h;
 * D+D- -> -(4/h^2) sin^2(pi k_j / n_j); a = rho/dt + (4 mu/h^2) sum_j sin^2.
 * If |s|^2 > 0: p^ = -i (s.w^)/|s|^2, u'^ = (w^ - s (s.w^)/|s|^2) / a;
 * else p^ = 0, u'^ = w^ / a.   w, u_new: [3][G]; p: [G] or NULL.
 * ------------------------------------------------------------------------ */
void or_solve(const or_grid *g, const double *w, double *u_new, double *p)
{
    int64_t G = grid_size(g);
    double h = g->h;
    double *re = malloc(sizeof(double) * 4 * G), *im = malloc(sizeof(double) * 4 * G);
    for (int c = 0; c < 3; c++) {
        memcpy(re + c * G, w + c * G, sizeof(double) * G);
        memset(im + c * G, 0, sizeof(double) * G);
        or_dft3(g, re + c * G, im + c * G, -1);
    }
    for (int64_t kz = 0; kz < g->n[2]; kz++)
        for (int64_t ky = 0; ky < g->n[1]; ky++)
            for (int64_t kx = 0; kx < g->n[0]; kx++) {
                int64_t q = (kz * g->n[1] + ky) * g->n[0] + kx;
                int64_t kk[3] = {kx, ky, kz};
                double s[3], a = g->rho / g->dt, s2 = 0.0;
                for (int j = 0; j < 3; j++) {
                    /* sin(2 pi k / n) is exactly zero at k = 0 and k = n/2; the
                     * rounded pi would give ~1e-16 there and wrongly switch on
                     * the projection of a mode that D0 does not see. */
                    s[j] = (2 * kk[j]) % g->n[j] == 0 ? 0.0
                                                     : sin(2.0 * M_PI * (double)kk[j] / (double)g->n[j]) / h;
                    double sn = sin(M_PI * (double)kk[j] / (double)g->n[j]);
                    a += 4.0 * g->mu / (h * h) * sn * sn;
                    s2 += s[j] * s[j];
                }
                cplx wh[3], sw = 0.0;
                for (int c = 0; c < 3; c++) {
                    wh[c] = re[c * G + q] + im[c * G + q] * I;
                    sw += s[c] * wh[c];
                }
                cplx ph = 0.0;
                for (int c = 0; c < 3; c++) {
                    cplx uh = s2 > 0.0 ? (wh[c] - s[c] * sw / s2) / a : wh[c] / a;
                    re[c * G + q] = creal(uh);
                    im[c * G + q] = cimag(uh);
                }
                if (s2 > 0.0) ph = -I * sw / s2;
                re[3 * G + q] = creal(ph);
                im[3 * G + q] = cimag(ph);
            }
    for (int c = 0; c < 4; c++) {
        if (c == 3 && !p) break;
        or_dft3(g, re + c * G, im + c * G, +1);
        double *dst = c < 3 ? u_new + c * G : p;
        for (int64_t q = 0; q < G; q++) dst[q] = re[c * G + q] / (double)G;
    }
    free(re);
    free(im);
}

/* Step 3 of the time step: u^{n+1} (and p^{n+1}) from u^n and F^n. */
void or_fluid_solve(const or_grid *g, const double *u, const double *F, double *u_new, double *p)
{
    int64_t G = grid_size(g);
    double *w = malloc(sizeof(double) * 3 * G);
    or_rhs(g, u, F, w);
    or_solve(g, w, u_new, p);
    free(w);
}

/* ------------------------------------------------------------------------
 * The first-order IB time step (Section 3.2, steps 1-4), nsteps times:
 *  1. f^n from X^n (or_forces) plus the external marker force at t^n;
 *  2. F^n = spread of f^n at X^n (Eq. discreteF) plus the body force at t^n;
 *  3. u^{n+1} from u^n and F^n (Eqs. discreteNS1-2);
 *  4. X^{n+1} = X^n + dt * interp of u^{n+1} at X^n (Eq. discreteX),
 *     carried as D^{n+1} = D^n + dt * U with X = X0 + D.
 * D: [3][m] displacement from s->X0, u: [3][G], t: scalar (all updated).
 * ------------------------------------------------------------------------ */
void or_step(const or_grid *g, const or_structure *s, double *D, double *u, double *t, int64_t nsteps)
{
    int64_t G = grid_size(g), m = s->m;
    int64_t mm = m > 0 ? m : 1;
    double *f = malloc(sizeof(double) * 3 * mm);
    double *U = malloc(sizeof(double) * 3 * mm);
    double *X = malloc(sizeof(double) * 3 * mm);
    double *F = malloc(sizeof(double) * 3 * G);
    double *un = malloc(sizeof(double) * 3 * G);
    for (int64_t n = 0; n < nsteps; n++) {
        for (int64_t q = 0; q < 3 * m; q++) X[q] = s->X0[q] + D[q];
        or_forces(s, D, f);
        or_marker_forcing(s, *t, f);
        or_spread(g, m, X, f, F);
        or_body_force(g, &s->forcing, g->rho, *t, F);
        or_fluid_solve(g, u, F, un, NULL);
        memcpy(u, un, sizeof(double) * 3 * G);
        or_interp(g, m, X, u, U);
        for (int64_t q = 0; q < 3 * m; q++) D[q] += g->dt * U[q];
        *t += g->dt;
    }
    free(f);
    free(U);
    free(X);
    free(F);
    free(un);
}

/* ========================================================================
 * Adjoint of one time step: the exact transpose of the linearisation of
 * steps 1-4 above, taken term by term from the forward definitions.
 * ======================================================================== */

/* phi'(r), from the two branches of phi (Section 3.2, definition of delta_h):
 * inner a = |r| <= 1: d/da (3 - 2a + sqrt(1 + 4a - 4a^2))/8
 *                   = (-2 + (2 - 4a)/sqrt(1 + 4a - 4a^2))/8;
 * outer 1 <= a <= 2: d/da (1/2 - phi(2 - a)) = phi_inner'(2 - a). */
static double phi_inner_d(double a)
{
    return (-2.0 + (2.0 - 4.0 * a) / sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
}

double or_phi_d(double r)
{
    double a = fabs(r), sg = r < 0.0 ? -1.0 : 1.0;
    if (a <= 1.0) return sg * phi_inner_d(a);
    if (a <= 2.0) return sg * phi_inner_d(2.0 - a);
    return 0.0;
}

/* Stencil weights and their derivatives d/ds (s = x/h) of one coordinate. */
static void stencil_d(double x, double inv_h, int64_t *i0, double w[4], double dw[4])
{
    double s = x * inv_h;
    int64_t b = (int64_t)floor(s);
    *i0 = b - 1;
    for (int a = 0; a < 4; a++) {
        w[a] = or_phi(s - (double)(*i0 + a));
        dw[a] = or_phi_d(s - (double)(*i0 + a));
    }
}

/* out_l += scale * sum_x sum_c v_c(l) u_c(x) grad_{X_l} [phi phi phi](X_l/h - x/h),
 * the derivative of interpolation with respect to the marker position,
 * contracted with a per-marker vector v.  X, v, out: [3][m]; u: [3][G]. */
void or_interp_grad(const or_grid *g, int64_t m, const double *X, const double *u, const double *v, double scale,
                    double *out)
{
    int64_t G = grid_size(g);
    double inv_h = 1.0 / g->h;
    for (int64_t l = 0; l < m; l++) {
        int64_t i0[3];
        double w[3][4], dw[3][4];
        for (int c = 0; c < 3; c++)
            stencil_d(X[c * m + l], inv_h, &i0[c], w[c], dw[c]);
        double acc[3] = {0.0, 0.0, 0.0};
        for (int c3 = 0; c3 < 4; c3++)
            for (int c2 = 0; c2 < 4; c2++)
                for (int c1 = 0; c1 < 4; c1++) {
                    int64_t q = node(g, i0[0] + c1, i0[1] + c2, i0[2] + c3);
                    double sv = 0.0;
                    for (int c = 0; c < 3; c++) sv += v[c * m + l] * u[c * G + q];
                    acc[0] += sv * dw[0][c1] * w[1][c2] * w[2][c3] * inv_h;
                    acc[1] += sv * w[0][c1] * dw[1][c2] * w[2][c3] * inv_h;
                    acc[2] += sv * w[0][c1] * w[1][c2] * dw[2][c3] * inv_h;
                }
        for (int a = 0; a < 3; a++) out[a * m + l] += scale * acc[a];
    }
}

/* out = (dA/du)^T lam for the upwind term A of Eq. (discreteNS1), where
 * A_i(c) = sum_k u_k(c) Dpm_k u_i(c) with the branch chosen by the sign of
 * u_k(c) (held fixed: the derivative where it exists).  Written as the
 * transpose of the forward loop: every forward dependence scatters back. */
void or_advection_adjoint(const or_grid *g, const double *u, const double *lam, double *out)
{
    int64_t G = grid_size(g);
    double h = g->h;
    memset(out, 0, sizeof(double) * 3 * G);
    for (int64_t k = 0; k < g->n[2]; k++)
        for (int64_t j = 0; j < g->n[1]; j++)
            for (int64_t i = 0; i < g->n[0]; i++) {
                int64_t q = node(g, i, j, k);
                int64_t minus[3] = {node(g, i - 1, j, k), node(g, i, j - 1, k), node(g, i, j, k - 1)};
                int64_t plus[3] = {node(g, i + 1, j, k), node(g, i, j + 1, k), node(g, i, j, k + 1)};
                for (int c = 0; c < 3; c++) {
                    double L = lam[c * G + q];
                    for (int d = 0; d < 3; d++) {
                        double uk = u[d * G + q];
                        if (uk > 0.0) {
                            double diff = (u[c * G + q] - u[c * G + minus[d]]) / h;
                            out[d * G + q] += L * diff;              /* d/du_k(c) */
                            out[c * G + q] += L * uk / h;            /* d/du_i(c) */
                            out[c * G + minus[d]] -= L * uk / h;     /* d/du_i(c - e_k) */
                        } else if (uk < 0.0) {
                            double diff = (u[c * G + plus[d]] - u[c * G + q]) / h;
                            out[d * G + q] += L * diff;
                            out[c * G + plus[d]] += L * uk / h;
                            out[c * G + q] -= L * uk / h;
                        }
                    }
                }
            }
}

/* out = (df/dD) lam (= its transpose: f = -grad E is a Hessian product).
 * Springs: with e = X_j - X_i, r = |e|, the force k (r - L0) e / r has the
 * Jacobian K = k [(1 - L0/r) I + (L0/r) e e^T / r^2] with respect to e, so
 * out_i += K (lam_j - lam_i), out_j -= the same.  Tethers: -k lam_i.
 * Bending is linear in D: the bending force evaluated at displacement lam. */
void or_forces_lin(const or_structure *s, const double *D, const double *lam, double *out)
{
    int64_t m = s->m;
    memset(out, 0, sizeof(double) * 3 * m);
    for (int64_t e = 0; e < s->n_spring; e++) {
        int64_t i = s->spring_ij[2 * e], j = s->spring_ij[2 * e + 1];
        double d[3], r2 = 0.0, dl[3], ed = 0.0;
        for (int c = 0; c < 3; c++) {
            d[c] = pos_diff(s, D, c, j, i);
            r2 += d[c] * d[c];
            dl[c] = lam[c * m + j] - lam[c * m + i];
        }
        double r = sqrt(r2), L0 = s->spring_L0[e], k = s->spring_k[e];
        for (int c = 0; c < 3; c++) ed += d[c] * dl[c];
        for (int c = 0; c < 3; c++) {
            double v = k * ((1.0 - L0 / r) * dl[c] + (L0 / r) * d[c] * ed / r2);
            out[c * m + i] += v;
            out[c * m + j] -= v;
        }
    }
    for (int64_t e = 0; e < s->n_tether; e++) {
        int64_t i = s->tether_i[e];
        for (int c = 0; c < 3; c++) out[c * m + i] += -s->tether_k[e] * lam[c * m + i];
    }
    for (int q = 0; q < s->n_sheet; q++) {
        const or_sheet *sh = &s->sheets[q];
        for (int32_t a = 0; a < sh->n2; a++)
            for (int32_t i = 1; i + 1 < sh->n1; i++) {
                int64_t im = sh->first + (int64_t)(i - 1) * sh->n2 + a;
                int64_t i0 = sh->first + (int64_t)i * sh->n2 + a;
                int64_t ip = sh->first + (int64_t)(i + 1) * sh->n2 + a;
                double cb = s->bend_b[sh->seg_of_row[i]] * sh->dw[i] / (sh->ds * sh->ds * sh->ds);
                for (int c = 0; c < 3; c++) {
                    double gv = cb * (lam[c * m + ip] - 2.0 * lam[c * m + i0] + lam[c * m + im]);
                    out[c * m + im] -= gv;
                    out[c * m + i0] += 2.0 * gv;
                    out[c * m + ip] -= gv;
                }
            }
    }
}

/* grad[seg] += lam . df/db_seg: the bending force is linear in b, with
 * df/db = (dw_i/ds^3) times the bending pattern of row i's deviation. */
void or_forces_dbend(const or_structure *s, const double *D, const double *lam, double *grad)
{
    int64_t m = s->m;
    for (int q = 0; q < s->n_sheet; q++) {
        const or_sheet *sh = &s->sheets[q];
        for (int32_t a = 0; a < sh->n2; a++)
            for (int32_t i = 1; i + 1 < sh->n1; i++) {
                int64_t im = sh->first + (int64_t)(i - 1) * sh->n2 + a;
                int64_t i0 = sh->first + (int64_t)i * sh->n2 + a;
                int64_t ip = sh->first + (int64_t)(i + 1) * sh->n2 + a;
                double unit = sh->dw[i] / (sh->ds * sh->ds * sh->ds);
                double acc = 0.0;
                for (int c = 0; c < 3; c++) {
                    double v = bend_dev(s, D, c, im, i0, ip);
                    acc += unit * v * (-lam[c * m + im] + 2.0 * lam[c * m + i0] - lam[c * m + ip]);
                }
                grad[sh->seg_of_row[i]] += acc;
            }
    }
}

/* ------------------------------------------------------------------------
 * Reverse of one time step (steps 1-4 of or_step) about the state
 * (u^n, D^n, t^n).  Given the sensitivities lam_u1 = dJ/du^{n+1} [3][G] and
 * lam_D1 = dJ/dD^{n+1} [3][m] of a scalar J, returns lam_u0 = dJ/du^n,
 * lam_D0 = dJ/dD^n and adds dJ/db_seg to grad_b [n_seg].  Backwards through
 * the forward definitions (S = spread with delta_h, I = interp, L = the
 * solve of Eqs. discreteNS1-2, a real symmetric operator):
 *   D' = D + dt I(X) u'          lam_U = dt lam_D1
 *                                g     = lam_u1 + I(X)^T lam_U = lam_u1 + S(X)(h^3 lam_U)
 *                                lam_X = [d/dX I(X) u']^T lam_U
 *   u' = L w                     lam_w = L lam_u1'  (L^T = L)
 *   w = rho u/dt - rho A(u) + F  lam_u0 = rho lam_w/dt - rho (dA/du)^T lam_w
 *   F = S(X) f + body(t)         lam_f = S(X)^T lam_w = h^-3 I(X) lam_w
 *                                lam_X += [d/dX S(X) f]^T lam_w
 *   f = f(D; b)                  lam_D0 = lam_D1 + lam_X + (df/dD)^T lam_f
 *                                grad_b += (df/db)^T lam_f
 * The forward step is recomputed here to obtain f^n and u^{n+1}.
 * ------------------------------------------------------------------------ */
void or_adjoint_step(const or_grid *g, const or_structure *s, const double *D, const double *u, double t,
                     const double *lam_u1, const double *lam_D1, double *lam_u0, double *lam_D0, double *grad_b)
{
    int64_t G = grid_size(g), m = s->m;
    int64_t mm = m > 0 ? m : 1;
    double h3 = g->h * g->h * g->h;
    double *X = malloc(sizeof(double) * 3 * mm), *f = malloc(sizeof(double) * 3 * mm);
    double *lU = malloc(sizeof(double) * 3 * mm), *lX = calloc(3 * mm, sizeof(double));
    double *lf = malloc(sizeof(double) * 3 * mm), *kf = malloc(sizeof(double) * 3 * mm);
    double *F = malloc(sizeof(double) * 3 * G), *un = malloc(sizeof(double) * 3 * G);
    double *gw = malloc(sizeof(double) * 3 * G), *lw = malloc(sizeof(double) * 3 * G);
    double *adv = calloc(3 * G, sizeof(double));

    /* forward recompute: X^n, f^n, F^n, u^{n+1} */
    for (int64_t q = 0; q < 3 * m; q++) X[q] = s->X0[q] + D[q];
    or_forces(s, D, f);
    or_marker_forcing(s, t, f);
    or_spread(g, m, X, f, F);
    or_body_force(g, &s->forcing, g->rho, t, F);
    or_fluid_solve(g, u, F, un, NULL);

    /* step 4 reversed */
    for (int64_t q = 0; q < 3 * m; q++) lU[q] = g->dt * lam_D1[q] * h3;
    or_spread(g, m, X, lU, gw);                       /* S(X)(h^3 lam_U) = I^T lam_U */
    for (int64_t q = 0; q < 3 * G; q++) gw[q] += lam_u1[q];
    for (int64_t q = 0; q < 3 * m; q++) lU[q] = g->dt * lam_D1[q];
    or_interp_grad(g, m, X, un, lU, 1.0, lX);

    /* step 3 reversed */
    or_solve(g, gw, lw, NULL);
    if (!g->no_advection) or_advection_adjoint(g, u, lw, adv);
    for (int64_t q = 0; q < 3 * G; q++) lam_u0[q] = g->rho * lw[q] / g->dt - g->rho * adv[q];

    /* step 2 reversed (the body force does not depend on the state) */
    or_interp(g, m, X, lw, lf);
    for (int64_t q = 0; q < 3 * m; q++) lf[q] /= h3;
    or_interp_grad(g, m, X, lw, f, 1.0 / h3, lX);

    /* step 1 reversed */
    or_forces_lin(s, D, lf, kf);
    for (int64_t q = 0; q < 3 * m; q++) lam_D0[q] = lam_D1[q] + lX[q] + kf[q];
    or_forces_dbend(s, D, lf, grad_b);

    free(X); free(f); free(lU); free(lX); free(lf); free(kf);
    free(F); free(un); free(gw); free(lw); free(adv);
}
