// Internal declarations shared by the translation units of libibgb.so.
// Not part of the public ABI (see include/ib.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "ib.h"

namespace ibgb {

// Programmatic dependent launch.  Kernels of the step are launched with
// launch_pdl, which lets a kernel be scheduled while its predecessor in the
// stream drains; every such kernel starts with PDL_ENTRY(), a wait that
// returns once the predecessor grid has completed and its memory is visible
// (a no-op for a plain launch).  Completion is transitive: a kernel past the
// wait sees the results of all earlier work.  Kernels do not trigger their
// successors early: resident waiting blocks cost more than the launch
// latency they hide (measured on the step's graph).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
#define PDL_ENTRY() pdl_wait()

template <class... KArgs, class... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args &&...args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Markers are binned by grid tile (TILE^3 cells).  Spreading works per bin,
// on at most CHUNK markers per work item; a bin's stencils cover the padded
// box of PAD^3 cells starting one cell below the tile.
constexpr int TILE = 8;
constexpr int PAD = TILE + 3;
constexpr int PAD3 = PAD * PAD * PAD;
constexpr int CHUNK = 512;
// Radix sort of the marker keys: 8-bit digits, RS_CHUNK keys per block
// (RS_ROUNDS rounds of RS_THREADS); the digit-count scan takes SCAN_TILE
// counts per block.
constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 4;
constexpr int RS_CHUNK = RS_THREADS * RS_ROUNDS;
constexpr int SCAN_TILE = 4096;

template <class T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <class T> using cplx_t = typename cplx_of<T>::type;

// Per-marker record in sorted order: the separable delta weights of the
// 4-point stencil along x, y, z (Section 3.2, definition of delta_h) and the
// marker force.  The stencil's first node is base cell - 1.
template <class T> struct alignas(16) Record {
    T w[3][4];
    T f[3];
    T pad;
};

// Four consecutive values of a 16-byte aligned record row (shared or global
// memory) in one (float) or two (double) vector loads.
__device__ __forceinline__ void ld4(const float *p, float (&v)[4])
{
    const float4 q = *reinterpret_cast<const float4 *>(p);
    v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
}
__device__ __forceinline__ void ld4(const double *p, double (&v)[4])
{
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
}

// Tile variant of each FFT pass family (index into the compiled variants):
// x = rows per block of the x passes, y / z = columns per block.
struct FftTune {
    int x = 0, y = 0, z = 0;
};

// Device-side error flags (bit mask), read back by ib_sync: a non-finite
// interpolated marker velocity; a bounded wait for an asynchronous copy that
// ran out (async_copy.cuh); a non-finite marker position or one whose cell
// index would not fit 32 bits (the key kernels).
enum : int { DEV_NONFINITE = 1, DEV_TIMEOUT = 2, DEV_RANGE = 4 };

struct GridDims {
    int nx, ny, nz;
    int ntx, nty, ntz;       // tiles per axis (TILE cells each)
    int ntiles;              // ntx*nty*ntz
    long long G;             // nx*ny*nz
    int nmark;               // marker count (set where a kernel needs it)
};

// Tile-major cell key: tiles in (z, y, x) order, cells within a tile in
// (z, y, x) order.  Sorting by it keeps each tile's markers contiguous and
// the markers of one cell adjacent.
__host__ __device__ __forceinline__ int tile_key(const GridDims &g, int bx, int by, int bz)
{
    const int tile = ((bz / TILE) * g.nty + by / TILE) * g.ntx + bx / TILE;
    return tile * (TILE * TILE * TILE) + ((bz % TILE) * TILE + by % TILE) * TILE + bx % TILE;
}

__host__ __device__ __forceinline__ void key_cell(const GridDims &g, int key, int &bx, int &by, int &bz)
{
    const int tile = key / (TILE * TILE * TILE), l = key % (TILE * TILE * TILE);
    const int tx = tile % g.ntx, ty = (tile / g.ntx) % g.nty, tz = tile / (g.ntx * g.nty);
    bx = tx * TILE + (l % TILE);
    by = ty * TILE + (l / TILE) % TILE;
    bz = tz * TILE + l / (TILE * TILE);
}

// Marker-side device arrays of one context (T = float or double).
struct MarkerArrays {
    int64_t m = 0;
    // state: FP64 reference positions; FP32 contexts add base cell + fraction
    double *X0 = nullptr;        // [3][m] (internal numbering, see qmap)
    int32_t *qmap = nullptr;     // [m] caller's marker id of each internal marker
    int32_t *qinv = nullptr;     // [m] internal index of each caller's marker id
    int32_t *cell0 = nullptr;    // [3][m]   floor(X0/h)           (FP32 contexts)
    void *r0 = nullptr;          // [3][m] T X0/h - cell0           (FP32 contexts)
    void *d = nullptr;           // [3][m] T displacement X - X0
    // springs, one CSR row per marker (each link appears in both end rows)
    int32_t *sp_off = nullptr;   // [m+1]
    int32_t *sp_j = nullptr;     // [nnz] other end
    void *sp_k = nullptr;        // [nnz] T
    void *sp_L0 = nullptr;       // [nnz] T
    void *sp_e0 = nullptr;       // [3][nnz] T  X0_j - X0_i
    void *sp_c0 = nullptr;       // [nnz] T  |e0|^2 - L0^2
    int64_t nnz = 0;
    void *tk = nullptr;          // [m] T tether stiffness (0: none)
    void *mf_dir = nullptr;      // [3][m] T direction of the external marker force (null: none)
    int32_t *bslot = nullptr;    // [m] bending slot or -1
    int32_t *bn = nullptr;       // [5][nb] neighbours along the line (-1: none)
    void *bc = nullptr;          // [3][nb] T c_{i-1}, c_i, c_{i+1} (0 where no term)
    int64_t nb = 0;
    // work space
    int32_t *key = nullptr;      // [m] cell key by marker id
    int32_t *key_alt = nullptr;  // [m] radix ping-pong
    int32_t *key_s = nullptr;    // [m] sorted keys
    int32_t *perm_alt = nullptr; // [m] radix ping-pong
    int32_t *perm = nullptr;     // [m] marker id at each sorted position
    int32_t *hist = nullptr;                        // radix digit histograms
    int64_t hist_len = 0;
    void *rfrac = nullptr;       // [3][m] T fractional offset of X/h in its base cell
    void *rec = nullptr;         // [m] Record<T>, sorted order
    void *f = nullptr;           // [3][m] T marker forces (ABI spread input)
    void *U = nullptr;           // [3][m] T interpolated velocity (ABI interp output)
    void *Us = nullptr;          // [3][m] T interpolated velocity in sorted order
    double *Xtmp = nullptr;      // [3][m] positions staged for ABI calls
    // reverse step (allocated by the first ib_adjoint_step)
    void *lamD = nullptr;        // [3][m] T dJ/dD^{n+1}, internal numbering
    void *lamDo = nullptr;       // [3][m] T dJ/dD^n
    void *rec2 = nullptr;        // [m] Record<T>: weights + h^3 dt lamD (the interp transpose as a spread)
    void *lf_s = nullptr;        // [3][m] T dJ/df by sorted position
    void *lX_s = nullptr;        // [3][m] T dJ/dX (explicit part) by sorted position
    void *lf = nullptr;          // [3][m] T dJ/df by marker
    void *lX = nullptr;          // [3][m] T dJ/dX by marker
    // bending-stiffness gradient: the term of the line centred at a slot's
    // marker has coefficient b_seg * unit; its contribution is summed per
    // segment in FP64 in a fixed order (CSR of slots per segment)
    int n_seg = 0;
    double *bunit = nullptr;     // [3][nb] dw / ds^3 of the terms centred at rows i-1, i, i+1 (0: none)
    int32_t *bseg = nullptr;     // [3][nb] their segments (-1: none)
    double *gterm = nullptr;     // [nb] per-term contribution
    int32_t *seg_off = nullptr;  // [n_seg+1]
    int32_t *seg_slot = nullptr; // [terms]
    double *gseg = nullptr;      // [n_seg]
    // host copies to rebuild bc when the stiffness changes: segment (-1: no
    // term), width dw and spacing ds of the terms centred at rows i-1, i, i+1
    // of each slot, [3][nb]
    std::vector<int32_t> h_bseg3;
    std::vector<double> h_bdw3, h_bds3;
};

struct Forcing {
    int active = 0;
    double dir[3] = {0, 0, 0};
    double mag = 0;              // rho*amp*omega
    double omega = 0;
    double mamp = 0, momega = 0; // external marker force amplitude (dyn) and angular frequency
    int2 *rows = nullptr;        // [nz*ny] (x_lo, x_hi) of forced cells, x_lo > x_hi: none
};

}  // namespace ibgb

struct ib_ctx {
    ib_grid_desc desc{};
    ibgb::GridDims dim{};
    bool fp64 = false;
    bool tc_fft = false;         // IB_FP32_TCFFT: y passes on the tensor cores (ny = 256)
    int elt = 4;                 // bytes per real
    int device = 0;
    cudaStream_t stream = nullptr;      // caller's stream
    cudaStream_t cap = nullptr;         // private stream for graph capture
    // grid fields
    void *u = nullptr;           // [3][G] state velocity
    void *F = nullptr;           // [3][G] spread force (tile-sparse in the step)
    void *ubuf = nullptr;        // [3][G] staging for ABI calls
    void *Fbuf = nullptr;        // [3][G] staging for ABI calls
    uint8_t *touched = nullptr;  // [ntiles] tiles some marker's stencil reaches
    int *tile_list = nullptr;    // [ntiles] touched tiles, compacted
    int *tile_count = nullptr;   // number of touched tiles
    int *tile_next = nullptr;    // spreading scatter's work counter (tile_count + 1)
    int32_t *bin_start = nullptr;   // [ntiles+1] first sorted marker of each tile (counts before the scan)
    int32_t *item_start = nullptr;  // [ntiles+1] first spreading work item of each tile
    int2 *items = nullptr;          // [max_items] (tile, chunk) spreading work items
    int *item_ctl = nullptr;        // [4] item count, work counters of the interpolation and its transpose
    int2 *bscan_tmp_plan = nullptr; // [ntiles/1024 + 1] bin planning partial sums
    void *partial = nullptr;        // [max_items][3][PAD^3] per-item padded force boxes
    int64_t max_items = 0;
    void *spec = nullptr;        // [4][nz][ny][nx/2] complex half spectrum (4th: pressure)
    void *nyq = nullptr;         // [4][nz][ny] complex, kx = nx/2
    void *p = nullptr;           // [G] pressure staging
    void *tw[3] = {nullptr, nullptr, nullptr};   // forward twiddles W_n^j, j < n, per axis
    void *sym_s[3] = {nullptr, nullptr, nullptr};    // sin(2 pi k/n)/h per axis (exact 0 at 0, n/2)
    void *sym_a[3] = {nullptr, nullptr, nullptr};    // (4 mu/h^2) sin^2(pi k/n) per axis
    int32_t *bscan_tmp = nullptr;
    int64_t bscan_tmp_len = 0;
    ibgb::Forcing forcing;
    ibgb::MarkerArrays mk;
    bool have_structure = false;
    double *d_time = nullptr;    // device [t, rho A w cos(w t) (body force), mamp cos(momega t) (markers), 0,
                                 //  mean velocity (3, FP64; FP32 contexts), 0]
    double *qpart = nullptr;     // FP32 contexts: [3][blocks] per-block sums for the FP64 mean mode
    double *d_tparams = nullptr; // device [dt, rho A w, w, mamp, momega]: advancing d_time
    double t = 0.0;
    double t_pair[4] = {0.0, 0.0, 0.0, 0.0};  // host staging of d_time
    int *d_status = nullptr;     // device error flags
    cudaGraphExec_t graph = nullptr;
    bool sort_from_state = false; // the last marker sort was made from the context's state (internal numbering)
    ibgb::FftTune fft_tune;      // FFT tile variants (ib_set_tuning)
    uint64_t version = 0;        // bumped when captured work goes stale (structure, tuning)
    int marker_blocks = 0;       // grid of the persistent marker kernels (0: every SM, full occupancy)
    // marker probe (ib_set_probe): normal displacements of chosen markers
    // recorded on the device every `every` steps into a ring of records
    int32_t probe_n = 0, probe_every = 0, probe_cap = 0;
    int32_t *probe_idx = nullptr;   // [n] internal marker ids
    double *probe_dir = nullptr;    // [3][n]
    double *probe_ring = nullptr;   // [cap][n]
    double *probe_t = nullptr;      // [cap] time of each record
    double *probe_env = nullptr;    // [n] max |eta| over the records so far
    long long *probe_ctl = nullptr; // [steps since ib_set_probe, records produced]
    long long probe_read = 0;       // records already returned by ib_read_probe
    void *adj_u1 = nullptr;      // [3][G] u^{n+1} recomputed or staged by the reverse step
    void *adj_lw = nullptr;      // [3][G] dJ/dw of the reverse step
};

namespace ibgb {

// Blocks of a persistent marker kernel (scatter, interp): the tuned count if
// set, else `full` (every SM at full occupancy), never more than `full`.
inline int persistent_grid(const ib_ctx *c, int full)
{
    return (c->marker_blocks > 0 && c->marker_blocks < full) ? c->marker_blocks : full;
}

// ---- launchers (k_markers.cu) ----------------------------------------------
// Keys and fractional offsets from the context's state (X0 + d).
void launch_keys_state(ib_ctx *c, cudaStream_t s);
// Keys and fractional offsets from explicit FP64 positions X [3][m].
void launch_keys_X(ib_ctx *c, const double *X, cudaStream_t s);
// Stable LSD radix sort of marker ids by tile (key / TILE^3) -> mk.key_s
// (full keys in sorted order), mk.perm.
void launch_sort(ib_ctx *c, cudaStream_t s);
// Bin starts (scan of the per-tile counts the key kernels made) and the list
// of spreading work items.
void launch_bin_plan(ib_ctx *c, cudaStream_t s);
// Records in sorted order: weights + forces.  mode 0: zero forces, 1: forces
// from the structure and the displacement, 2: fscale * f [3][m] (marker order).
// rec: output array (null: the context's mk.rec).
void launch_records(ib_ctx *c, int mode, const void *f, cudaStream_t s, void *rec = nullptr, double fscale = 1.0);
int sort_passes(long long G);
// Stable radix sort by tile of keys key[0..m) (cell keys < G) with caller-provided
// buffers: kbuf0/kbuf1/vbuf0 [m] work space, vout [m] receives the marker ids
// in sorted order (kbuf1 the sorted keys), hist [256*ceil(m/RS_CHUNK)+1] and
// scan_tmp [hist/SCAN_TILE+4] work space.
void radix_sort_raw(const int32_t *key, int m, long long G, int32_t *kbuf0, int32_t *kbuf1, int32_t *vbuf0,
                    int32_t *vout, int32_t *hist, int32_t *scan_tmp, cudaStream_t s);
// Interpolate u at the sorted markers (needs the bin plan): step mode adds
// dt*U to d, else writes U (k_spread.cu).
void launch_interp(ib_ctx *c, const void *u, void *U, bool step_mode, cudaStream_t s);

// ---- spread (k_spread.cu) ----------------------------------------------------
// Records -> F [3][G]: per-bin padded partial boxes, then a fixed-order sum
// per touched tile.  dense: F is zeroed first (every node written); else only
// touched tiles are written and c->touched flags them.  rec: the records to
// spread (null: the context's mk.rec).
void launch_spread(ib_ctx *c, void *F, bool dense, cudaStream_t s, const void *rec = nullptr);
int64_t spread_max_items(const GridDims &g, int64_t m);

// ---- fluid solve (k_fft.cu) --------------------------------------------------
// u_n, F -> u_np1 (may alias u_n); p optional.  use_touched: read F only on
// touched tiles; step_mode: also add the body force at *d_time and advance it.
// ev (nullable): 4 events recorded after the x-fwd, y-fwd, z and y-inv passes.
void launch_fluid(ib_ctx *c, const void *u_n, const void *F, void *u_np1, void *p, bool use_touched,
                  bool step_mode, cudaStream_t s, cudaEvent_t *ev = nullptr);

// Right-hand side and time handling of a fluid solve.
enum FluidMode : int {
    FLUID_PLAIN = 0,    // w = rho u/dt - rho A(u) + F
    FLUID_STEP = 1,     // PLAIN plus the body force at d_time; advances d_time by dt
    FLUID_REPLAY = 2,   // STEP without advancing d_time (recomputing a step)
    FLUID_DIRECT = 3,   // w = u + F: no advection, no body force (the adjoint solve)
};
void launch_fluid_mode(ib_ctx *c, const void *u_n, const void *F, void *u_np1, void *p, bool use_touched, int mode,
                       cudaStream_t s, cudaEvent_t *ev = nullptr);

bool fft_length_supported(int n);

// The main tiles of a y pass (ny = 256) as tensor-core DFT products
// (k_tcfft.cu); false when the shape is not supported.
bool launch_ytc(float2 *spec, int nxh, int nz, int ncomp, const float2 *tw, int dir, int *status, int nsm,
                cudaStream_t s);

// ---- reverse step (k_adjoint.cu) ---------------------------------------------
// Needs the bin plan and both record arrays (mk.rec: forces f^n, mk.rec2:
// h^3 dt lamD).  lw = dJ/dw [3][G], u1 = u^{n+1}:
//  lam_u_out = rho lw/dt - rho (dA/du^n)^T lw;
//  mk.lf = h^-3 interp(lw), mk.lX = d/dX [interp(u1) . lamU + h^-3 interp(lw) . f];
//  mk.lamDo = mk.lamD + mk.lX + (df/dD) mk.lf and the per-term gradient mk.gterm;
//  mk.gseg = per-segment sums of mk.gterm.
void launch_adv_adjoint(ib_ctx *c, const void *lw, void *lam_u_out, cudaStream_t s);
void launch_adj_markers(ib_ctx *c, const void *u1, const void *lw, cudaStream_t s);
// grad_b [n_seg] (device) += mk.gseg
void launch_grad_accumulate(ib_ctx *c, double *grad_b, cudaStream_t s);

// The probe's per-step kernel (no-op without a probe), k_probe.cu.
void launch_probe(ib_ctx *c, cudaStream_t s);
void free_probe(ib_ctx *c);

// One block waiting, at most `polls` polls, on an mbarrier nothing arrives on:
// sets DEV_TIMEOUT in *status (k_waitcheck.cu).
void launch_wait_check(int *status, int polls, cudaStream_t s);

// One forward step of c enqueued on stream s (what ib_step captures).
void enqueue_step_on(ib_ctx *c, cudaStream_t s);

// Record msg as the calling thread's ib_last_error() and return st.
ib_status set_error(ib_status st, const char *msg);

}  // namespace ibgb
