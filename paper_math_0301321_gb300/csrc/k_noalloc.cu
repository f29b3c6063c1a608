// Allocation-free marker bin sort.
//
// Some callers cannot call cudaMalloc: code running while a CUDA graph is
// being captured in global mode, hosts embedded in a runtime that owns all
// device memory through its own pool and forbids outside allocations, or
// real-time loops that may not take the allocator's locks.  For them this
// file offers ib_bin_sort_noalloc: the same stable cell sort as ib_bin_sort,
// but with no context and no allocation.  The caller passes device buffers
// for the positions and the two outputs; the radix sort's work space lives
// in one file-scope device array of fixed size, allocated when the library
// is loaded and held by every GPU that loads it until the process exits.
#include <mutex>

#include "ib_internal.cuh"

namespace ibgb {

namespace {

constexpr long long kMaxMarkers = 1LL << 20;                     // IB_NOALLOC_MAX_MARKERS
constexpr long long kChunks = (kMaxMarkers + RS_CHUNK - 1) / RS_CHUNK;
constexpr long long kHist = 256 * kChunks + 1;
constexpr long long kScanTmp = kHist / SCAN_TILE + 4;
// int32 slots: three [kMaxMarkers] buffers, the digit histogram, scan partials
constexpr long long kScratchInts = 3 * kMaxMarkers + kHist + kScanTmp;

// Shared by every call on a device; holds the last call's contents.
static __device__ __align__(256) int32_t g_sort_scratch[kScratchInts];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int32_t *g_addr[kMaxDevices] = {};

// tile-major key of the cell floor(X * (1/h)) (indices wrapped), as the
// context entry points compute it
__global__ void k_keys_noalloc(int m, GridDims g, const double *__restrict__ X, double inv_h,
                               int32_t *__restrict__ key)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= m) return;
    const int n[3] = {g.nx, g.ny, g.nz};
    int b[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double s = __dmul_rn(X[(long long)c * m + l], inv_h);
        int v = (int)floor(s) % n[c];
        b[c] = v < 0 ? v + n[c] : v;
    }
    key[l] = tile_key(g, b[0], b[1], b[2]);
}

}  // namespace
}  // namespace ibgb

using namespace ibgb;

extern "C" ib_status ib_bin_sort_noalloc(const int32_t n[3], double h, int64_t m, const double *X, int32_t *key,
                                         int32_t *perm, void *stream)
{
    if (!n || !(h > 0)) return set_error(IB_ERR_ARG, "ib_bin_sort_noalloc: null grid size or h <= 0");
    if (m < 0 || m > kMaxMarkers)
        return set_error(IB_ERR_ARG, "ib_bin_sort_noalloc: marker count outside [0, IB_NOALLOC_MAX_MARKERS = 1048576]");
    if (m > 0 && (!X || !key || !perm)) return set_error(IB_ERR_ARG, "ib_bin_sort_noalloc: null buffer");
    for (int j = 0; j < 3; ++j)
        if (n[j] < TILE || n[j] % TILE) return set_error(IB_ERR_ARG, "ib_bin_sort_noalloc: grid sizes must be multiples of 8");
    const long long G = (long long)n[0] * n[1] * n[2];
    if (G >= (1LL << 31)) return set_error(IB_ERR_ARG, "ib_bin_sort_noalloc: grid has 2^31 cells or more");
    if (m == 0) return IB_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return set_error(IB_ERR_CUDA, "ib_bin_sort_noalloc: no usable CUDA device");
    int32_t *base = nullptr;
    {
        // once per device, with that device current: the device address of the array
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess) {
                cudaGetLastError();
                return set_error(IB_ERR_CUDA, "ib_bin_sort_noalloc: cudaGetSymbolAddress failed");
            }
            g_addr[dev] = static_cast<int32_t *>(p);
        }
        base = g_addr[dev];
    }
    int32_t *kbuf0 = base;
    int32_t *kbuf1 = base + kMaxMarkers;
    int32_t *vbuf0 = base + 2 * kMaxMarkers;
    int32_t *hist = base + 3 * kMaxMarkers;
    int32_t *scan_tmp = hist + kHist;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int mi = (int)m;
    GridDims g{};
    g.nx = n[0];
    g.ny = n[1];
    g.nz = n[2];
    g.ntx = n[0] / TILE;
    g.nty = n[1] / TILE;
    g.ntz = n[2] / TILE;
    g.ntiles = g.ntx * g.nty * g.ntz;
    g.G = G;
    k_keys_noalloc<<<(mi + 255) / 256, 256, 0, s>>>(mi, g, X, 1.0 / h, key);
    radix_sort_raw(key, mi, G, kbuf0, kbuf1, vbuf0, perm, hist, scan_tmp, s);
    if (cudaGetLastError() != cudaSuccess) return set_error(IB_ERR_CUDA, "ib_bin_sort_noalloc: launch failed");
    return IB_OK;
}
