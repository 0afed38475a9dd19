// The neighbour list of one point set, without any device allocation.
//
// Some callers cannot call cudaMalloc: a solver embedded in a host program
// whose own allocator owns all of the GPU's memory and refuses allocations
// from anyone else, and time-critical loops that must not stall, since
// cudaMalloc and cudaFree can synchronise the whole device.  For them,
// sph_neighbour_list_static takes the positions and the three output arrays
// from the caller and keeps every other array it needs (keys and values in id
// order, the sort's ping-pong buffers, its digit histograms and the scan
// partials) in one file-scope device array of fixed size, g_nl_scratch.
//
// In host code the name g_nl_scratch is only a stand-in for the device
// symbol, not a device address: a kernel given it would fault (or silently
// touch host memory where the GPU can reach it).  Every call therefore looks
// up the real address with cudaGetSymbolAddress, with the caller's device
// current, and gives kernels that address.  The lookup is not cached: a cached
// address would outlive a cudaDeviceReset or a new primary context, and the
// lookup costs little next to the sort.
//
// The work is the same as the fluid part of sph_neighbour_list (cell of each
// point, stable radix sort by (cell, id), first index of every cell) and uses
// the same kernels, so the two give identical results.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "sph_internal.cuh"

namespace sph {

namespace {

constexpr int64_t kMaxPoints = SPH_STATIC_MAX_POINTS;
constexpr int64_t kMaxCells = SPH_STATIC_MAX_CELLS;
constexpr int64_t kTiles = (kMaxPoints + kRadixTile - 1) / kRadixTile;
constexpr int64_t kHistWords = 256 * kTiles;
constexpr int64_t kScanMax = kHistWords > kMaxCells + 2 ? kHistWords : kMaxCells + 2;
constexpr int64_t kPartWords = (kScanMax + kScanTile - 1) / kScanTile + 1;
// key and value in id order, key and value ping-pong, histograms, partials
constexpr int64_t kScratchWords = 4 * kMaxPoints + kHistWords + kPartWords;
static __device__ __align__(256) uint32_t g_nl_scratch[kScratchWords];

// Device address of g_nl_scratch on the current device.
int scratch_address(uint32_t **out)
{
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_nl_scratch) != cudaSuccess || !p) return SPH_ERR_CUDA;
    *out = (uint32_t *)p;
    return SPH_OK;
}

}  // namespace

}  // namespace sph

using namespace sph;

extern "C" int sph_neighbour_list_static(const sph_params *p, int64_t n, const double *pos,
                                         uint32_t *sorted_id, uint32_t *cell,
                                         int32_t *cell_start, void *stream)
{
    if (!p || n < 0 || !cell_start) return SPH_ERR_INVALID_ARG;
    if (n > 0 && (!pos || !sorted_id || !cell)) return SPH_ERR_INVALID_ARG;
    int dims[3];
    uint32_t nc = 0;
    int rc = validate_params(p, n, 0, dims, &nc);
    if (rc) return rc;
    if (n > kMaxPoints || (int64_t)nc > kMaxCells) return SPH_ERR_TOO_LARGE;
    uint32_t *base = nullptr;
    rc = scratch_address(&base);
    if (rc) return rc;
    uint32_t *key_in = base, *val_in = base + kMaxPoints;
    uint32_t *key_tmp = base + 2 * kMaxPoints, *val_tmp = base + 3 * kMaxPoints;

    // A host-side context that only carries what the sort and the scan read:
    // the stream and the scratch arrays (all inside g_nl_scratch).
    sph_ctx ctx;
    memset(&ctx, 0, sizeof(ctx));
    ctx.stream = (cudaStream_t)stream;
    ctx.w.radix_hist = base + 4 * kMaxPoints;
    ctx.w.scan_part = ctx.w.radix_hist + kHistWords;
    const DevParams P = derive_params(*p, dims, nc);
    cudaStream_t st = ctx.stream;

    // Cell counts are accumulated straight into the caller's cell_start,
    // which starts at zero; the scan then turns them into first indices.
    if (check_cuda(cudaMemsetAsync(cell_start, 0, ((size_t)nc + 2) * sizeof(int32_t), st)))
        return SPH_ERR_CUDA;
    if (n > 0) {
        const int T = 256;
        SPH_LAUNCH(&ctx, k_boundary_hash, (unsigned)((n + T - 1) / T), T, 0, st, pos, 0u, (int)n, P,
                   key_in, val_in, (uint32_t *)cell_start);
        rc = radix_sort(&ctx, key_in, val_in, key_tmp, val_tmp, cell, sorted_id, (int)n,
                        key_passes_for(nc), st);
        if (rc) return rc;
    }
    rc = exclusive_scan_u32(&ctx, (uint32_t *)cell_start, (uint32_t *)cell_start,
                            (int64_t)nc + 2, ctx.w.scan_part, st);
    if (rc) return rc;
    return check_cuda(cudaGetLastError());
}
