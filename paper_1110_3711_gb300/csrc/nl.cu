// NL stage (Sections 2 and 4.1 of the paper): cell-linked list on the GPU.
//
// Fluid (every step), a counting sort by cell:
//   k_hash        cell of every particle: c_d = floor((x_d - min_d) / s), linear
//                 id cx + nx (cy + ny cz) (cells follow X, Y, Z; Section 4.4),
//                 the per-cell counts and a slot inside the cell (atomics),
//                 and the counts per scan tile of kScanTile cells.
//   k_scan_items  exclusive scan of the per-cell counts: start[c] = number of
//                 particles in cells below c, i.e. CellBeginEnd of Fig. 8 with
//                 empty cells as equal begin and end; its tile sums come from
//                 k_hash, so the scan is one down-sweep; the same kernel
//                 appends the PI work items of the cells it scans.
//   k_place       cell-grouped order start[c] + slot (arbitrary inside a cell).
//   k_reorder     rank by id inside the cell, which gives the (cell, id) order
//                 whatever the order before; copy of the fluid state (x, y, z
//                 and the {v, rho} records of both levels) to that place, the
//                 packed PI input {pos, P/rho^2} of Section 4.3 (the other
//                 one, {v, rho}, is the state record itself) and the largest
//                 sound speed (Section 4.1 maxima).
// Boundary (once) and the static entry point: a stable LSD radix sort of the
// keys in id order, 8-bit digits: k_radix_hist (tile histograms), exclusive
// scan (digit-major), k_radix_scatter (ranks from warp match + per-warp digit
// counters, no atomics, stable).
// All kernels are HBM-bound; grids are sized from the particle count.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sph_internal.cuh"

namespace sph {

constexpr int kHashBlock = 512;   // threads (particles) per k_hash block
constexpr int kHashTiles = 4;     // scan tiles a block counts in shared memory

// ------------------------------------------------------------------ cells --

// float32 value of x with its 24 leading significand bits (the rest cut off,
// so |xf - x| < 2^-23 |x|), built from the bit pattern with integer operations
// only; 0 below the normal float range, NaN above it and for inf or NaN.
__device__ __forceinline__ float trunc_to_float(double x)
{
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const uint32_t e = (hi >> 20) & 0x7ffu;
    if (e < 897u) return 0.0f;
    if (e > 1150u) return __int_as_float(0x7fffffff);
    return __uint_as_float((hi & 0x80000000u) | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) |
                           (lo >> 29));
}

// floor((x - mn) / s) as the float64 definition gives it: d = x - mn rounded,
// then d / s with IEEE division, then floor; -1 outside [0, n).
//
// Fast path, float32 and integer operations only: e = xf (1/s) - mn/s with the
// float32 constants a = RN(1/s), b = RN(mn/s).  Each of xf, a, b and the fused
// multiply-add is within 2^-23 (relative) of its exact value, so
// |e - (x - mn)/s| < 2^-20 (|e| + |mn/s|).  The margin E below is twice that,
// plus eabs >= 2^-124 / s, the largest error of an input below the float range
// flushed to 0; when e - E and e + E floor
// to the same integer, no integer lies within the error of e, so floor(e) is
// floor((x - mn)/s), and also floor of the rounded float64 quotient, whose
// relative error (about 2^-52) is far inside the margin.  Otherwise (a
// quotient within about 2^-19 relative of an integer, |e| >= 2^22, NaN) the
// float64 path decides: reciprocal, and a true division when the quotient is
// within 1e-9 of an integer (the only case where the two can round to
// different sides).
__device__ __forceinline__ int axis_cell(double x, double mn, double s, double inv_s, int n,
                                         float a, float b, float babs, float eabs)
{
    const float e = fmaf(trunc_to_float(x), a, -b);
    if (fabsf(e) < 4194304.0f) {  // 2^22; false for NaN
        const float E = fmaf(0x1p-19f, fabsf(e) + babs, eabs);
        const int lo = __float2int_rd(e - E), hi = __float2int_rd(e + E);
        if (lo == hi) return (lo >= 0 && lo < n) ? lo : -1;
    }
    double d = x - mn;
    double t = d * inv_s;
    double f = floor(t);
    if (t - f < 1e-9 || (f + 1.0) - t < 1e-9) f = floor(__ddiv_rn(d, s));
    if (!(f >= 0.0) || f >= (double)n) return -1;
    return (int)f;
}

__device__ __forceinline__ uint32_t cell_of(const DevParams &P, double x, double y, double z)
{
    int cx = axis_cell(x, P.dom_min[0], P.s, P.inv_s, P.nx, P.cell_af, P.cell_bf[0], P.cell_babsf[0],
                       P.cell_eabsf);
    int cy = axis_cell(y, P.dom_min[1], P.s, P.inv_s, P.ny, P.cell_af, P.cell_bf[1], P.cell_babsf[1],
                       P.cell_eabsf);
    int cz = axis_cell(z, P.dom_min[2], P.s, P.inv_s, P.nz, P.cell_af, P.cell_bf[2], P.cell_babsf[2],
                       P.cell_eabsf);
    if (cx < 0 || cy < 0 || cz < 0) return P.ncells;
    return (uint32_t)cx + (uint32_t)P.nx * ((uint32_t)cy + (uint32_t)P.ny * (uint32_t)cz);
}

// One thread per particle (current order i): its cell (cell_i[i]), its slot
// among the particles of that cell (slot_i[i]) and count[cell] += 1.  The
// slots come from one atomic per distinct cell of the warp (consecutive
// particles mostly share a cell), so their order inside a cell is arbitrary;
// k_reorder restores the id order inside every cell.
__global__ void __launch_bounds__(kHashBlock)
k_hash(const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
       int n, DevParams P, uint32_t *__restrict__ cell_i, uint32_t *__restrict__ slot_i,
       uint32_t *__restrict__ count, uint32_t *__restrict__ tile_count, Scalars *sc)
{
    __shared__ uint32_t tsum[kHashTiles];
    __shared__ uint32_t tbase;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    // lanes past the end take a key no particle has, so the warp stays whole
    const uint32_t c = i < n ? cell_of(P, x[i], y[i], z[i]) : 0xffffffffu;
    if (threadIdx.x < kHashTiles) tsum[threadIdx.x] = 0u;
    if (threadIdx.x == 0) tbase = i < n ? c / (uint32_t)kScanTile : 0u;
    const unsigned peers = __match_any_sync(0xffffffffu, c);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (i < n && lane == leader) base = atomicAdd(&count[c], (uint32_t)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    // The same counts per scan tile of kScanTile cells: the tile sums of the
    // cell-start scan, so that it needs only its down-sweep.  The block's
    // particles (consecutive in the previous sorted order) lie in a few
    // consecutive tiles, counted in shared memory from the tile of its first
    // particle; one global atomic per tile and block (a tile holds tens of
    // thousands of particles, so per-warp global atomics would queue on a
    // few addresses).
    __syncthreads();
    const uint32_t tile = i < n ? c / (uint32_t)kScanTile : 0xffffffffu;
    const unsigned tpeers = __match_any_sync(0xffffffffu, tile);
    if (i < n && lane == __ffs(tpeers) - 1) {
        const uint32_t d = tile - tbase;
        if (d < (uint32_t)kHashTiles) atomicAdd(&tsum[d], (uint32_t)__popc(tpeers));
        else atomicAdd(&tile_count[tile], (uint32_t)__popc(tpeers));
    }
    __syncthreads();
    if (threadIdx.x < kHashTiles && tsum[threadIdx.x] != 0u)
        atomicAdd(&tile_count[tbase + threadIdx.x], tsum[threadIdx.x]);
    if (i < n) {
        cell_i[i] = c;
        slot_i[i] = base + (uint32_t)__popc(peers & ((1u << lane) - 1u));
        if (c == P.ncells) atomicOr(&sc->flags, SPH_FLAG_OUT_OF_GRID);
    }
}

// One thread per particle (current order i): position q = start[cell] + slot in
// the cell-grouped order; cell_q[q] = cell, src_q[q] = i, id_q[q] = id.
__global__ void k_place(int n, const uint32_t *__restrict__ cell_i,
                        const uint32_t *__restrict__ slot_i, const uint32_t *__restrict__ id,
                        const int32_t *__restrict__ start, uint32_t *__restrict__ cell_q,
                        uint32_t *__restrict__ src_q, uint32_t *__restrict__ id_q)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t c = cell_i[i];
    const uint32_t q = (uint32_t)start[c] + slot_i[i];
    cell_q[q] = c;
    src_q[q] = (uint32_t)i;
    id_q[q] = id[i];
}

// ------------------------------------------------------------- radix sort --

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_IPT = 8;
constexpr int RS_TILE = RS_THREADS * RS_IPT;
static_assert(RS_TILE == kRadixTile, "tile size shared with the static-scratch neighbour list");

int radix_tiles(int64_t n) { return (int)((n + RS_TILE - 1) / RS_TILE); }

__global__ void __launch_bounds__(RS_THREADS)
k_radix_hist(const uint32_t *__restrict__ keys, int n, int shift, int tiles,
             uint32_t *__restrict__ hist)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int base = blockIdx.x * RS_TILE;
#pragma unroll
    for (int k = 0; k < RS_IPT; ++k) {
        int idx = base + k * RS_THREADS + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one tile.  Warp w owns elements [w*256, (w+1)*256) of the
// tile, visited as 8 rounds of 32 consecutive elements, so (warp, round, lane)
// is the element order; an element's rank is the count of equal digits before
// it: earlier warps (prefix of the per-warp counters), earlier rounds of its
// warp (the counter before this round) and lower lanes of its round (match).
__global__ void __launch_bounds__(RS_THREADS)
k_radix_scatter(const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                uint32_t *__restrict__ kout, uint32_t *__restrict__ vout, int n, int shift,
                int tiles, const uint32_t *__restrict__ off)
{
    __shared__ uint32_t whist[RS_WARPS][256];
    __shared__ uint32_t goff[256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < RS_WARPS * 256; t += RS_THREADS) (&whist[0][0])[t] = 0;
    goff[threadIdx.x] = off[threadIdx.x * tiles + blockIdx.x];
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    const int base = blockIdx.x * RS_TILE + warp * (RS_IPT * 32);
    uint32_t key[RS_IPT], val[RS_IPT], rank[RS_IPT];
#pragma unroll
    for (int k = 0; k < RS_IPT; ++k) {
        int idx = base + k * 32 + lane;
        bool valid = idx < n;
        key[k] = valid ? kin[idx] : 0u;
        val[k] = valid ? vin[idx] : 0u;
        uint32_t d = valid ? ((key[k] >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = valid ? whist[warp][d] : 0u;
        rank[k] = before + __popc(peers & lt);
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) whist[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        uint32_t sum = 0;
        const int d = threadIdx.x;  // RS_THREADS == 256 digits
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            uint32_t t = whist[w][d];
            whist[w][d] = sum;
            sum += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < RS_IPT; ++k) {
        int idx = base + k * 32 + lane;
        if (idx < n) {
            uint32_t d = (key[k] >> shift) & 255u;
            uint32_t pos = goff[d] + whist[warp][d] + rank[k];
            kout[pos] = key[k];
            vout[pos] = val[k];
        }
    }
}

// ------------------------------------------------------------------- scan --

// exclusive scan of one block's tile; returns the tile total to thread 0
__device__ __forceinline__ uint32_t block_exclusive(uint32_t v, uint32_t *smem)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) smem[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int nw = blockDim.x >> 5;
        uint32_t s = lane < nw ? smem[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        if (lane < nw) smem[lane] = s;  // inclusive per warp
    }
    __syncthreads();
    uint32_t warp_prefix = warp ? smem[warp - 1] : 0u;
    uint32_t total = smem[(blockDim.x >> 5) - 1];
    __syncthreads();
    smem[32] = total;
    return warp_prefix + x - v;
}

__global__ void __launch_bounds__(kScanBlock)
k_scan_reduce(const uint32_t *__restrict__ in, int64_t n, uint32_t *__restrict__ part)
{
    __shared__ uint32_t red[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += in[base + k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t t = red[threadIdx.x];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) part[blockIdx.x] = t;
    }
}

// Down-sweep: every block adds the sum of the partials of the blocks before it
// (a block reduction over at most a few thousand values) to its own exclusive
// scan, so no separate pass over the partials is needed.
__global__ void __launch_bounds__(kScanBlock)
k_scan_down(const uint32_t *in, uint32_t *out, int64_t n, const uint32_t *__restrict__ part)
{
    __shared__ uint32_t smem[33];
    __shared__ uint32_t base_s;
    uint32_t b = 0;
    for (int k = threadIdx.x; k < (int)blockIdx.x; k += kScanBlock) b += part[k];
    for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
    if ((threadIdx.x & 31) == 0) smem[threadIdx.x >> 5] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kScanBlock / 32; ++w) t += smem[w];
        base_s = t;
    }
    __syncthreads();
    const uint32_t base = base_s;
    int64_t start = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = start + k < n ? in[start + k] : 0u;
        s += v[k];
    }
    uint32_t ex = block_exclusive(s, smem) + base;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (start + k < n) out[start + k] = ex;
        ex += v[k];
    }
}

// The down-sweep of k_scan_down over the fluid cell counts (start = the cell
// starts, n = ncells + 2 entries), which also appends the PI work items of
// the fluid list: a cell of m particles (c < ncells; the particles outside the
// grid get none) gives ceil(m / 32) items {first particle, number of
// particles} of up to 32 targets of that cell (the paper's GPU kernel gives
// one thread per particle, Section 4; here one warp per item).  The items of
// a block are appended with one atomic, so their order between blocks is
// arbitrary (the sums of a target do not depend on it).
__global__ void __launch_bounds__(kScanBlock)
k_scan_items(const uint32_t *count, uint32_t *start, int64_t n, const uint32_t *__restrict__ part,
             uint32_t ncells, uint32_t *__restrict__ items, uint32_t *__restrict__ n_items)
{
    __shared__ uint32_t smem[33];
    __shared__ uint32_t base_s, ibase_s;
    uint32_t b = 0;
    for (int k = threadIdx.x; k < (int)blockIdx.x; k += kScanBlock) b += part[k];
    for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
    if ((threadIdx.x & 31) == 0) smem[threadIdx.x >> 5] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kScanBlock / 32; ++w) t += smem[w];
        base_s = t;
    }
    __syncthreads();
    const int64_t c0 = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0, ni = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = c0 + k < n ? count[c0 + k] : 0u;
        s += v[k];
        if (c0 + k < (int64_t)ncells) ni += (v[k] + 31u) >> 5;
    }
    const uint32_t ex0 = block_exclusive(s, smem) + base_s;
    uint32_t ex = ex0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (c0 + k < n) start[c0 + k] = ex;
        ex += v[k];
    }
    // the block's items: exclusive position of this thread's, then one atomic
    uint32_t it = block_exclusive(ni, smem);
    if (threadIdx.x == kScanBlock - 1) {
        const uint32_t tot = it + ni;
        ibase_s = tot ? atomicAdd(n_items, tot) : 0u;
    }
    __syncthreads();
    it += ibase_s;
    ex = ex0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (c0 + k < (int64_t)ncells) {
            for (uint32_t o = 0; o < v[k]; o += 32u, ++it) {
                items[2 * (size_t)it] = ex + o;
                items[2 * (size_t)it + 1] = min(32u, v[k] - o);
            }
        }
        ex += v[k];
    }
}

size_t scan_partials(int64_t n) { return (size_t)((n + kScanTile - 1) / kScanTile) + 1; }

int exclusive_scan_u32(sph_ctx *ctx, const uint32_t *in, uint32_t *out, int64_t n,
                       uint32_t *partials, cudaStream_t st)
{
    if (n <= 0) return SPH_OK;
    int64_t blocks = (n + kScanTile - 1) / kScanTile;
    SPH_LAUNCH(ctx, k_scan_reduce, (unsigned)blocks, kScanBlock, 0, st, in, n, partials);
    SPH_LAUNCH(ctx, k_scan_down, (unsigned)blocks, kScanBlock, 0, st, in, out, n, partials);
    return check_cuda(cudaGetLastError());
}

// Sort (key, val) pairs of length n with `passes` 8-bit passes; the result is
// in (kout, vout).  tmp buffers have length n.
int radix_sort(sph_ctx *ctx, const uint32_t *kin, const uint32_t *vin, uint32_t *ktmp,
                      uint32_t *vtmp, uint32_t *kout, uint32_t *vout, int n, int passes,
                      cudaStream_t st)
{
    if (n <= 0) return SPH_OK;
    Workspace &w = ctx->w;
    int tiles = radix_tiles(n);
    // ping-pong so that the last pass lands in (kout, vout)
    const uint32_t *ks = kin, *vs = vin;
    for (int p = 0; p < passes; ++p) {
        bool to_out = ((passes - 1 - p) % 2) == 0;
        uint32_t *kd = to_out ? kout : ktmp;
        uint32_t *vd = to_out ? vout : vtmp;
        int shift = 8 * p;
        SPH_LAUNCH(ctx, k_radix_hist, tiles, RS_THREADS, 0, st, ks, n, shift, tiles, w.radix_hist);
        int rc = exclusive_scan_u32(ctx, w.radix_hist, w.radix_hist, (int64_t)256 * tiles,
                                    w.scan_part, st);
        if (rc) return rc;
        SPH_LAUNCH(ctx, k_radix_scatter, tiles, RS_THREADS, 0, st, ks, vs, kd, vd, n, shift,
                   tiles, w.radix_hist);
        ks = kd;
        vs = vd;
    }
    return check_cuda(cudaGetLastError());
}

// ---------------------------------------------------------------- reorder --

template <typename Real> using Vec4 = Real4T<Real>;

// Tait pressure over rho^2 and sound speed, float64 form.
__device__ __forceinline__ void eos64(const DevParams &P, double rho, double *pr, double *c)
{
    double r = rho * P.inv_rho0;
    double pw, cs;
    if (P.gamma_is_7) {
        double r2 = r * r;
        double r3 = r2 * r;
        pw = r3 * r3 * r;
        cs = r3;
    } else {
        pw = pow(r, P.gamma);
        cs = pow(r, 0.5 * (P.gamma - 1.0));
    }
    *pr = P.B * (pw - 1.0) / (rho * rho);
    *c = P.c0 * cs;
}

// Tait pressure over rho^2 and sound speed, float32 form: with delta = rho/rho0
// - 1 (small), (1 + delta)^7 - 1 is evaluated by its binomial expansion to
// avoid the cancellation of pow(...) - 1 in float32.
__device__ __forceinline__ void eos32(const DevParams &P, float rho, float *pr, float *c)
{
    float d = (rho - (float)P.rho0) * P.inv_rho0f;
    float pw1, cs;
    if (P.gamma_is_7) {
        pw1 = d * fmaf(d, fmaf(d, fmaf(d, fmaf(d, fmaf(d, d + 7.0f, 21.0f), 35.0f), 35.0f), 21.0f), 7.0f);
        float r = 1.0f + d;
        cs = r * r * r;
    } else {
        float l = log1pf(d);
        pw1 = expm1f((float)P.gamma * l);
        cs = expf(0.5f * ((float)P.gamma - 1.0f) * l);
    }
    *pr = P.Bf * pw1 / (rho * rho);
    *c = P.c0f * cs;
}

// Origin of every cell column along each axis, min_d + c s, written once per
// context so that the per-step kernels do not spend the float64 unit on it.
__global__ void k_fill_origins(DevParams P, double *origin)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < P.nx) origin[k] = P.dom_min[0] + (double)k * P.s;
    else if (k < P.nx + P.ny) origin[k] = P.dom_min[1] + (double)(k - P.nx) * P.s;
    else if (k < P.nx + P.ny + P.nz) origin[k] = P.dom_min[2] + (double)(k - P.nx - P.ny) * P.s;
}

int fill_origins(sph_ctx *ctx)
{
    const int n = ctx->dp.nx + ctx->dp.ny + ctx->dp.nz, T = 256;
    SPH_LAUNCH(ctx, k_fill_origins, (n + T - 1) / T, T, 0, ctx->stream, ctx->dp, ctx->w.origin);
    return check_cuda(cudaGetLastError());
}

__device__ __forceinline__ void cell_origin(const DevParams &P, const double *__restrict__ origin,
                                            uint32_t c, double *ox, double *oy, double *oz)
{
    uint32_t cx = c % (uint32_t)P.nx;
    uint32_t t = c / (uint32_t)P.nx;
    uint32_t cy = t % (uint32_t)P.ny;
    uint32_t cz = t / (uint32_t)P.ny;
    *ox = origin[cx];
    *oy = origin[P.nx + cy];
    *oz = origin[P.nx + P.ny + cz];
}

// Threads [0, nf): particle q of the cell-grouped order (cell_q, src_q, id_q
// from k_place) takes position p = start[c] + (number of particles of its cell
// with a smaller id), which is its place in the (cell, id) order; its fluid
// state (x, y, z, the records V and VM, id) is copied from buffer `src` to
// position p of buffer `dst`, and its packed position record written.  The ids
// of a cell are contiguous in id_q, so the rank
// reads them from L1 (about 27 per cell at rest density; the cost grows with
// the square of a cell's population).  Threads [nf, nf+nb): refresh the packed
// pressure/density of boundary particle (i - nf).  Block max of the sound
// speed goes to sc->mx.c.
template <typename Real, bool SPLIT>
__global__ void __launch_bounds__(256)
k_reorder(int nf, int nb, DevParams P, const uint32_t *__restrict__ cell_q,
          const uint32_t *__restrict__ src_q, const uint32_t *__restrict__ id_q,
          const double *__restrict__ sx, const double *__restrict__ sy, const double *__restrict__ sz,
          const typename Vec4<Real>::T *__restrict__ sV, const typename Vec4<Real>::T *__restrict__ sVM,
          double *__restrict__ dx, double *__restrict__ dy, double *__restrict__ dz,
          typename Vec4<Real>::T *__restrict__ dV, typename Vec4<Real>::T *__restrict__ dVM,
          uint32_t *__restrict__ did, typename Vec4<Real>::T *__restrict__ posp,
          uint32_t *__restrict__ cell, const Real *__restrict__ brho,
          typename Vec4<Real>::T *__restrict__ bposp, typename Vec4<Real>::T *__restrict__ bvelr,
          const int32_t *__restrict__ bstart, const int32_t *__restrict__ fstart,
          const double *__restrict__ origin, float4 *__restrict__ posf, Scalars *sc)
{
    __shared__ double red[32];
    __shared__ float redf[32];
    typedef typename Vec4<Real>::T V4;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    // the largest sound speed, in the precision of the form
    Real cmax = 0;
    int p = 0;  // destination of thread i
    if (i < nf) {
        const uint32_t s = src_q[i];
        const uint32_t c = cell_q[i];
        const uint32_t myid = id_q[i];
        // the source loads are issued before the rank loop, which hides their latency
        const double x = sx[s], y = sy[s], z = sz[s];
        const V4 vv = sV[s], vm = sVM[s];
        const int b = fstart[c], e = fstart[c + 1];
        int r = 0;
#pragma unroll 4
        for (int k = b; k < e; ++k) r += id_q[k] < myid ? 1 : 0;
        p = b + r;
        dx[p] = x; dy[p] = y; dz[p] = z;
        dV[p] = vv;   // also the PI input velr = {v, rho}
        dVM[p] = vm;
        did[p] = myid;
        cell[p] = c;
        const Real rho = vv.w;
        V4 pp;
        if (SPLIT) {
            float pr, cs;
            eos32(P, (float)rho, &pr, &cs);
            double ox = 0.0, oy = 0.0, oz = 0.0;
            if (c < P.ncells) cell_origin(P, origin, c, &ox, &oy, &oz);
            pp.x = (Real)(x - ox); pp.y = (Real)(y - oy); pp.z = (Real)(z - oz); pp.w = (Real)pr;
            if (c < P.ncells) cmax = (Real)cs;
        } else {
            double pr, cs;
            eos64(P, (double)rho, &pr, &cs);
            pp.x = (Real)x; pp.y = (Real)y; pp.z = (Real)z; pp.w = (Real)pr;
            if (c < P.ncells) {
                cmax = (Real)cs;
                double ox, oy, oz;
                cell_origin(P, origin, c, &ox, &oy, &oz);
                posf[p] = make_float4((float)(x - ox), (float)(y - oy), (float)(z - oz), 0.f);
            }
        }
        posp[p] = pp;
    } else if (i < nf + nb) {
        int j = i - nf;
        if (j < bstart[P.ncells]) {
            Real rho = brho[j];
            V4 pp = bposp[j];
            V4 vv;
            vv.x = 0; vv.y = 0; vv.z = 0; vv.w = rho;
            if (SPLIT) {
                float pr, cs;
                eos32(P, (float)rho, &pr, &cs);
                pp.w = (Real)pr;
                cmax = (Real)cs;
            } else {
                double pr, cs;
                eos64(P, (double)rho, &pr, &cs);
                pp.w = (Real)pr;
                cmax = (Real)cs;
            }
            bposp[j] = pp;
            bvelr[j] = vv;
        }
    }
    if (SPLIT) block_max_to_f(&sc->mx.c, (float)cmax, redf);
    else block_max_to(&sc->mx.c, (double)cmax, red);
}

// Boundary list (built once): gather the id-ordered boundary state staged in
// `in_*` into sorted order, with packed positions.
template <typename Real, bool SPLIT>
__global__ void k_boundary_place(int nb, uint32_t nf, DevParams P,
                                 const uint32_t *__restrict__ key_sorted,
                                 const uint32_t *__restrict__ val_sorted,
                                 const double *__restrict__ in_pos, const double *__restrict__ in_rho,
                                 const double *__restrict__ in_rhom,
                                 double *bx, double *by, double *bz, Real *brho, Real *brhom,
                                 uint32_t *bid, uint32_t *bcell,
                                 typename Vec4<Real>::T *bposp, typename Vec4<Real>::T *bvelr,
                                 const double *__restrict__ origin, float4 *__restrict__ bposf)
{
    typedef typename Vec4<Real>::T V4;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    uint32_t k = val_sorted[i];
    uint32_t c = key_sorted[i];
    double x = in_pos[3 * (size_t)(nf + k)], y = in_pos[3 * (size_t)(nf + k) + 1],
           z = in_pos[3 * (size_t)(nf + k) + 2];
    bx[i] = x; by[i] = y; bz[i] = z;
    brho[i] = (Real)in_rho[nf + k];
    brhom[i] = (Real)in_rhom[nf + k];
    bid[i] = nf + k;
    bcell[i] = c;
    V4 pp, vv;
    if (SPLIT) {
        double ox = 0.0, oy = 0.0, oz = 0.0;
        if (c < P.ncells) cell_origin(P, origin, c, &ox, &oy, &oz);
        pp.x = (Real)(x - ox); pp.y = (Real)(y - oy); pp.z = (Real)(z - oz);
    } else {
        pp.x = (Real)x; pp.y = (Real)y; pp.z = (Real)z;
        if (c < P.ncells) {
            double ox, oy, oz;
            cell_origin(P, origin, c, &ox, &oy, &oz);
            bposf[i] = make_float4((float)(x - ox), (float)(y - oy), (float)(z - oz), 0.f);
        }
    }
    pp.w = 0;
    vv.x = 0; vv.y = 0; vv.z = 0; vv.w = (Real)in_rho[nf + k];
    bposp[i] = pp;
    bvelr[i] = vv;
}

__global__ void k_boundary_hash(const double *__restrict__ pos, uint32_t nf, int nb, DevParams P,
                                uint32_t *key_by_id, uint32_t *val_by_id, uint32_t *count)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nb) return;
    size_t g = (size_t)(nf + k);
    uint32_t c = cell_of(P, pos[3 * g], pos[3 * g + 1], pos[3 * g + 2]);
    key_by_id[k] = c;
    val_by_id[k] = (uint32_t)k;
    atomicAdd(&count[c], 1u);
}

int key_passes_for(uint32_t ncells);

static int key_passes(uint32_t ncells)
{
    int bits = 0;
    while (bits < 32 && ((uint64_t)1 << bits) <= (uint64_t)ncells) ++bits;
    return bits <= 8 ? 1 : (bits + 7) / 8;
}

// ------------------------------------------------------------ entry points --

template <typename Real, bool SPLIT>
static int nl_fluid_t(sph_ctx *ctx)
{
    Workspace &w = ctx->w;
    cudaStream_t st = ctx->stream;
    int nf = (int)ctx->nf, nb = (int)ctx->nb;
    int src = ctx->cur, dst = 1 - ctx->cur;
    const int T = 256;
    // one memset clears the cell counts, their tile sums and the work-item
    // counters of this step (they follow each other in the workspace)
    const int64_t ftiles = scan_tiles((int64_t)ctx->ncells + 2);
    if (check_cuda(cudaMemsetAsync(w.count, 0,
                                   sizeof(uint32_t) * (ctx->ncells + 2 + ftiles + kCtrReset), st)))
        return SPH_ERR_CUDA;
    // cell and slot of every particle (key_tmp, val_tmp), counts per cell and
    // per scan tile
    if (nf > 0)
        SPH_LAUNCH(ctx, k_hash, (nf + kHashBlock - 1) / kHashBlock, kHashBlock, 0, st, w.x[src],
                   w.y[src], w.z[src], nf, ctx->dp, w.key_tmp, w.val_tmp, w.count, w.fpart, w.sc);
    // cell starts and the PI work items (up to 32 particles of one cell each)
    SPH_LAUNCH(ctx, k_scan_items, (unsigned)ftiles, kScanBlock, 0, st, w.count,
               (uint32_t *)w.fstart, (int64_t)ctx->ncells + 2, w.fpart, ctx->ncells, w.items_f,
               &w.ctr[0]);
    // cell-grouped order: cell (key_sorted), source (val_sorted), id (key_by_id)
    if (nf > 0)
        SPH_LAUNCH(ctx, k_place, (nf + T - 1) / T, T, 0, st, nf, w.key_tmp, w.val_tmp, w.id[src],
                   w.fstart, w.key_sorted, w.val_sorted, w.key_by_id);
    int tot = nf + nb;
    if (tot > 0) {
        typedef typename Vec4<Real>::T V4;
        SPH_LAUNCH(ctx, (k_reorder<Real, SPLIT>), (tot + T - 1) / T, T, 0, st, nf, nb, ctx->dp,
                   w.key_sorted, w.val_sorted, w.key_by_id, w.x[src], w.y[src], w.z[src],
                   (const V4 *)w.V[src], (const V4 *)w.VM[src], w.x[dst], w.y[dst], w.z[dst],
                   (V4 *)w.V[dst], (V4 *)w.VM[dst], w.id[dst], (V4 *)w.posp, w.cell,
                   (const Real *)w.brho, (V4 *)w.bposp, (V4 *)w.bvelr, w.bstart, w.fstart,
                   w.origin, w.posf, w.sc);
    }
    ctx->cur = dst;
    return check_cuda(cudaGetLastError());
}

int nl_fluid(sph_ctx *ctx)
{
    if (ctx->precision == SPH_FP32_SPLIT) return nl_fluid_t<float, true>(ctx);
    return nl_fluid_t<double, false>(ctx);
}

// Build the boundary list from the id-ordered state staged in w.stage
// (pos 3N | vel 3N | rho N | velm 3N | rhom N).
template <typename Real, bool SPLIT>
static int nl_boundary_t(sph_ctx *ctx)
{
    Workspace &w = ctx->w;
    cudaStream_t st = ctx->stream;
    int nf = (int)ctx->nf, nb = (int)ctx->nb;
    size_t N = (size_t)(nf + nb);
    const double *in_pos = w.stage;
    const double *in_rho = w.stage + 6 * N;
    const double *in_rhom = w.stage + 10 * N;
    const int T = 256;
    if (check_cuda(cudaMemsetAsync(w.count, 0,
                                   sizeof(uint32_t) * (ctx->ncells + 2 +
                                                       scan_tiles((int64_t)ctx->ncells + 2) +
                                                       kCtrWords),
                                   st)))
        return SPH_ERR_CUDA;
    if (nb > 0) {
        SPH_LAUNCH(ctx, k_boundary_hash, (nb + T - 1) / T, T, 0, st, in_pos, (uint32_t)nf, nb,
                   ctx->dp, w.key_by_id, w.val_by_id, w.count);
        int rc = radix_sort(ctx, w.key_by_id, w.val_by_id, w.key_tmp, w.val_tmp, w.key_sorted,
                            w.val_sorted, nb, ctx->nl_passes, st);
        if (rc) return rc;
        SPH_LAUNCH(ctx, (k_boundary_place<Real, SPLIT>), (nb + T - 1) / T, T, 0, st, nb,
                   (uint32_t)nf, ctx->dp, w.key_sorted, w.val_sorted, in_pos, in_rho, in_rhom,
                   w.bx, w.by, w.bz, (Real *)w.brho, (Real *)w.brhom, w.bid, w.bcell,
                   (typename Vec4<Real>::T *)w.bposp, (typename Vec4<Real>::T *)w.bvelr, w.origin,
                   w.bposf);
    }
    int rc = exclusive_scan_u32(ctx, w.count, (uint32_t *)w.bstart, (int64_t)ctx->ncells + 2,
                                w.scan_part, st);
    if (rc) return rc;
    rc = boundary_items_launch(ctx);
    if (rc) return rc;
    return check_cuda(cudaGetLastError());
}

int key_passes_for(uint32_t ncells) { return key_passes(ncells); }

int nl_boundary_build(sph_ctx *ctx)
{
    ctx->nl_passes = key_passes(ctx->ncells);
    if (ctx->precision == SPH_FP32_SPLIT) return nl_boundary_t<float, true>(ctx);
    return nl_boundary_t<double, false>(ctx);
}

}  // namespace sph
