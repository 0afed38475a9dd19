// Internal declarations of libsph (not part of the ABI).
//
// Data layout in HBM (one context):
//   fluid state, double-buffered (NL gathers buffer `cur` into `1-cur`), in
//   sorted (cell, id) order:  x y z (f64, one array each) | V = {vx, vy, vz,
//   rho} | VM = {vx, vy, vz, rho} of the previous level (Real4 records, Real =
//   f64 in SPH_FP64, f32 in SPH_FP32_SPLIT) | id (u32).
//   packed PI inputs of Section 4.3: posp = {x, y, z, P/rho^2} (written by NL)
//   and velr = {vx, vy, vz, rho}, which is V of the current buffer itself; in
//   SPH_FP32_SPLIT the position is the f32 offset from the origin of the
//   particle's cell, in SPH_FP64 it is absolute.  cell (u32) per particle.
//   PI output acc = {ax, ay, az, drho/dt} per fluid particle.
//   boundary state (never moves, sorted once): x y z (f64), rho rhom (Real),
//   id (u32), packed posp/velr like the fluid, ar (Real) output.
//   NL scratch: cell and in-cell slot per particle, the cell-grouped cell /
//   source / id arrays (fluid, every step); keys/values by id and their
//   sorted copies (boundary radix sort, once); per-cell counts and first
//   indices (fluid and boundary), radix-sort tile histograms.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sph.h"

namespace sph {

// Largest value of each time-step maximum, stored as the bit pattern of a
// non-negative double (so atomicMax on the integer is a max on the value).
struct Maxima {
    unsigned long long f2;    // max |f_a|^2 over fluid
    unsigned long long c;     // max c_a over all particles in the grid
    unsigned long long visc;  // max |h v.r / (r^2 + eta^2)| over pairs
};

struct Scalars {
    Maxima mx;
    double dt_last;
    double time;
    long long step;     // completed steps
    uint32_t flags;
    uint32_t bmoved;    // set when a staged boundary position differs from the list's
};

// Constants every kernel needs, passed by value.
struct DevParams {
    double h, s, inv_s, rho0, inv_rho0, gamma, c0, alpha, eta2, cfl, mass, B, fixed_dt;
    double invh, kA64, kB64;  // 1/h and the grad-W factor constants (see pi.cu)
    double kc64;              // -alpha c0 / rho0^3 (viscosity factor for gamma = 7, see pi.cu)
    double kcu64;             // c0 / rho0^3 (the same without -alpha, for d/d alpha in the adjoint)
    double g[3];
    double dom_min[3];
    int nx, ny, nz;
    uint32_t ncells;
    int euler_every;
    int reach;            // cells searched on each side: 1 (cell >= 2h) or 2 (h <= cell < 2h)
    int clamp;
    int gamma_is_7;
    int tensile;          // tensile correction on
    int tensile_n;
    double tens_eps, tens_pos, inv_wdp;   // inv_wdp = 1 / W(dp)
    // float copies for the FP32 path
    float hf, invhf, four_h2f, eta2f, massf, alphaf, c0f, inv_rho0f, Bf, sf;
    float kA, kB;   // grad-W factor constants (see pi.cu)
    float aDf, tens_epsf, tens_posf, inv_wdpf;  // 1/(pi h^3) and the tensile constants
    // the warp FP32 PI kernel works in units of h (see pi32.cu): s/h, eta^2/h^2,
    // the grad-W branch q < 1 as F'' = gw1 q + gw0, the per-target factors
    // -m kB (momentum) and m kB (continuity), and -alpha c0 / rho0^3
    float s_hf, eta2_h2f, gw1, gw0, nmkBf, mkBf, kcf, nalphaf;
    // cell of a position from a float32 estimate (see nl.cu): 1/s, min/s and
    // |min/s| per axis, and the error bound of positions flushed to 0
    float cell_af, cell_bf[3], cell_babsf[3], cell_eabsf;
    float gf[3];
};

struct Workspace {
    // fluid state
    double *x[2], *y[2], *z[2];
    void *V[2], *VM[2];       // Real4 {vx, vy, vz, rho} of this and of the previous level
    uint32_t *id[2];
    char *state_chunk[2];
    size_t state_chunk_bytes;
    // packed PI inputs / outputs (fluid); the velocity record is V[cur]
    void *posp, *acc;
    float4 *posf, *bposf;     // SPH_FP64: float32 offsets from the cell origin (pre-test of PI)
    uint32_t *cell;
    // boundary
    double *bx, *by, *bz;
    void *brho, *brhom, *bposp, *bvelr, *bar;
    uint32_t *bid, *bcell;
    char *bstate_chunk;
    size_t bstate_chunk_bytes;
    // NL scratch.  Fluid: key_tmp / val_tmp = cell / slot per particle,
    // key_sorted / val_sorted / key_by_id = cell / source / id in the
    // cell-grouped order.  Boundary: the radix sort's keys and values.
    uint32_t *key_by_id, *val_by_id, *key_tmp, *val_tmp, *key_sorted, *val_sorted;
    uint32_t *count;          // [ncells + 2], then fpart, then the work-item counters ctr
    uint32_t *fpart;          // fluid NL: particles per scan tile of kScanTile cells (k_hash)
    uint32_t *ctr;            // [0] fluid items, [1] next item of the PI queue, [2] spare, [3] boundary items
    uint32_t *items_f, *items_b;  // PI work items, {first, count} pairs: fluid, up to 32
                                  // particles of one cell (k_scan_items); boundary, packed
                                  // cells of one x row (k_pack_boundary_items)
    int4 *franges, *branges;      // per-cell x-run tables (SPH_PI_THREAD_FASTCELLS)
    int32_t *fstart, *bstart; // [ncells + 2]
    double *origin;           // cell origins min_d + c s along x (nx), y (ny), z (nz)
    uint32_t *radix_hist;     // [256 * tiles]
    uint32_t *scan_part;      // scan partials
    // adjoint scratch (SPH_FP64 contexts): cotangents of F and D, the adjoint
    // in sorted order (11 doubles per particle), dJ/dalpha partial sums (per
    // work item at its first target, or per block)
    double *adj_gF, *adj_gD, *adj_lam, *adj_part;
    double *sens_p, *sens_den;  // sensor pressures and Shepard denominators
    double *front;              // front position: max x and the sum of exp((x - max) / tau)
    // host exchange staging: 11 doubles per particle
    double *stage;
    Scalars *sc;
    unsigned long long *counts4;  // validation counters
};

}  // namespace sph

struct sph_ctx {
    sph_params prm;
    sph::DevParams dp;
    int64_t nf, nb;
    int dims[3];
    uint32_t ncells;
    int precision;
    size_t real_size;
    cudaStream_t stream;
    sph::Workspace w;
    int cur;                 // current fluid buffer
    int nl_passes;           // radix passes of 8 bits
    bool nl_valid, pi_valid;
    long long launches;
    int device;
    int pi_grid_f;              // persistent grid size of the warp PI kernels
    int adj_grid;               // persistent grid size of the work-item adjoint kernel
    bool branges_ready;         // boundary x-run table built for the current boundary list
    bool boundary_built;        // the boundary list exists (built at least once)
    // sph_run_graph: executable graphs of two consecutive steps, one per value
    // of `cur` at the start, and the number of kernels each launches
    cudaGraphExec_t graph[2];
    long long graph_launches[2];
};

namespace sph {

// {v, rho} records of the current fluid state: the PI input velr of Section 4.3.
inline void *velr_of(const sph_ctx *ctx) { return ctx->w.V[ctx->cur]; }

// Four-component record of the precision of a form.
template <typename Real> struct Real4T;
template <> struct Real4T<float> { typedef float4 T; };
template <> struct Real4T<double> { typedef double4_32a T; };

// workspace planning (api.cu)
size_t plan_workspace(const sph_params &p, int64_t nf, int64_t nb, int dims[3], uint32_t *ncells,
                      Workspace *w, char *base);

// parameter checks and derived constants (api.cu)
int validate_params(const sph_params *p, int64_t nf, int64_t nb, int dims[3], uint32_t *ncells);
DevParams derive_params(const sph_params &p, const int dims[3], uint32_t ncells);

// NL (nl.cu)
int nl_fluid(sph_ctx *ctx);
int radix_sort(sph_ctx *ctx, const uint32_t *kin, const uint32_t *vin, uint32_t *ktmp,
               uint32_t *vtmp, uint32_t *kout, uint32_t *vout, int n, int passes,
               cudaStream_t st);
int key_passes_for(uint32_t ncells);
__global__ void k_boundary_hash(const double *__restrict__ pos, uint32_t nf, int nb, DevParams P,
                                uint32_t *key_by_id, uint32_t *val_by_id, uint32_t *count);
int nl_boundary_build(sph_ctx *ctx);
void nl_boundary_refresh_launch(sph_ctx *ctx, cudaStream_t st);
int radix_tiles(int64_t n);
size_t scan_partials(int64_t n);

// PI (pi.cu, pi32.cu)
int pi_launch(sph_ctx *ctx);
int pi32_launch(sph_ctx *ctx);
int pi32_thread_launch(sph_ctx *ctx);
int pi32_setup(sph_ctx *ctx);
int fill_origins(sph_ctx *ctx);
int pi32_sym_launch(sph_ctx *ctx);
int pi32_sym_setup(sph_ctx *ctx);
int pi64_setup(sph_ctx *ctx);
int adjoint_setup(sph_ctx *ctx);   // adjoint.cu
int boundary_items_launch(sph_ctx *ctx);
int count_work_launch(sph_ctx *ctx);
constexpr int kCtrWords = 4;     // work-item counters after the cell counts
constexpr int kCtrReset = 3;     // counters cleared by every fluid NL

// SU (su.cu)
int su_launch(sph_ctx *ctx);

// id-order exchange (api.cu)
int check_cuda(cudaError_t e);

// generic helpers
constexpr int kRadixTile = 2048;   // keys per radix-sort tile (nl.cu)
constexpr int kMaxSensors = 4096;  // sensor points per objective call
constexpr int kScanBlock = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanBlock * kScanItems;

int exclusive_scan_u32(sph_ctx *ctx, const uint32_t *in, uint32_t *out, int64_t n,
                       uint32_t *partials, cudaStream_t st);
// Tiles of kScanTile entries in a scan of n entries.
inline int64_t scan_tiles(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *dst, double v)
{
    // non-negative doubles (and +inf / NaN, which compare above) order like
    // their bit patterns.  The stored maximum only grows, so a value not above
    // the one already read needs no atomic (most blocks of a large grid skip
    // it instead of queueing on the one address).
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    if (b > *(volatile unsigned long long *)dst) atomicMax(dst, b);
}

__device__ __forceinline__ double warp_max(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ float warp_maxf(float v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide max of a non-negative float, one atomic per block (the float64
// unit is used once per block).
__device__ __forceinline__ void block_max_to_f(unsigned long long *dst, float v, float *smem32)
{
    bool nan = v != v;
    unsigned anynan = __syncthreads_or(nan);
    float m = warp_maxf(nan ? 0.0f : v);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) smem32[wid] = m;
    __syncthreads();
    if (wid == 0) {
        int nw = (blockDim.x + 31) >> 5;
        float t = lane < nw ? smem32[lane] : 0.0f;
        t = warp_maxf(t);
        if (lane == 0)
            atomic_max_nonneg(dst, anynan ? __longlong_as_double(0x7ff8000000000000LL) : (double)t);
    }
    __syncthreads();
}

// Block-wide max of a non-negative value followed by one atomic per block.
// Every thread of the block must call it.  NaN is propagated (fmax drops NaN,
// so it is tracked separately).
__device__ __forceinline__ void block_max_to(unsigned long long *dst, double v, double *smem32)
{
    bool nan = v != v;
    unsigned anynan = __syncthreads_or(nan);
    double m = warp_max(nan ? 0.0 : v);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) smem32[wid] = m;
    __syncthreads();
    if (wid == 0) {
        int nw = (blockDim.x + 31) >> 5;
        double t = lane < nw ? smem32[lane] : 0.0;
        t = warp_max(t);
        if (lane == 0) atomic_max_nonneg(dst, anynan ? __longlong_as_double(0x7ff8000000000000LL) : t);
    }
    __syncthreads();
}

}  // namespace sph

#define SPH_LAUNCH(ctx, kernel, grid, block, smem, st, ...)                       \
    do {                                                                          \
        kernel<<<(grid), (block), (smem), (st)>>>(__VA_ARGS__);                   \
        (ctx)->launches++;                                                        \
    } while (0)
