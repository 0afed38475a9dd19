// PI, SPH_FP32_SPLIT form, in the paper's GPU design (Section 4, Fig. 11): one
// thread per target particle walks its own neighbour ranges and evaluates the
// pair terms under a per-candidate branch; F-F and F-B in one kernel, B-F in
// its own (Section 4.5).  Two ways of finding the ranges (Section 4.4):
//   pi_kernel = 1  the 27 cells from CellBeginEnd inside the kernel (Fig. 11 top);
//                  with cells of edge in [h, 2h) (Section 4.6, optimisation F; the paper's
//                  finer cells) the 125 cells as 25 x-runs of 5 cells
//   pi_kernel = 2  "FastCells": 9 x-run ranges per cell precomputed after NL by
//                  k_cell_ranges and read by the kernel (Fig. 11 bottom)
// Kept as selectable variants of sph_interact so that the paper's GPU
// optimisations can be measured on GB300 beside the warp-cooperative kernel
// (pi_kernel = 0, pi32.cu); the arithmetic of a pair is the same (pair_t).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "pair32.cuh"
#include "sph_internal.cuh"

namespace sph {

namespace {

// The pair terms of the warp kernel (pair32.cuh, units of h) for r_ab in
// metres; rho2a = rho_a^2.
template <bool MOMENTUM>
__device__ __forceinline__ void pair_t(const DevParams &P, const float4 &pa, const float4 &va,
                                       float rho2a, const float4 &pb, const float4 &vb, float rx,
                                       float ry, float rz, Acc32 &o)
{
    pair_acc32<MOMENTUM, false>(P, rx * P.invhf, ry * P.invhf, rz * P.invhf, pa.w, va, rho2a, vb,
                                pb.w, o);
}

// Candidates of one x-run: each gets the shift of its own cell x + k
// (k = -R .. R), found from the first indices of cells x - R + 1 .. x + R
// (cut[0 .. 2R-1]): k = -R + the number of cuts at or below j.
template <bool MOMENTUM, int R>
__device__ __forceinline__ void walk_range(const DevParams &P, const float4 &pa, const float4 &va,
                                           float ca, int j0, int j1, const int (&cut)[2 * R],
                                           int dy, int dz, const float4 *__restrict__ posp,
                                           const float4 *__restrict__ velr, Acc32 &o)
{
    const float ya = pa.y - (float)dy * P.sf;
    const float za = pa.z - (float)dz * P.sf;
    for (int j = j0; j < j1; ++j) {
        int k = -R;
#pragma unroll
        for (int u = 0; u < 2 * R; ++u) k += j >= cut[u] ? 1 : 0;
        const float xa = pa.x - (float)k * P.sf;
        float4 pb = posp[j];
        float rx = xa - pb.x, ry = ya - pb.y, rz = za - pb.z;
        float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
        if (r2 < P.four_h2f) pair_t<MOMENTUM>(P, pa, va, ca, pb, velr[j], rx, ry, rz, o);
    }
}

// The (2R+1)^2 x-runs of one list around cell (cx, cy, cz).  FAST (R = 1)
// reads the run bounds from the per-cell table (9 x {begin, first of cell x,
// first of cell x+1, end}); otherwise they come from the cell first indices.
// Cut indices clamp to the row (cells left of x = 0 hold nothing; the first
// index of cell nx of a row is the end of the row).
template <bool MOMENTUM, bool FAST, int R>
__device__ __forceinline__ void runs_t(const DevParams &P, const float4 &pa, const float4 &va,
                                       float ca, uint32_t cell, int cx, int cy, int cz,
                                       const float4 *__restrict__ posp,
                                       const float4 *__restrict__ velr,
                                       const int32_t *__restrict__ start,
                                       const int4 *__restrict__ ranges, Acc32 &o)
{
    constexpr int W = 2 * R + 1;
    for (int q = 0; q < W * W; ++q) {
        const int dz = q / W - R, dy = q % W - R;
        int j0, j1, cut[2 * R];
        if (FAST) {
            const int4 rg = ranges[(size_t)cell * 9 + q];
            j0 = rg.x;
            cut[0] = rg.y;
            cut[2 * R - 1] = rg.z;
            j1 = rg.w;
        } else {
            const int y = cy + dy, z = cz + dz;
            if (y < 0 || y >= P.ny || z < 0 || z >= P.nz) continue;
            const int row = P.nx * (y + P.ny * z);
            j0 = start[row + max(cx - R, 0)];
            j1 = start[row + min(cx + R, P.nx - 1) + 1];
#pragma unroll
            for (int u = 0; u < 2 * R; ++u) cut[u] = start[row + min(max(cx - R + 1 + u, 0), P.nx)];
        }
        if (j0 >= j1) continue;
        walk_range<MOMENTUM, R>(P, pa, va, ca, j0, j1, cut, dy, dz, posp, velr, o);
    }
}

template <bool FAST, int R>
__global__ void __launch_bounds__(128)
k_pi_thread_fluid(int nf, DevParams P, const float4 *__restrict__ posp,
                  const float4 *__restrict__ velr, const uint32_t *__restrict__ cell,
                  const int32_t *__restrict__ fstart, const int4 *__restrict__ franges,
                  const float4 *__restrict__ bposp, const float4 *__restrict__ bvelr,
                  const int32_t *__restrict__ bstart, const int4 *__restrict__ branges,
                  float4 *__restrict__ acc, Scalars *sc)
{
    __shared__ double red[32];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int nvalid = fstart[P.ncells];
    double f2 = 0.0, vis = 0.0;
    if (i < nvalid) {
        const float4 pa = posp[i], va = velr[i];
        const uint32_t c = cell[i];
        const uint32_t t = c / (uint32_t)P.nx;
        const int cx = (int)(c - t * (uint32_t)P.nx), cy = (int)(t % (uint32_t)P.ny),
                  cz = (int)(t / (uint32_t)P.ny);
        const float ca = va.w * va.w;  // rho_a^2
        Acc32 o = {0.f, 0.f, 0.f, 0.f, 0.f};
        runs_t<true, FAST, R>(P, pa, va, ca, c, cx, cy, cz, posp, velr, fstart, franges, o);
        runs_t<true, FAST, R>(P, pa, va, ca, c, cx, cy, cz, bposp, bvelr, bstart, branges, o);
        const float ax = fmaf(P.nmkBf, o.ax, P.gf[0]);
        const float ay = fmaf(P.nmkBf, o.ay, P.gf[1]);
        const float az = fmaf(P.nmkBf, o.az, P.gf[2]);
        acc[i] = make_float4(ax, ay, az, P.mkBf * o.ar);
        f2 = (double)ax * ax + (double)ay * ay + (double)az * az;
        vis = (double)o.vis;
        if (!(f2 < INFINITY) || !(o.ar == o.ar)) atomicOr(&sc->flags, SPH_FLAG_NAN);
    }
    block_max_to(&sc->mx.f2, f2, red);
    block_max_to(&sc->mx.visc, vis, red);
}

template <bool FAST, int R>
__global__ void __launch_bounds__(128)
k_pi_thread_boundary(int nb, DevParams P, const float4 *__restrict__ bposp,
                     const float4 *__restrict__ bvelr, const uint32_t *__restrict__ bcell,
                     const int32_t *__restrict__ bstart, const float4 *__restrict__ posp,
                     const float4 *__restrict__ velr, const int32_t *__restrict__ fstart,
                     const int4 *__restrict__ franges, float *__restrict__ bar, Scalars *sc)
{
    __shared__ double red[32];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int nvalid = bstart[P.ncells];
    double vis = 0.0;
    if (i < nvalid) {
        const float4 pa = bposp[i], va = bvelr[i];
        const uint32_t c = bcell[i];
        const uint32_t t = c / (uint32_t)P.nx;
        const int cx = (int)(c - t * (uint32_t)P.nx), cy = (int)(t % (uint32_t)P.ny),
                  cz = (int)(t / (uint32_t)P.ny);
        Acc32 o = {0.f, 0.f, 0.f, 0.f, 0.f};
        runs_t<false, FAST, R>(P, pa, va, 0.f, c, cx, cy, cz, posp, velr, fstart, franges, o);
        bar[i] = P.mkBf * o.ar;
        vis = (double)o.vis;
    }
    block_max_to(&sc->mx.visc, vis, red);
}

// FastCells table: for every cell and each of its 9 (dy, dz) rows, {first index
// of the run, first of cell x, first of cell x+1, end of the run}; rows outside
// the grid get an empty range.
__global__ void k_cell_ranges(DevParams P, const int32_t *__restrict__ start,
                              int4 *__restrict__ ranges)
{
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)P.ncells * 9) return;
    const uint32_t c = (uint32_t)(t / 9);
    const int q = (int)(t % 9);
    const uint32_t u = c / (uint32_t)P.nx;
    const int cx = (int)(c - u * (uint32_t)P.nx), cy = (int)(u % (uint32_t)P.ny),
              cz = (int)(u / (uint32_t)P.ny);
    const int y = cy + q % 3 - 1, z = cz + q / 3 - 1;
    int4 rg = make_int4(0, 0, 0, 0);
    if (y >= 0 && y < P.ny && z >= 0 && z < P.nz) {
        const int row = P.nx * (y + P.ny * z);
        rg = make_int4(start[row + max(cx - 1, 0)], start[row + cx], start[row + cx + 1],
                       start[row + min(cx + 1, P.nx - 1) + 1]);
    }
    ranges[t] = rg;
}

}  // namespace

int pi32_thread_launch(sph_ctx *ctx)
{
    Workspace &w = ctx->w;
    cudaStream_t st = ctx->stream;
    const int nf = (int)ctx->nf, nb = (int)ctx->nb;
    const int T = 128;
    const bool fast = ctx->prm.pi_kernel == SPH_PI_THREAD_FASTCELLS;
    if (fast) {
        const size_t n9 = (size_t)ctx->ncells * 9;
        const unsigned g = (unsigned)((n9 + 255) / 256);
        SPH_LAUNCH(ctx, k_cell_ranges, g, 256, 0, st, ctx->dp, w.fstart, w.franges);
        if (!ctx->branges_ready) {
            SPH_LAUNCH(ctx, k_cell_ranges, g, 256, 0, st, ctx->dp, w.bstart, w.branges);
            ctx->branges_ready = true;
        }
    }
    if (nf > 0) {
        if (fast)
            SPH_LAUNCH(ctx, (k_pi_thread_fluid<true, 1>), (nf + T - 1) / T, T, 0, st, nf, ctx->dp,
                       (const float4 *)w.posp, (const float4 *)velr_of(ctx), w.cell, w.fstart, w.franges,
                       (const float4 *)w.bposp, (const float4 *)w.bvelr, w.bstart, w.branges,
                       (float4 *)w.acc, w.sc);
        else if (ctx->dp.reach == 1)
            SPH_LAUNCH(ctx, (k_pi_thread_fluid<false, 1>), (nf + T - 1) / T, T, 0, st, nf, ctx->dp,
                       (const float4 *)w.posp, (const float4 *)velr_of(ctx), w.cell, w.fstart,
                       (const int4 *)nullptr, (const float4 *)w.bposp, (const float4 *)w.bvelr,
                       w.bstart, (const int4 *)nullptr, (float4 *)w.acc, w.sc);
        else
            SPH_LAUNCH(ctx, (k_pi_thread_fluid<false, 2>), (nf + T - 1) / T, T, 0, st, nf, ctx->dp,
                       (const float4 *)w.posp, (const float4 *)velr_of(ctx), w.cell, w.fstart,
                       (const int4 *)nullptr, (const float4 *)w.bposp, (const float4 *)w.bvelr,
                       w.bstart, (const int4 *)nullptr, (float4 *)w.acc, w.sc);
    }
    if (nb > 0) {
        if (fast)
            SPH_LAUNCH(ctx, (k_pi_thread_boundary<true, 1>), (nb + T - 1) / T, T, 0, st, nb, ctx->dp,
                       (const float4 *)w.bposp, (const float4 *)w.bvelr, w.bcell, w.bstart,
                       (const float4 *)w.posp, (const float4 *)velr_of(ctx), w.fstart, w.franges,
                       (float *)w.bar, w.sc);
        else if (ctx->dp.reach == 1)
            SPH_LAUNCH(ctx, (k_pi_thread_boundary<false, 1>), (nb + T - 1) / T, T, 0, st, nb, ctx->dp,
                       (const float4 *)w.bposp, (const float4 *)w.bvelr, w.bcell, w.bstart,
                       (const float4 *)w.posp, (const float4 *)velr_of(ctx), w.fstart,
                       (const int4 *)nullptr, (float *)w.bar, w.sc);
        else
            SPH_LAUNCH(ctx, (k_pi_thread_boundary<false, 2>), (nb + T - 1) / T, T, 0, st, nb, ctx->dp,
                       (const float4 *)w.bposp, (const float4 *)w.bvelr, w.bcell, w.bstart,
                       (const float4 *)w.posp, (const float4 *)velr_of(ctx), w.fstart,
                       (const int4 *)nullptr, (float *)w.bar, w.sc);
    }
    return check_cuda(cudaGetLastError());
}

}  // namespace sph
