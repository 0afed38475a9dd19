// PI stage (Sections 2, 4.3-4.5 of the paper): particle interactions.
//
// Float64 form, two designs.  k_pi64w (default for cells of edge 2h or more):
// one warp per work item with float32 lockstep candidate tests and float64
// pairs in per-lane hit walks (warp_items.cuh), fluid and boundary items in
// one launch.  k_pi_fluid64 / k_pi_boundary64: one thread per target particle
// (Section 4): its own data stay in registers and its sums are written once at
// the end (Section 4.5); fluid targets evaluate F-F and F-B in one kernel
// (Section 4.5, optimisation E), boundary targets have their own B-F kernel
// (continuity only).  Candidates are the
// particles of the 27 surrounding cells, visited as the 9 x-runs of Fig. 10 /
// Fig. 11 (cells x-1, x, x+1 of one (y, z) row are contiguous after NL); with
// cells of edge in [h, 2h) (the paper's finer cells, Section 4.6, optimisation F) the 125
// surrounding cells as 25 x-runs of 5 cells (P.reach = 2).
//
// Per ordered pair a <- b with r_ab = x_a - x_b, r = |r_ab| < 2h, q = r/h:
//   grad_a W_ab = F r_ab,  F = aD/h^2 (-3 + 2.25 q)         (q < 1)
//                            = -0.75 aD/h (2 - q)^2 / r       (1 <= q < 2), aD = 1/(pi h^3)
//   mu = h v_ab.r_ab / (r^2 + eta^2);  Pi = -alpha (c_a + c_b) mu / (rho_a + rho_b) if v_ab.r_ab < 0
//     (gamma = 7: -alpha (c_a + c_b)/(rho_a + rho_b) = -alpha c0/rho0^3 (rho_a^2 - rho_a rho_b + rho_b^2))
//   ace_a += -m (P_a/rho_a^2 + P_b/rho_b^2 + Pi) F r_ab      (fluid targets)
//   ar_a  +=  m F v_ab.r_ab
//   visc   = max(visc, |mu|)
// then ace_a += g; the block maxima of |ace|^2 and visc feed the time step.
//
// SPH_FP64: absolute float64 positions, every operation in float64.
// SPH_FP32_SPLIT: float32 positions relative to the origin of the particle's
// cell; a candidate in the neighbouring cell (dx, dy, dz) is shifted by
// (dx, dy, dz) * s, so all differences stay small and float32-accurate.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sph_internal.cuh"
#include "warp_items.cuh"

namespace sph {

__device__ __forceinline__ void cell_xyz(const DevParams &P, uint32_t c, int *cx, int *cy, int *cz)
{
    uint32_t t = c / (uint32_t)P.nx;
    *cx = (int)(c - t * (uint32_t)P.nx);
    *cy = (int)(t % (uint32_t)P.ny);
    *cz = (int)(t / (uint32_t)P.ny);
}

// ------------------------------------------------------------------ FP64 --

struct Acc64 {
    double ax, ay, az, ar, vis;
};

// Tensile correction of Monaghan (2000): R_ab (W(r)/W(dp))^n, with pr = P/rho^2
// (same sign as P) of the two particles.
__device__ __forceinline__ double tensile64(const DevParams &P, double q, double pra, double prb)
{
    double aD = P.kA64 * P.h * P.h;
    double w = q < 1.0 ? aD * (1.0 - 1.5 * q * q + 0.75 * q * q * q)
                       : aD * 0.25 * (2.0 - q) * (2.0 - q) * (2.0 - q);
    double f = w * P.inv_wdp, fn = 1.0;
    for (int k = 0; k < P.tensile_n; ++k) fn *= f;
    double R = (pra > 0.0 && prb > 0.0)
                   ? P.tens_pos * (pra + prb)
                   : P.tens_eps * (fmax(-pra, 0.0) + fmax(-prb, 0.0));
    return R * fn;
}

template <bool MOMENTUM>
__device__ __forceinline__ void pair64(const DevParams &P, const double4_32a &pa, const double4_32a &va,
                                       double ca, const double4_32a &pb, const double4_32a &vb, double rx,
                                       double ry, double rz, double r2, Acc64 &o)
{
    double rinv = rsqrt(r2);
    double r = r2 * rinv;
    double q = r * P.invh;
    double F = q < 1.0 ? P.kA64 * (-3.0 + 2.25 * q) : P.kB64 * (2.0 - q) * (2.0 - q) * rinv;
    double dvx = va.x - vb.x, dvy = va.y - vb.y, dvz = va.z - vb.z;
    double vdr = dvx * rx + dvy * ry + dvz * rz;
    double mu;
    if (MOMENTUM) {
        double Pi = 0.0;
        const double hv = P.h * vdr;
        if (P.gamma_is_7) {
            // with c = c0 (rho/rho0)^3, -alpha (c_a + c_b) / (rho_a + rho_b) equals
            // kc64 (rho_a^2 - rho_a rho_b + rho_b^2) (a^3 + b^3 = (a + b)(a^2 - ab + b^2)),
            // so Pi_ab = kc64 (...) mu_ab needs the one reciprocal of mu_ab only
            mu = hv / (r2 + P.eta2);
            if (vdr < 0.0) Pi = P.kc64 * fma(vb.w, vb.w - va.w, va.w * va.w) * mu;
        } else {
            // one reciprocal for both quotients: d = 1/((r^2 + eta^2)(rho_a + rho_b))
            const double S = va.w + vb.w;
            const double d = 1.0 / ((r2 + P.eta2) * S);
            mu = hv * S * d;
            if (vdr < 0.0) {
                const double rb = vb.w * P.inv_rho0;
                const double cb = P.c0 * pow(rb, 0.5 * (P.gamma - 1.0));
                Pi = -P.alpha * (ca + cb) * hv * d;
            }
        }
        if (P.tensile) Pi += tensile64(P, q, pa.w, pb.w);
        double coef = -(pa.w + pb.w + Pi) * F;
        o.ax += coef * rx;
        o.ay += coef * ry;
        o.az += coef * rz;
    } else {
        mu = P.h * vdr / (r2 + P.eta2);
    }
    o.ar += vdr * F;
    o.vis = fmax(o.vis, fabs(mu));
}

// The candidates of the (2R+1)^2 x-runs around cell (cx, cy, cz).  A float32
// pre-test on the cell-relative offsets (candidate offset + its cell delta *
// s against the target's offset) drops the candidates that are certainly
// outside the support: its threshold 4h^2 (1 + 1e-5) lies above the float32
// error of the offsets (about 1e-6 of 4h^2) and the float64 test that follows
// decides every pair exactly as before, so the pairs and every float64 result
// are those of the float64 test alone; the float64 unit, the scarce resource
// here, evaluates only the candidates near the support.
template <bool MOMENTUM>
__device__ __forceinline__ void runs64(const DevParams &P, int self, const double4_32a &pa,
                                       const float4 &fa, const double4_32a &va, double ca, int cx,
                                       int cy, int cz, const double4_32a *__restrict__ posp,
                                       const float4 *__restrict__ posf,
                                       const double4_32a *__restrict__ velr,
                                       const int32_t *__restrict__ start, Acc64 &o)
{
    const double s2 = 4.0 * P.h * P.h;
    const float s2f = P.four_h2f * (1.0f + 1e-5f);
    const int R = P.reach;
    int x0 = max(cx - R, 0), x1 = min(cx + R, P.nx - 1);
    for (int dz = -R; dz <= R; ++dz) {
        int z = cz + dz;
        if (z < 0 || z >= P.nz) continue;
        const float za = fa.z - (float)dz * P.sf;
        for (int dy = -R; dy <= R; ++dy) {
            int y = cy + dy;
            if (y < 0 || y >= P.ny) continue;
            const float ya = fa.y - (float)dy * P.sf;
            int row = P.nx * (y + P.ny * z);
            int j0 = start[row + x0], j1 = start[row + x1 + 1];
            // first index of cells x-R+1 .. x+R: a candidate lies in cell
            // x - R + (number of these at or below its index)
            int cut[4];
            for (int u = 0; u < 2 * R; ++u) cut[u] = start[row + min(max(cx - R + 1 + u, 0), P.nx)];
            for (int j = j0; j < j1; ++j) {
                if (j == self) continue;
                int k = -R;
                for (int u = 0; u < 2 * R; ++u) k += j >= cut[u] ? 1 : 0;
                const float4 fb = posf[j];
                const float ex = fa.x - (float)k * P.sf - fb.x, ey = ya - fb.y, ez = za - fb.z;
                if (!(fmaf(ex, ex, fmaf(ey, ey, ez * ez)) < s2f)) continue;
                double4_32a pb = posp[j];
                double rx = pa.x - pb.x, ry = pa.y - pb.y, rz = pa.z - pb.z;
                double r2 = rx * rx + ry * ry + rz * rz;
                if (r2 < s2) pair64<MOMENTUM>(P, pa, va, ca, pb, velr[j], rx, ry, rz, r2, o);
            }
        }
    }
}

__device__ __forceinline__ double sound64(const DevParams &P, double rho)
{
    double r = rho * P.inv_rho0;
    return P.gamma_is_7 ? P.c0 * r * r * r : P.c0 * pow(r, 0.5 * (P.gamma - 1.0));
}

__global__ void __launch_bounds__(128)
k_pi_fluid64(int nf, DevParams P, const double4_32a *__restrict__ posp,
             const double4_32a *__restrict__ velr, const uint32_t *__restrict__ cell,
             const int32_t *__restrict__ fstart, const double4_32a *__restrict__ bposp,
             const double4_32a *__restrict__ bvelr, const int32_t *__restrict__ bstart,
             const float4 *__restrict__ posf, const float4 *__restrict__ bposf,
             double4_32a *__restrict__ acc, Scalars *sc)
{
    __shared__ double red[32];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int nvalid = fstart[P.ncells];
    double f2 = 0.0, vis = 0.0;
    if (i < nvalid) {
        double4_32a pa = posp[i], va = velr[i];
        const float4 fa = posf[i];
        int cx, cy, cz;
        cell_xyz(P, cell[i], &cx, &cy, &cz);
        double ca = sound64(P, va.w);
        Acc64 o = {0.0, 0.0, 0.0, 0.0, 0.0};
        runs64<true>(P, i, pa, fa, va, ca, cx, cy, cz, posp, posf, velr, fstart, o);
        runs64<true>(P, -1, pa, fa, va, ca, cx, cy, cz, bposp, bposf, bvelr, bstart, o);
        double ax = P.mass * o.ax + P.g[0];
        double ay = P.mass * o.ay + P.g[1];
        double az = P.mass * o.az + P.g[2];
        acc[i] = make_double4_32a(ax, ay, az, P.mass * o.ar);
        f2 = __dadd_rn(__dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay)), __dmul_rn(az, az));
        vis = o.vis;
        if (!(f2 < INFINITY) || !(o.ar == o.ar)) atomicOr(&sc->flags, SPH_FLAG_NAN);
    } else if (i < nf) {
        acc[i] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    }
    block_max_to(&sc->mx.f2, f2, red);
    block_max_to(&sc->mx.visc, vis, red);
}

__global__ void __launch_bounds__(128)
k_pi_boundary64(int nb, DevParams P, const double4_32a *__restrict__ bposp,
                const double4_32a *__restrict__ bvelr, const uint32_t *__restrict__ bcell,
                const int32_t *__restrict__ bstart, const double4_32a *__restrict__ posp,
                const double4_32a *__restrict__ velr, const int32_t *__restrict__ fstart,
                const float4 *__restrict__ bposf, const float4 *__restrict__ posf,
                double *__restrict__ bar, Scalars *sc)
{
    __shared__ double red[32];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int nvalid = bstart[P.ncells];
    double vis = 0.0;
    if (i < nvalid) {
        double4_32a pa = bposp[i], va = bvelr[i];
        const float4 fa = bposf[i];
        int cx, cy, cz;
        cell_xyz(P, bcell[i], &cx, &cy, &cz);
        Acc64 o = {0.0, 0.0, 0.0, 0.0, 0.0};
        runs64<false>(P, -1, pa, fa, va, 0.0, cx, cy, cz, posp, posf, velr, fstart, o);
        bar[i] = P.mass * o.ar;
        vis = o.vis;
    } else if (i < nb) {
        bar[i] = 0.0;
    }
    block_max_to(&sc->mx.visc, vis, red);
}

// -------------------------------------------------------- validation pass --

// Exact counts in float64 with the products and sums rounded one by one (no
// contraction), the same arithmetic as a plain CPU evaluation of
// dx*dx + dy*dy + dz*dz < 4h^2 on absolute positions.
__device__ __forceinline__ void count_runs(const DevParams &P, double xa, double ya, double za,
                                           int self, int cx, int cy, int cz,
                                           const double *__restrict__ x,
                                           const double *__restrict__ y,
                                           const double *__restrict__ z,
                                           const int32_t *__restrict__ start,
                                           unsigned long long &cand, unsigned long long &pairs)
{
    const double s2 = 4.0 * P.h * P.h;
    const int R = P.reach;
    int x0 = max(cx - R, 0), x1 = min(cx + R, P.nx - 1);
    for (int dz = -R; dz <= R; ++dz) {
        int zz = cz + dz;
        if (zz < 0 || zz >= P.nz) continue;
        for (int dy = -R; dy <= R; ++dy) {
            int yy = cy + dy;
            if (yy < 0 || yy >= P.ny) continue;
            int row = P.nx * (yy + P.ny * zz);
            int j0 = start[row + x0], j1 = start[row + x1 + 1];
            for (int j = j0; j < j1; ++j) {
                if (j == self) continue;
                double rx = __dsub_rn(xa, x[j]), ry = __dsub_rn(ya, y[j]), rz = __dsub_rn(za, z[j]);
                double r2 = __dadd_rn(__dadd_rn(__dmul_rn(rx, rx), __dmul_rn(ry, ry)), __dmul_rn(rz, rz));
                cand++;
                if (r2 < s2) pairs++;
            }
        }
    }
}

__global__ void k_count_work(int nf, int nb, DevParams P, const double *__restrict__ x,
                             const double *__restrict__ y, const double *__restrict__ z,
                             const uint32_t *__restrict__ cell, const int32_t *__restrict__ fstart,
                             const double *__restrict__ bx, const double *__restrict__ by,
                             const double *__restrict__ bz, const uint32_t *__restrict__ bcell,
                             const int32_t *__restrict__ bstart, unsigned long long *counts)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long c = 0, p = 0;
    int cx, cy, cz;
    if (i < nf) {
        if (i < fstart[P.ncells]) {
            cell_xyz(P, cell[i], &cx, &cy, &cz);
            count_runs(P, x[i], y[i], z[i], i, cx, cy, cz, x, y, z, fstart, c, p);
            count_runs(P, x[i], y[i], z[i], -1, cx, cy, cz, bx, by, bz, bstart, c, p);
            atomicAdd(&counts[0], c);
            atomicAdd(&counts[1], p);
        }
    } else if (i < nf + nb) {
        int j = i - nf;
        if (j < bstart[P.ncells]) {
            cell_xyz(P, bcell[j], &cx, &cy, &cz);
            count_runs(P, bx[j], by[j], bz[j], -1, cx, cy, cz, x, y, z, fstart, c, p);
            atomicAdd(&counts[2], c);
            atomicAdd(&counts[3], p);
        }
    }
}

// ------------------------------------------------- FP64, warp per work item --
//
// The work items of the FP32 warp kernel with float64 pairs (warp_items.cuh):
// float32 lockstep tests of the staged cell-relative offsets, then each lane
// walks its own hits with the float64 test and the float64 pair of pair64, so
// the float64 unit works on near neighbours with the lanes of the warp busy
// together (the thread-per-target kernel above runs its pair branch with the
// lanes whose candidate passed).  Cells of edge 2h or more only.

namespace {

constexpr int W64_WARPS = 4;

template <bool MOMENTUM>
__device__ __forceinline__ void pi64_item(
    const DevParams &P, witems::Smem &S, int lane, uint32_t it, const uint32_t *__restrict__ items,
    const double4_32a *__restrict__ tposp, const double4_32a *__restrict__ tvelr,
    const float4 *__restrict__ tposf, const uint32_t *__restrict__ tcell,
    const int32_t *__restrict__ tstart, const double4_32a *__restrict__ fposp,
    const double4_32a *__restrict__ fvelr, const float4 *__restrict__ fposf,
    const int32_t *__restrict__ fstart, const double4_32a *__restrict__ bposp,
    const double4_32a *__restrict__ bvelr, const float4 *__restrict__ bposf,
    const int32_t *__restrict__ bstart, const uint32_t *__restrict__ fcell,
    double4_32a *__restrict__ acc, double *__restrict__ bar, double *part, double &f2max,
    double &vismax, bool &bad)
{
    const witems::Item I = witems::item_of(P, items, it, tcell, lane);
    const int i = I.i;
    const witems::Frame Fr = witems::frame_of(P, I, tposf[i], tcell, 4.0004f);
    const double s2 = 4.0 * P.h * P.h;
    // the target this lane works for in the balanced walk, its sums, and the
    // lane's own target's total
    int wi = i;
    double4_32a pa, va;
    double ca = 0.0;
    Acc64 w = {0.0, 0.0, 0.0, 0.0, 0.0}, o = {0.0, 0.0, 0.0, 0.0, 0.0};
    witems::for_each_hit_balanced<MOMENTUM>(
        P, S, lane, I, Fr, fstart, fposf, bstart, bposf, fcell,
        [&](int t) {
            wi = I.i0 + t;
            pa = tposp[wi];
            va = tvelr[wi];
            ca = MOMENTUM ? sound64(P, va.w) : 0.0;
            w = {0.0, 0.0, 0.0, 0.0, 0.0};
        },
        [&](int j, bool blist) {
            if (MOMENTUM && !blist && j == wi) return;   // the target itself
            const double4_32a pb = blist ? bposp[j] : fposp[j];
            const double rx = pa.x - pb.x, ry = pa.y - pb.y, rz = pa.z - pb.z;
            const double r2 = rx * rx + ry * ry + rz * rz;
            if (r2 < s2)
                pair64<MOMENTUM>(P, pa, va, ca, pb, blist ? bvelr[j] : fvelr[j], rx, ry, rz, r2,
                                 w);
        },
        [&](int, int slot) {
            double *ps = part + 5 * slot;
            ps[0] = w.ax; ps[1] = w.ay; ps[2] = w.az; ps[3] = w.ar; ps[4] = w.vis;
        },
        [&](int slot) {
            const double *ps = part + 5 * slot;
            o.ax += ps[0]; o.ay += ps[1]; o.az += ps[2]; o.ar += ps[3];
            o.vis = fmax(o.vis, ps[4]);
        });
    if (I.active) {
        if (MOMENTUM) {
            const double ax = P.mass * o.ax + P.g[0];
            const double ay = P.mass * o.ay + P.g[1];
            const double az = P.mass * o.az + P.g[2];
            acc[i] = make_double4_32a(ax, ay, az, P.mass * o.ar);
            const double f2 =
                __dadd_rn(__dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay)), __dmul_rn(az, az));
            f2max = fmax(f2max, f2);
            bad |= !(f2 < INFINITY) || !(o.ar == o.ar);
        } else {
            bar[i] = P.mass * o.ar;
            bad |= !(o.ar == o.ar);
        }
        vismax = fmax(vismax, o.vis);
    }
}

// One queue: the nfi fluid items, then the boundary items (as k_pi32).  The
// particles outside the grid have no item; their outputs are zeroed here.
// Registers are held to 3 resident CTAs per SM (without the bound the compiler
// takes 128 and spills).
__global__ void __launch_bounds__(W64_WARPS * 32, 3)
k_pi64w(DevParams P, int nf, int nb, const uint32_t *__restrict__ items_f,
        const uint32_t *__restrict__ items_b,
        const uint32_t *__restrict__ ctr, int use_b, uint32_t *__restrict__ next_p,
        const double4_32a *__restrict__ posp, const double4_32a *__restrict__ velr,
        const float4 *__restrict__ posf, const uint32_t *__restrict__ cell,
        const int32_t *__restrict__ fstart, const double4_32a *__restrict__ bposp,
        const double4_32a *__restrict__ bvelr, const float4 *__restrict__ bposf,
        const uint32_t *__restrict__ bcell, const int32_t *__restrict__ bstart,
        double4_32a *__restrict__ acc, double *__restrict__ bar, Scalars *sc)
{
    __shared__ witems::Smem smem[W64_WARPS];
    __shared__ double partsm[W64_WARPS][5 * witems::NSLOT];   // balanced-walk partial sums
    __shared__ double red[32];
    const int lane = threadIdx.x & 31;
    witems::Smem &S = smem[threadIdx.x >> 5];
    double *part = partsm[threadIdx.x >> 5];
    const uint32_t nfi = ctr[0];
    const uint32_t n_items = nfi + (use_b ? ctr[3] : 0u);
    double f2max = 0.0, vismax = 0.0;
    bool bad = false;
    for (;;) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(next_p, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;
        if (it < nfi)
            pi64_item<true>(P, S, lane, it, items_f, posp, velr, posf, cell, fstart, posp, velr,
                            posf, fstart, bposp, bvelr, bposf, bstart, cell, acc, bar, part,
                            f2max, vismax, bad);
        else
            pi64_item<false>(P, S, lane, it - nfi, items_b, bposp, bvelr, bposf, bcell, bstart,
                             posp, velr, posf, fstart, nullptr, nullptr, nullptr, bstart, cell,
                             acc, bar, part, f2max, vismax, bad);
    }
    const int g = blockIdx.x * blockDim.x + threadIdx.x, G = gridDim.x * blockDim.x;
    for (int k = fstart[P.ncells] + g; k < nf; k += G) acc[k] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    if (use_b)
        for (int k = bstart[P.ncells] + g; k < nb; k += G) bar[k] = 0.0;
    if (bad) atomicOr(&sc->flags, SPH_FLAG_NAN);
    block_max_to(&sc->mx.f2, f2max, red);
    block_max_to(&sc->mx.visc, vismax, red);
}

}  // namespace

// ------------------------------------------------------------ entry points --

int pi_launch(sph_ctx *ctx)
{
    Workspace &w = ctx->w;
    cudaStream_t st = ctx->stream;
    int nf = (int)ctx->nf, nb = (int)ctx->nb;
    const int T = 128;
    if (ctx->precision == SPH_FP32_SPLIT) {
        if (ctx->prm.pi_kernel == SPH_PI_WARP) return pi32_launch(ctx);
        if (ctx->prm.pi_kernel == SPH_PI_WARP_SYM) return pi32_sym_launch(ctx);
        return pi32_thread_launch(ctx);
    } else if (ctx->dp.reach == 1 && ctx->prm.pi_kernel == SPH_PI_WARP) {
        if (nf + nb == 0) return SPH_OK;
        if (check_cuda(cudaMemsetAsync(&w.ctr[1], 0, sizeof(uint32_t), st))) return SPH_ERR_CUDA;
        SPH_LAUNCH(ctx, k_pi64w, ctx->pi_grid_f, W64_WARPS * 32, 0, st, ctx->dp, nf, nb,
                   w.items_f, w.items_b, w.ctr, nb > 0 ? 1 : 0, &w.ctr[1],
                   (const double4_32a *)w.posp, (const double4_32a *)velr_of(ctx), w.posf, w.cell,
                   w.fstart, (const double4_32a *)w.bposp, (const double4_32a *)w.bvelr, w.bposf,
                   w.bcell, w.bstart, (double4_32a *)w.acc, (double *)w.bar, w.sc);
    } else {
        if (nf > 0)
            SPH_LAUNCH(ctx, k_pi_fluid64, (nf + T - 1) / T, T, 0, st, nf, ctx->dp,
                       (const double4_32a *)w.posp, (const double4_32a *)velr_of(ctx), w.cell, w.fstart,
                       (const double4_32a *)w.bposp, (const double4_32a *)w.bvelr, w.bstart,
                       w.posf, w.bposf, (double4_32a *)w.acc, w.sc);
        if (nb > 0)
            SPH_LAUNCH(ctx, k_pi_boundary64, (nb + T - 1) / T, T, 0, st, nb, ctx->dp,
                       (const double4_32a *)w.bposp, (const double4_32a *)w.bvelr, w.bcell, w.bstart,
                       (const double4_32a *)w.posp, (const double4_32a *)velr_of(ctx), w.fstart, w.bposf,
                       w.posf, (double *)w.bar, w.sc);
    }
    return check_cuda(cudaGetLastError());
}

// Persistent grid of the FP64 warp kernel: one resident set of CTAs.
int pi64_setup(sph_ctx *ctx)
{
    int dev = 0, sms = 0, nblk = 0;
    if (check_cuda(cudaGetDevice(&dev))) return SPH_ERR_CUDA;
    if (check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
        return SPH_ERR_CUDA;
    if (check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nblk, k_pi64w, W64_WARPS * 32,
                                                                0)))
        return SPH_ERR_CUDA;
    ctx->pi_grid_f = sms * (nblk > 0 ? nblk : 1);
    return SPH_OK;
}

int count_work_launch(sph_ctx *ctx)
{
    Workspace &w = ctx->w;
    cudaStream_t st = ctx->stream;
    int nf = (int)ctx->nf, nb = (int)ctx->nb;
    int cur = ctx->cur;
    if (check_cuda(cudaMemsetAsync(w.counts4, 0, 4 * sizeof(unsigned long long), st)))
        return SPH_ERR_CUDA;
    int tot = nf + nb;
    if (tot == 0) return SPH_OK;
    const int T = 128;
    SPH_LAUNCH(ctx, k_count_work, (tot + T - 1) / T, T, 0, st, nf, nb, ctx->dp, w.x[cur], w.y[cur],
               w.z[cur], w.cell, w.fstart, w.bx, w.by, w.bz, w.bcell, w.bstart, w.counts4);
    return check_cuda(cudaGetLastError());
}

}  // namespace sph
