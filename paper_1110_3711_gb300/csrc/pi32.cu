// PI stage, SPH_FP32_SPLIT form: warp-cooperative particle interaction.
//
// The paper's GPU kernel (Section 4, Fig. 11) gives every target particle its
// own thread and its own walk over the 27 cells; the pair body then runs under
// a divergent branch (a warp idles whenever any lane has a false neighbour,
// Section 4 "code divergence").  Here one warp owns a work item: up to 32
// target particles of one cell, or for boundary targets of consecutive cells
// of one x row (cells follow X, Y, Z after NL, so they are a contiguous
// range).  For that item the warp
//   1. builds the table of its 9 fluid x-runs (and 9 boundary x-runs for
//      fluid targets): cells x-1..x+1 of every (y, z) row are one index range
//      (Section 4.4, Fig. 10);
//   2. stages the candidates of those runs that lie within 2h of the bounding
//      box of its targets (the others cannot be neighbours of any of them) in
//      shared memory, already shifted into the frame of the target cell and
//      measured in units of h ((candidate offset + cell delta * s) / h), with
//      |x_b|^2 beside them;
//   3. tests all candidates against all 32 targets in lockstep: the warp reads
//      one candidate (a shared-memory broadcast) and each lane evaluates
//      |x_b|^2 - 2 x_a.x_b - (4 - |x_a|^2) (three FMAs and a subtraction; it
//      is negative exactly when |x_a - x_b| < 2h up to float32 rounding)
//      and shifts its sign bit into a hit mask;
//   4. walks its own hit bits (about 112 real neighbours per lane, so lanes
//      stay balanced) and evaluates the pair terms of the oracle (cubic-spline
//      gradient, Tait pressure, artificial viscosity, continuity) from the
//      staged data, recomputing r_ab exactly from the shifted offsets.
// An item of at most 16 targets (a thinly filled cell, the free surface)
// would leave half the lanes idle through the walk: there each target has two
// lanes, l and l + 16, and at most 8 targets four lanes, l + 8 j; the lanes of
// a target take the candidates k = j mod 2 (or mod 4) of every chunk, and
// their sums are joined in a fixed order by shuffles at the end.
// Work items are taken from a list built by NL with an atomic counter, so the
// grid is persistent (one resident set of CTAs) and balances itself.  Fluid
// items hold the particles of one cell (about 27 at rest; a fuller cell gives
// items of 32).  Boundary targets (B-F) come in packed items: consecutive
// cells of one x row with at most 32 particles together (a boundary cell holds
// about 10), the candidates being the fluid of the union of their
// neighbourhoods (x-runs from the first cell - 1 to the last + 1); each
// candidate is shifted by its own cell's x distance from the first cell, each
// target by its cell's.  Fluid and boundary items form one queue (fluid first)
// served by one launch.  Sums of a target are accumulated in candidate order
// by one lane (or by each of its lanes, then joined), so results do not depend
// on the order the items are processed in.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "pair32.cuh"
#include "sph_internal.cuh"
#include "warp_items.cuh"

// Staged candidates per warp and set.  224 (36.8 KB of shared memory per CTA
// of 4 warps) admits 6 CTAs, 24 warps, per SM; 256 admitted 5 (PI 2.7 %
// slower at 1M on GB300), and 160 with 7 or 8 CTAs (72 or 64 registers) was
// 7 % slower: fuller sets count for more than more resident warps.
#ifndef SPH_PI_CAP
#define SPH_PI_CAP 224
#endif
#ifndef SPH_PI_WARPS
#define SPH_PI_WARPS 4
#endif
// Resident CTAs per SM the register allocation is held to: 6 CTAs of 128
// threads need at most 85 registers per thread (the compiler takes 80).
#ifndef SPH_PI_MINB
#define SPH_PI_MINB 6
#endif

namespace sph {

namespace {

constexpr int CAP = SPH_PI_CAP;   // staged candidates per warp and pass
constexpr int NCH = CAP / 32;     // 32-candidate chunks per pass
constexpr int WARPS = SPH_PI_WARPS;
constexpr int RAW_PER_PASS = 2 * CAP;  // candidates sampled per pass (before the box test)
static_assert(CAP % 32 == 0, "CAP must be a multiple of 32");

struct WarpSmem {
    float4 A[CAP];        // shifted candidate offset {x, y, z} and |x|^2, then P / rho^2
    float4 V[CAP];        // candidate {vx, vy, vz, rho}
    float Pr[CAP];        // candidate P / rho^2
    uint32_t M[NCH][32];  // hit bits of lane l for chunk q
    witems::RunTable T;   // x-runs
};

// One work item, processed by the whole warp.  MOMENTUM: fluid targets (F-F
// and F-B, acc out).  !MOMENTUM: boundary targets (B-F continuity only, bar
// out).  t* are the target arrays, f* the fluid candidates, b* the boundary
// candidates (fluid targets only).
template <bool MOMENTUM, bool TENSILE>
__device__ __forceinline__ void pi32_item(
    const DevParams &P, WarpSmem &S, int lane, uint32_t it, const uint32_t *__restrict__ items,
    const float4 *__restrict__ tposp, const float4 *__restrict__ tvelr,
    const uint32_t *__restrict__ tcell, const int32_t *__restrict__ tstart,
    const float4 *__restrict__ fposp, const float4 *__restrict__ fvelr,
    const int32_t *__restrict__ fstart, const float4 *__restrict__ bposp,
    const float4 *__restrict__ bvelr, const int32_t *__restrict__ bstart,
    float4 *__restrict__ acc, float *__restrict__ bar, const uint32_t *__restrict__ fcell,
    double &f2max, float &vismax, bool &bad)
{
    // ---- the item: targets [i0, i0 + nt) of cells c .. c + (cx1 - cx) of one x row
    witems::Item I = witems::item_of(P, items, it, tcell, lane);
    // g lanes per target: 2 for at most 16 targets, 4 for at most 8; target
    // t has lanes t + (32 / g) j, j < g, and lane j of a target keeps the hits
    // at chunk bits b = j mod g
    const int g = I.nt <= 8 ? 4 : (I.nt <= 16 ? 2 : 1);
    if (g > 1) {
        const int tl = lane & (32 / g - 1);
        I.active = tl < I.nt;
        I.i = I.i0 + (I.active ? tl : 0);
    }
    const uint32_t keep = g == 1 ? 0xffffffffu
                        : (g == 2 ? 0x55555555u << (lane >> 4) : 0x11111111u << (lane >> 3));
    const int i = I.i;
    const float4 pa = tposp[i], va = tvelr[i];
    // the target in the item's frame, units of h; the lockstep test decides
    // the pairs (threshold 4 h^2)
    const witems::Frame F = witems::frame_of(P, I, pa, tcell, 4.0f);
    const float rho2a = va.w * va.w;

    const int K = witems::build_runs<MOMENTUM>(P, S.T, lane, I, fstart, bstart);
    const witems::Box B = witems::target_box(F);

    // staged data of a kept candidate: offset (A, from the position record),
    // {v, rho} (V) and P/rho^2 (Pr); both loads are issued together (the
    // velocity is wasted on a candidate the box test drops, but waits on nothing)
    struct Cand {
        float4 pos, v;
    };
    auto load = [&](int j, bool blist, bool) {
        Cand c;
        c.pos = blist ? bposp[j] : fposp[j];
        c.v = blist ? bvelr[j] : fvelr[j];
        return c;
    };
    auto store = [&](int slot, const float4 &a, const Cand &c) {
        S.A[slot] = a;
        S.V[slot] = c.v;
        S.Pr[slot] = c.pos.w;
    };

    Acc32 o = {0.f, 0.f, 0.f, 0.f, 0.f};
    // Pass p takes the blocks p, p + npass, p + 2 npass, ... of candidates:
    // every pass samples the whole neighbourhood, so every lane finds about
    // 1/npass of its neighbours in each pass and the hit walks stay balanced.
    // Only candidates within 2h of the targets' bounding box are staged; the
    // staged set is tested and walked whenever it may not take another 32.
    const int npass = (K + RAW_PER_PASS - 1) / RAW_PER_PASS;
    for (int pass = 0; pass < npass; ++pass) {
        const int np = witems::pass_slots(K, npass, pass);
        int k0 = 0, r = 0;
        while (k0 < np) {
            const int n = witems::stage_set<MOMENTUM>(P, S.T, B, lane, CAP, pass, npass, np, K,
                                                      k0, r, fcell, load, store);
            // far candidates fill the last chunk
            const int nch = (n + 31) >> 5;
            if (n + lane < nch * 32) {
                S.A[n + lane] = make_float4(0.f, 0.f, 0.f, INFINITY);
                S.V[n + lane] = make_float4(0.f, 0.f, 0.f, 1.f);
                S.Pr[n + lane] = 0.f;
            }
            __syncwarp();
            // ---- lockstep distance tests, one hit bit per candidate
            uint32_t cm = witems::lockstep_tests<true>(S.A, S.M, n, lane, F, keep);
            // |x|^2 has served the tests: the pair walk reads P/rho^2 from its place
            __syncwarp();
            for (int q2 = 0; q2 < nch; ++q2) S.A[q2 * 32 + lane].w = S.Pr[q2 * 32 + lane];
            __syncwarp();
            // ---- every lane walks its own hits (about 112 per lane in all), in
            // staging order: candidate k of chunk q is bit 31 - k of its mask.
            // cm has bit q set when chunk q holds a hit of this lane, so a lane
            // that has finished a chunk moves to its next one in one step (no
            // loop over empty chunks while the rest of the warp waits)
            int qb = 0;
            uint32_t m = 0u;
            for (;;) {
                if (m == 0u) {
                    if (cm == 0u) break;
                    const int q = __ffs(cm) - 1;
                    cm &= cm - 1u;
                    m = S.M[q][lane];
                    qb = q * 32;
                }
                const int k = __clz(m);
                m &= 0x7fffffffu >> k;
                const int ls = qb + k;
                const float4 b = S.A[ls];
                pair_acc32<MOMENTUM, TENSILE>(P, F.x - b.x, F.y - b.y, F.z - b.z, pa.w, va, rho2a,
                                              S.V[ls], b.w, o);
            }
            __syncwarp();
        }
    }

    if (g > 1) {
        // lane t collects the sums of lanes t + 16 (and t + 8, t + 24): a fixed
        // tree over the lanes of target t
        for (int d = 16; d >= 32 / g; d >>= 1) {
            o.ax += __shfl_down_sync(0xffffffffu, o.ax, d);
            o.ay += __shfl_down_sync(0xffffffffu, o.ay, d);
            o.az += __shfl_down_sync(0xffffffffu, o.az, d);
            o.ar += __shfl_down_sync(0xffffffffu, o.ar, d);
            o.vis = fmaxf(o.vis, __shfl_down_sync(0xffffffffu, o.vis, d));
        }
    }
    if (I.active && lane < 32 / g) {
        if (MOMENTUM) {
            const float ax = fmaf(P.nmkBf, o.ax, P.gf[0]);
            const float ay = fmaf(P.nmkBf, o.ay, P.gf[1]);
            const float az = fmaf(P.nmkBf, o.az, P.gf[2]);
            const float ar = P.mkBf * o.ar;
            acc[i] = make_float4(ax, ay, az, ar);
            const double f2 = (double)ax * ax + (double)ay * ay + (double)az * az;
            f2max = fmax(f2max, f2);
            bad |= !(f2 < INFINITY) || !(ar == ar);
        } else {
            const float ar = P.mkBf * o.ar;
            bar[i] = ar;
            bad |= !(ar == ar);
        }
        vismax = fmaxf(vismax, o.vis);
    }
}

// PI over one queue of work items: the nf_items fluid items first (F-F + F-B),
// then the nb_items packed boundary items (B-F), taken by the warps of a
// persistent grid from one atomic counter, so that boundary items fill the
// tail of the fluid work instead of following it in a second launch.
template <bool TENSILE>
__global__ void __launch_bounds__(WARPS * 32, SPH_PI_MINB)
k_pi32(DevParams P, const uint32_t *__restrict__ items_f, const uint32_t *__restrict__ items_b,
       const uint32_t *__restrict__ ctr, int use_b, uint32_t *__restrict__ next_p,
       const float4 *__restrict__ posp, const float4 *__restrict__ velr,
       const uint32_t *__restrict__ cell, const int32_t *__restrict__ fstart,
       const float4 *__restrict__ bposp, const float4 *__restrict__ bvelr,
       const uint32_t *__restrict__ bcell, const int32_t *__restrict__ bstart,
       float4 *__restrict__ acc, float *__restrict__ bar, Scalars *sc)
{
    __shared__ WarpSmem smem[WARPS];
    __shared__ double red[32];
    const int lane = threadIdx.x & 31;
    WarpSmem &S = smem[threadIdx.x >> 5];
    const uint32_t nfi = ctr[0];
    const uint32_t n_items = nfi + (use_b ? ctr[3] : 0u);
    double f2max = 0.0;
    float vismax = 0.0f;
    bool bad = false;
    for (;;) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(next_p, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;
        if (it < nfi)
            pi32_item<true, TENSILE>(P, S, lane, it, items_f, posp, velr, cell, fstart, posp,
                                     velr, fstart, bposp, bvelr, bstart, acc, bar, cell, f2max,
                                     vismax, bad);
        else
            pi32_item<false, false>(P, S, lane, it - nfi, items_b, bposp, bvelr, bcell, bstart,
                                    posp, velr, fstart, nullptr, nullptr, bstart, acc, bar, cell,
                                    f2max, vismax, bad);
    }
    if (bad) atomicOr(&sc->flags, SPH_FLAG_NAN);
    block_max_to(&sc->mx.f2, f2max, red);
    block_max_to(&sc->mx.visc, (double)vismax, red);
}

// Work items of the boundary list (built once per list), one thread: runs of
// consecutive cells of one x row are packed into an item while their particles
// number 32 at most; a cell of more than 32 particles gives items of 32.  Each
// item is {first particle, number of particles}; *count is the number of items.
__global__ void k_pack_boundary_items(DevParams P, const uint32_t *__restrict__ bcell,
                                      const int32_t *__restrict__ bstart,
                                      uint32_t *__restrict__ items, uint32_t *__restrict__ count)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const int n = bstart[P.ncells];  // particles inside the grid
    uint32_t k = 0;
    int i = 0;
    while (i < n) {
        uint32_t c = bcell[i];
        int m = bstart[c + 1] - i;
        if (m > 32) {
            for (int o = 0; o < m; o += 32) {
                items[2 * k] = (uint32_t)(i + o);
                items[2 * k + 1] = (uint32_t)min(32, m - o);
                ++k;
            }
            i += m;
            continue;
        }
        const int first = i;
        int nt = m;
        i += m;
        while (i < n) {
            const uint32_t c2 = bcell[i];
            const int m2 = bstart[c2 + 1] - i;
            if (c2 != c + 1 || (c2 % (uint32_t)P.nx) == 0u || nt + m2 > 32) break;
            nt += m2;
            c = c2;
            i += m2;
        }
        items[2 * k] = (uint32_t)first;
        items[2 * k + 1] = (uint32_t)nt;
        ++k;
    }
    *count = k;
}

}  // namespace

int pi32_setup(sph_ctx *ctx)
{
    int dev = 0, sms = 0, nblk = 0;
    if (check_cuda(cudaGetDevice(&dev))) return SPH_ERR_CUDA;
    if (check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
        return SPH_ERR_CUDA;
    if (ctx->dp.tensile) {
        if (check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nblk, k_pi32<true>,
                                                                    WARPS * 32, 0)))
            return SPH_ERR_CUDA;
    } else if (check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nblk, k_pi32<false>,
                                                                       WARPS * 32, 0))) {
        return SPH_ERR_CUDA;
    }
    ctx->pi_grid_f = sms * (nblk > 0 ? nblk : 1);
    return SPH_OK;
}

int boundary_items_launch(sph_ctx *ctx)
{
    int nb = (int)ctx->nb;
    if (nb == 0) return SPH_OK;
    Workspace &w = ctx->w;
    const int T = 256;
    (void)T;
    SPH_LAUNCH(ctx, k_pack_boundary_items, 1, 32, 0, ctx->stream, ctx->dp, w.bcell, w.bstart,
               w.items_b, &w.ctr[3]);
    return check_cuda(cudaGetLastError());
}

int pi32_launch(sph_ctx *ctx)
{
    Workspace &w = ctx->w;
    cudaStream_t st = ctx->stream;
    if (ctx->nf == 0 && ctx->nb == 0) return SPH_OK;
    // clear the "next item" counter of the queue
    if (check_cuda(cudaMemsetAsync(&w.ctr[1], 0, sizeof(uint32_t), st))) return SPH_ERR_CUDA;
    const int use_b = ctx->nb > 0 ? 1 : 0;
    if (ctx->dp.tensile)
        SPH_LAUNCH(ctx, k_pi32<true>, ctx->pi_grid_f, WARPS * 32, 0, st, ctx->dp, w.items_f,
                   w.items_b, w.ctr, use_b, &w.ctr[1], (const float4 *)w.posp,
                   (const float4 *)velr_of(ctx), w.cell, w.fstart, (const float4 *)w.bposp,
                   (const float4 *)w.bvelr, w.bcell, w.bstart, (float4 *)w.acc, (float *)w.bar,
                   w.sc);
    else
        SPH_LAUNCH(ctx, k_pi32<false>, ctx->pi_grid_f, WARPS * 32, 0, st, ctx->dp, w.items_f,
                   w.items_b, w.ctr, use_b, &w.ctr[1], (const float4 *)w.posp,
                   (const float4 *)velr_of(ctx), w.cell, w.fstart, (const float4 *)w.bposp,
                   (const float4 *)w.bvelr, w.bcell, w.bstart, (float4 *)w.acc, (float *)w.bar,
                   w.sc);
    return check_cuda(cudaGetLastError());
}

}  // namespace sph
