// PI stage, SPH_FP32_SPLIT form, symmetric variant (pi_kernel =
// SPH_PI_WARP_SYM): every interacting pair between different cells is
// evaluated once and its terms are added to both particles.
//
// The pair terms are antisymmetric in the momentum and symmetric in the
// continuity equation: with f = (P_a/rho_a^2 + P_b/rho_b^2 + Pi_ab) F, the
// momentum sums get -m f r_ab at a and +m f r_ab at b, both continuity sums get
// m F v_ab.r_ab, and the viscous dt term |mu_ab| is the same from both sides
// (Section 3.1, optimisation A, applies this on the CPU).  The paper keeps the
// GPU kernel one-sided because threads cannot scatter to b without conflicts
// (Section 4); here the conflicts are resolved by ordered updates in shared
// memory and atomic additions in global memory.
//
// Work items are those of the warp kernel (pi32.cu: up to 32 targets of one
// cell, one warp each).  The candidates of an item are
//   fluid:     the 13 cells after the target cell in (z, y, x) order -- the
//              three rows (dy, +1), the row (+1, 0) and the cell x+1 of the own
//              row -- evaluated for both particles; and the target cell itself,
//              evaluated for the target only (each of its particles is a target
//              of an item of this cell, so each ordered pair there is visited
//              once as now);
//   boundary:  all 9 rows, evaluated for both particles (the B-F continuity
//              term of a boundary particle is the b side of an F-B pair), so no
//              separate boundary-target kernel runs.
// The work-item search is that of the warp kernel (warp_items.cuh: run table
// with the half-shell runs, candidates within 2h of the targets' bounding box
// staged in passes of 8-candidate blocks, lockstep distance tests), and the
// per-lane hit walk and pair terms are those of the warp kernel, in units of h
// with the constants folded out of the loop.
// The b-side terms of a staged set are summed per candidate in shared memory
// (lanes that reach the same candidate in the same iteration take turns, the
// turn decided by the last lane id written to the slot's tag; shared-memory
// float atomics cost more than the pairs they save), then every candidate with
// a non-zero sum adds it to the particle's global sums with one vector atomic;
// the a-side
// sums of the targets are added the same way at the end of the item.  The
// global sums start at (g, 0) (k_sym_init) and the largest |a|^2 is taken after
// the kernel (k_sym_max).
//
// The order of the global atomic additions depends on scheduling: results agree with
// the one-sided kernels to float32 rounding but are not reproducible bit for
// bit from run to run.  Cells of edge >= 2h only; no tensile correction.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "pair32.cuh"
#include "sph_internal.cuh"
#include "warp_items.cuh"

namespace sph {

namespace {

constexpr int CAP = 160;          // staged candidates per warp and set
constexpr int NCH = CAP / 32;
constexpr int WARPS = 4;
constexpr int RAW_PER_PASS = 2 * CAP;  // candidates sampled per pass (before the box test)
static_assert(CAP % 32 == 0, "CAP must be a multiple of 32");

// Staged candidate index flags: boundary list, evaluated for both particles.
constexpr uint32_t J_BOUNDARY = 0x80000000u;
constexpr uint32_t J_BOTH = 0x40000000u;
constexpr uint32_t J_INDEX = 0x3fffffffu;

struct WarpSmem {
    float4 A[CAP];        // shifted candidate offset {x, y, z} / h and |x|^2
    float4 V[CAP];        // candidate {vx, vy, vz, rho}
    float4 B[CAP];        // b-side sums of the set: (-f r'), (v.r') F''
    float Pr[CAP];        // candidate P / rho^2
    uint32_t J[CAP];      // candidate index and its J_ flags
    int tag[CAP];         // lane allowed to add to the slot in the current round
    uint32_t M[NCH][32];  // hit bits of lane l for chunk q
    uint32_t symF[NCH];   // fluid candidates evaluated for both particles
    uint32_t isB[NCH];    // boundary candidates (always both particles)
    witems::RunTable T;   // the half-shell x-runs
};

__device__ __forceinline__ void red_add_v4(float4 *p, float a, float b, float c, float d)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b),
                 "f"(c), "f"(d)
                 : "memory");
}

// Pair terms in units of h (the same arithmetic as the warp kernel): returns
// f'' = (P_a/rho_a^2 + P_b/rho_b^2 + Pi) F'' and (v_ab . r') F''; the momentum
// term of a is -m kB f'' r', that of b +m kB f'' r'; both continuity terms are
// m kB (v.r') F''.
__device__ __forceinline__ void pair_sym(const DevParams &P, float rx, float ry, float rz,
                                         float pra, const float4 &va, float rho2a, const float4 &vb,
                                         float prb, float &coef, float &cF, float &vis)
{
    float vdr, F;
    pair_terms32<true, false>(P, rx, ry, rz, pra, va, rho2a, vb, prb, coef, vdr, F, vis);
    cF = vdr * F;
}

__global__ void __launch_bounds__(WARPS * 32)
k_pi32_sym(DevParams P, const uint32_t *__restrict__ items, const uint32_t *__restrict__ n_items_p,
           uint32_t *__restrict__ next_p, const float4 *__restrict__ fposp,
           const float4 *__restrict__ fvelr, const uint32_t *__restrict__ fcell,
           const int32_t *__restrict__ fstart, const float4 *__restrict__ bposp,
           const float4 *__restrict__ bvelr, const int32_t *__restrict__ bstart,
           float4 *__restrict__ acc, float *__restrict__ bar, Scalars *sc)
{
    __shared__ WarpSmem smem[WARPS];
    __shared__ double red[32];
    const int lane = threadIdx.x & 31;
    WarpSmem &S = smem[threadIdx.x >> 5];
    const uint32_t n_items = *n_items_p;
    float vismax = 0.0f;

    for (;;) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(next_p, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;

        // ---- the item: the targets of one cell (fluid items hold one cell)
        const witems::Item I = witems::item_of(P, items, it, fcell, lane);
        const int i = I.i;
        const float4 pa = fposp[i], va = fvelr[i];
        const witems::Frame F = witems::frame_of(P, I, pa, fcell, 4.0f);
        const float rho2a = va.w * va.w;
        const int K = witems::build_runs<true, witems::RUNS_HALF>(P, S.T, lane, I, fstart, bstart);
        const witems::Box Bx = witems::target_box(F);

        struct Cand {
            float4 pos, v;
            uint32_t jj;
        };
        auto load = [&](int j, bool blist, bool own) {
            Cand c;
            c.pos = blist ? bposp[j] : fposp[j];
            c.v = blist ? bvelr[j] : fvelr[j];
            // own row: the target cell is one-sided, cell x+1 symmetric
            c.jj = (uint32_t)j | (blist ? J_BOUNDARY : (own ? 0u : J_BOTH));
            return c;
        };
        auto store = [&](int slot, const float4 &a, const Cand &c) {
            S.A[slot] = a;
            S.V[slot] = c.v;
            S.Pr[slot] = c.pos.w;
            S.J[slot] = c.jj;
            S.B[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
        };

        float ax = 0.f, ay = 0.f, az = 0.f, ar = 0.f;
        const int npass = (K + RAW_PER_PASS - 1) / RAW_PER_PASS;
        for (int pass = 0; pass < npass; ++pass) {
            const int np = witems::pass_slots(K, npass, pass);
            int k0 = 0, r = 0;
            while (k0 < np) {
                const int n = witems::stage_set<true, witems::RUNS_HALF>(
                    P, S.T, Bx, lane, CAP, pass, npass, np, K, k0, r, fcell, load, store);
                // far candidates fill the last chunk
                const int nch = (n + 31) >> 5;
                if (n + lane < nch * 32) {
                    S.A[n + lane] = make_float4(0.f, 0.f, 0.f, INFINITY);
                    S.V[n + lane] = make_float4(0.f, 0.f, 0.f, 1.f);
                    S.Pr[n + lane] = 0.f;
                    S.J[n + lane] = 0u;
                    S.B[n + lane] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                __syncwarp();
                for (int q = 0; q < nch; ++q) {
                    const uint32_t jj = S.J[q * 32 + lane];
                    const uint32_t bf = __ballot_sync(0xffffffffu, (jj & J_BOTH) != 0u);
                    const uint32_t bb = __ballot_sync(0xffffffffu, (jj & J_BOUNDARY) != 0u);
                    if (lane == 0) {
                        S.symF[q] = bf;
                        S.isB[q] = bb;
                    }
                }
                __syncwarp();
                // ---- lockstep distance tests, one hit bit per candidate
                witems::lockstep_tests<false>(S.A, S.M, n, lane, F);
                __syncwarp();
                // ---- every lane walks its own hits; b-side terms to the candidate's
                // slot.  All lanes iterate together (until no lane has a hit left)
                // so that the warp-wide turns below are well defined.
                int q = 0;
                uint32_t m = nch > 0 ? S.M[0][lane] : 0u, sf = nch > 0 ? S.symF[0] : 0u,
                         sb = nch > 0 ? S.isB[0] : 0u;
                for (;;) {
                    while (m == 0u && q + 1 < nch) {
                        ++q;
                        m = S.M[q][lane];
                        sf = S.symF[q];
                        sb = S.isB[q];
                    }
                    const bool has = m != 0u;
                    if (!__any_sync(0xffffffffu, has)) break;
                    int ls = 0;
                    bool two = false;
                    float4 add = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (has) {
                        const int bit = __ffs(m) - 1;
                        m &= m - 1u;
                        ls = q * 32 + bit;
                        const float4 b = S.A[ls];
                        const float rx = F.x - b.x, ry = F.y - b.y, rz = F.z - b.z;
                        float coef, cF;
                        pair_sym(P, rx, ry, rz, pa.w, va, rho2a, S.V[ls], S.Pr[ls], coef, cF,
                                 vismax);
                        ax = fmaf(coef, rx, ax);
                        ay = fmaf(coef, ry, ay);
                        az = fmaf(coef, rz, az);
                        ar += cF;
                        if ((sf >> bit) & 1u) {
                            two = true;
                            add = make_float4(-coef * rx, -coef * ry, -coef * rz, cF);
                        } else if ((sb >> bit) & 1u) {
                            two = true;
                            add.w = cF;
                        }
                    }
                    // lanes that reached the same candidate take turns: each lane
                    // with something to add writes its id to the slot's tag, and
                    // the lane whose id is read back adds; the others try again
                    bool todo = two;
                    while (__any_sync(0xffffffffu, todo)) {
                        if (todo) S.tag[ls] = lane;
                        __syncwarp();
                        const bool mine = todo && S.tag[ls] == lane;
                        if (mine) {
                            float4 t = S.B[ls];
                            t.x += add.x;
                            t.y += add.y;
                            t.z += add.z;
                            t.w += add.w;
                            S.B[ls] = t;
                            todo = false;
                        }
                        __syncwarp();
                    }
                }
                __syncwarp();
                // ---- b-side sums of the set to the particles
                for (int mm = 0; mm < nch; ++mm) {
                    const int ls = lane + 32 * mm;
                    const float4 bs = S.B[ls];
                    const uint32_t jj = S.J[ls];
                    const uint32_t j = jj & J_INDEX;
                    if (jj & J_BOTH) {
                        if (bs.x != 0.f || bs.y != 0.f || bs.z != 0.f || bs.w != 0.f)
                            red_add_v4(acc + j, P.nmkBf * bs.x, P.nmkBf * bs.y, P.nmkBf * bs.z,
                                       P.mkBf * bs.w);
                    } else if (jj & J_BOUNDARY) {
                        if (bs.w != 0.f) atomicAdd(bar + j, P.mkBf * bs.w);
                    }
                }
                __syncwarp();
            }
        }
        if (I.active) red_add_v4(acc + i, P.nmkBf * ax, P.nmkBf * ay, P.nmkBf * az, P.mkBf * ar);
    }
    block_max_to(&sc->mx.visc, (double)vismax, red);
}

// Global sums before the symmetric kernel: (g, 0) for fluid, 0 for boundary.
__global__ void k_sym_init(int nf, int nb, DevParams P, float4 *__restrict__ acc,
                           float *__restrict__ bar)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nf) acc[i] = make_float4(P.gf[0], P.gf[1], P.gf[2], 0.f);
    else if (i < nf + nb) bar[i - nf] = 0.f;
}

// After the symmetric kernel: the largest |a|^2 over fluid particles in the
// grid and the NaN flag.
__global__ void k_sym_max(int nf, int nb, DevParams P, const int32_t *__restrict__ fstart,
                          const int32_t *__restrict__ bstart, const float4 *__restrict__ acc,
                          const float *__restrict__ bar, Scalars *sc)
{
    __shared__ double red[32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double f2 = 0.0;
    bool bad = false;
    if (i < nf) {
        if (i < fstart[P.ncells]) {
            const float4 a = acc[i];
            f2 = (double)a.x * a.x + (double)a.y * a.y + (double)a.z * a.z;
            bad = !(f2 < INFINITY) || !(a.w == a.w);
        }
    } else if (i < nf + nb) {
        if (i - nf < bstart[P.ncells]) {
            const float b = bar[i - nf];
            bad = !(b == b);
        }
    }
    if (bad) atomicOr(&sc->flags, SPH_FLAG_NAN);
    block_max_to(&sc->mx.f2, f2, red);
}

}  // namespace

int pi32_sym_setup(sph_ctx *ctx)
{
    int dev = 0, sms = 0, b = 0;
    if (check_cuda(cudaGetDevice(&dev))) return SPH_ERR_CUDA;
    if (check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
        return SPH_ERR_CUDA;
    if (check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pi32_sym, WARPS * 32, 0)))
        return SPH_ERR_CUDA;
    ctx->pi_grid_f = sms * (b > 0 ? b : 1);
    return SPH_OK;
}

int pi32_sym_launch(sph_ctx *ctx)
{
    Workspace &w = ctx->w;
    cudaStream_t st = ctx->stream;
    const int nf = (int)ctx->nf, nb = (int)ctx->nb, T = 256;
    if (nf + nb == 0) return SPH_OK;
    SPH_LAUNCH(ctx, k_sym_init, (nf + nb + T - 1) / T, T, 0, st, nf, nb, ctx->dp, (float4 *)w.acc,
               (float *)w.bar);
    if (nf > 0) {
        if (check_cuda(cudaMemsetAsync(&w.ctr[1], 0, sizeof(uint32_t), st))) return SPH_ERR_CUDA;
        SPH_LAUNCH(ctx, k_pi32_sym, ctx->pi_grid_f, WARPS * 32, 0, st, ctx->dp, w.items_f,
                   &w.ctr[0], &w.ctr[1], (const float4 *)w.posp, (const float4 *)velr_of(ctx), w.cell,
                   w.fstart, (const float4 *)w.bposp, (const float4 *)w.bvelr, w.bstart,
                   (float4 *)w.acc, (float *)w.bar, w.sc);
    }
    SPH_LAUNCH(ctx, k_sym_max, (nf + nb + T - 1) / T, T, 0, st, nf, nb, ctx->dp, w.fstart, w.bstart,
               (const float4 *)w.acc, (const float *)w.bar, w.sc);
    return check_cuda(cudaGetLastError());
}

}  // namespace sph
