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
// The lockstep distance test (warp_items.cuh) and the per-lane hit walk are those of
// the warp kernel, in units of h with the constants folded out of the loop.
// The b-side terms of a pass are summed per staged candidate in shared memory
// (lanes that reach the same candidate in the same iteration take turns, the
// turn decided by the last lane id written to the slot's tag; shared-memory
// float atomics cost more than the pairs they save), then every candidate with
// a non-zero
// sum adds it to the particle's global sums with one vector atomic; the a-side
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

constexpr int CAP = 160;          // staged candidates per warp and pass
constexpr int NCH = CAP / 32;
constexpr int WARPS = 4;
constexpr int NRUN = 14;          // 5 fluid + 9 boundary x-runs
static_assert(CAP % 32 == 0, "CAP must be a multiple of 32");

struct WarpSmem {
    float4 A[CAP];        // shifted candidate offset {x, y, z} / h and |x|^2
    float4 V[CAP];        // candidate {vx, vy, vz, rho}
    float4 B[CAP];        // b-side sums of the pass: (-f r'), (v.r') F''
    float Pr[CAP];        // candidate P / rho^2
    int J[CAP];           // candidate index in its list
    int tag[CAP];         // lane allowed to add to the slot in the current round
    uint32_t M[NCH][32];  // hit bits of lane l for chunk q
    uint32_t symF[NCH];   // fluid candidates evaluated for both particles
    uint32_t isB[NCH];    // boundary candidates (always both particles)
    int4 run[NRUN];       // {inclusive end slot, first index, start of cell x, start of cell x+1}
    int code[NRUN];       // list (bit 0), dy+1 (bits 1-2), dz+1 (bits 3-4), own row (bit 5)
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
                                         float pra, const float4 &va, float cpa, const float4 &vb,
                                         float prb, float &coef, float &cF, float &vis)
{
    float vdr, F;
    pair_terms32<true, false>(P, rx, ry, rz, pra, va, cpa, vb, prb, coef, vdr, F, vis);
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

        // ---- the item: targets [i0, i0 + nt) of cell c
        // fluid items hold the particles of one cell
        const int i0 = (int)items[2 * it];
        const uint32_t c = fcell[i0];
        const int nt = (int)items[2 * it + 1];
        const bool active = lane < nt;
        const int i = i0 + (active ? lane : 0);
        const float4 pa = fposp[i], va = fvelr[i];
        const uint32_t cyz = c / (uint32_t)P.nx;
        const int cx = (int)(c - cyz * (uint32_t)P.nx);
        const int cy = (int)(cyz % (uint32_t)P.ny);
        const int cz = (int)(cyz / (uint32_t)P.ny);
        const float xa = pa.x * P.invhf, ya = pa.y * P.invhf, za = pa.z * P.invhf;
        const float thr = active ? 4.0f - fmaf(xa, xa, fmaf(ya, ya, za * za)) : -INFINITY;
        const float ra = va.w * P.inv_rho0f;
        const float cpa = P.nalphaf * (P.c0f * ra * ra * ra);

        // ---- run table: lane r describes run r
        int K;
        {
            const int r = lane;
            int L = 0, j0 = 0, b1 = 0, b2 = 0, code = 0;
            if (r < NRUN) {
                int list, dy, dz, x0, x1;
                if (r < 5) {
                    // fluid: rows (-1, +1), (0, +1), (+1, +1), (+1, 0) whole,
                    // and cells x, x+1 of the own row
                    list = 0;
                    dy = r < 3 ? r - 1 : (r == 3 ? 1 : 0);
                    dz = r < 3 ? 1 : 0;
                    x0 = r == 4 ? cx : max(cx - 1, 0);
                } else {
                    list = 1;
                    dz = (r - 5) / 3 - 1;
                    dy = (r - 5) % 3 - 1;
                    x0 = max(cx - 1, 0);
                }
                x1 = min(cx + 1, P.nx - 1);
                const int y = cy + dy, z = cz + dz;
                code = list | ((dy + 1) << 1) | ((dz + 1) << 3) | (r == 4 ? 32 : 0);
                if (y >= 0 && y < P.ny && z >= 0 && z < P.nz) {
                    const int32_t *st = list ? bstart : fstart;
                    const int row = P.nx * (y + P.ny * z);
                    j0 = st[row + x0];
                    L = st[row + x1 + 1] - j0;
                    b1 = st[row + cx];
                    b2 = st[row + cx + 1];
                }
            }
            int pe = L;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(0xffffffffu, pe, o);
                if (lane >= o) pe += t;
            }
            if (r < NRUN) {
                S.run[r] = make_int4(pe, j0, b1, b2);
                S.code[r] = code;
            }
            K = __shfl_sync(0xffffffffu, pe, NRUN - 1);
        }
        __syncwarp();

        float ax = 0.f, ay = 0.f, az = 0.f, ar = 0.f;
        const int npass = (K + CAP - 1) / CAP;
        for (int pass = 0; pass < npass; ++pass) {
            const int np = (K - pass + npass - 1) / npass;
            const int nch = (np + 31) >> 5;
            // ---- stage the candidates of this pass (pass p takes p, p + npass, ...)
            int r = 0;
            for (int m = 0; m < nch; ++m) {
                const int ls = lane + 32 * m;
                const int s = ls < np ? pass + npass * ls : K;
                float4 a, v;
                float pr;
                int j = 0;
                bool symf = false, isb = false;
                if (s < K) {
                    while (s >= S.run[r].x) ++r;
                    const int4 ri = S.run[r];
                    const int prev = r ? S.run[r - 1].x : 0;
                    j = ri.y + (s - prev);
                    const int cd = S.code[r];
                    const float sx = j < ri.z ? -P.s_hf : (j < ri.w ? 0.0f : P.s_hf);
                    const float sy = (float)(((cd >> 1) & 3) - 1) * P.s_hf;
                    const float sz = (float)(((cd >> 3) & 3) - 1) * P.s_hf;
                    float4 p;
                    if (cd & 1) {
                        p = bposp[j];
                        v = bvelr[j];
                        isb = true;
                    } else {
                        p = fposp[j];
                        v = fvelr[j];
                        // own row: the target cell is one-sided, cell x+1 symmetric
                        symf = !(cd & 32) || j >= ri.w;
                    }
                    a.x = fmaf(p.x, P.invhf, sx);
                    a.y = fmaf(p.y, P.invhf, sy);
                    a.z = fmaf(p.z, P.invhf, sz);
                    a.w = fmaf(a.x, a.x, fmaf(a.y, a.y, a.z * a.z));
                    pr = p.w;
                } else {
                    a = make_float4(0.f, 0.f, 0.f, INFINITY);
                    v = make_float4(0.f, 0.f, 0.f, 1.f);
                    pr = 0.f;
                }
                S.A[ls] = a;
                S.V[ls] = v;
                S.Pr[ls] = pr;
                S.J[ls] = j;
                S.B[ls] = make_float4(0.f, 0.f, 0.f, 0.f);
                const uint32_t bf = __ballot_sync(0xffffffffu, symf);
                const uint32_t bb = __ballot_sync(0xffffffffu, isb);
                if (lane == 0) {
                    S.symF[m] = bf;
                    S.isB[m] = bb;
                }
            }
            __syncwarp();
            // ---- lockstep distance tests, one hit bit per candidate
            witems::lockstep_tests<false>(S.A, S.M, np, lane, witems::Frame{xa, ya, za, thr});
            // ---- every lane walks its own hits; b-side terms to the candidate's
            // slot.  All lanes iterate together (until no lane has a hit left)
            // so that the warp-wide match below is well defined.
            int q = 0;
            uint32_t m = S.M[0][lane], sf = S.symF[0], sb = S.isB[0];
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
                    const float rx = xa - b.x, ry = ya - b.y, rz = za - b.z;
                    float coef, cF;
                    pair_sym(P, rx, ry, rz, pa.w, va, cpa, S.V[ls], S.Pr[ls], coef, cF, vismax);
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
            // ---- b-side sums of the pass to the particles
            for (int mm = 0; mm < nch; ++mm) {
                const int ls = lane + 32 * mm;
                const float4 bs = S.B[ls];
                if ((S.symF[mm] >> lane) & 1u) {
                    if (bs.x != 0.f || bs.y != 0.f || bs.z != 0.f || bs.w != 0.f)
                        red_add_v4(acc + S.J[ls], P.nmkBf * bs.x, P.nmkBf * bs.y, P.nmkBf * bs.z,
                                   P.mkBf * bs.w);
                } else if ((S.isB[mm] >> lane) & 1u) {
                    if (bs.w != 0.f) atomicAdd(bar + S.J[ls], P.mkBf * bs.w);
                }
            }
            __syncwarp();
        }
        if (active) red_add_v4(acc + i, P.nmkBf * ax, P.nmkBf * ay, P.nmkBf * az, P.mkBf * ar);
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
