// PI stage, SPH_FP32_SPLIT form: warp-cooperative particle interaction.
//
// The paper's GPU kernel (Section 4, Fig. 11) gives every target particle its
// own thread and its own walk over the 27 cells; the pair body then runs under
// a divergent branch (a warp idles whenever any lane has a false neighbour,
// Section 4 "code divergence").  Here one warp owns a work item: up to 32
// target particles of one cell (cells follow X, Y, Z after NL, so they are a
// contiguous range).  For that item the warp
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
// Work items are taken from a list built by NL with an atomic counter, so the
// grid is persistent (one resident set of CTAs) and balances itself.  Boundary
// targets (B-F) come in packed items: consecutive cells of one x row with at
// most 32 particles together (a boundary cell holds about 10), the candidates
// being the fluid of the union of their neighbourhoods (x-runs from the first
// cell - 1 to the last + 1); each candidate is shifted by its own cell's x
// distance from the first cell, each target by its cell's.  Fluid and boundary
// items form one queue (fluid first) served by one launch.  Sums of a target
// are accumulated by one lane in candidate order, so results do not depend on
// the order the items are processed in.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sph_internal.cuh"

#ifndef SPH_PI_CAP
#define SPH_PI_CAP 256
#endif
#ifndef SPH_PI_WARPS
#define SPH_PI_WARPS 4
#endif
// Resident CTAs per SM the register allocation is held to: shared memory
// (about 42.7 KB per CTA) admits 5 per SM, and 5 CTAs of 128 threads need at
// most 96 registers per thread.
#ifndef SPH_PI_MINB
#define SPH_PI_MINB 5
#endif

namespace sph {

namespace {

constexpr int CAP = SPH_PI_CAP;   // staged candidates per warp and pass
constexpr int NCH = CAP / 32;     // 32-candidate chunks per pass
constexpr int WARPS = SPH_PI_WARPS;
constexpr int NRUN = 18;          // 9 fluid + 9 boundary x-runs
constexpr int RAW_PER_PASS = 2 * CAP;  // candidates sampled per pass (before the box test)
static_assert(CAP % 32 == 0, "CAP must be a multiple of 32");

struct WarpSmem {
    float4 A[CAP];        // shifted candidate offset {x, y, z} and |x|^2
    float4 V[CAP];        // candidate {vx, vy, vz, rho}
    float Pr[CAP];        // candidate P / rho^2
    uint32_t M[NCH][32];  // hit bits of lane l for chunk q
    int4 run[NRUN];       // {inclusive end slot, first index, start of cell x, start of cell x+1}
    int code[NRUN];       // list (bit 0), dy+1 (bits 1-2), dz+1 (bits 3-4)
    float box[6];         // targets' bounding box: min x, max x, min y, max y, min z, max z
};

struct Acc {
    float ax, ay, az, ar, vis;
};

// Approximate reciprocal and reciprocal square root (PTX rcp.approx and
// rsqrt.approx, relative error about 2^-23).  Their arguments here are normal
// numbers (densities, r'^2 + eta^2/h^2 >= eta^2/h^2, r'^2 clamped at 1e-30),
// so flushing subnormals changes nothing.
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Terms of one ordered pair a <- b (see the oracle): momentum sum, continuity
// sum and the viscous dt term, in units of h.  With r' = r / h and
// q = |r'|, the cubic-spline gradient is grad_a W = F r with
// F = (kB / h) F'', F'' = (kA h / kB)(2.25 q - 3) for q < 1 and (2 - q)^2 / q
// for 1 <= q < 2, so that
//   momentum:   -(P_a/rho_a^2 + P_b/rho_b^2 + Pi_ab) F r   = -kB (...) F'' r'
//   continuity:  v_ab . F r                                =  kB (v_ab . r') F''
//   viscosity:  mu_ab = h v_ab.r / (r^2 + eta^2)          = v_ab.r' / (q^2 + eta^2/h^2)
//   Pi_ab = -alpha (c_a + c_b) mu_ab / (rho_a + rho_b)     (mu_ab < 0, else 0).
// The sums hold (...) F'' r' and (v_ab . r') F''; the constant factors -m kB
// and m kB are applied once per target.  cpa = -alpha c_a; -alpha c_b is
// kcf rho_b^3 (Tait sound speed with gamma = 7, c = c0 (rho / rho0)^3).
// Tensile correction of Monaghan (2000): R_ab (W(r)/W(dp))^n (see the FP64 form).
__device__ __forceinline__ float tensile32(const DevParams &P, float q, float pra, float prb)
{
    float t = 2.0f - q;
    float w = q < 1.0f ? P.aDf * fmaf(q * q, fmaf(0.75f, q, -1.5f), 1.0f) : P.aDf * 0.25f * t * t * t;
    float f = w * P.inv_wdpf, fn = 1.0f;
    for (int k = 0; k < P.tensile_n; ++k) fn *= f;
    float R = (pra > 0.0f && prb > 0.0f) ? P.tens_posf * (pra + prb)
                                          : P.tens_epsf * (fmaxf(-pra, 0.0f) + fmaxf(-prb, 0.0f));
    return R * fn;
}

template <bool MOMENTUM, bool TENSILE>
__device__ __forceinline__ void pair(const DevParams &P, float xa, float ya, float za,
                                     const float4 &pa, const float4 &va, float cpa,
                                     const float4 &b, const float4 &vb, float prb, Acc &o)
{
    const float rx = xa - b.x, ry = ya - b.y, rz = za - b.z;
    const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
    const float rinv = rsqrt_approx(fmaxf(r2, 1e-30f));
    const float q = r2 * rinv;
    const float t = 2.0f - q;
    const float F = q < 1.0f ? fmaf(P.gw1, q, P.gw0) : t * t * rinv;
    const float dvx = va.x - vb.x, dvy = va.y - vb.y, dvz = va.z - vb.z;
    const float vdr = fmaf(dvx, rx, fmaf(dvy, ry, dvz * rz));
    const float mu = vdr * rcp_approx(r2 + P.eta2_h2f);
    if (MOMENTUM) {
        const float cc = fmaf(P.kcf, vb.w * vb.w * vb.w, cpa);
        float coef;
        if (TENSILE) {
            const float Pi = cc * fminf(mu, 0.0f) * rcp_approx(va.w + vb.w) +
                             tensile32(P, q, pa.w, prb);
            coef = (pa.w + prb + Pi) * F;
        } else {
            coef = fmaf(cc * fminf(mu, 0.0f), rcp_approx(va.w + vb.w), pa.w + prb) * F;
        }
        o.ax = fmaf(coef, rx, o.ax);
        o.ay = fmaf(coef, ry, o.ay);
        o.az = fmaf(coef, rz, o.az);
    }
    o.ar = fmaf(vdr, F, o.ar);
    o.vis = fmaxf(o.vis, fabsf(mu));
}

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
    const int nlists = MOMENTUM ? 2 : 1;
    {
        // ---- the item: fluid targets [i0, i0 + nt) of cell c; boundary
        // targets [i0, i0 + nt) of cells c .. c + (cx1 - cx) of one x row
        int i0, nt;
        if (MOMENTUM) {
            i0 = (int)items[it];
            nt = min(32, tstart[tcell[i0] + 1] - i0);
        } else {
            i0 = (int)items[2 * it];
            nt = (int)items[2 * it + 1];
        }
        const uint32_t c = tcell[i0];
        const bool active = lane < nt;
        const int i = i0 + (active ? lane : 0);
        const float4 pa = tposp[i], va = tvelr[i];
        const uint32_t cyz = c / (uint32_t)P.nx;
        const int cx = (int)(c - cyz * (uint32_t)P.nx);
        const int cy = (int)(cyz % (uint32_t)P.ny);
        const int cz = (int)(cyz / (uint32_t)P.ny);
        // last cell of the item (same row) and the target's own x distance
        const int cx1 = MOMENTUM ? cx : cx + (int)(tcell[i0 + nt - 1] - c);
        const float tshift = MOMENTUM ? 0.0f : (float)(int)(tcell[i] - c) * P.s_hf;
        const float xa = fmaf(pa.x, P.invhf, tshift), ya = pa.y * P.invhf, za = pa.z * P.invhf;
        const float m2x = -2.0f * xa, m2y = -2.0f * ya, m2z = -2.0f * za;
        const float thr = active ? 4.0f - fmaf(xa, xa, fmaf(ya, ya, za * za)) : -INFINITY;
        const float ra = va.w * P.inv_rho0f;
        const float cpa = P.nalphaf * (P.c0f * ra * ra * ra);

        // ---- run table: lane r describes run r
        int K;
        {
            const int r = lane;
            int L = 0, j0 = 0, b1 = 0, b2 = 0, code = 0;
            if (r < 9 * nlists) {
                const int list = r / 9, q = r % 9;
                const int dz = q / 3 - 1, dy = q % 3 - 1;
                const int y = cy + dy, z = cz + dz;
                code = list | ((dy + 1) << 1) | ((dz + 1) << 3);
                if (y >= 0 && y < P.ny && z >= 0 && z < P.nz) {
                    const int32_t *st = list ? bstart : fstart;
                    const int row = P.nx * (y + P.ny * z);
                    const int x0 = max(cx - 1, 0), x1 = min(cx1 + 1, P.nx - 1);
                    j0 = st[row + x0];
                    L = st[row + x1 + 1] - j0;
                    if (MOMENTUM) {
                        b1 = st[row + cx];
                        b2 = st[row + cx + 1];
                    } else {
                        b1 = row + cx;  // cell id of the item's first cell in this row
                    }
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

        // bounding box of the item's targets (units of h, item frame)
        float bx0 = active ? xa : INFINITY, bx1 = active ? xa : -INFINITY;
        float by0 = active ? ya : INFINITY, by1 = active ? ya : -INFINITY;
        float bz0 = active ? za : INFINITY, bz1 = active ? za : -INFINITY;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            bx0 = fminf(bx0, __shfl_xor_sync(0xffffffffu, bx0, o));
            bx1 = fmaxf(bx1, __shfl_xor_sync(0xffffffffu, bx1, o));
            by0 = fminf(by0, __shfl_xor_sync(0xffffffffu, by0, o));
            by1 = fmaxf(by1, __shfl_xor_sync(0xffffffffu, by1, o));
            bz0 = fminf(bz0, __shfl_xor_sync(0xffffffffu, bz0, o));
            bz1 = fmaxf(bz1, __shfl_xor_sync(0xffffffffu, bz1, o));
        }
        if (lane == 0) {
            S.box[0] = bx0; S.box[1] = bx1;
            S.box[2] = by0; S.box[3] = by1;
            S.box[4] = bz0; S.box[5] = bz1;
        }
        __syncwarp();

        Acc o = {0.f, 0.f, 0.f, 0.f, 0.f};
        // Pass p takes candidates p, p + npass, p + 2 npass, ...: every pass
        // samples the whole neighbourhood, so every lane finds about 1/npass of
        // its neighbours in each pass and the hit walks stay balanced.  Only
        // candidates within 2h of the targets' bounding box are staged (the
        // others cannot be within 2h of any target; the box test's threshold
        // 4.0004 h^2 lies above its float32 error and that of the lockstep
        // test), packed with a ballot; the staged set is tested and walked
        // whenever it may not take another 32.
        const int npass = (K + RAW_PER_PASS - 1) / RAW_PER_PASS;
        for (int pass = 0; pass < npass; ++pass) {
            const int np = (K - pass + npass - 1) / npass;
            int k0 = 0, r = 0;
            while (k0 < np) {
                // ---- stage the candidates near the box, at most CAP
                int n = 0;
                while (k0 < np && n <= CAP - 32) {
                    const int ls = k0 + lane;
                    bool keep = false;
                    float4 a, v;
                    float pr = 0.f;
                    if (ls < np) {
                        const int sidx = pass + npass * ls;
                        while (sidx >= S.run[r].x) ++r;
                        const int4 ri = S.run[r];
                        const int prev = r ? S.run[r - 1].x : 0;
                        const int j = ri.y + (sidx - prev);
                        const int cd = S.code[r];
                        const float sx =
                            MOMENTUM ? (j < ri.z ? -P.s_hf : (j < ri.w ? 0.0f : P.s_hf))
                                     : (float)((int)fcell[j] - ri.z) * P.s_hf;
                        const float sy = (float)(((cd >> 1) & 3) - 1) * P.s_hf;
                        const float sz = (float)(((cd >> 3) & 3) - 1) * P.s_hf;
                        const bool blist = MOMENTUM && (cd & 1);
                        // both loads issued together (the velocity is wasted on a
                        // candidate the box test drops, but waits on nothing)
                        const float4 p = blist ? bposp[j] : fposp[j];
                        v = blist ? bvelr[j] : fvelr[j];
                        a.x = fmaf(p.x, P.invhf, sx);
                        a.y = fmaf(p.y, P.invhf, sy);
                        a.z = fmaf(p.z, P.invhf, sz);
                        const float dx = fmaxf(fmaxf(S.box[0] - a.x, a.x - S.box[1]), 0.0f);
                        const float dy = fmaxf(fmaxf(S.box[2] - a.y, a.y - S.box[3]), 0.0f);
                        const float dz = fmaxf(fmaxf(S.box[4] - a.z, a.z - S.box[5]), 0.0f);
                        keep = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < 4.0004f;
                        if (keep) {
                            a.w = fmaf(a.x, a.x, fmaf(a.y, a.y, a.z * a.z));
                            pr = p.w;
                        }
                    }
                    const unsigned ball = __ballot_sync(0xffffffffu, keep);
                    if (keep) {
                        const int slot = n + __popc(ball & ((1u << lane) - 1u));
                        S.A[slot] = a;
                        S.V[slot] = v;
                        S.Pr[slot] = pr;
                    }
                    n += __popc(ball);
                    k0 += 32;
                }
                // far candidates fill the last chunk
                const int nch = (n + 31) >> 5;
                if (n + lane < nch * 32) {
                    S.A[n + lane] = make_float4(0.f, 0.f, 0.f, INFINITY);
                    S.V[n + lane] = make_float4(0.f, 0.f, 0.f, 1.f);
                    S.Pr[n + lane] = 0.f;
                }
                __syncwarp();
                // ---- lockstep distance tests, one hit bit per candidate
                for (int q = 0; q < nch; ++q) {
                    // the sign of t - thr is the hit bit; it is shifted into two
                    // independent 16-candidate masks (candidate k lands at bit 15 - k
                    // of its half), which are joined and bit-reversed so that
                    // candidate k ends at bit k
                    uint32_t lo = 0u, hi = 0u;
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const float4 a = S.A[q * 32 + k];
                        const float4 b = S.A[q * 32 + 16 + k];
                        const float ta = fmaf(m2x, a.x, fmaf(m2y, a.y, fmaf(m2z, a.z, a.w))) - thr;
                        const float tb = fmaf(m2x, b.x, fmaf(m2y, b.y, fmaf(m2z, b.z, b.w))) - thr;
                        lo = __funnelshift_l(__float_as_uint(ta), lo, 1);
                        hi = __funnelshift_l(__float_as_uint(tb), hi, 1);
                    }
                    S.M[q][lane] = __brev((lo << 16) | hi);
                }
                // |x|^2 has served the tests: the pair walk reads P/rho^2 from its place
                __syncwarp();
                for (int q2 = 0; q2 < nch; ++q2) S.A[q2 * 32 + lane].w = S.Pr[q2 * 32 + lane];
                __syncwarp();
                // ---- every lane walks its own hits (about 112 per lane in all)
                int q = 0;
                uint32_t m = nch > 0 ? S.M[0][lane] : 0u;
                for (;;) {
                    while (m == 0u && q + 1 < nch) {
                        ++q;
                        m = S.M[q][lane];
                    }
                    if (m == 0u) break;
                    const int ls = q * 32 + __ffs(m) - 1;
                    m &= m - 1u;
                    const float4 b = S.A[ls];
                    pair<MOMENTUM, TENSILE>(P, xa, ya, za, pa, va, cpa, b, S.V[ls], b.w, o);
                }
                __syncwarp();
            }
        }

        if (active) {
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
                   (const float4 *)w.velr, w.cell, w.fstart, (const float4 *)w.bposp,
                   (const float4 *)w.bvelr, w.bcell, w.bstart, (float4 *)w.acc, (float *)w.bar,
                   w.sc);
    else
        SPH_LAUNCH(ctx, k_pi32<false>, ctx->pi_grid_f, WARPS * 32, 0, st, ctx->dp, w.items_f,
                   w.items_b, w.ctr, use_b, &w.ctr[1], (const float4 *)w.posp,
                   (const float4 *)w.velr, w.cell, w.fstart, (const float4 *)w.bposp,
                   (const float4 *)w.bvelr, w.bcell, w.bstart, (float4 *)w.acc, (float *)w.bar,
                   w.sc);
    return check_cuda(cudaGetLastError());
}

}  // namespace sph
