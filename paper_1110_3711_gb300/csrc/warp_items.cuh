// Warp-per-work-item candidate search shared by the float64 kernels (PI and
// its adjoint).
//
// A work item is up to 32 fluid targets of one cell (items_f, one entry per
// first target) or up to 32 boundary targets of consecutive cells of one x
// row (items_b, {first, count} pairs).  For an item the warp
//   1. builds the table of its x-runs (Section 4.4, Fig. 10): for every
//      (dy, dz) of the 9 neighbour rows, cells x-1 .. x+1 (of the item's first
//      and last cell) are one index range of the fluid list, and for fluid
//      targets of the boundary list too;
//   2. stages the candidates of those runs that lie within 2h of the targets'
//      bounding box in shared memory, as their float32 cell-relative offsets
//      shifted into the frame of the item's first cell, in units of h, with
//      |x|^2 beside them, and their indices;
//   3. tests every candidate against every target in lockstep, in float32,
//      against 4 (1 + 1e-4) (units of h^2): the float32 error of the offsets
//      and of the test is below 1e-5 of 4, so every pair of the float64 test
//      r^2 < 4h^2 is a hit (the float64 test then decides);
//   4. lets every lane walk its own hits in staging order, calling the
//      caller's hit function with the candidate's index and list.
// Neighbourhoods of more candidates than a pass holds take several passes;
// pass p samples candidates p, p + npass, ..., so that each pass holds about
// 1/npass of every lane's neighbours.  The walk order depends only on the item, so
// sums accumulated in it are deterministic.  Cells of edge 2h or more only.
#pragma once

#include "sph_internal.cuh"

namespace sph {
namespace witems {

constexpr int CAP = 256;
constexpr int NCH = CAP / 32;
constexpr int NRUN = 18;   // 9 fluid + 9 boundary x-runs

constexpr int RAW_PER_PASS = 2 * CAP;  // candidates sampled per pass (before the box test)

struct Smem {
    float4 A[CAP];          // shifted offset {x, y, z} (units of h) and |x|^2
    uint32_t J[CAP];        // candidate index, bit 31 set for the boundary list
    uint32_t M[NCH][32];    // hit bits of lane l for chunk q
    int4 run[NRUN];         // {inclusive end slot, first index, b1, b2}
    int code[NRUN];         // list (bit 0), dy+1 (bits 1-2), dz+1 (bits 3-4)
    float box[6];           // targets' bounding box: min x, max x, min y, max y, min z, max z
    int hincl[32];          // balanced walk: hits of targets 0 .. t of the tested set
};

constexpr int NSLOT = 63;   // partial-sum slots of the balanced walk (lane + target)

// The item's targets as one lane sees them.
struct Item {
    int i0, nt;             // first target, number of targets
    int i;                  // this lane's target (i0 for lanes past nt)
    bool active;            // lane < nt
    uint32_t c;             // cell of the first target
    int cx, cy, cz, cx1;    // its coordinates; cx1: x of the item's last cell
};

template <bool FLUID_TARGETS>
__device__ __forceinline__ Item item_of(const DevParams &P, const uint32_t *__restrict__ items,
                                        uint32_t it, const uint32_t *__restrict__ tcell,
                                        const int32_t *__restrict__ tstart, int lane)
{
    Item I;
    if (FLUID_TARGETS) {
        I.i0 = (int)items[it];
        I.nt = min(32, tstart[tcell[I.i0] + 1] - I.i0);
    } else {
        I.i0 = (int)items[2 * it];
        I.nt = (int)items[2 * it + 1];
    }
    I.c = tcell[I.i0];
    I.active = lane < I.nt;
    I.i = I.i0 + (I.active ? lane : 0);
    const uint32_t t = I.c / (uint32_t)P.nx;
    I.cx = (int)(I.c - t * (uint32_t)P.nx);
    I.cy = (int)(t % (uint32_t)P.ny);
    I.cz = (int)(t / (uint32_t)P.ny);
    I.cx1 = FLUID_TARGETS ? I.cx : I.cx + (int)(tcell[I.i0 + I.nt - 1] - I.c);
    return I;
}

// Lane's target in the item's frame (units of h): x, y, z and the test
// threshold 4 (1 + 1e-4) - |x|^2 (-inf for idle lanes).
struct Frame {
    float x, y, z, thr;
};

template <bool FLUID_TARGETS>
__device__ __forceinline__ Frame frame_of(const DevParams &P, const Item &I, const float4 &fa,
                                          const uint32_t *__restrict__ tcell)
{
    Frame F;
    const float tshift = FLUID_TARGETS ? 0.0f : (float)(int)(tcell[I.i] - I.c) * P.s_hf;
    F.x = fmaf(fa.x, P.invhf, tshift);
    F.y = fa.y * P.invhf;
    F.z = fa.z * P.invhf;
    F.thr = I.active ? 4.0004f - fmaf(F.x, F.x, fmaf(F.y, F.y, F.z * F.z)) : -INFINITY;
    return F;
}

// Steps 1-3 above; after each staged set is tested, flush(nch) runs with the
// hit masks of its nch chunks in S.M (lane l's bit k of S.M[q][l]: candidate
// q * 32 + k is a hit of target l).  Every lane of the warp must call it.
template <bool FLUID_TARGETS, class Flush>
__device__ __forceinline__ void stage_and_test(const DevParams &P, Smem &S, int lane,
                                               const Item &I, const Frame &F,
                                               const int32_t *__restrict__ fstart,
                                               const float4 *__restrict__ fposf,
                                               const int32_t *__restrict__ bstart,
                                               const float4 *__restrict__ bposf,
                                               const uint32_t *__restrict__ fcell, Flush &&flush)
{
    const int nlists = FLUID_TARGETS ? 2 : 1;
    int K;
    {
        const int r = lane;
        int L = 0, j0 = 0, b1 = 0, b2 = 0, code = 0;
        if (r < 9 * nlists) {
            const int list = r / 9, q = r % 9;
            const int dz = q / 3 - 1, dy = q % 3 - 1;
            const int y = I.cy + dy, z = I.cz + dz;
            code = list | ((dy + 1) << 1) | ((dz + 1) << 3);
            if (y >= 0 && y < P.ny && z >= 0 && z < P.nz) {
                const int32_t *st = list ? bstart : fstart;
                const int row = P.nx * (y + P.ny * z);
                const int x0 = max(I.cx - 1, 0), x1 = min(I.cx1 + 1, P.nx - 1);
                j0 = st[row + x0];
                L = st[row + x1 + 1] - j0;
                if (FLUID_TARGETS) {
                    b1 = st[row + I.cx];       // first index of cell x
                    b2 = st[row + I.cx + 1];   // first index of cell x + 1
                } else {
                    b1 = row + I.cx;           // cell id of the item's first cell in this row
                }
            }
        }
        int pe = L;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, pe, o);
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
    {
        const bool act = F.thr > -INFINITY;
        float b[6] = {act ? F.x : INFINITY, act ? F.x : -INFINITY, act ? F.y : INFINITY,
                      act ? F.y : -INFINITY, act ? F.z : INFINITY, act ? F.z : -INFINITY};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                b[2 * d] = fminf(b[2 * d], __shfl_xor_sync(0xffffffffu, b[2 * d], o));
                b[2 * d + 1] = fmaxf(b[2 * d + 1], __shfl_xor_sync(0xffffffffu, b[2 * d + 1], o));
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int d = 0; d < 6; ++d) S.box[d] = b[d];
        }
        __syncwarp();
    }

    const float m2x = -2.0f * F.x, m2y = -2.0f * F.y, m2z = -2.0f * F.z;
    // Pass p takes candidates p, p + npass, ... (an interleaved sample of the
    // whole neighbourhood); only those within 2h of the targets' bounding box
    // are staged (the box test's threshold 4.0004 h^2 lies above its float32
    // error), packed with a ballot, and the staged set is tested and walked
    // whenever it may not take another 32.
    const int npass = (K + RAW_PER_PASS - 1) / RAW_PER_PASS;
    for (int pass = 0; pass < npass; ++pass) {
        const int np = (K - pass + npass - 1) / npass;
        int k0 = 0, r = 0;
        while (k0 < np) {
            int n = 0;
            while (k0 < np && n <= CAP - 32) {
                const int ls = k0 + lane;
                bool keep = false;
                float4 a;
                uint32_t jj = 0;
                if (ls < np) {
                    const int sidx = pass + npass * ls;
                    while (sidx >= S.run[r].x) ++r;
                    const int4 ri = S.run[r];
                    const int prev = r ? S.run[r - 1].x : 0;
                    const int j = ri.y + (sidx - prev);
                    const int cd = S.code[r];
                    const float sx = FLUID_TARGETS
                                         ? (j < ri.z ? -P.s_hf : (j < ri.w ? 0.0f : P.s_hf))
                                         : (float)((int)fcell[j] - ri.z) * P.s_hf;
                    const float sy = (float)(((cd >> 1) & 3) - 1) * P.s_hf;
                    const float sz = (float)(((cd >> 3) & 3) - 1) * P.s_hf;
                    const bool blist = FLUID_TARGETS && (cd & 1);
                    const float4 f = blist ? bposf[j] : fposf[j];
                    a.x = fmaf(f.x, P.invhf, sx);
                    a.y = fmaf(f.y, P.invhf, sy);
                    a.z = fmaf(f.z, P.invhf, sz);
                    const float dx = fmaxf(fmaxf(S.box[0] - a.x, a.x - S.box[1]), 0.0f);
                    const float dy = fmaxf(fmaxf(S.box[2] - a.y, a.y - S.box[3]), 0.0f);
                    const float dz = fmaxf(fmaxf(S.box[4] - a.z, a.z - S.box[5]), 0.0f);
                    keep = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < 4.0004f;
                    a.w = fmaf(a.x, a.x, fmaf(a.y, a.y, a.z * a.z));
                    jj = (uint32_t)j | (blist ? 0x80000000u : 0u);
                }
                const unsigned ball = __ballot_sync(0xffffffffu, keep);
                if (keep) {
                    const int slot = n + __popc(ball & ((1u << lane) - 1u));
                    S.A[slot] = a;
                    S.J[slot] = jj;
                }
                n += __popc(ball);
                k0 += 32;
            }
            // far candidates fill the last chunk
            const int nch = (n + 31) >> 5;
            if (n + lane < nch * 32) {
                S.A[n + lane] = make_float4(0.f, 0.f, 0.f, INFINITY);
                S.J[n + lane] = 0u;
            }
            __syncwarp();
            // lockstep tests: the sign of t - thr is the hit bit, shifted into two
            // 16-candidate masks that are joined and bit-reversed (candidate k at bit k)
            for (int q = 0; q < nch; ++q) {
                uint32_t lo = 0u, hi = 0u;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const float4 a = S.A[q * 32 + k];
                    const float4 b = S.A[q * 32 + 16 + k];
                    const float ta = fmaf(m2x, a.x, fmaf(m2y, a.y, fmaf(m2z, a.z, a.w))) - F.thr;
                    const float tb = fmaf(m2x, b.x, fmaf(m2y, b.y, fmaf(m2z, b.z, b.w))) - F.thr;
                    lo = __funnelshift_l(__float_as_uint(ta), lo, 1);
                    hi = __funnelshift_l(__float_as_uint(tb), hi, 1);
                }
                S.M[q][lane] = __brev((lo << 16) | hi);
            }
            __syncwarp();
            flush(nch);
            __syncwarp();
        }
    }
}

// Steps 1-4 above; hit(j, blist) runs for every hit of this lane (blist:
// candidate j of the boundary list).  Every lane of the warp must call it.
template <bool FLUID_TARGETS, class Hit>
__device__ __forceinline__ void for_each_hit(const DevParams &P, Smem &S, int lane, const Item &I,
                                             const Frame &F, const int32_t *__restrict__ fstart,
                                             const float4 *__restrict__ fposf,
                                             const int32_t *__restrict__ bstart,
                                             const float4 *__restrict__ bposf,
                                             const uint32_t *__restrict__ fcell, Hit &&hit)
{
    stage_and_test<FLUID_TARGETS>(P, S, lane, I, F, fstart, fposf, bstart, bposf, fcell,
                                  [&](int nch) {
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
            const uint32_t jj = S.J[ls];
            hit((int)(jj & 0x7fffffffu), FLUID_TARGETS && (jj >> 31) != 0u);
        }
    });
}

// Steps 1-3 above, then a balanced walk: the hits of a tested set, taken in
// target order (target t is lane t of the item) and staging order within a
// target, are dealt to the 32 lanes in equal consecutive shares, so every
// lane walks the same number of hits whatever the targets' counts (the
// float64 pipe, which takes about 19 cycles per warp instruction on GB300,
// then works with all lanes busy).  A lane whose share spans several targets
// switches target in between:
//   begin(t)        the lane now works for target t (load it, clear the sums);
//   hit(j, blist)   a hit of that target;
//   end(t, slot)    the lane's partial sums for t go to partial slot `slot`;
// slots are lane + t, unique along the staircase the shares form.  Then the
// lane of every target with hits adds its slots in lane order,
//   combine(slot),
// so the result depends only on the item, not on scheduling.
template <bool FLUID_TARGETS, class Begin, class Hit, class End, class Combine>
__device__ __forceinline__ void for_each_hit_balanced(
    const DevParams &P, Smem &S, int lane, const Item &I, const Frame &F,
    const int32_t *__restrict__ fstart, const float4 *__restrict__ fposf,
    const int32_t *__restrict__ bstart, const float4 *__restrict__ bposf,
    const uint32_t *__restrict__ fcell, Begin &&begin, Hit &&hit, End &&end, Combine &&combine)
{
    stage_and_test<FLUID_TARGETS>(P, S, lane, I, F, fstart, fposf, bstart, bposf, fcell,
                                  [&](int nch) {
        // hits per target and their inclusive prefix over the lanes
        int c = 0;
        for (int q = 0; q < nch; ++q) c += __popc(S.M[q][lane]);
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        S.hincl[lane] = incl;
        const int T = __shfl_sync(0xffffffffu, incl, 31);
        __syncwarp();
        if (T == 0) return;
        const int sh = (T + 31) >> 5;
        const int g0 = min(lane * sh, T), g1 = min(g0 + sh, T);
        if (g0 < g1) {
            // the target holding hit g0: the smallest t with incl[t] > g0
            int lo = 0, hi = 31;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (S.hincl[mid] > g0) hi = mid;
                else lo = mid + 1;
            }
            int t = lo;
            int o = g0 - (t ? S.hincl[t - 1] : 0);   // hits of t before g0
            int q = 0;
            uint32_t m = S.M[0][t];
            while (o >= __popc(m)) {
                o -= __popc(m);
                m = S.M[++q][t];
            }
            for (; o > 0; --o) m &= m - 1u;
            begin(t);
            for (int g = g0; g < g1; ++g) {
                while (m == 0u) {
                    if (++q == nch) {
                        end(t, lane + t);
                        // the next target with hits (one exists: g < g1 <= T)
                        do {
                            ++t;
                        } while (S.hincl[t] == S.hincl[t - 1]);
                        begin(t);
                        q = 0;
                    }
                    m = S.M[q][t];
                }
                const int ls = q * 32 + __ffs(m) - 1;
                m &= m - 1u;
                const uint32_t jj = S.J[ls];
                hit((int)(jj & 0x7fffffffu), FLUID_TARGETS && (jj >> 31) != 0u);
            }
            end(t, lane + t);
        }
        __syncwarp();
        // the target of this lane adds the partial sums of its shares in lane order
        if (c > 0) {
            const int first = incl - c, last = incl - 1;
            for (int L = first / sh; L <= last / sh; ++L) combine(L + lane);
        }
    });
}

}  // namespace witems
}  // namespace sph
