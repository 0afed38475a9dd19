// Warp-per-work-item candidate search of the PI kernels: the float32 warp
// kernel (pi32.cu), the float64 PI (pi.cu) and its adjoint (adjoint.cu); the
// symmetric float32 variant (pi32_sym.cu) shares the lockstep test.
//
// A work item is up to 32 fluid targets of one cell (items_f) or up to 32
// boundary targets of consecutive cells of one x row (items_b), both as
// {first, count} pairs.  For an item the warp
//   1. builds the table of its x-runs (Section 4.4, Fig. 10): for every
//      (dy, dz) of the 9 neighbour rows, cells x-1 .. x+1 (of the item's first
//      and last cell) are one index range of the fluid list, and for fluid
//      targets of the boundary list too (build_runs);
//   2. stages the candidates of those runs that lie within 2h of the targets'
//      bounding box (target_box) in shared memory, as their float32
//      cell-relative offsets shifted into the frame of the item's first cell,
//      in units of h, with |x|^2 beside them, and whatever else the kernel
//      needs of them (stage_set);
//   3. tests every candidate against every target in lockstep (lockstep_tests):
//      the warp reads one candidate (a shared-memory broadcast) and each lane
//      evaluates |x_b|^2 - 2 x_a.x_b - (thr0 - |x_a|^2), negative when
//      |x_a - x_b|^2 < thr0 h^2 up to float32 rounding, and shifts its sign
//      into a hit mask.  The float32 kernel takes thr0 = 4 (the test decides
//      its pairs); the float64 kernels take 4 (1 + 1e-4): the float32 error of
//      the offsets and of the test is below 1e-5 of 4, so every pair of their
//      float64 test r^2 < 4h^2 is a hit (the float64 test then decides);
//   4. lets every lane walk its own hits in staging order.
// Neighbourhoods of more candidates than a pass holds take several passes;
// pass p samples blocks p, p + npass, ... of BLK consecutive candidates, so
// that each pass holds about 1/npass of every lane's neighbours.  The walk order depends only on the item, so
// sums accumulated in it are deterministic.  Cells of edge 2h or more only.
#pragma once

#include "sph_internal.cuh"

namespace sph {
namespace witems {

constexpr int CAP = 256;
constexpr int NCH = CAP / 32;
constexpr int NRUN = 18;   // 9 fluid + 9 boundary x-runs

constexpr int RAW_PER_PASS = 2 * CAP;  // candidates sampled per pass (before the box test)

// Passes sample the item's candidates in blocks of BLK consecutive ones: pass
// p takes blocks p, p + npass, p + 2 npass, ...  A block of 8 records of 16
// bytes is one 128-byte line, so each pass loads whole lines and no sector is
// fetched by two passes, while every pass still samples the whole
// neighbourhood (the hit walks stay balanced).
#ifndef SPH_PASS_BLOCK
#define SPH_PASS_BLOCK 8
#endif
constexpr int BLK = SPH_PASS_BLOCK;

// Sample slots of pass `pass` of npass over K candidates (a multiple of BLK;
// slots past the last candidate are empty).
__device__ __forceinline__ int pass_slots(int K, int npass, int pass)
{
    const int nblk = (K + BLK - 1) / BLK;
    return nblk > pass ? BLK * ((nblk - pass + npass - 1) / npass) : 0;
}

// Candidate index (0 .. K-1 over the item's runs) of sample slot ls of a pass.
__device__ __forceinline__ int pass_candidate(int ls, int npass, int pass)
{
    return (pass + npass * (ls / BLK)) * BLK + ls % BLK;
}

// Box-test threshold (units of h^2): above the float32 error of the box
// distance and of the lockstep test, so that no hit of either form is lost.
constexpr float BOX_THR = 4.0004f;

// A candidate sampled by a pass is a block of BLK consecutive ones, and the
// 32 lanes of a staging round take 32 consecutive sample slots.
static_assert(32 % BLK == 0, "a staging round must hold whole pass blocks");

// The item's x-runs.
struct RunTable {
    int4 run[NRUN];         // {inclusive end slot, first index - first slot, b1, b2}
    float2 sh[NRUN];        // y and z shift of the run's row into the item frame (units of h)
};

// The bounding box of the item's targets: centre and half extent along x, y, z
// (units of h, item frame), the same in every lane.
struct Box {
    float cx, ex, cy, ey, cz, ez;
};

// Staged candidates of the float64 kernels.
struct Smem {
    float4 A[CAP];          // shifted offset {x, y, z} (units of h) and |x|^2
    uint32_t J[CAP];        // candidate index, bit 31 set for the boundary list
    uint32_t M[NCH][32];    // hit bits of lane l for chunk q
    RunTable T;
    Box B;                  // the targets' box (kept here, not in registers, during the walks)
    int hincl[32];          // balanced walk: hits of targets 0 .. t of the tested set
};

constexpr int NSLOT = 63;   // partial-sum slots of the balanced walk (lane + target)

// The item's targets as one lane sees them.  Items of both kinds are
// {first target, number of targets}: up to 32 particles of one cell (fluid
// items) or of consecutive non-empty cells of one x row (boundary items), or
// a chunk of 32 of a fuller cell.
struct Item {
    int i0, nt;             // first target, number of targets
    int i;                  // this lane's target (i0 for lanes past nt)
    bool active;            // lane < nt
    bool multi;             // the targets span more than one cell
    uint32_t c;             // cell of the first target
    int cx, cy, cz, cx1;    // its coordinates; cx1: x of the item's last cell
};

__device__ __forceinline__ Item item_of(const DevParams &P, const uint32_t *__restrict__ items,
                                        uint32_t it, const uint32_t *__restrict__ tcell, int lane)
{
    Item I;
    I.i0 = (int)items[2 * it];
    I.nt = (int)items[2 * it + 1];
    I.c = tcell[I.i0];
    I.active = lane < I.nt;
    I.i = I.i0 + (I.active ? lane : 0);
    const uint32_t t = I.c / (uint32_t)P.nx;
    I.cx = (int)(I.c - t * (uint32_t)P.nx);
    I.cy = (int)(t % (uint32_t)P.ny);
    I.cz = (int)(t / (uint32_t)P.ny);
    I.cx1 = I.cx + (int)(tcell[I.i0 + I.nt - 1] - I.c);
    I.multi = I.cx1 != I.cx;
    return I;
}

// Lane's target in the item's frame (units of h; the frame of the item's
// first cell): x, y, z and the test threshold thr0 - |x|^2 (-inf for idle
// lanes).
struct Frame {
    float x, y, z, thr;
};

__device__ __forceinline__ Frame frame_of(const DevParams &P, const Item &I, const float4 &fa,
                                          const uint32_t *__restrict__ tcell, float thr0)
{
    Frame F;
    const float tshift = I.multi ? (float)(int)(tcell[I.i] - I.c) * P.s_hf : 0.0f;
    F.x = fmaf(fa.x, P.invhf, tshift);
    F.y = fa.y * P.invhf;
    F.z = fa.z * P.invhf;
    F.thr = I.active ? thr0 - fmaf(F.x, F.x, fmaf(F.y, F.y, F.z * F.z)) : -INFINITY;
    return F;
}

// Which x-runs an item searches.  RUNS_FULL: the 9 (dy, dz) rows of the fluid
// list (runs 0-8) and, for fluid targets, of the boundary list (runs 9-17),
// cells x-1 .. x+1 each.  RUNS_HALF (fluid targets of one cell, symmetric pair
// evaluation): the fluid cells after the item's own cell in (z, y, x) order,
// i.e. the rows (dy, dz) = (-1, +1), (0, +1), (+1, +1), (+1, 0) whole (runs
// 0-3) and cells x, x+1 of the own row (run 4), then the 9 boundary rows
// (runs 5-13).
constexpr int RUNS_FULL = 0;
constexpr int RUNS_HALF = 1;

// First run of the boundary list.
template <bool FLUID_TARGETS, int RUNS>
__device__ __forceinline__ constexpr int first_boundary_run()
{
    return !FLUID_TARGETS ? NRUN : (RUNS == RUNS_HALF ? 5 : 9);
}

// Step 1: lane r describes run r of the table; returns the number of
// candidates K.  b1, b2 of a run: for fluid targets (an item of one cell) the
// first indices of cells x and x + 1 of its row (a candidate's x shift follows
// from its index); for boundary targets the cell id of the item's first cell
// in that row (a candidate's x shift follows from its own cell).
template <bool FLUID_TARGETS, int RUNS = RUNS_FULL>
__device__ __forceinline__ int build_runs(const DevParams &P, RunTable &T, int lane, const Item &I,
                                          const int32_t *__restrict__ fstart,
                                          const int32_t *__restrict__ bstart)
{
    static_assert(RUNS == RUNS_FULL || FLUID_TARGETS, "half-shell runs need fluid targets");
    const int nruns = RUNS == RUNS_HALF ? 14 : (FLUID_TARGETS ? 18 : 9);
    const int r = lane;
    int L = 0, j0 = 0, b1 = 0, b2 = 0, dy = 0, dz = 0;
    if (r < nruns) {
        const int fb = first_boundary_run<FLUID_TARGETS, RUNS>();
        const int list = r >= fb ? 1 : 0;
        int x0off = -1;
        if (RUNS == RUNS_HALF && !list) {
            dz = r < 3 ? 1 : 0;
            dy = r < 3 ? r - 1 : (r == 3 ? 1 : 0);
            if (r == 4) x0off = 0;
        } else {
            const int q = list ? r - fb : r;
            dz = q / 3 - 1;
            dy = q % 3 - 1;
        }
        const int y = I.cy + dy, z = I.cz + dz;
        if (y >= 0 && y < P.ny && z >= 0 && z < P.nz) {
            const int32_t *st = list ? bstart : fstart;
            const int row = P.nx * (y + P.ny * z);
            const int x0 = max(I.cx + x0off, 0), x1 = min(I.cx1 + 1, P.nx - 1);
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
        // candidate at sample index sidx of this run: index sidx + (j0 - first slot)
        T.run[r] = make_int4(pe, j0 - (pe - L), b1, b2);
        T.sh[r] = make_float2((float)dy * P.s_hf, (float)dz * P.s_hf);
    }
    const int K = __shfl_sync(0xffffffffu, pe, NRUN - 1);
    __syncwarp();
    return K;
}

// The bounding box of the item's active targets, reduced over the warp so that
// every lane holds it.
__device__ __forceinline__ Box target_box(const Frame &F)
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
    Box B;
    B.cx = 0.5f * (b[0] + b[1]);
    B.ex = 0.5f * (b[1] - b[0]);
    B.cy = 0.5f * (b[2] + b[3]);
    B.ey = 0.5f * (b[3] - b[2]);
    B.cz = 0.5f * (b[4] + b[5]);
    B.ez = 0.5f * (b[5] - b[4]);
    return B;
}

// Step 3 for the n staged candidates in A (their w is |x|^2; slots n .. of the
// last chunk hold far candidates): bit k of M[q][lane] (MSB_FIRST: bit 31 - k)
// is set when candidate q * 32 + k is a hit of this lane's target.  The sign
// of t - thr is shifted into two independent 16-candidate masks (candidate k
// lands at bit 15 - k of its half), which are joined (and bit-reversed unless
// MSB_FIRST).  A last chunk of at most 16 candidates tests one half.  Only
// the bits set in keep are kept (a lane that shares its target with other
// lanes takes a share of the candidates).  Returns the lane's non-empty
// chunks: bit q set when M[q][lane] != 0.
template <bool MSB_FIRST>
__device__ __forceinline__ uint32_t lockstep_tests(const float4 *A, uint32_t (*M)[32], int n,
                                                   int lane, const Frame &F,
                                                   uint32_t keep = 0xffffffffu)
{
    uint32_t cm = 0u;
    const float m2x = -2.0f * F.x, m2y = -2.0f * F.y, m2z = -2.0f * F.z;
    const int nch = (n + 31) >> 5;
    for (int q = 0; q < nch; ++q) {
        uint32_t lo = 0u, hi = 0u;
        if (n - 32 * q > 16) {
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const float4 a = A[q * 32 + k];
                const float4 b = A[q * 32 + 16 + k];
                const float ta = fmaf(m2x, a.x, fmaf(m2y, a.y, fmaf(m2z, a.z, a.w))) - F.thr;
                const float tb = fmaf(m2x, b.x, fmaf(m2y, b.y, fmaf(m2z, b.z, b.w))) - F.thr;
                lo = __funnelshift_l(__float_as_uint(ta), lo, 1);
                hi = __funnelshift_l(__float_as_uint(tb), hi, 1);
            }
        } else {
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const float4 a = A[q * 32 + k];
                const float ta = fmaf(m2x, a.x, fmaf(m2y, a.y, fmaf(m2z, a.z, a.w))) - F.thr;
                lo = __funnelshift_l(__float_as_uint(ta), lo, 1);
            }
        }
        const uint32_t w = ((lo << 16) | hi) & keep;
        M[q][lane] = MSB_FIRST ? w : __brev(w);
        cm |= (w != 0u ? 1u : 0u) << q;
    }
    return cm;
}

// Step 2 for one set: sample slots k0, k0 + 1, ... of pass `pass` (np slots,
// K candidates in the item) are taken 32 at a time while the set may take
// another 32 (at most cap); the candidates within 2h of the box are packed by
// a ballot into slots 0 .. n-1 and n is returned.  k0 and r (the current run,
// which only moves forward) carry over to the next set.
// A candidate's x shift into the item's frame comes from its index (fluid
// targets: an item of one cell) or from its own cell (boundary targets, whose
// items may span several cells: fcell is the cell of every fluid particle).
//   load(j, blist, own) issues the loads of candidate j of its list and
//                  returns them; its member pos is the float32 offset record
//                  (metres); own: a candidate of the item's own cell in the
//                  RUNS_HALF search (evaluated for the target side only)
//   store(slot, a, c) writes the kept candidate: a = shifted offset {x, y, z}
//                  in units of h and |x|^2, c what load returned
template <bool FLUID_TARGETS, int RUNS = RUNS_FULL, class Load, class Store>
__device__ __forceinline__ int stage_set(const DevParams &P, const RunTable &T, const Box &Bx,
                                         int lane, int cap, int pass, int npass, int np, int K,
                                         int &k0, int &r, const uint32_t *__restrict__ fcell,
                                         Load &&load, Store &&store)
{
    typedef decltype(load(0, false, false)) Cand;
    // the box is uniform over the warp: held in registers for the set
    const Box B = Bx;
    // sample index of slot k0 + lane: rounds of 32 slots hold whole blocks, so
    // it advances by 32 npass per round
    int sidx = pass_candidate(lane, npass, pass) + k0 * npass;
    int n = 0;
    while (k0 < np && n <= cap - 32) {
        const int ls = k0 + lane;
        bool keep = false;
        float4 a;
        Cand c;
        if (ls < np && sidx < K) {
            while (sidx >= T.run[r].x) ++r;
            const int4 ri = T.run[r];
            const int j = sidx + ri.y;
            const float2 sh = T.sh[r];
            const bool blist = r >= first_boundary_run<FLUID_TARGETS, RUNS>();
            const bool own = RUNS == RUNS_HALF && r == 4 && j < ri.w;
            const float sx = FLUID_TARGETS ? (j < ri.z ? -P.s_hf : (j < ri.w ? 0.0f : P.s_hf))
                                           : (float)((int)fcell[j] - ri.z) * P.s_hf;
            c = load(j, blist, own);
            a.x = fmaf(c.pos.x, P.invhf, sx);
            a.y = fmaf(c.pos.y, P.invhf, sh.x);
            a.z = fmaf(c.pos.z, P.invhf, sh.y);
            // distance to the box along each axis: |a - centre| - half extent, or 0 inside
            const float dx = fmaxf(fabsf(a.x - B.cx) - B.ex, 0.0f);
            const float dy = fmaxf(fabsf(a.y - B.cy) - B.ey, 0.0f);
            const float dz = fmaxf(fabsf(a.z - B.cz) - B.ez, 0.0f);
            keep = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < BOX_THR;
            if (keep) a.w = fmaf(a.x, a.x, fmaf(a.y, a.y, a.z * a.z));
        }
        const unsigned ball = __ballot_sync(0xffffffffu, keep);
        if (keep) store(n + __popc(ball & ((1u << lane) - 1u)), a, c);
        n += __popc(ball);
        k0 += 32;
        sidx += 32 * npass;
    }
    return n;
}

// Steps 1-3 above for the float64 kernels (candidates from the float32
// offsets fposf / bposf); after each staged set is tested, flush(nch) runs
// with the hit masks of its nch chunks in S.M (lane l's bit k of S.M[q][l]:
// candidate q * 32 + k is a hit of target l) and the candidates' indices in
// S.J.  Every lane of the warp must call it.
template <bool FLUID_TARGETS, class Flush>
__device__ __forceinline__ void stage_and_test(const DevParams &P, Smem &S, int lane,
                                               const Item &I, const Frame &F,
                                               const int32_t *__restrict__ fstart,
                                               const float4 *__restrict__ fposf,
                                               const int32_t *__restrict__ bstart,
                                               const float4 *__restrict__ bposf,
                                               const uint32_t *__restrict__ fcell, Flush &&flush)
{
    const int K = build_runs<FLUID_TARGETS>(P, S.T, lane, I, fstart, bstart);
    {
        const Box B = target_box(F);
        if (lane == 0) S.B = B;
        __syncwarp();
    }
    struct Cand {
        float4 pos;
        uint32_t jj;
    };
    auto load = [&](int j, bool blist, bool) {
        Cand c;
        c.pos = blist ? bposf[j] : fposf[j];
        c.jj = (uint32_t)j | (blist ? 0x80000000u : 0u);
        return c;
    };
    auto store = [&](int slot, const float4 &a, const Cand &c) {
        S.A[slot] = a;
        S.J[slot] = c.jj;
    };
    const int npass = (K + RAW_PER_PASS - 1) / RAW_PER_PASS;
    for (int pass = 0; pass < npass; ++pass) {
        const int np = pass_slots(K, npass, pass);
        int k0 = 0, r = 0;
        while (k0 < np) {
            const int n = stage_set<FLUID_TARGETS>(P, S.T, S.B, lane, CAP, pass, npass, np, K,
                                                   k0, r, fcell, load, store);
            // far candidates fill the last chunk
            const int nch = (n + 31) >> 5;
            if (n + lane < nch * 32) {
                S.A[n + lane] = make_float4(0.f, 0.f, 0.f, INFINITY);
                S.J[n + lane] = 0u;
            }
            __syncwarp();
            lockstep_tests<false>(S.A, S.M, n, lane, F);
            __syncwarp();
            flush(nch);
            __syncwarp();
        }
    }
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
    const uint32_t *__restrict__ fcell, Begin &&begin, Hit &&hit, End &&end,
    Combine &&combine)
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
