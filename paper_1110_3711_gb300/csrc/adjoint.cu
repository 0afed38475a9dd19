// Hand-written adjoint of one fixed-dt time step (PI + SU) and of the sensor
// objective, SPH_FP64 form.
//
// Forward step n (Table 1 formulation; state x, v, u = v^{n-1}, rho,
// sig = rho^{n-1}; F = fluid acceleration, D = density rate from PI):
//   x' = x + dt v + dt^2/2 F      v' = u + 2dt F  (Euler step: v + dt F)
//   u' = v                         rho' = sig + 2dt D (Euler: rho + dt D)
//   sig' = rho                     boundary rho' clamped at rho0
// Its adjoint, given the adjoint lam' of the state after the step:
//   gF = dt^2/2 lam_x' + cv dt lam_v'        gD = cv dt lam_rho'   (cv = 2, Euler 1)
//   lam_x = lam_x' + (PI terms)              lam_v = dt lam_x' + lam_u' [+ lam_v'] + (PI terms)
//   lam_u = lam_v' [Euler: 0]                lam_rho = lam_sig' [+ lam_rho'] + (PI terms)
//   lam_sig = lam_rho' [Euler: 0]
// and the PI terms are the vector-Jacobian product of the pair sums with the
// cotangents (gF, gD).  For an ordered pair a <- b, L = gF_a . f_ab + gD_a d_ab
// depends on r_ab, v_ab, rho_a, rho_b and alpha; because the neighbour
// relation is symmetric, every particle collects the derivatives of the
// pairs it receives (a = self) and of the pairs it sources (b = self) by
// walking its own 27 cells once: a gather, no atomics, deterministic.  With
// cells of edge 2h the walk runs on the warp work items of the float64 PI
// (warp_items.cuh) and dJ/dalpha is summed per item; with finer cells one
// thread walks per particle and dJ/dalpha is summed per block.  The partial
// sums are added in a fixed order.
//
// Arrays exchanged with the caller (lam, lam_next) are float64 in
// persistent-id order with the layout of sph_get_state:
//   [x: 3N][v: 3N][rho: N][v_prev: 3N][rho_prev: N]   (boundary x, v rows unused).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sph_internal.cuh"
#include "warp_items.cuh"

namespace sph {

namespace {

constexpr int kAdjThreads = 128;

// Adjoint sums of one target particle over its pairs.
struct SelfAdj {
    double rx, ry, rz;  // lam_x
    double vx, vy, vz;  // lam_v
    double rho;         // lam_rho
    double alpha;       // dJ/dalpha of the pairs the target receives
};

__device__ __forceinline__ double sound_of(const DevParams &P, double rho)
{
    double r = rho * P.inv_rho0;
    return P.gamma_is_7 ? P.c0 * r * r * r : P.c0 * pow(r, 0.5 * (P.gamma - 1.0));
}

// Terms of one target particle that its pair derivatives use, formed once:
// rho, P/rho^2, the sound speed c, d(P/rho^2)/drho = (c^2 - 2 rho P/rho^2) / rho^2
// and dc/drho = c (gamma - 1) / (2 rho).
struct PartTerms {
    double rho, pr, c, dpr, dc;
};

__device__ __forceinline__ PartTerms part_terms(const DevParams &P, double rho, double pr)
{
    PartTerms t;
    const double ir = 1.0 / rho;
    t.rho = rho;
    t.pr = pr;
    t.c = sound_of(P, rho);
    t.dpr = ir * ir * (t.c * t.c - 2.0 * pr * rho);
    t.dc = 0.5 * (P.gamma - 1.0) * t.c * ir;
    return t;
}

// Kernel factor of grad_a W = F r_ab and (dF/dr) / r, from one reciprocal
// square root of r^2.
__device__ __forceinline__ void kernel_factor(const DevParams &P, double r2, double *F,
                                              double *dFr)
{
    const double irl = rsqrt(r2);
    const double q = r2 * irl * P.invh;
    if (q < 1.0) {
        *F = P.kA64 * (-3.0 + 2.25 * q);
        *dFr = P.kA64 * 2.25 * P.invh * irl;
    } else {
        const double t = 2.0 - q;
        *F = P.kB64 * t * t * irl;
        *dFr = P.kB64 * (-2.0 * t * P.invh * irl - t * t * irl * irl) * irl;
    }
}

// Both ordered pairs of {a, b} at once, as seen by a (self).  For the ordered
// pair a <- b,
//   L_ab = gF_a . f_ab + gD_a d_ab,
//   f_ab = -m Q F r,  Q = P_a/rho_a^2 + P_b/rho_b^2 + Pi,  d_ab = m (v.r) F,
// with r = r_ab, v = v_ab, grad_a W = F r, Pi = K mu (K = -alpha (c_a + c_b) /
// (rho_a + rho_b), mu = h v.r / (r^2 + eta^2), only where v.r < 0).  L_ba is
// the same function of r_ba = -r and v_ba = -v, under which F, v.r, mu and Q
// do not change and grad_r F = (dF/dr / r) r, dQ/dr = kv v + kr r (kv = K h /
// (r^2 + eta^2), kr = -2 kv v.r / (r^2 + eta^2)) change sign.  So
//   d(L_ab + L_ba)/dx_a = m (gD_a + gD_b) (F v + v.r grad_r F)
//                         - m Q (dG.r) grad_r F - m Q F dG - m F (dG.r) dQ/dr,
//   d(L_ab + L_ba)/dv_a = (m (gD_a + gD_b) F - m F (dG.r) kv) r,
//   d(L_ab + L_ba)/drho_a = -m F (dG.r) (d(P/rho^2)/drho_a + dPi/drho_a),
// with dG = gF_a - gF_b (gF_b = 0 where b is a boundary particle: its pair
// b <- a has no momentum term).  dJ/dalpha takes L_ab only, so that every
// ordered pair counts once over all targets.  One reciprocal square root and
// one reciprocal d = 1/((r^2 + eta^2)(rho_a + rho_b)) per pair; every other
// quotient is a product.
template <bool FLUID_B>
__device__ __forceinline__ void pair_adj(const DevParams &P, double rx, double ry, double rz,
                                         double vx, double vy, double vz, const PartTerms &A,
                                         double rho_b, double pr_b, double c_b, double gFax,
                                         double gFay, double gFaz, double gFbx, double gFby,
                                         double gFbz, double gDs, SelfAdj &l)
{
    const double m = P.mass;
    const double r2 = rx * rx + ry * ry + rz * rz;
    double F, dFr;
    kernel_factor(P, r2, &F, &dFr);
    const double vdr = vx * rx + vy * ry + vz * rz;
    const double den = r2 + P.eta2;
    // K = -alpha (c_a + c_b) / (rho_a + rho_b); for gamma = 7 the polynomial
    // kc64 (rho_a^2 - rho_a rho_b + rho_b^2) (pi.cu), so only 1/den is needed
    double iden, iS = 0.0, t = 0.0;
    if (P.gamma_is_7) {
        iden = 1.0 / den;
        t = fma(rho_b, rho_b - A.rho, A.rho * A.rho);
    } else {
        const double S = A.rho + rho_b;
        const double d = 1.0 / (den * S);
        iden = d * S;
        iS = d * den;
    }
    const double mu = P.h * vdr * iden;
    const double dGx = FLUID_B ? gFax - gFbx : gFax;
    const double dGy = FLUID_B ? gFay - gFby : gFay;
    const double dGz = FLUID_B ? gFaz - gFbz : gFaz;
    const double s1 = gFax * rx + gFay * ry + gFaz * rz;
    const double sd = dGx * rx + dGy * ry + dGz * rz;
    const double cs = A.c + c_b;
    double K = 0.0, Pi = 0.0;
    if (vdr < 0.0) {
        K = P.gamma_is_7 ? P.kc64 * t : -P.alpha * cs * iS;
        Pi = K * mu;
    }
    const double Q = A.pr + pr_b + Pi;
    const double mF = m * F;
    const double cg = m * gDs;       // continuity, both directions
    const double Aq = -m * Q * sd;   // times grad_r F
    const double Bc = -mF * Q;       // times dG
    const double Cc = -mF * sd;      // times dQ
    const double kv = K * P.h * iden, kr = -2.0 * kv * vdr * iden;
    const double gx = dFr * rx, gy = dFr * ry, gz = dFr * rz;  // grad_r F
    l.rx += cg * (F * vx + vdr * gx) + Aq * gx + Bc * dGx + Cc * (kv * vx + kr * rx);
    l.ry += cg * (F * vy + vdr * gy) + Aq * gy + Bc * dGy + Cc * (kv * vy + kr * ry);
    l.rz += cg * (F * vz + vdr * gz) + Aq * gz + Bc * dGz + Cc * (kv * vz + kr * rz);
    const double cvv = cg * F + Cc * kv;
    l.vx += cvv * rx;
    l.vy += cvv * ry;
    l.vz += cvv * rz;
    double dPi = 0.0;
    if (vdr < 0.0) {
        if (P.gamma_is_7) {
            // dK/drho_a = kc64 (2 rho_a - rho_b); dPi/dalpha = -(c0/rho0^3) t mu
            dPi = P.kc64 * fma(2.0, A.rho, -rho_b) * mu;
            l.alpha += mF * s1 * P.kcu64 * t * mu;   // (-m F s1) dPi/dalpha
        } else {
            dPi = -P.alpha * mu * (A.dc * iS - cs * iS * iS);
            l.alpha += mF * s1 * cs * mu * iS;   // (-m F s1) (-(c_a + c_b) mu / (rho_a + rho_b))
        }
    }
    l.rho += Cc * (A.dpr + dPi);
}

// d L_ab / d rho_b for the ordered pair a <- b (a fluid, b the boundary
// target): -m F (gF_a . r) (d(P/rho^2)/drho_b + dPi/drho_b).
__device__ __forceinline__ double pair_adj_rho_b(const DevParams &P, double rx, double ry,
                                                 double rz, double vx, double vy, double vz,
                                                 const PartTerms &B, double rho_a, double c_a,
                                                 double gFx, double gFy, double gFz)
{
    const double r2 = rx * rx + ry * ry + rz * rz;
    double F, dFr;
    kernel_factor(P, r2, &F, &dFr);
    const double Cc = -P.mass * F * (gFx * rx + gFy * ry + gFz * rz);
    const double vdr = vx * rx + vy * ry + vz * rz;
    double dPi = 0.0;
    if (vdr < 0.0) {
        const double den = r2 + P.eta2;
        if (P.gamma_is_7) {
            // dK/drho_b = kc64 (2 rho_b - rho_a) (pair_adj)
            const double mu = P.h * vdr / den;
            dPi = P.kc64 * fma(2.0, B.rho, -rho_a) * mu;
        } else {
            const double S = rho_a + B.rho;
            const double d = 1.0 / (den * S);
            const double iS = d * den, mu = P.h * vdr * d * S;
            const double cs = c_a + B.c;
            dPi = -P.alpha * mu * (B.dc * iS - cs * iS * iS);
        }
    }
    return Cc * (B.dpr + dPi);
}

__device__ __forceinline__ void cell_coords(const DevParams &P, uint32_t c, int *cx, int *cy,
                                            int *cz)
{
    uint32_t t = c / (uint32_t)P.nx;
    *cx = (int)(c - t * (uint32_t)P.nx);
    *cy = (int)(t % (uint32_t)P.ny);
    *cz = (int)(t / (uint32_t)P.ny);
}

// Visit the candidates j of the x-runs of a list around cell (cx, cy, cz): 9
// runs of 3 cells, or 25 runs of 5 cells when cells are finer than 2h.
#define FOR_RUNS(P, cx, cy, cz, start, j, ...)                                    \
    {                                                                              \
        const int R_ = (P).reach;                                                  \
        int x0_ = max((cx) - R_, 0), x1_ = min((cx) + R_, (P).nx - 1);             \
        for (int dz_ = -R_; dz_ <= R_; ++dz_) {                                    \
            int z_ = (cz) + dz_;                                                   \
            if (z_ < 0 || z_ >= (P).nz) continue;                                  \
            for (int dy_ = -R_; dy_ <= R_; ++dy_) {                                \
                int y_ = (cy) + dy_;                                               \
                if (y_ < 0 || y_ >= (P).ny) continue;                              \
                int row_ = (P).nx * (y_ + (P).ny * z_);                            \
                int e_ = (start)[row_ + x1_ + 1];                                  \
                for (int j = (start)[row_ + x0_]; j < e_; ++j) { __VA_ARGS__ }     \
            }                                                                      \
        }                                                                          \
    }

// FOR_RUNS with the float32 pre-test of the float64 PI (pi.cu): a candidate
// whose cell-relative float32 offset lies certainly outside the support of the
// target's offset fa (threshold 4h^2 (1 + 1e-5), above the float32 error of
// the offsets) is skipped before the body, which keeps its exact float64 test,
// so the pairs and the results are unchanged.
#define FOR_RUNS_F(P, cx, cy, cz, start, fa, posf, j, ...)                            \
    {                                                                                  \
        const int R_ = (P).reach;                                                      \
        const float s2f_ = (P).four_h2f * (1.0f + 1e-5f);                              \
        int x0_ = max((cx) - R_, 0), x1_ = min((cx) + R_, (P).nx - 1);                 \
        for (int dz_ = -R_; dz_ <= R_; ++dz_) {                                        \
            int z_ = (cz) + dz_;                                                       \
            if (z_ < 0 || z_ >= (P).nz) continue;                                      \
            const float za_ = (fa).z - (float)dz_ * (P).sf;                            \
            for (int dy_ = -R_; dy_ <= R_; ++dy_) {                                    \
                int y_ = (cy) + dy_;                                                   \
                if (y_ < 0 || y_ >= (P).ny) continue;                                  \
                const float ya_ = (fa).y - (float)dy_ * (P).sf;                        \
                int row_ = (P).nx * (y_ + (P).ny * z_);                                \
                int cut_[4];                                                           \
                for (int u_ = 0; u_ < 2 * R_; ++u_)                                    \
                    cut_[u_] = (start)[row_ + min(max((cx) - R_ + 1 + u_, 0), (P).nx)]; \
                int e_ = (start)[row_ + x1_ + 1];                                      \
                for (int j = (start)[row_ + x0_]; j < e_; ++j) {                       \
                    int k_ = -R_;                                                      \
                    for (int u_ = 0; u_ < 2 * R_; ++u_) k_ += j >= cut_[u_] ? 1 : 0;   \
                    const float4 fb_ = (posf)[j];                                      \
                    const float ex_ = (fa).x - (float)k_ * (P).sf - fb_.x;             \
                    const float ey_ = ya_ - fb_.y, ez_ = za_ - fb_.z;                  \
                    if (!(fmaf(ex_, ex_, fmaf(ey_, ey_, ez_ * ez_)) < s2f_)) continue; \
                    { __VA_ARGS__ }                                                    \
                }                                                                      \
            }                                                                          \
        }                                                                              \
    }

// ---- adjoint SU ------------------------------------------------------------

__global__ void k_adj_su_fluid(int nf, size_t N, DevParams P, const int32_t *__restrict__ fstart,
                               const uint32_t *__restrict__ id,
                               const double *__restrict__ lam_next, double *__restrict__ lam_s,
                               double *__restrict__ gF, double *__restrict__ gD,
                               const Scalars *__restrict__ sc)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    const bool euler = ((sc->step + 1) % P.euler_every) == 0;
    const double dt = P.fixed_dt;
    const size_t k = id[i];
    const double *lx = lam_next + 3 * k, *lv = lam_next + 3 * N + 3 * k,
                 *lu = lam_next + 7 * N + 3 * k;
    const double lr = lam_next[6 * N + k], ls = lam_next[10 * N + k];
    double *ox = lam_s + 3 * (size_t)i, *ov = lam_s + 3 * N + 3 * (size_t)i,
           *ou = lam_s + 7 * N + 3 * (size_t)i;
    if (i < fstart[P.ncells]) {
        const double cv = euler ? 1.0 : 2.0;
        for (int d = 0; d < 3; ++d) {
            gF[3 * (size_t)i + d] = 0.5 * dt * dt * lx[d] + cv * dt * lv[d];
            ox[d] = lx[d];
            ov[d] = dt * lx[d] + lu[d] + (euler ? lv[d] : 0.0);
            ou[d] = euler ? 0.0 : lv[d];
        }
        gD[i] = cv * dt * lr;
        lam_s[6 * N + i] = ls + (euler ? lr : 0.0);
        lam_s[10 * N + i] = euler ? 0.0 : lr;
    } else {  // outside the grid: the forward step left the particle unchanged
        for (int d = 0; d < 3; ++d) {
            gF[3 * (size_t)i + d] = 0.0;
            ox[d] = lx[d];
            ov[d] = lv[d];
            ou[d] = lu[d];
        }
        gD[i] = 0.0;
        lam_s[6 * N + i] = lr;
        lam_s[10 * N + i] = ls;
    }
}

__global__ void k_adj_su_boundary(int nf, int nb, size_t N, DevParams P,
                                  const int32_t *__restrict__ bstart,
                                  const uint32_t *__restrict__ bid,
                                  const double *__restrict__ brho, const double *__restrict__ brhom,
                                  const double *__restrict__ bar,
                                  const double *__restrict__ lam_next, double *__restrict__ lam_s,
                                  double *__restrict__ gD, const Scalars *__restrict__ sc)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nb) return;
    const bool euler = ((sc->step + 1) % P.euler_every) == 0;
    const double sdt = P.fixed_dt;
    const size_t k = bid[j];
    const size_t s = (size_t)nf + j;
    const double lr = lam_next[6 * N + k], ls = lam_next[10 * N + k];
    for (int d = 0; d < 3; ++d) {
        lam_s[3 * s + d] = 0.0;
        lam_s[3 * N + 3 * s + d] = 0.0;
        lam_s[7 * N + 3 * s + d] = 0.0;
    }
    if (j < bstart[P.ncells]) {
        // the forward density update, evaluated as in the forward kernel, decides the clamp
        const double dtr = sdt;
        double r = brho[j];
        double nr = euler ? r + dtr * bar[j] : brhom[j] + (2.0 * sdt) * bar[j];
        const double mask = (P.clamp && nr < P.rho0) ? 0.0 : 1.0;
        const double cv = euler ? 1.0 : 2.0;
        gD[s] = cv * sdt * mask * lr;
        lam_s[6 * N + s] = ls + (euler ? mask * lr : 0.0);
        lam_s[10 * N + s] = euler ? 0.0 : mask * lr;
    } else {
        gD[s] = 0.0;
        lam_s[6 * N + s] = lr;
        lam_s[10 * N + s] = ls;
    }
}

// ---- adjoint PI --------------------------------------------------------------

__global__ void __launch_bounds__(kAdjThreads)
k_adj_pi_fluid(int nf, size_t N, DevParams P, const double4_32a *__restrict__ posp,
               const double4_32a *__restrict__ velr, const uint32_t *__restrict__ cell,
               const int32_t *__restrict__ fstart, const double4_32a *__restrict__ bposp,
               const double4_32a *__restrict__ bvelr, const int32_t *__restrict__ bstart,
               const double *__restrict__ gF, const double *__restrict__ gD,
               double *__restrict__ lam_s, double *__restrict__ part,
               const float4 *__restrict__ posf, const float4 *__restrict__ bposf)
{
    __shared__ double red[kAdjThreads / 32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double dal = 0.0;
    if (i < fstart[P.ncells]) {
        const double4_32a pa = posp[i], va = velr[i];
        const PartTerms ta = part_terms(P, va.w, pa.w);
        const double gFx = gF[3 * (size_t)i], gFy = gF[3 * (size_t)i + 1],
                     gFz = gF[3 * (size_t)i + 2], gDa = gD[i];
        SelfAdj l = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        const double s2 = 4.0 * P.h * P.h;
        int cx, cy, cz;
        cell_coords(P, cell[i], &cx, &cy, &cz);
        const float4 fa = posf[i];
        // fluid neighbours: F-F in both directions
        FOR_RUNS_F(P, cx, cy, cz, fstart, fa, posf, j, {
            if (j == i) continue;
            const double4_32a pb = posp[j];
            const double rx = pa.x - pb.x, ry = pa.y - pb.y, rz = pa.z - pb.z;
            const double r2 = rx * rx + ry * ry + rz * rz;
            if (!(r2 < s2)) continue;
            const double4_32a vb = velr[j];
            pair_adj<true>(P, rx, ry, rz, va.x - vb.x, va.y - vb.y, va.z - vb.z, ta, vb.w, pb.w,
                           sound_of(P, vb.w), gFx, gFy, gFz, gF[3 * (size_t)j],
                           gF[3 * (size_t)j + 1], gF[3 * (size_t)j + 2], gDa + gD[j], l);
        })
        // boundary neighbours: F-B (momentum + continuity) and B-F (continuity)
        FOR_RUNS_F(P, cx, cy, cz, bstart, fa, bposf, j, {
            const double4_32a pb = bposp[j];
            const double rx = pa.x - pb.x, ry = pa.y - pb.y, rz = pa.z - pb.z;
            const double r2 = rx * rx + ry * ry + rz * rz;
            if (!(r2 < s2)) continue;
            const double rho_b = bvelr[j].w;
            pair_adj<false>(P, rx, ry, rz, va.x, va.y, va.z, ta, rho_b, pb.w, sound_of(P, rho_b),
                            gFx, gFy, gFz, 0.0, 0.0, 0.0, gDa + gD[(size_t)nf + j], l);
        })
        dal = l.alpha;
        double *ox = lam_s + 3 * (size_t)i, *ov = lam_s + 3 * N + 3 * (size_t)i;
        ox[0] += l.rx; ox[1] += l.ry; ox[2] += l.rz;
        ov[0] += l.vx; ov[1] += l.vy; ov[2] += l.vz;
        lam_s[6 * N + i] += l.rho;
    }
    // deterministic block sum of dJ/dalpha
    for (int o = 16; o > 0; o >>= 1) dal += __shfl_xor_sync(0xffffffffu, dal, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dal;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kAdjThreads / 32; ++w) s += red[w];
        part[blockIdx.x] = s;
    }
}

// boundary particle j: the F-B pairs it sources give it a density adjoint
__global__ void __launch_bounds__(kAdjThreads)
k_adj_pi_boundary(int nf, int nb, size_t N, DevParams P, const double4_32a *__restrict__ bposp,
                  const double4_32a *__restrict__ bvelr, const uint32_t *__restrict__ bcell,
                  const int32_t *__restrict__ bstart, const double4_32a *__restrict__ posp,
                  const double4_32a *__restrict__ velr, const int32_t *__restrict__ fstart,
                  const double *__restrict__ gF, const double *__restrict__ gD,
                  double *__restrict__ lam_s, const float4 *__restrict__ posf,
                  const float4 *__restrict__ bposf)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nb || j >= bstart[P.ncells]) return;
    const double4_32a pb = bposp[j], vb = bvelr[j];
    const PartTerms tb = part_terms(P, vb.w, pb.w);
    const double s2 = 4.0 * P.h * P.h;
    int cx, cy, cz;
    cell_coords(P, bcell[j], &cx, &cy, &cz);
    double lr = 0.0;
    const float4 fb = bposf[j];
    FOR_RUNS_F(P, cx, cy, cz, fstart, fb, posf, i, {
        const double4_32a pa = posp[i];
        const double rx = pa.x - pb.x, ry = pa.y - pb.y, rz = pa.z - pb.z;
        const double r2 = rx * rx + ry * ry + rz * rz;
        if (!(r2 < s2)) continue;
        const double4_32a va = velr[i];
        lr += pair_adj_rho_b(P, rx, ry, rz, va.x, va.y, va.z, tb, va.w, sound_of(P, va.w),
                             gF[3 * (size_t)i], gF[3 * (size_t)i + 1], gF[3 * (size_t)i + 2]);
    })
    lam_s[6 * N + (size_t)nf + j] += lr;
}

// sorted-order adjoint -> persistent-id order
__global__ void k_adj_out(int nf, int nb, size_t N, const uint32_t *__restrict__ id,
                          const uint32_t *__restrict__ bid, const double *__restrict__ lam_s,
                          double *__restrict__ lam)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf + nb) return;
    size_t k = i < nf ? id[i] : bid[i - nf];
    for (int d = 0; d < 3; ++d) {
        lam[3 * k + d] = lam_s[3 * (size_t)i + d];
        lam[3 * N + 3 * k + d] = lam_s[3 * N + 3 * (size_t)i + d];
        lam[7 * N + 3 * k + d] = lam_s[7 * N + 3 * (size_t)i + d];
    }
    lam[6 * N + k] = lam_s[6 * N + i];
    lam[10 * N + k] = lam_s[10 * N + i];
}

// ---- adjoint PI on the warp work items (cells of edge 2h or more) -------------
//
// The candidate search of the float64 PI kernel (warp_items.cuh): every lane
// walks the hits of its own target and sums pair_adj (fluid targets, F-F and
// F-B with their B-F counterparts) or pair_adj_rho_b (boundary targets) in
// the item's fixed order.  dJ/dalpha of an item is summed over its lanes in a
// fixed order and stored at its first target, so the total does not depend on
// the order the items are processed in.

constexpr int kAdjWarps = 4;

__device__ __forceinline__ void adj_fluid_item(
    const DevParams &P, witems::Smem &S, int lane, uint32_t it, int nf, size_t N,
    const uint32_t *__restrict__ items, const double4_32a *__restrict__ posp,
    const double4_32a *__restrict__ velr, const float4 *__restrict__ posf,
    const uint32_t *__restrict__ cell, const int32_t *__restrict__ fstart,
    const double4_32a *__restrict__ bposp, const double4_32a *__restrict__ bvelr,
    const float4 *__restrict__ bposf, const int32_t *__restrict__ bstart,
    const double *__restrict__ gF, const double *__restrict__ gD, double *__restrict__ lam_s,
    double *__restrict__ part, double *slots)
{
    const witems::Item I = witems::item_of(P, items, it, cell, lane);
    const int i = I.i;
    const witems::Frame Fr = witems::frame_of(P, I, posf[i], cell, 4.0004f);
    const double s2 = 4.0 * P.h * P.h;
    // the target this lane works for in the balanced walk, its sums (w), and
    // the total of the lane's own target (l)
    int wi = i;
    double4_32a pa, va;
    PartTerms ta;
    double gFx = 0.0, gFy = 0.0, gFz = 0.0, gDa = 0.0;
    SelfAdj w = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    SelfAdj l = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    witems::for_each_hit_balanced<true>(
        P, S, lane, I, Fr, fstart, posf, bstart, bposf, cell,
        [&](int t) {
            wi = I.i0 + t;
            pa = posp[wi];
            va = velr[wi];
            ta = part_terms(P, va.w, pa.w);
            gFx = gF[3 * (size_t)wi];
            gFy = gF[3 * (size_t)wi + 1];
            gFz = gF[3 * (size_t)wi + 2];
            gDa = gD[wi];
            w = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        },
        [&](int j, bool blist) {
            if (!blist) {
                if (j == wi) return;
                const double4_32a pb = posp[j];
                const double rx = pa.x - pb.x, ry = pa.y - pb.y, rz = pa.z - pb.z;
                if (!(rx * rx + ry * ry + rz * rz < s2)) return;
                const double4_32a vb = velr[j];
                pair_adj<true>(P, rx, ry, rz, va.x - vb.x, va.y - vb.y, va.z - vb.z, ta, vb.w,
                               pb.w, sound_of(P, vb.w), gFx, gFy, gFz, gF[3 * (size_t)j],
                               gF[3 * (size_t)j + 1], gF[3 * (size_t)j + 2], gDa + gD[j], w);
            } else {
                const double4_32a pb = bposp[j];
                const double rx = pa.x - pb.x, ry = pa.y - pb.y, rz = pa.z - pb.z;
                if (!(rx * rx + ry * ry + rz * rz < s2)) return;
                const double rho_b = bvelr[j].w;
                pair_adj<false>(P, rx, ry, rz, va.x, va.y, va.z, ta, rho_b, pb.w,
                                sound_of(P, rho_b), gFx, gFy, gFz, 0.0, 0.0, 0.0,
                                gDa + gD[(size_t)nf + j], w);
            }
        },
        [&](int, int slot) {
            double *ps = slots + 8 * slot;
            ps[0] = w.rx; ps[1] = w.ry; ps[2] = w.rz;
            ps[3] = w.vx; ps[4] = w.vy; ps[5] = w.vz;
            ps[6] = w.rho; ps[7] = w.alpha;
        },
        [&](int slot) {
            const double *ps = slots + 8 * slot;
            l.rx += ps[0]; l.ry += ps[1]; l.rz += ps[2];
            l.vx += ps[3]; l.vy += ps[4]; l.vz += ps[5];
            l.rho += ps[6]; l.alpha += ps[7];
        });
    if (I.active) {
        double *ox = lam_s + 3 * (size_t)i, *ov = lam_s + 3 * N + 3 * (size_t)i;
        ox[0] += l.rx; ox[1] += l.ry; ox[2] += l.rz;
        ov[0] += l.vx; ov[1] += l.vy; ov[2] += l.vz;
        lam_s[6 * N + i] += l.rho;
    }
    double a = I.active ? l.alpha : 0.0;
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) part[I.i0] = a;
}

__device__ __forceinline__ void adj_boundary_item(
    const DevParams &P, witems::Smem &S, int lane, uint32_t it, int nf, size_t N,
    const uint32_t *__restrict__ items, const double4_32a *__restrict__ bposp,
    const double4_32a *__restrict__ bvelr, const float4 *__restrict__ bposf,
    const uint32_t *__restrict__ bcell, const int32_t *__restrict__ bstart,
    const double4_32a *__restrict__ posp, const double4_32a *__restrict__ velr,
    const float4 *__restrict__ posf, const uint32_t *__restrict__ cell,
    const int32_t *__restrict__ fstart, const double *__restrict__ gF,
    double *__restrict__ lam_s, double *slots)
{
    const witems::Item I = witems::item_of(P, items, it, bcell, lane);
    const int j = I.i;
    const witems::Frame Fr = witems::frame_of(P, I, bposf[j], bcell, 4.0004f);
    const double s2 = 4.0 * P.h * P.h;
    // balanced walk: the boundary target this lane works for, its sum (w) and
    // the total of the lane's own target (lr)
    int wj = j;
    double4_32a pb;
    PartTerms tb;
    double w = 0.0, lr = 0.0;
    witems::for_each_hit_balanced<false>(
        P, S, lane, I, Fr, fstart, posf, bstart, bposf, cell,
        [&](int t) {
            wj = I.i0 + t;
            pb = bposp[wj];
            tb = part_terms(P, bvelr[wj].w, pb.w);
            w = 0.0;
        },
        [&](int i, bool) {
            const double4_32a pa = posp[i];
            const double rx = pa.x - pb.x, ry = pa.y - pb.y, rz = pa.z - pb.z;
            if (!(rx * rx + ry * ry + rz * rz < s2)) return;
            const double4_32a va = velr[i];
            w += pair_adj_rho_b(P, rx, ry, rz, va.x, va.y, va.z, tb, va.w, sound_of(P, va.w),
                                gF[3 * (size_t)i], gF[3 * (size_t)i + 1], gF[3 * (size_t)i + 2]);
        },
        [&](int, int slot) { slots[8 * slot] = w; },
        [&](int slot) { lr += slots[8 * slot]; });
    if (I.active) lam_s[6 * N + (size_t)nf + j] += lr;
}

// One queue: the fluid items, then the boundary items, over a persistent grid.
__global__ void __launch_bounds__(kAdjWarps * 32)
k_adj_pi_w(int nf, size_t N, DevParams P, const uint32_t *__restrict__ items_f,
           const uint32_t *__restrict__ items_b, const uint32_t *__restrict__ ctr, int use_b,
           uint32_t *__restrict__ next_p, const double4_32a *__restrict__ posp,
           const double4_32a *__restrict__ velr, const float4 *__restrict__ posf,
           const uint32_t *__restrict__ cell, const int32_t *__restrict__ fstart,
           const double4_32a *__restrict__ bposp, const double4_32a *__restrict__ bvelr,
           const float4 *__restrict__ bposf, const uint32_t *__restrict__ bcell,
           const int32_t *__restrict__ bstart, const double *__restrict__ gF,
           const double *__restrict__ gD, double *__restrict__ lam_s, double *__restrict__ part)
{
    __shared__ witems::Smem smem[kAdjWarps];
    __shared__ double slotsm[kAdjWarps][8 * witems::NSLOT];   // balanced-walk partial sums
    const int lane = threadIdx.x & 31;
    witems::Smem &S = smem[threadIdx.x >> 5];
    double *slots = slotsm[threadIdx.x >> 5];
    const uint32_t nfi = ctr[0];
    const uint32_t n_items = nfi + (use_b ? ctr[3] : 0u);
    for (;;) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(next_p, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;
        if (it < nfi)
            adj_fluid_item(P, S, lane, it, nf, N, items_f, posp, velr, posf, cell, fstart, bposp,
                           bvelr, bposf, bstart, gF, gD, lam_s, part, slots);
        else
            adj_boundary_item(P, S, lane, it - nfi, nf, N, items_b, bposp, bvelr, bposf, bcell,
                              bstart, posp, velr, posf, cell, fstart, gF, lam_s, slots);
    }
}

// dJ/dalpha += sum of part[0 .. n): one block, each thread sums a fixed strided
// subset in order, then a fixed-order tree: deterministic.
__global__ void __launch_bounds__(1024) k_adj_alpha(const double *__restrict__ part, int n,
                                                    double *dalpha)
{
    __shared__ double t[1024];
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += 1024) s += part[k];
    t[threadIdx.x] = s;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) t[threadIdx.x] += t[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *dalpha += t[0];
}

// ---- sensor objective ---------------------------------------------------------

__device__ __forceinline__ double kernel_w(const DevParams &P, double r)
{
    double aD = P.kA64 * P.h * P.h;
    double q = r * P.invh;
    if (q < 1.0) return aD * (1.0 - 1.5 * q * q + 0.75 * q * q * q);
    if (q < 2.0) {
        double t = 2.0 - q;
        return aD * 0.25 * t * t * t;
    }
    return 0.0;
}

__device__ __forceinline__ double pressure_of(const DevParams &P, double rho)
{
    double r = rho * P.inv_rho0;
    double pw;
    if (P.gamma_is_7) {
        double r3 = r * r * r;
        pw = r3 * r3 * r;
    } else {
        pw = pow(r, P.gamma);
    }
    return P.B * (pw - 1.0);
}

__device__ __forceinline__ int sensor_axis(double x, double mn, double inv_s, int n)
{
    double t = floor((x - mn) * inv_s);
    if (!(t >= 0.0) || t >= (double)n) return -1;
    return (int)t;
}

// One warp per sensor: Shepard sum over the fluid particles within 2h.
template <typename Real>
__global__ void k_sensor(int S, DevParams P, const double *__restrict__ spos,
                         const double *__restrict__ x, const double *__restrict__ y,
                         const double *__restrict__ z, const typename Real4T<Real>::T *__restrict__ V,
                         const int32_t *__restrict__ fstart, double *__restrict__ p_out,
                         double *__restrict__ den_out)
{
    const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= S) return;
    const double xs = spos[3 * s], ys = spos[3 * s + 1], zs = spos[3 * s + 2];
    int cx = sensor_axis(xs, P.dom_min[0], P.inv_s, P.nx);
    int cy = sensor_axis(ys, P.dom_min[1], P.inv_s, P.ny);
    int cz = sensor_axis(zs, P.dom_min[2], P.inv_s, P.nz);
    double num = 0.0, den = 0.0;
    if (cx >= 0 && cy >= 0 && cz >= 0) {
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
                int e = fstart[row + x1 + 1];
                for (int b = fstart[row + x0] + lane; b < e; b += 32) {
                    double dx = xs - x[b], dy2 = ys - y[b], dz2 = zs - z[b];
                    double r2 = dx * dx + dy2 * dy2 + dz2 * dz2;
                    if (r2 < s2) {
                        double rb = (double)V[b].w;
                        double w = kernel_w(P, sqrt(r2)) * P.mass / rb;
                        num += w * pressure_of(P, rb);
                        den += w;
                    }
                }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_xor_sync(0xffffffffu, num, o);
        den += __shfl_xor_sync(0xffffffffu, den, o);
    }
    if (lane == 0) {
        p_out[s] = den > 0.0 ? num / den : 0.0;
        if (den_out) den_out[s] = den;
    }
}

// dJ/d(x_b, rho_b) of J = sum_s g_s P_s, added into lam (id order), one thread
// per fluid particle (the sensor set is small):
//   dP_s/drho_b = (w_sb c_b^2 - (P_b - P_s) w_sb / rho_b) / den_s
//   dP_s/dx_b   = (P_b - P_s) (m / rho_b) F(r_sb) (x_b - x_s) / den_s
__global__ void k_sensor_adj(int nf, size_t N, int S, DevParams P, const double *__restrict__ spos,
                             const double *__restrict__ g, const double *__restrict__ ps,
                             const double *__restrict__ dens, const double *__restrict__ x,
                             const double *__restrict__ y, const double *__restrict__ z,
                             const double4_32a *__restrict__ V, const uint32_t *__restrict__ id,
                             const int32_t *__restrict__ fstart, double *__restrict__ lam)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf || i >= fstart[P.ncells]) return;
    const double xi = x[i], yi = y[i], zi = z[i], rb = V[i].w;
    const double Pb = pressure_of(P, rb), cb = sound_of(P, rb);
    const double s2 = 4.0 * P.h * P.h;
    double lx = 0, ly = 0, lz = 0, lr = 0;
    for (int s = 0; s < S; ++s) {
        double dx = xi - spos[3 * s], dy = yi - spos[3 * s + 1], dz = zi - spos[3 * s + 2];
        double r2 = dx * dx + dy * dy + dz * dz;
        if (!(r2 < s2) || !(dens[s] > 0.0)) continue;
        double r = sqrt(r2);
        double w = kernel_w(P, r) * P.mass / rb;
        double coef = g[s] / dens[s];
        double dPs = Pb - ps[s];
        lr += coef * (w * cb * cb - dPs * w / rb);
        double q = r * P.invh;
        double F = q < 1.0 ? P.kA64 * (-3.0 + 2.25 * q)
                           : P.kB64 * (2.0 - q) * (2.0 - q) / r;
        double f = coef * dPs * (P.mass / rb) * F;
        lx += f * dx;
        ly += f * dy;
        lz += f * dz;
    }
    const size_t k = id[i];
    lam[3 * k] += lx;
    lam[3 * k + 1] += ly;
    lam[3 * k + 2] += lz;
    lam[6 * N + k] += lr;
}

template <typename Real>
int sensor_launch(sph_ctx *ctx, const double *spos, int S, double *p_out, double *den_out)
{
    Workspace &w = ctx->w;
    const int c = ctx->cur;
    const int T = 128;
    SPH_LAUNCH(ctx, k_sensor<Real>, (S * 32 + T - 1) / T, T, 0, ctx->stream, S, ctx->dp, spos,
               w.x[c], w.y[c], w.z[c], (const typename Real4T<Real>::T *)w.V[c], w.fstart, p_out,
               den_out);
    return check_cuda(cudaGetLastError());
}

}  // namespace

// Front of the fluid: the smooth maximum J = tau log sum_a exp(x_a / tau) of
// the fluid x coordinates, computed as m + tau log sum_a exp((x_a - m) / tau)
// with m = max_a x_a (no overflow).  One block, so every sum is formed in the
// same order.  Writes front[0] = m, front[1] = the sum and, if J is given, *J.
__global__ void __launch_bounds__(1024)
k_front(int nf, double tau, const double *__restrict__ x, double *__restrict__ front,
        double *__restrict__ J)
{
    __shared__ double red[32];
    __shared__ double sm;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double m = -INFINITY;
    for (int i = threadIdx.x; i < nf; i += blockDim.x) m = fmax(m, x[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) red[warp] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = red[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
        sm = t;
    }
    __syncthreads();
    m = sm;
    double s = 0.0;
    for (int i = threadIdx.x; i < nf; i += blockDim.x) s += exp((x[i] - m) / tau);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __syncthreads();
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        front[0] = m;
        front[1] = t;
        if (J) *J = m + tau * log(t);
    }
}

// dJ/dx_a of dj * J_front: dj exp((x_a - m) / tau) / sum, added to the
// position adjoint of particle a (persistent-id layout).
__global__ void k_front_adj(int nf, double tau, double dj, const double *__restrict__ x,
                            const uint32_t *__restrict__ id, const double *__restrict__ front,
                            double *__restrict__ lam)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    lam[3 * (size_t)id[i]] += dj * exp((x[i] - front[0]) / tau) / front[1];
}

}  // namespace sph

using namespace sph;

extern "C" int sph_sensor_pressure(sph_ctx *ctx, const double *sensors, int64_t n_sensors,
                                   double *pressure)
{
    if (!ctx || n_sensors < 0 || (n_sensors > 0 && (!sensors || !pressure)))
        return SPH_ERR_INVALID_ARG;
    if (n_sensors > kMaxSensors) return SPH_ERR_TOO_LARGE;
    if (!ctx->nl_valid) return SPH_ERR_SEQUENCE;
    if (n_sensors == 0) return SPH_OK;
    if (ctx->precision == SPH_FP32_SPLIT)
        return sensor_launch<float>(ctx, sensors, (int)n_sensors, pressure, nullptr);
    return sensor_launch<double>(ctx, sensors, (int)n_sensors, pressure, nullptr);
}

extern "C" int sph_sensor_adjoint(sph_ctx *ctx, const double *sensors, int64_t n_sensors,
                                  const double *dj_dp, double *lam)
{
    if (!ctx || n_sensors < 0 || (n_sensors > 0 && (!sensors || !dj_dp || !lam)))
        return SPH_ERR_INVALID_ARG;
    if (ctx->precision != SPH_FP64) return SPH_ERR_INVALID_ARG;
    if (n_sensors > kMaxSensors) return SPH_ERR_TOO_LARGE;
    if (!ctx->nl_valid) return SPH_ERR_SEQUENCE;
    if (n_sensors == 0 || ctx->nf == 0) return SPH_OK;
    Workspace &w = ctx->w;
    int rc = sensor_launch<double>(ctx, sensors, (int)n_sensors, w.sens_p, w.sens_den);
    if (rc) return rc;
    const int c = ctx->cur, nf = (int)ctx->nf;
    const size_t N = (size_t)(ctx->nf + ctx->nb);
    const int T = 128;
    SPH_LAUNCH(ctx, k_sensor_adj, (nf + T - 1) / T, T, 0, ctx->stream, nf, N, (int)n_sensors,
               ctx->dp, sensors, dj_dp, w.sens_p, w.sens_den, w.x[c], w.y[c], w.z[c],
               (const double4_32a *)w.V[c], w.id[c], w.fstart, lam);
    return check_cuda(cudaGetLastError());
}

// Persistent grid of the work-item adjoint kernel: one resident set of CTAs.
int sph::adjoint_setup(sph_ctx *ctx)
{
    int dev = 0, sms = 0, nblk = 0;
    if (check_cuda(cudaGetDevice(&dev))) return SPH_ERR_CUDA;
    if (check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
        return SPH_ERR_CUDA;
    if (check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nblk, k_adj_pi_w,
                                                                kAdjWarps * 32, 0)))
        return SPH_ERR_CUDA;
    ctx->adj_grid = sms * (nblk > 0 ? nblk : 1);
    return SPH_OK;
}

extern "C" int sph_adjoint_step(sph_ctx *ctx, const double *lam_next, double *lam, double *dalpha)
{
    if (!ctx || !lam_next || !lam || !dalpha || lam_next == lam) return SPH_ERR_INVALID_ARG;
    if (ctx->precision != SPH_FP64 || !(ctx->prm.fixed_dt > 0.0) || ctx->dp.tensile)
        return SPH_ERR_INVALID_ARG;
    // forward NL and PI of the loaded state: the neighbour lists, packed inputs
    // and (for the boundary clamp) the density rates of this step
    int rc = sph_neighbour_list(ctx);
    if (!rc) rc = sph_interact(ctx);
    if (rc) return rc;
    Workspace &w = ctx->w;
    cudaStream_t st = ctx->stream;
    const int nf = (int)ctx->nf, nb = (int)ctx->nb, c = ctx->cur;
    const size_t N = (size_t)(nf + nb);
    const int T = kAdjThreads;
    const int blocks_f = (nf + T - 1) / T;
    if (nf > 0)
        SPH_LAUNCH(ctx, k_adj_su_fluid, blocks_f, T, 0, st, nf, N, ctx->dp, w.fstart, w.id[c],
                   lam_next, w.adj_lam, w.adj_gF, w.adj_gD, w.sc);
    if (nb > 0)
        SPH_LAUNCH(ctx, k_adj_su_boundary, (nb + T - 1) / T, T, 0, st, nf, nb, N, ctx->dp,
                   w.bstart, w.bid, (const double *)w.brho, (const double *)w.brhom,
                   (const double *)w.bar, lam_next, w.adj_lam, w.adj_gD, w.sc);
    int nparts = blocks_f;
    if (ctx->dp.reach == 1 && nf > 0) {
        // work items of this step's NL (cells of edge 2h or more)
        if (check_cuda(cudaMemsetAsync(w.adj_part, 0, sizeof(double) * (size_t)nf, st)))
            return SPH_ERR_CUDA;
        if (check_cuda(cudaMemsetAsync(&w.ctr[1], 0, sizeof(uint32_t), st))) return SPH_ERR_CUDA;
        SPH_LAUNCH(ctx, k_adj_pi_w, ctx->adj_grid, kAdjWarps * 32, 0, st, nf, N, ctx->dp,
                   w.items_f, w.items_b, w.ctr, nb > 0 ? 1 : 0, &w.ctr[1],
                   (const double4_32a *)w.posp, (const double4_32a *)velr_of(ctx), w.posf, w.cell,
                   w.fstart, (const double4_32a *)w.bposp, (const double4_32a *)w.bvelr, w.bposf,
                   w.bcell, w.bstart, w.adj_gF, w.adj_gD, w.adj_lam, w.adj_part);
        nparts = nf;
    } else {
        if (nf > 0)
            SPH_LAUNCH(ctx, k_adj_pi_fluid, blocks_f, T, 0, st, nf, N, ctx->dp,
                       (const double4_32a *)w.posp, (const double4_32a *)velr_of(ctx), w.cell, w.fstart,
                       (const double4_32a *)w.bposp, (const double4_32a *)w.bvelr, w.bstart,
                       w.adj_gF, w.adj_gD, w.adj_lam, w.adj_part, w.posf, w.bposf);
        if (nb > 0 && nf > 0)
            SPH_LAUNCH(ctx, k_adj_pi_boundary, (nb + T - 1) / T, T, 0, st, nf, nb, N, ctx->dp,
                       (const double4_32a *)w.bposp, (const double4_32a *)w.bvelr, w.bcell,
                       w.bstart, (const double4_32a *)w.posp, (const double4_32a *)velr_of(ctx),
                       w.fstart, w.adj_gF, w.adj_gD, w.adj_lam, w.posf, w.bposf);
    }
    if (N > 0)
        SPH_LAUNCH(ctx, k_adj_out, (unsigned)((N + T - 1) / T), T, 0, st, nf, nb, N, w.id[c],
                   w.bid, w.adj_lam, lam);
    if (nf > 0) SPH_LAUNCH(ctx, k_adj_alpha, 1, 1024, 0, st, w.adj_part, nparts, dalpha);
    return check_cuda(cudaGetLastError());
}

extern "C" int sph_front_position(sph_ctx *ctx, double tau, double *J)
{
    if (!ctx || !J || !(tau > 0.0) || ctx->nf <= 0) return SPH_ERR_INVALID_ARG;
    Workspace &w = ctx->w;
    SPH_LAUNCH(ctx, k_front, 1, 1024, 0, ctx->stream, (int)ctx->nf, tau, w.x[ctx->cur], w.front, J);
    return check_cuda(cudaGetLastError());
}

extern "C" int sph_front_adjoint(sph_ctx *ctx, double tau, double dj, double *lam)
{
    if (!ctx || !lam || !(tau > 0.0) || ctx->nf <= 0) return SPH_ERR_INVALID_ARG;
    if (ctx->precision != SPH_FP64) return SPH_ERR_INVALID_ARG;
    Workspace &w = ctx->w;
    const int nf = (int)ctx->nf, c = ctx->cur, T = 256;
    SPH_LAUNCH(ctx, k_front, 1, 1024, 0, ctx->stream, nf, tau, w.x[c], w.front, (double *)nullptr);
    SPH_LAUNCH(ctx, k_front_adj, (nf + T - 1) / T, T, 0, ctx->stream, nf, tau, dj, w.x[c], w.id[c],
               w.front, lam);
    return check_cuda(cudaGetLastError());
}
