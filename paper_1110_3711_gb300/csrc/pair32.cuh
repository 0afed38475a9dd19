// Pair terms of the float32 PI kernels (SPH_FP32_SPLIT), shared by the warp
// kernel (pi32.cu), its symmetric variant (pi32_sym.cu) and the
// thread-per-particle kernels (pi32_thread.cu).
//
// One ordered pair a <- b of the oracle's interaction (cubic-spline gradient,
// Tait pressure, artificial viscosity of Monaghan 1992, continuity; Table 1),
// in units of h.  With r' = r_ab / h and q = |r'|, the kernel gradient is
// grad_a W = F r_ab with F = (kB / h) F'',
//   F'' = (kA h / kB)(2.25 q - 3)   for q < 1,   F'' = (2 - q)^2 / q   for 1 <= q < 2,
// so that
//   momentum:    -(P_a/rho_a^2 + P_b/rho_b^2 + Pi_ab) F r_ab  = -kB (...) F'' r'
//   continuity:   v_ab . F r_ab                               =  kB (v_ab . r') F''
//   viscosity:    mu_ab = h v_ab.r_ab / (r^2 + eta^2)        =  v_ab.r' / (q^2 + eta^2/h^2)
//   Pi_ab = -alpha (c_a + c_b) mu_ab / (rho_a + rho_b)  for mu_ab < 0, else 0.
// The kernels sum (...) F'' r' and (v_ab . r') F'' and apply the constant
// factors -m kB and m kB once per target.  The float32 form needs gamma = 7,
// whose Tait sound speed is c = c0 (rho / rho0)^3; with
// a^3 + b^3 = (a + b)(a^2 - a b + b^2) the viscosity factor is
//   -alpha (c_a + c_b) / (rho_a + rho_b) = kcf (rho_a^2 - rho_a rho_b + rho_b^2),
// kcf = -alpha c0 / rho0^3, so the pair needs no reciprocal of rho_a + rho_b;
// rho2a = rho_a^2 is a per-target constant.
#pragma once

#include "sph_internal.cuh"

namespace sph {

// Approximate reciprocal and reciprocal square root (PTX rcp.approx and
// rsqrt.approx, relative error about 2^-23).  Their arguments in the pair
// terms are normal numbers (r'^2 + eta^2/h^2 >= eta^2/h^2, r'^2 + 1e-30), so
// flushing subnormals changes nothing.
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

// Sums of one target: momentum (x, y, z), continuity and max |mu|.
struct Acc32 {
    float ax, ay, az, ar, vis;
};

// Tensile correction of Monaghan (2000): R_ab (W(r) / W(dp))^n, with
// R_ab = eps_pos (P_a/rho_a^2 + P_b/rho_b^2) for two positive pressures and
// eps (|P|/rho^2 summed over the negative ones) otherwise.
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

// The terms of pair a <- b from r' = (rx, ry, rz) (units of h):
//   coef = (P_a/rho_a^2 + P_b/rho_b^2 + Pi_ab [+ T_ab]) F''   (MOMENTUM only)
//   vdr  = v_ab . r',  F = F''  (the continuity term is vdr F)
// and vis = max(vis, |mu_ab|).  pra, prb: P/rho^2 of a and b; va, vb:
// {vx, vy, vz, rho}; rho2a = rho_a^2.
template <bool MOMENTUM, bool TENSILE>
__device__ __forceinline__ void pair_terms32(const DevParams &P, float rx, float ry, float rz,
                                             float pra, const float4 &va, float rho2a,
                                             const float4 &vb, float prb, float &coef,
                                             float &vdr_out, float &F_out, float &vis)
{
    // 1e-30 keeps the reciprocal square root finite for r = 0 (the pair a = a,
    // whose terms vanish with r'); for r'^2 of the pairs it is far below rounding
    const float r2 = fmaf(rx, rx, fmaf(ry, ry, fmaf(rz, rz, 1e-30f)));
    const float rinv = rsqrt_approx(r2);
    const float q = r2 * rinv;
    const float t = 2.0f - q;
    const float F = q < 1.0f ? fmaf(P.gw1, q, P.gw0) : t * t * rinv;
    const float dvx = va.x - vb.x, dvy = va.y - vb.y, dvz = va.z - vb.z;
    const float vdr = fmaf(dvx, rx, fmaf(dvy, ry, dvz * rz));
    const float mu = vdr * rcp_approx(r2 + P.eta2_h2f);
    if (MOMENTUM) {
        // rho_b^2 - rho_a rho_b + rho_a^2; rho_b - rho_a is exact (two densities
        // within a factor of two of each other)
        const float kq = P.kcf * fmaf(vb.w, vb.w - va.w, rho2a);
        if (TENSILE) {
            const float Pi = kq * fminf(mu, 0.0f) + tensile32(P, q, pra, prb);
            coef = (pra + prb + Pi) * F;
        } else {
            coef = fmaf(kq, fminf(mu, 0.0f), pra + prb) * F;
        }
    }
    vdr_out = vdr;
    F_out = F;
    vis = fmaxf(vis, fabsf(mu));
}

// pair_terms32 accumulated into the sums of target a.
template <bool MOMENTUM, bool TENSILE>
__device__ __forceinline__ void pair_acc32(const DevParams &P, float rx, float ry, float rz,
                                           float pra, const float4 &va, float rho2a,
                                           const float4 &vb, float prb, Acc32 &o)
{
    float coef = 0.0f, vdr, F;
    pair_terms32<MOMENTUM, TENSILE>(P, rx, ry, rz, pra, va, rho2a, vb, prb, coef, vdr, F, o.vis);
    if (MOMENTUM) {
        o.ax = fmaf(coef, rx, o.ax);
        o.ay = fmaf(coef, ry, o.ay);
        o.az = fmaf(coef, rz, o.az);
    }
    o.ar = fmaf(vdr, F, o.ar);
}

}  // namespace sph
