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
// factors -m kB and m kB once per target.  cpa = -alpha c_a is a per-target
// constant; -alpha c_b is kcf rho_b^3 (Tait sound speed with gamma = 7,
// c = c0 (rho / rho0)^3).
#pragma once

#include "sph_internal.cuh"

namespace sph {

// Approximate reciprocal and reciprocal square root (PTX rcp.approx and
// rsqrt.approx, relative error about 2^-23).  Their arguments in the pair
// terms are normal numbers (densities, r'^2 + eta^2/h^2 >= eta^2/h^2, r'^2
// clamped at 1e-30), so flushing subnormals changes nothing.
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
// {vx, vy, vz, rho}.
template <bool MOMENTUM, bool TENSILE>
__device__ __forceinline__ void pair_terms32(const DevParams &P, float rx, float ry, float rz,
                                             float pra, const float4 &va, float cpa,
                                             const float4 &vb, float prb, float &coef,
                                             float &vdr_out, float &F_out, float &vis)
{
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
        if (TENSILE) {
            const float Pi = cc * fminf(mu, 0.0f) * rcp_approx(va.w + vb.w) +
                             tensile32(P, q, pra, prb);
            coef = (pra + prb + Pi) * F;
        } else {
            coef = fmaf(cc * fminf(mu, 0.0f), rcp_approx(va.w + vb.w), pra + prb) * F;
        }
    }
    vdr_out = vdr;
    F_out = F;
    vis = fmaxf(vis, fabsf(mu));
}

// pair_terms32 accumulated into the sums of target a.
template <bool MOMENTUM, bool TENSILE>
__device__ __forceinline__ void pair_acc32(const DevParams &P, float rx, float ry, float rz,
                                           float pra, const float4 &va, float cpa,
                                           const float4 &vb, float prb, Acc32 &o)
{
    float coef = 0.0f, vdr, F;
    pair_terms32<MOMENTUM, TENSILE>(P, rx, ry, rz, pra, va, cpa, vb, prb, coef, vdr, F, o.vis);
    if (MOMENTUM) {
        o.ax = fmaf(coef, rx, o.ax);
        o.ay = fmaf(coef, ry, o.ay);
        o.az = fmaf(coef, rz, o.az);
    }
    o.ar = fmaf(vdr, F, o.ar);
}

}  // namespace sph
