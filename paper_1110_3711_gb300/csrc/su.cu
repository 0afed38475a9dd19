// SU stage (Section 4.1, Table 1 of the paper): time step and integration.
//
// The variable time step (Monaghan & Kos) uses the three maxima PI and NL left
// in device memory:
//   dt = CFL * min( sqrt(h / max|f|),  h / (max c + max |h v.r/(r^2+eta^2)|) )
// computed in float64 once per block from the same bits, so every block and
// the finaliser agree exactly.  Verlet (Table 1) with an Euler step when
// (step + 1) % N_s == 0:
//   v^{n+1} = v^{n-1} + 2 dt F^n  (Euler: v^n + dt F^n),  same for rho with D^n
//   x^{n+1} = x^n + dt v^n + dt^2 F^n / 2   (always float64)
// Boundary particles update rho only and never drop below rho0 (dynamic
// boundaries).  k_finalize then advances time and step and clears the maxima.
// HBM-bound: one read and one write of the state per particle.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sph_internal.cuh"

namespace sph {

__device__ __forceinline__ double step_dt(const DevParams &P, const Scalars *sc)
{
    if (P.fixed_dt > 0.0) return P.fixed_dt;
    double f = sqrt(__longlong_as_double((long long)sc->mx.f2));
    double dtf = sqrt(P.h / f);
    double dtcv = P.h / (__longlong_as_double((long long)sc->mx.c) +
                         __longlong_as_double((long long)sc->mx.visc));
    return P.cfl * fmin(dtf, dtcv);
}

// Exact float -> double through the bit pattern (exponent rebiased,
// significand widened), so the split form's position increments reach the
// float64 accumulation without a conversion on the float64 unit, the scarce
// resource of this kernel.  Subnormal floats (below 1.2e-38) become 0; inf
// and NaN stay inf and NaN.
__device__ __forceinline__ double widen(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xffu;
    const uint32_t sign = u & 0x80000000u;
    if (e == 0u) return __hiloint2double((int)sign, 0);
    const uint32_t ex = e == 255u ? 0x7ffu : e + 896u;
    return __hiloint2double((int)(sign | (ex << 20) | ((u & 0x7fffffu) >> 3)), (int)(u << 29));
}
__device__ __forceinline__ double widen(double f) { return f; }

// Fluid particles in blocks [0, fblocks), boundary particles after them.
template <typename Real>
__global__ void __launch_bounds__(256)
k_su(int nf, int nb, int fblocks, DevParams P, const int32_t *__restrict__ fstart,
     const int32_t *__restrict__ bstart, double *__restrict__ x, double *__restrict__ y,
     double *__restrict__ z, typename Real4T<Real>::T *__restrict__ V,
     typename Real4T<Real>::T *__restrict__ VM, const typename Real4T<Real>::T *__restrict__ acc,
     Real *__restrict__ brho, Real *__restrict__ brhom, const Real *__restrict__ bar, Scalars *sc)
{
    typedef typename Real4T<Real>::T R4;
    // dt and its multiples in the precision of the form, once per block
    __shared__ Real sdt[3];
    __shared__ int seuler;
    if (threadIdx.x == 0) {
        const double dt = step_dt(P, sc);
        sdt[0] = (Real)dt;
        sdt[1] = (Real)(2.0 * dt);
        sdt[2] = (Real)(0.5 * dt * dt);
        seuler = ((sc->step + 1) % P.euler_every) == 0;
    }
    __syncthreads();
    const Real dtr = sdt[0], dt2 = sdt[1], hdt2 = sdt[2];
    bool nan = false;
    if ((int)blockIdx.x < fblocks) {
        const int i = blockIdx.x * blockDim.x + threadIdx.x;
        if (i < nf && i < fstart[P.ncells]) {
            const R4 f = acc[i];
            const R4 v = V[i];
            // x^{n+1} = x^n + (dt v^n + dt^2/2 F^n): the increment in the precision
            // of the form, the accumulation always in float64
            x[i] = x[i] + widen(dtr * v.x + hdt2 * f.x);
            y[i] = y[i] + widen(dtr * v.y + hdt2 * f.y);
            z[i] = z[i] + widen(dtr * v.z + hdt2 * f.z);
            R4 nv;
            if (seuler) {
                nv.x = v.x + dtr * f.x;
                nv.y = v.y + dtr * f.y;
                nv.z = v.z + dtr * f.z;
                nv.w = v.w + dtr * f.w;
            } else {
                const R4 u = VM[i];
                nv.x = u.x + dt2 * f.x;
                nv.y = u.y + dt2 * f.y;
                nv.z = u.z + dt2 * f.z;
                nv.w = u.w + dt2 * f.w;
            }
            VM[i] = v;
            V[i] = nv;
            nan = !(nv.w == nv.w) || !(nv.x == nv.x) || !(nv.y == nv.y) || !(nv.z == nv.z);
        }
    } else {
        const int i = (blockIdx.x - fblocks) * blockDim.x + threadIdx.x;
        if (i < nb && i < bstart[P.ncells]) {
            Real r = brho[i];
            Real nr = seuler ? r + dtr * bar[i] : brhom[i] + dt2 * bar[i];
            if (P.clamp && nr < (Real)P.rho0) nr = (Real)P.rho0;
            brhom[i] = r;
            brho[i] = nr;
            nan = !(nr == nr);
        }
    }
    if (nan) atomicOr(&sc->flags, SPH_FLAG_NAN);
}

// One thread, after the update: advance time and step, clear the maxima.
__global__ void k_finalize(DevParams P, Scalars *sc)
{
    double dt = step_dt(P, sc);
    sc->dt_last = dt;
    sc->time += dt;
    sc->step += 1;
    sc->mx.f2 = 0ull;
    sc->mx.c = 0ull;
    sc->mx.visc = 0ull;
    if (!(dt >= 1e-12)) atomicOr(&sc->flags, SPH_FLAG_DT_TOO_SMALL);
}

template <typename Real>
static int su_t(sph_ctx *ctx)
{
    Workspace &w = ctx->w;
    cudaStream_t st = ctx->stream;
    int nf = (int)ctx->nf, nb = (int)ctx->nb;
    int c = ctx->cur;
    const int T = 256;
    const int fblocks = (nf + T - 1) / T, bblocks = (nb + T - 1) / T;
    SPH_LAUNCH(ctx, k_su<Real>, fblocks + bblocks > 0 ? fblocks + bblocks : 1, T, 0, st, nf, nb,
               fblocks, ctx->dp, w.fstart, w.bstart, w.x[c], w.y[c], w.z[c],
               (typename Real4T<Real>::T *)w.V[c], (typename Real4T<Real>::T *)w.VM[c],
               (const typename Real4T<Real>::T *)w.acc, (Real *)w.brho, (Real *)w.brhom,
               (const Real *)w.bar, w.sc);
    SPH_LAUNCH(ctx, k_finalize, 1, 1, 0, st, ctx->dp, w.sc);
    return check_cuda(cudaGetLastError());
}

int su_launch(sph_ctx *ctx)
{
    if (ctx->precision == SPH_FP32_SPLIT) return su_t<float>(ctx);
    return su_t<double>(ctx);
}

}  // namespace sph
