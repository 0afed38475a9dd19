// C ABI of libsph (include/sph.h): workspace carving, context life cycle, the
// three stage calls and the persistent-id-order exchange of particle data.
// The library allocates no device memory: every array lives in the caller's
// workspace, carved here with 256-byte alignment.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "sph_internal.cuh"

namespace sph {

int check_cuda(cudaError_t e) { return e == cudaSuccess ? SPH_OK : SPH_ERR_CUDA; }

namespace {

struct Bump {
    char *base;
    size_t off;
    template <typename T> T *take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? (T *)(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

// Cells searched on each side of a particle's own cell: the support 2h spans
// one cell of edge >= 2h and two cells of edge in [h, 2h).
int cell_reach(const sph_params &p)
{
    return p.cell_size >= 2.0 * p.h * (1.0 - 1e-12) ? 1 : 2;
}

int validate(const sph_params *p, int64_t nf, int64_t nb, int dims[3], uint32_t *ncells)
{
    if (!p || nf < 0 || nb < 0) return SPH_ERR_INVALID_ARG;
    if (!(p->h > 0) || !(p->cell_size >= p->h * (1.0 - 1e-12)) || !(p->rho0 > 0) ||
        !(p->gamma > 0) || !(p->c0 > 0) || !(p->mass > 0) || !(p->cfl > 0) ||
        !(p->alpha >= 0) || !(p->eta2_coef > 0) || p->verlet_euler_every < 1 ||
        (p->precision != SPH_FP64 && p->precision != SPH_FP32_SPLIT) ||
        p->pi_kernel < SPH_PI_WARP || p->pi_kernel > SPH_PI_WARP_SYM)
        return SPH_ERR_INVALID_ARG;
    // the float32 PI kernels take the sound speed as c0 (rho / rho0)^3, the
    // Tait form of gamma = 7 (Table 1)
    if (p->precision == SPH_FP32_SPLIT && p->gamma != 7.0) return SPH_ERR_INVALID_ARG;
    // cells below the support 2h (the paper's finer cells, Section 4.6, optimisation F):
    // searched by the float64 kernels and the thread-per-particle kernel only
    if (cell_reach(*p) > 1 && p->precision == SPH_FP32_SPLIT && p->pi_kernel != SPH_PI_THREAD)
        return SPH_ERR_INVALID_ARG;
    // float64: the warp-per-item kernel or one thread per particle
    if (p->precision == SPH_FP64 && p->pi_kernel != SPH_PI_WARP && p->pi_kernel != SPH_PI_THREAD)
        return SPH_ERR_INVALID_ARG;
    const bool tensile = p->tensile_eps != 0.0 || p->tensile_pos != 0.0;
    if (tensile && (p->tensile_n < 1 || p->tensile_n > 16 || !(p->dp > 0) ||
                    (p->precision == SPH_FP32_SPLIT && p->pi_kernel != SPH_PI_WARP)))
        return SPH_ERR_INVALID_ARG;
    uint64_t nc = 1;
    for (int d = 0; d < 3; ++d) {
        double span = p->dom_max[d] - p->dom_min[d];
        if (!(span > 0) || !isfinite(span)) return SPH_ERR_INVALID_ARG;
        double n = ceil(span / p->cell_size);
        if (n > 2.0e9) return SPH_ERR_TOO_LARGE;
        dims[d] = (int)n;
        nc *= (uint64_t)dims[d];
    }
    if (nc + 3 > (uint64_t)INT32_MAX) return SPH_ERR_TOO_LARGE;
    if (nf + nb > (int64_t)INT32_MAX / 16) return SPH_ERR_TOO_LARGE;
    *ncells = (uint32_t)nc;
    return SPH_OK;
}

DevParams derive(const sph_params &p, const int dims[3], uint32_t ncells)
{
    DevParams d;
    memset(&d, 0, sizeof(d));
    d.h = p.h;
    d.s = p.cell_size;
    d.inv_s = 1.0 / p.cell_size;
    d.rho0 = p.rho0;
    d.inv_rho0 = 1.0 / p.rho0;
    d.gamma = p.gamma;
    d.c0 = p.c0;
    d.alpha = p.alpha;
    d.eta2 = p.eta2_coef * p.h * p.h;
    d.cfl = p.cfl;
    d.mass = p.mass;
    d.B = p.c0 * p.c0 * p.rho0 / p.gamma;
    d.fixed_dt = p.fixed_dt;
    d.invh = 1.0 / p.h;
    double aD = 1.0 / (M_PI * p.h * p.h * p.h);
    d.kA64 = aD / (p.h * p.h);
    d.kB64 = -0.75 * aD / p.h;
    d.kcu64 = p.c0 / (p.rho0 * p.rho0 * p.rho0);
    d.kc64 = -p.alpha * d.kcu64;
    d.cell_af = (float)(1.0 / p.cell_size);
    d.cell_eabsf = (float)fmax(0x1p-60, 0x1p-124 / p.cell_size);  // inf: always the float64 path
    for (int k = 0; k < 3; ++k) {
        d.cell_bf[k] = (float)(p.dom_min[k] / p.cell_size);
        d.cell_babsf[k] = fabsf(d.cell_bf[k]);
        d.g[k] = p.g[k];
        d.dom_min[k] = p.dom_min[k];
        d.gf[k] = (float)p.g[k];
    }
    d.nx = dims[0];
    d.ny = dims[1];
    d.nz = dims[2];
    d.ncells = ncells;
    d.euler_every = (int)p.verlet_euler_every;
    d.reach = cell_reach(p);
    d.clamp = p.clamp_boundary_rho ? 1 : 0;
    d.gamma_is_7 = p.gamma == 7.0;
    d.hf = (float)p.h;
    d.invhf = (float)(1.0 / p.h);
    d.four_h2f = (float)(4.0 * p.h * p.h);
    d.eta2f = (float)d.eta2;
    d.massf = (float)p.mass;
    d.alphaf = (float)p.alpha;
    d.c0f = (float)p.c0;
    d.inv_rho0f = (float)(1.0 / p.rho0);
    d.Bf = (float)d.B;
    d.sf = (float)p.cell_size;
    d.kA = (float)d.kA64;
    d.kB = (float)d.kB64;
    d.aDf = (float)aD;
    d.s_hf = (float)(p.cell_size / p.h);
    d.eta2_h2f = (float)p.eta2_coef;
    d.gw1 = (float)(2.25 * d.kA64 * p.h / d.kB64);
    d.gw0 = (float)(-3.0 * d.kA64 * p.h / d.kB64);
    d.nmkBf = (float)(-p.mass * d.kB64);
    d.mkBf = (float)(p.mass * d.kB64);
    d.kcf = (float)(-p.alpha * p.c0 / (p.rho0 * p.rho0 * p.rho0));
    d.nalphaf = (float)(-p.alpha);
    d.tensile = (p.tensile_eps != 0.0 || p.tensile_pos != 0.0) ? 1 : 0;
    d.tensile_n = (int)p.tensile_n;
    d.tens_eps = p.tensile_eps;
    d.tens_pos = p.tensile_pos;
    if (d.tensile) {
        // W(dp) of the cubic spline (the reference spacing of the correction)
        double q = p.dp / p.h, w;
        if (q < 1.0) w = aD * (1.0 - 1.5 * q * q + 0.75 * q * q * q);
        else if (q < 2.0) w = aD * 0.25 * (2.0 - q) * (2.0 - q) * (2.0 - q);
        else w = 0.0;
        d.inv_wdp = w > 0.0 ? 1.0 / w : 0.0;
    }
    d.tens_epsf = (float)d.tens_eps;
    d.tens_posf = (float)d.tens_pos;
    d.inv_wdpf = (float)d.inv_wdp;
    return d;
}

}  // namespace

int validate_params(const sph_params *p, int64_t nf, int64_t nb, int dims[3], uint32_t *ncells)
{
    return validate(p, nf, nb, dims, ncells);
}

DevParams derive_params(const sph_params &p, const int dims[3], uint32_t ncells)
{
    return derive(p, dims, ncells);
}

size_t plan_workspace(const sph_params &p, int64_t nf, int64_t nb, int dims[3], uint32_t *ncells,
                      Workspace *w, char *base)
{
    (void)dims;
    Workspace tmp;
    Workspace &W = w ? *w : tmp;
    memset(&W, 0, sizeof(W));
    const size_t R = p.precision == SPH_FP32_SPLIT ? 4 : 8;
    const size_t V4 = 4 * R;
    Bump b{base, 0};
    for (int k = 0; k < 2; ++k) {
        size_t start = (b.off + 255) & ~(size_t)255;
        W.x[k] = b.take<double>(nf);
        W.y[k] = b.take<double>(nf);
        W.z[k] = b.take<double>(nf);
        W.V[k] = b.take<char>(V4 * nf);
        W.VM[k] = b.take<char>(V4 * nf);
        W.id[k] = b.take<uint32_t>(nf);
        b.off = (b.off + 255) & ~(size_t)255;
        W.state_chunk[k] = base ? base + start : nullptr;
        W.state_chunk_bytes = b.off - start;
    }
    W.posp = b.take<char>(V4 * nf);
    W.acc = b.take<char>(V4 * nf);
    W.cell = b.take<uint32_t>(nf);
    {
        size_t start = (b.off + 255) & ~(size_t)255;
        W.brho = b.take<char>(R * nb);
        W.brhom = b.take<char>(R * nb);
        b.off = (b.off + 255) & ~(size_t)255;
        W.bstate_chunk = base ? base + start : nullptr;
        W.bstate_chunk_bytes = b.off - start;
    }
    W.bx = b.take<double>(nb);
    W.by = b.take<double>(nb);
    W.bz = b.take<double>(nb);
    W.bid = b.take<uint32_t>(nb);
    W.bcell = b.take<uint32_t>(nb);
    W.bposp = b.take<char>(V4 * nb);
    if (p.precision == SPH_FP64) {
        W.posf = b.take<float4>(nf > 0 ? nf : 1);
        W.bposf = b.take<float4>(nb > 0 ? nb : 1);
    }
    W.bvelr = b.take<char>(V4 * nb);
    W.bar = b.take<char>(R * nb);
    int64_t m = nf > nb ? nf : nb;
    W.key_by_id = b.take<uint32_t>(m);
    W.val_by_id = b.take<uint32_t>(m);
    W.key_tmp = b.take<uint32_t>(m);
    W.val_tmp = b.take<uint32_t>(m);
    W.key_sorted = b.take<uint32_t>(m);
    W.val_sorted = b.take<uint32_t>(m);
    const size_t ftiles = (size_t)scan_tiles((int64_t)*ncells + 2);
    W.count = b.take<uint32_t>((size_t)*ncells + 2 + ftiles + kCtrWords);
    W.fpart = W.count ? W.count + *ncells + 2 : nullptr;
    W.ctr = W.count ? W.fpart + ftiles : nullptr;
    W.items_f = b.take<uint32_t>(2 * (size_t)(nf > 0 ? nf : 1));  // {first, count} pairs
    W.items_b = b.take<uint32_t>(2 * (size_t)(nb > 0 ? nb : 1));  // {first, count} pairs
    if (p.precision == SPH_FP32_SPLIT && p.pi_kernel == SPH_PI_THREAD_FASTCELLS) {
        W.franges = b.take<int4>((size_t)*ncells * 9);
        W.branges = b.take<int4>((size_t)*ncells * 9);
    }
    W.fstart = b.take<int32_t>((size_t)*ncells + 2);
    W.origin = b.take<double>((size_t)dims[0] + dims[1] + dims[2]);
    W.bstart = b.take<int32_t>((size_t)*ncells + 2);
    int64_t hist = (int64_t)256 * radix_tiles(m > 0 ? m : 1);
    W.radix_hist = b.take<uint32_t>((size_t)hist);
    int64_t scan_n = hist > (int64_t)*ncells + 2 ? hist : (int64_t)*ncells + 2;
    W.scan_part = b.take<uint32_t>(scan_partials(scan_n));
    if (p.precision == SPH_FP64) {
        W.adj_gF = b.take<double>(3 * (size_t)nf + 1);
        W.adj_gD = b.take<double>((size_t)(nf + nb) + 1);
        W.adj_lam = b.take<double>((size_t)11 * (size_t)(nf + nb) + 1);
        W.adj_part = b.take<double>((size_t)nf + 2);   // dJ/dalpha per work item (first target)
    }
    W.sens_p = b.take<double>(kMaxSensors);
    W.sens_den = b.take<double>(kMaxSensors);
    W.front = b.take<double>(2);
    W.stage = b.take<double>((size_t)11 * (size_t)(nf + nb) + 1);
    W.sc = b.take<Scalars>(1);
    W.counts4 = b.take<unsigned long long>(4);
    return (b.off + 255) & ~(size_t)255;
}

// ------------------------------------------------------ exchange kernels --

template <typename Real>
__global__ void k_scatter_in(int nf, size_t N, const double *__restrict__ stage, double *x,
                             double *y, double *z, typename Real4T<Real>::T *V,
                             typename Real4T<Real>::T *VM, uint32_t *id)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    const double *pos = stage, *vel = stage + 3 * N, *r = stage + 6 * N, *vm = stage + 7 * N,
                 *rm = stage + 10 * N;
    x[i] = pos[3 * (size_t)i];
    y[i] = pos[3 * (size_t)i + 1];
    z[i] = pos[3 * (size_t)i + 2];
    typename Real4T<Real>::T v, u;
    v.x = (Real)vel[3 * (size_t)i];
    v.y = (Real)vel[3 * (size_t)i + 1];
    v.z = (Real)vel[3 * (size_t)i + 2];
    v.w = (Real)r[i];
    u.x = (Real)vm[3 * (size_t)i];
    u.y = (Real)vm[3 * (size_t)i + 1];
    u.z = (Real)vm[3 * (size_t)i + 2];
    u.w = (Real)rm[i];
    V[i] = v;
    VM[i] = u;
    id[i] = (uint32_t)i;
}

template <typename Real>
__global__ void k_gather_out(int nf, int nb, size_t N, double *__restrict__ stage,
                             const double *x, const double *y, const double *z,
                             const typename Real4T<Real>::T *V,
                             const typename Real4T<Real>::T *VM, const uint32_t *id,
                             const double *bx, const double *by, const double *bz,
                             const Real *brho, const Real *brhom, const uint32_t *bid)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double *pos = stage, *vel = stage + 3 * N, *r = stage + 6 * N, *vm = stage + 7 * N,
           *rm = stage + 10 * N;
    if (i < nf) {
        size_t k = id[i];
        const typename Real4T<Real>::T v = V[i], u = VM[i];
        pos[3 * k] = x[i]; pos[3 * k + 1] = y[i]; pos[3 * k + 2] = z[i];
        vel[3 * k] = (double)v.x; vel[3 * k + 1] = (double)v.y; vel[3 * k + 2] = (double)v.z;
        vm[3 * k] = (double)u.x; vm[3 * k + 1] = (double)u.y; vm[3 * k + 2] = (double)u.z;
        r[k] = (double)v.w;
        rm[k] = (double)u.w;
    } else if (i < nf + nb) {
        int j = i - nf;
        size_t k = bid[j];
        pos[3 * k] = bx[j]; pos[3 * k + 1] = by[j]; pos[3 * k + 2] = bz[j];
        vel[3 * k] = 0.0; vel[3 * k + 1] = 0.0; vel[3 * k + 2] = 0.0;
        vm[3 * k] = 0.0; vm[3 * k + 1] = 0.0; vm[3 * k + 2] = 0.0;
        r[k] = (double)brho[j];
        rm[k] = (double)brhom[j];
    }
}

template <typename V4, typename Real>
__global__ void k_export_forces(int nf, int nb, size_t N, uint32_t ncells, const V4 *__restrict__ acc,
                                const Real *__restrict__ bar, const uint32_t *__restrict__ id,
                                const uint32_t *__restrict__ bid, const uint32_t *__restrict__ cell,
                                const uint32_t *__restrict__ bcell, double *__restrict__ stage)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double *ace = stage, *ar = stage + 3 * N;
    if (i < nf) {
        size_t k = id[i];
        V4 a = acc[i];
        bool in = cell[i] < ncells;   // particles outside the grid have no forces
        ace[3 * k] = in ? (double)a.x : 0.0;
        ace[3 * k + 1] = in ? (double)a.y : 0.0;
        ace[3 * k + 2] = in ? (double)a.z : 0.0;
        ar[k] = in ? (double)a.w : 0.0;
    } else if (i < nf + nb) {
        int j = i - nf;
        ar[bid[j]] = bcell[j] < ncells ? (double)bar[j] : 0.0;
    }
}

// Boundary particles whose staged position differs, bit for bit, from the one
// the current boundary list holds set sc->bmoved.
__global__ void k_boundary_same(int nb, const double *__restrict__ stage, const double *bx,
                                const double *by, const double *bz, const uint32_t *bid,
                                Scalars *sc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    const size_t g = bid[i];
    const bool same = __double_as_longlong(stage[3 * g]) == __double_as_longlong(bx[i]) &&
                      __double_as_longlong(stage[3 * g + 1]) == __double_as_longlong(by[i]) &&
                      __double_as_longlong(stage[3 * g + 2]) == __double_as_longlong(bz[i]);
    if (!same) sc->bmoved = 1u;
}

// Densities of the boundary particles from the staged state (list unchanged).
template <typename Real>
__global__ void k_boundary_rho(int nb, size_t N, const double *__restrict__ stage,
                               const uint32_t *__restrict__ bid, Real *brho, Real *brhom)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    const size_t g = bid[i];
    brho[i] = (Real)stage[6 * N + g];
    brhom[i] = (Real)stage[10 * N + g];
}

}  // namespace sph

using namespace sph;

namespace {

template <typename Real> void launch_scatter_in(sph_ctx *ctx, int buf)
{
    Workspace &w = ctx->w;
    int nf = (int)ctx->nf;
    if (nf == 0) return;
    size_t N = (size_t)(ctx->nf + ctx->nb);
    const int T = 256;
    SPH_LAUNCH(ctx, k_scatter_in<Real>, (nf + T - 1) / T, T, 0, ctx->stream, nf, N, w.stage,
               w.x[buf], w.y[buf], w.z[buf], (typename Real4T<Real>::T *)w.V[buf],
               (typename Real4T<Real>::T *)w.VM[buf], w.id[buf]);
}

template <typename Real> void launch_gather_out(sph_ctx *ctx)
{
    Workspace &w = ctx->w;
    int nf = (int)ctx->nf, nb = (int)ctx->nb;
    int c = ctx->cur;
    size_t N = (size_t)(nf + nb);
    if (N == 0) return;
    const int T = 256;
    SPH_LAUNCH(ctx, k_gather_out<Real>, (unsigned)((N + T - 1) / T), T, 0, ctx->stream, nf, nb,
               N, w.stage, w.x[c], w.y[c], w.z[c], (const typename Real4T<Real>::T *)w.V[c],
               (const typename Real4T<Real>::T *)w.VM[c], w.id[c], w.bx, w.by, w.bz,
               (const Real *)w.brho, (const Real *)w.brhom, w.bid);
}

// Copy the caller's id-ordered state into the stage; missing previous levels
// are copied from the current ones.
int stage_in(sph_ctx *ctx, const double *pos, const double *vel, const double *rho,
             const double *velm, const double *rhom)
{
    size_t N = (size_t)(ctx->nf + ctx->nb);
    double *s = ctx->w.stage;
    cudaStream_t st = ctx->stream;
    if (N == 0) return SPH_OK;
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaMemcpyAsync(s, pos, 3 * N * sizeof(double), cudaMemcpyDefault, st);
    e = e ? e : cudaMemcpyAsync(s + 3 * N, vel, 3 * N * sizeof(double), cudaMemcpyDefault, st);
    e = e ? e : cudaMemcpyAsync(s + 6 * N, rho, N * sizeof(double), cudaMemcpyDefault, st);
    e = e ? e : cudaMemcpyAsync(s + 7 * N, velm ? velm : s + 3 * N, 3 * N * sizeof(double),
                                cudaMemcpyDefault, st);
    e = e ? e : cudaMemcpyAsync(s + 10 * N, rhom ? rhom : s + 6 * N, N * sizeof(double),
                                cudaMemcpyDefault, st);
    return check_cuda(e);
}

int load_state(sph_ctx *ctx, const double *pos, const double *vel, const double *rho,
               const double *velm, const double *rhom)
{
    int rc = stage_in(ctx, pos, vel, rho, velm, rhom);
    if (rc) return rc;
    ctx->cur = 0;
    if (ctx->precision == SPH_FP32_SPLIT) launch_scatter_in<float>(ctx, 0);
    else launch_scatter_in<double>(ctx, 0);
    Workspace &w = ctx->w;
    const int nb = (int)ctx->nb, T = 256;
    const size_t N = (size_t)(ctx->nf + ctx->nb);
    // Boundaries never move: when the new state keeps every boundary position,
    // the boundary list stands and only the densities are taken over.
    bool rebuild = !ctx->boundary_built;
    if (!rebuild && nb > 0) {
        uint32_t moved = 0;
        if (check_cuda(cudaMemsetAsync(&w.sc->bmoved, 0, sizeof(uint32_t), ctx->stream)))
            return SPH_ERR_CUDA;
        SPH_LAUNCH(ctx, k_boundary_same, (nb + T - 1) / T, T, 0, ctx->stream, nb, w.stage, w.bx,
                   w.by, w.bz, w.bid, w.sc);
        if (check_cuda(cudaMemcpyAsync(&moved, &w.sc->bmoved, sizeof(uint32_t),
                                       cudaMemcpyDeviceToHost, ctx->stream)) ||
            check_cuda(cudaStreamSynchronize(ctx->stream)))
            return SPH_ERR_CUDA;
        rebuild = moved != 0;
    }
    if (rebuild) {
        ctx->branges_ready = false;
        rc = nl_boundary_build(ctx);
        if (rc) return rc;
        ctx->boundary_built = true;
    } else if (nb > 0) {
        if (ctx->precision == SPH_FP32_SPLIT)
            SPH_LAUNCH(ctx, k_boundary_rho<float>, (nb + T - 1) / T, T, 0, ctx->stream, nb, N,
                       w.stage, w.bid, (float *)w.brho, (float *)w.brhom);
        else
            SPH_LAUNCH(ctx, k_boundary_rho<double>, (nb + T - 1) / T, T, 0, ctx->stream, nb, N,
                       w.stage, w.bid, (double *)w.brho, (double *)w.brhom);
    }
    ctx->nl_valid = ctx->pi_valid = false;
    return check_cuda(cudaStreamSynchronize(ctx->stream));
}

int sync_flags(sph_ctx *ctx)
{
    uint32_t flags = 0;
    if (check_cuda(cudaMemcpyAsync(&flags, &ctx->w.sc->flags, sizeof(flags),
                                   cudaMemcpyDeviceToHost, ctx->stream)))
        return SPH_ERR_CUDA;
    if (check_cuda(cudaStreamSynchronize(ctx->stream))) return SPH_ERR_CUDA;
    return flags ? SPH_ERR_DEVICE_FLAG : SPH_OK;
}

int copy_out(void *dst, const void *src, size_t bytes, cudaStream_t st)
{
    if (!dst || bytes == 0) return SPH_OK;
    return check_cuda(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
}

}  // namespace

extern "C" {

int sph_workspace_bytes(const sph_params *p, int64_t n_f, int64_t n_b, size_t *bytes)
{
    int dims[3];
    uint32_t nc;
    if (!bytes) return SPH_ERR_INVALID_ARG;
    int rc = validate(p, n_f, n_b, dims, &nc);
    if (rc) return rc;
    *bytes = plan_workspace(*p, n_f, n_b, dims, &nc, nullptr, nullptr);
    return SPH_OK;
}

int sph_create(const sph_params *p, int64_t n_f, int64_t n_b, const double *pos,
               const double *vel, const double *rho, void *workspace, size_t ws_bytes,
               void *stream, sph_ctx **out)
{
    if (!out) return SPH_ERR_INVALID_ARG;
    *out = nullptr;
    int dims[3];
    uint32_t nc;
    int rc = validate(p, n_f, n_b, dims, &nc);
    if (rc) return rc;
    if (n_f + n_b > 0 && (!pos || !vel || !rho)) return SPH_ERR_INVALID_ARG;
    size_t need = plan_workspace(*p, n_f, n_b, dims, &nc, nullptr, nullptr);
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace & 255)) return SPH_ERR_WORKSPACE;
    sph_ctx *ctx = (sph_ctx *)calloc(1, sizeof(sph_ctx));
    if (!ctx) return SPH_ERR_INVALID_ARG;
    ctx->prm = *p;
    ctx->nf = n_f;
    ctx->nb = n_b;
    for (int d = 0; d < 3; ++d) ctx->dims[d] = dims[d];
    ctx->ncells = nc;
    ctx->precision = p->precision;
    ctx->real_size = p->precision == SPH_FP32_SPLIT ? 4 : 8;
    ctx->stream = (cudaStream_t)stream;
    ctx->dp = derive(*p, dims, nc);
    cudaGetDevice(&ctx->device);
    plan_workspace(*p, n_f, n_b, dims, &nc, &ctx->w, (char *)workspace);
    rc = check_cuda(cudaMemsetAsync(ctx->w.sc, 0, sizeof(Scalars), ctx->stream));
    if (!rc) rc = fill_origins(ctx);
    if (!rc && ctx->precision == SPH_FP32_SPLIT)
        rc = p->pi_kernel == SPH_PI_WARP_SYM ? pi32_sym_setup(ctx) : pi32_setup(ctx);
    else if (!rc)
        rc = pi64_setup(ctx);
    if (!rc && ctx->precision == SPH_FP64) rc = adjoint_setup(ctx);
    if (!rc) rc = load_state(ctx, pos, vel, rho, nullptr, nullptr);
    if (rc) {
        free(ctx);
        return rc;
    }
    *out = ctx;
    return SPH_OK;
}

int sph_neighbour_list(sph_ctx *ctx)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    int rc = nl_fluid(ctx);
    if (rc) return rc;
    ctx->nl_valid = true;
    ctx->pi_valid = false;
    return SPH_OK;
}

int sph_interact(sph_ctx *ctx)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (!ctx->nl_valid) return SPH_ERR_SEQUENCE;
    int rc = pi_launch(ctx);
    if (rc) return rc;
    ctx->pi_valid = true;
    return SPH_OK;
}

int sph_update(sph_ctx *ctx, double *dt_out)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (!ctx->pi_valid) return SPH_ERR_SEQUENCE;
    int rc = su_launch(ctx);
    if (rc) return rc;
    ctx->nl_valid = ctx->pi_valid = false;
    if (dt_out) {
        if (check_cuda(cudaMemcpyAsync(dt_out, &ctx->w.sc->dt_last, sizeof(double),
                                       cudaMemcpyDefault, ctx->stream)))
            return SPH_ERR_CUDA;
        return sync_flags(ctx);
    }
    return SPH_OK;
}

int sph_run(sph_ctx *ctx, int64_t n_steps)
{
    if (!ctx || n_steps < 0) return SPH_ERR_INVALID_ARG;
    for (int64_t k = 0; k < n_steps; ++k) {
        int rc = sph_neighbour_list(ctx);
        if (!rc) rc = sph_interact(ctx);
        if (!rc) rc = sph_update(ctx, nullptr);
        if (rc) return rc;
    }
    return SPH_OK;
}

int sph_run_graph(sph_ctx *ctx, int64_t n_steps)
{
    if (!ctx || n_steps < 0) return SPH_ERR_INVALID_ARG;
    if (ctx->stream == nullptr || ctx->stream == cudaStreamLegacy ||
        ctx->stream == cudaStreamPerThread)
        return SPH_ERR_INVALID_ARG;
    int64_t k = 0;
    for (; k + 2 <= n_steps; k += 2) {
        const int c = ctx->cur;
        if (!ctx->graph[c]) {
            // capture two steps: the buffers swap every step, so the pair is periodic
            cudaGraph_t g = nullptr;
            long long before = ctx->launches;
            if (check_cuda(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal)))
                return SPH_ERR_CUDA;
            int rc = sph_run(ctx, 2);
            cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
            if (rc || e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                ctx->cur = c;
                return rc ? rc : SPH_ERR_CUDA;
            }
            e = cudaGraphInstantiate(&ctx->graph[c], g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                ctx->graph[c] = nullptr;
                ctx->cur = c;
                return SPH_ERR_CUDA;
            }
            ctx->graph_launches[c] = ctx->launches - before;
            ctx->launches = before;
            ctx->cur = c;   // capture recorded the work; nothing ran yet
        }
        if (check_cuda(cudaGraphLaunch(ctx->graph[c], ctx->stream))) return SPH_ERR_CUDA;
        ctx->launches += ctx->graph_launches[c];
        // the two steps leave cur where it started
    }
    if (k < n_steps) return sph_run(ctx, 1);
    ctx->nl_valid = ctx->pi_valid = false;
    return SPH_OK;
}

int sph_get_state(sph_ctx *ctx, double *pos, double *vel, double *rho, double *vel_prev,
                  double *rho_prev)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (ctx->precision == SPH_FP32_SPLIT) launch_gather_out<float>(ctx);
    else launch_gather_out<double>(ctx);
    size_t N = (size_t)(ctx->nf + ctx->nb);
    double *s = ctx->w.stage;
    cudaStream_t st = ctx->stream;
    int rc = copy_out(pos, s, 3 * N * sizeof(double), st);
    if (!rc) rc = copy_out(vel, s + 3 * N, 3 * N * sizeof(double), st);
    if (!rc) rc = copy_out(rho, s + 6 * N, N * sizeof(double), st);
    if (!rc) rc = copy_out(vel_prev, s + 7 * N, 3 * N * sizeof(double), st);
    if (!rc) rc = copy_out(rho_prev, s + 10 * N, N * sizeof(double), st);
    if (rc) return rc;
    return check_cuda(cudaStreamSynchronize(st));
}

int sph_set_state(sph_ctx *ctx, const double *pos, const double *vel, const double *rho,
                  const double *vel_prev, const double *rho_prev)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (ctx->nf + ctx->nb > 0 && (!pos || !vel || !rho)) return SPH_ERR_INVALID_ARG;
    return load_state(ctx, pos, vel, rho, vel_prev, rho_prev);
}

int sph_get_time(sph_ctx *ctx, double *time, double *last_dt, int64_t *steps)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    Scalars sc;
    if (check_cuda(cudaMemcpyAsync(&sc, ctx->w.sc, sizeof(sc), cudaMemcpyDeviceToHost, ctx->stream)))
        return SPH_ERR_CUDA;
    if (check_cuda(cudaStreamSynchronize(ctx->stream))) return SPH_ERR_CUDA;
    if (time) *time = sc.time;
    if (last_dt) *last_dt = sc.dt_last;
    if (steps) *steps = sc.step;
    return SPH_OK;
}

int sph_status(sph_ctx *ctx, uint32_t *flags, int clear)
{
    if (!ctx || !flags) return SPH_ERR_INVALID_ARG;
    if (check_cuda(cudaMemcpyAsync(flags, &ctx->w.sc->flags, sizeof(uint32_t),
                                   cudaMemcpyDeviceToHost, ctx->stream)))
        return SPH_ERR_CUDA;
    if (clear && check_cuda(cudaMemsetAsync(&ctx->w.sc->flags, 0, sizeof(uint32_t), ctx->stream)))
        return SPH_ERR_CUDA;
    return check_cuda(cudaStreamSynchronize(ctx->stream));
}

int sph_get_neighbour_list(sph_ctx *ctx, uint32_t *sorted_id, uint32_t *cell, int32_t *cell_start)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (!ctx->nl_valid && !ctx->pi_valid) return SPH_ERR_SEQUENCE;
    cudaStream_t st = ctx->stream;
    size_t nf = (size_t)ctx->nf;
    int rc = copy_out(sorted_id, ctx->w.id[ctx->cur], nf * sizeof(uint32_t), st);
    if (!rc) rc = copy_out(cell, ctx->w.cell, nf * sizeof(uint32_t), st);
    if (!rc) rc = copy_out(cell_start, ctx->w.fstart, ((size_t)ctx->ncells + 2) * sizeof(int32_t), st);
    if (rc) return rc;
    return check_cuda(cudaStreamSynchronize(st));
}

int sph_get_grid(sph_ctx *ctx, int64_t dims[3])
{
    if (!ctx || !dims) return SPH_ERR_INVALID_ARG;
    for (int d = 0; d < 3; ++d) dims[d] = ctx->dims[d];
    return SPH_OK;
}

int sph_get_forces(sph_ctx *ctx, double *ace, double *ar, double *maxima)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (!ctx->pi_valid) return SPH_ERR_SEQUENCE;
    Workspace &w = ctx->w;
    int nf = (int)ctx->nf, nb = (int)ctx->nb;
    size_t N = (size_t)(nf + nb);
    cudaStream_t st = ctx->stream;
    const int T = 256;
    if (N > 0) {
        if (ctx->precision == SPH_FP32_SPLIT)
            SPH_LAUNCH(ctx, (k_export_forces<float4, float>), (unsigned)((N + T - 1) / T), T, 0, st,
                       nf, nb, N, ctx->ncells, (const float4 *)w.acc, (const float *)w.bar,
                       w.id[ctx->cur], w.bid, w.cell, w.bcell, w.stage);
        else
            SPH_LAUNCH(ctx, (k_export_forces<double4_32a, double>), (unsigned)((N + T - 1) / T), T, 0,
                       st, nf, nb, N, ctx->ncells, (const double4_32a *)w.acc, (const double *)w.bar,
                       w.id[ctx->cur], w.bid, w.cell, w.bcell, w.stage);
    }
    int rc = copy_out(ace, w.stage, 3 * (size_t)nf * sizeof(double), st);
    if (!rc) rc = copy_out(ar, w.stage + 3 * N, N * sizeof(double), st);
    Maxima mx;
    if (!rc) rc = check_cuda(cudaMemcpyAsync(&mx, &w.sc->mx, sizeof(mx), cudaMemcpyDeviceToHost, st));
    if (rc) return rc;
    rc = check_cuda(cudaStreamSynchronize(st));
    if (!rc && maxima) {
        unsigned long long b[3] = {mx.f2, mx.c, mx.visc};
        double v[3];
        memcpy(v, b, sizeof(v));
        maxima[0] = sqrt(v[0]);
        maxima[1] = v[1];
        maxima[2] = v[2];
    }
    return rc;
}

int sph_count_work(sph_ctx *ctx, int64_t counts[4])
{
    if (!ctx || !counts) return SPH_ERR_INVALID_ARG;
    if (!ctx->nl_valid) return SPH_ERR_SEQUENCE;
    int rc = count_work_launch(ctx);
    if (rc) return rc;
    unsigned long long c[4];
    if (check_cuda(cudaMemcpyAsync(c, ctx->w.counts4, sizeof(c), cudaMemcpyDeviceToHost, ctx->stream)))
        return SPH_ERR_CUDA;
    if (check_cuda(cudaStreamSynchronize(ctx->stream))) return SPH_ERR_CUDA;
    for (int k = 0; k < 4; ++k) counts[k] = (int64_t)c[k];
    return SPH_OK;
}

int64_t sph_launch_count(const sph_ctx *ctx) { return ctx ? (int64_t)ctx->launches : 0; }

int sph_checkpoint_bytes(const sph_ctx *ctx, size_t *bytes)
{
    if (!ctx || !bytes) return SPH_ERR_INVALID_ARG;
    *bytes = ctx->w.state_chunk_bytes + ctx->w.bstate_chunk_bytes +
             ((sizeof(Scalars) + 255) & ~(size_t)255);
    return SPH_OK;
}

int sph_save_state(sph_ctx *ctx, void *dst)
{
    if (!ctx || !dst) return SPH_ERR_INVALID_ARG;
    Workspace &w = ctx->w;
    char *d = (char *)dst;
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaMemcpyAsync(d, w.state_chunk[ctx->cur], w.state_chunk_bytes,
                                    cudaMemcpyDefault, st);
    if (!e && w.bstate_chunk_bytes)
        e = cudaMemcpyAsync(d + w.state_chunk_bytes, w.bstate_chunk, w.bstate_chunk_bytes,
                            cudaMemcpyDefault, st);
    if (!e)
        e = cudaMemcpyAsync(d + w.state_chunk_bytes + w.bstate_chunk_bytes, w.sc, sizeof(Scalars),
                            cudaMemcpyDefault, st);
    return check_cuda(e);
}

int sph_load_state(sph_ctx *ctx, const void *src)
{
    if (!ctx || !src) return SPH_ERR_INVALID_ARG;
    Workspace &w = ctx->w;
    const char *s = (const char *)src;
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaMemcpyAsync(w.state_chunk[ctx->cur], s, w.state_chunk_bytes,
                                    cudaMemcpyDefault, st);
    if (!e && w.bstate_chunk_bytes)
        e = cudaMemcpyAsync(w.bstate_chunk, s + w.state_chunk_bytes, w.bstate_chunk_bytes,
                            cudaMemcpyDefault, st);
    if (!e)
        e = cudaMemcpyAsync(w.sc, s + w.state_chunk_bytes + w.bstate_chunk_bytes, sizeof(Scalars),
                            cudaMemcpyDefault, st);
    ctx->nl_valid = ctx->pi_valid = false;
    return check_cuda(e);
}

const char *sph_error_string(int code)
{
    switch (code) {
    case SPH_OK: return "ok";
    case SPH_ERR_INVALID_ARG: return "invalid argument";
    case SPH_ERR_WORKSPACE: return "workspace missing, too small or not 256-byte aligned";
    case SPH_ERR_CUDA: return "CUDA error";
    case SPH_ERR_DEVICE_FLAG: return "device status flag set (see sph_status)";
    case SPH_ERR_TOO_LARGE: return "particle count or cell grid exceeds 32-bit indices";
    case SPH_ERR_SEQUENCE: return "call out of order (NL -> PI -> SU)";
    default: return "unknown error";
    }
}

void sph_destroy(sph_ctx *ctx)
{
    if (!ctx) return;
    for (int k = 0; k < 2; ++k)
        if (ctx->graph[k]) cudaGraphExecDestroy(ctx->graph[k]);
    free(ctx);
}

}  // extern "C"
