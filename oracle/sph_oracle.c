/*
 * FP64 CPU oracle of the weakly compressible SPH time step (Sections 2 and 4 of
 * Dominguez, Crespo & Gomez-Gesteira, "Optimization strategies for parallel CPU
 * and GPU implementations of a meshfree particle method").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library under paper_1110_3711_gb300/
 * may include, link or call this file; only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark use it.  It shares no code, header or
 * constant with the CUDA path.
 *
 * It is deliberately plain: every particle array is in persistent-id order,
 * the neighbour search is the cell-linked list of Section 2 written with
 * explicit loops over the 27 cells, every formula is evaluated in double
 * precision in the order it is written, and compilation uses
 * -ffp-contract=off so that x86 and Arm hosts give identical bits.
 *
 * One step is the paper's three stages (Section 2, Fig. 1):
 *   NL  cell of every particle, a stable sort by (cell, id), the first index
 *       of every cell ("CellBeginEnd", Section 4.1, Fig. 8), one list for
 *       fluid and one for boundary particles (Section 2);
 *   PI  fluid-fluid, fluid-boundary and boundary-fluid interactions, never
 *       boundary-boundary (Section 2): momentum with the Tait pressure and
 *       Monaghan's artificial viscosity, continuity, with the cubic spline
 *       kernel (Table 1);
 *   SU  variable time step from the force and the sound speed/viscous limits
 *       (Table 1, Section 4.1) and the Verlet scheme with a periodic Euler step
 *       (Table 1).
 * The paper names these formulations (Table 1) but prints no equations; the
 * standard forms of its references are written out next to each function.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double dp, h, cell_size, rho0, gamma, c0, alpha, eta2_coef, cfl, mass;
    double g[3];
    double dom_min[3], dom_max[3];
    int64_t verlet_euler_every;
    double fixed_dt;
    int64_t clamp_boundary_rho;
    double tensile_eps, tensile_pos;
    int64_t tensile_n;
} or_params;

#define OR_PI 3.14159265358979323846

/* ---------------------------------------------------------------- grid ---- */

/* Number of cells along each axis: ceil((max - min) / cell_size). */
int or_grid(const or_params *p, int64_t dims[3])
{
    for (int d = 0; d < 3; ++d) {
        double span = p->dom_max[d] - p->dom_min[d];
        dims[d] = (int64_t)ceil(span / p->cell_size);
        if (dims[d] < 1) return -1;
    }
    return 0;
}

/* Cell of one position: c_d = floor((x_d - min_d) / s); linear id
 * cx + nx*(cy + ny*cz) with x fastest (the cells follow X, Y and Z, Section
 * 4.4).  A position outside the grid gets the id n_cells (excluded). */
static int64_t cell_of(const or_params *p, const int64_t dims[3], const double *x)
{
    int64_t c[3];
    for (int d = 0; d < 3; ++d) {
        double t = floor((x[d] - p->dom_min[d]) / p->cell_size);
        if (!(t >= 0.0) || t >= (double)dims[d]) return dims[0] * dims[1] * dims[2];
        c[d] = (int64_t)t;
    }
    return c[0] + dims[0] * (c[1] + dims[1] * c[2]);
}

void or_cells(const or_params *p, int64_t n, const double *pos, int64_t *cell)
{
    int64_t dims[3];
    or_grid(p, dims);
    for (int64_t i = 0; i < n; ++i) cell[i] = cell_of(p, dims, pos + 3 * i);
}

/* Stable counting sort of particle indices by cell (Section 4.1).  On return
 * order[k] is the k-th particle in (cell, id) order and start[c] is the number
 * of particles whose cell is below c, for c = 0 .. n_cells + 1, so cell c
 * holds order[start[c] .. start[c+1]) and an empty cell has
 * start[c] == start[c+1] (the CellBeginEnd array of Fig. 8). */
int or_list(const or_params *p, int64_t n, const int64_t *cell, int64_t *order, int64_t *start)
{
    int64_t dims[3];
    or_grid(p, dims);
    int64_t nc = dims[0] * dims[1] * dims[2];
    int64_t *fill = (int64_t *)calloc((size_t)(nc + 2), sizeof(int64_t));
    if (!fill) return -1;
    for (int64_t c = 0; c <= nc + 1; ++c) start[c] = 0;
    for (int64_t i = 0; i < n; ++i) start[cell[i] + 1] += 1;
    for (int64_t c = 1; c <= nc + 1; ++c) start[c] += start[c - 1];
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = cell[i];
        order[start[c] + fill[c]] = i;
        fill[c] += 1;
    }
    free(fill);
    return 0;
}

/* ------------------------------------------------------------- physics ---- */

/* Cubic spline kernel (Monaghan & Lattanzio 1985; Table 1), 3D, support 2h:
 *   W(q) = 1/(pi h^3) * (1 - 1.5 q^2 + 0.75 q^3)   for 0 <= q < 1
 *        = 1/(pi h^3) * 0.25 (2 - q)^3             for 1 <= q < 2
 *        = 0                                         otherwise,   q = r/h. */
double or_kernel_w(double h, double r)
{
    double q = r / h;
    double ad = 1.0 / (OR_PI * h * h * h);
    if (q < 1.0) return ad * (1.0 - 1.5 * q * q + 0.75 * q * q * q);
    if (q < 2.0) return ad * 0.25 * (2.0 - q) * (2.0 - q) * (2.0 - q);
    return 0.0;
}

/* Gradient factor F with grad_a W_ab = F * (x_a - x_b), i.e. F = (dW/dr)/r:
 *   dW/dq = 1/(pi h^3) * (-3 q + 2.25 q^2)     for q < 1
 *         = 1/(pi h^3) * (-0.75 (2 - q)^2)     for 1 <= q < 2
 *   F = (dW/dq) / (h r). */
double or_kernel_f(double h, double r)
{
    double q = r / h;
    double ad = 1.0 / (OR_PI * h * h * h);
    double dwdq;
    if (q < 1.0) dwdq = ad * (-3.0 * q + 2.25 * q * q);
    else if (q < 2.0) dwdq = ad * (-0.75 * (2.0 - q) * (2.0 - q));
    else return 0.0;
    return dwdq / (h * r);
}

/* Tait equation of state (Batchelor 1974; Table 1):
 *   P = B ((rho/rho0)^gamma - 1),  B = c0^2 rho0 / gamma,
 * and the speed of sound c = sqrt(dP/drho) = c0 (rho/rho0)^((gamma-1)/2). */
double or_pressure(const or_params *p, double rho)
{
    double B = p->c0 * p->c0 * p->rho0 / p->gamma;
    return B * (pow(rho / p->rho0, p->gamma) - 1.0);
}

double or_sound(const or_params *p, double rho)
{
    return p->c0 * pow(rho / p->rho0, 0.5 * (p->gamma - 1.0));
}

/* One ordered pair (a receives from b), r_ab = x_a - x_b, v_ab = v_a - v_b,
 * with the artificial viscosity of Monaghan (1992; Table 1):
 *   mu_ab = h v_ab.r_ab / (r^2 + eta^2),  eta^2 = 0.01 h^2
 *   Pi_ab = -alpha cbar_ab mu_ab / rhobar_ab  if v_ab.r_ab < 0, else 0
 *   momentum:   dv_a/dt   += -m_b (P_a/rho_a^2 + P_b/rho_b^2 + Pi_ab + T_ab) grad_a W_ab
 *   continuity: drho_a/dt += m_b v_ab . grad_a W_ab
 * and the viscous time-step term |h v_ab.r_ab / (r^2 + eta^2)|.
 * T_ab is the tensile correction of Monaghan (2000) (the "tensil" array of
 * Table 3; zero unless tensile_eps or tensile_pos is set):
 *   T_ab = R_ab (W(r_ab) / W(dp))^n,
 *   R_ab = tensile_pos (P_a/rho_a^2 + P_b/rho_b^2)      if P_a > 0 and P_b > 0,
 *        = R_a + R_b, R = tensile_eps |P|/rho^2 for P < 0 and 0 otherwise. */
typedef struct { double acc[3], ar, visc; } pair_out;

static double tensile_r(const or_params *p, double Pa, double rhoa, double Pb, double rhob)
{
    if (Pa > 0.0 && Pb > 0.0) return p->tensile_pos * (Pa / (rhoa * rhoa) + Pb / (rhob * rhob));
    double R = 0.0;
    if (Pa < 0.0) R += p->tensile_eps * fabs(Pa) / (rhoa * rhoa);
    if (Pb < 0.0) R += p->tensile_eps * fabs(Pb) / (rhob * rhob);
    return R;
}

static void pair_terms(const or_params *p, int momentum,
                       const double *xa, const double *va, double rhoa, double Pa, double ca,
                       const double *xb, const double *vb, double rhob, double Pb, double cb,
                       pair_out *o)
{
    double r_ab[3], v_ab[3];
    for (int d = 0; d < 3; ++d) { r_ab[d] = xa[d] - xb[d]; v_ab[d] = va[d] - vb[d]; }
    double r2 = r_ab[0] * r_ab[0] + r_ab[1] * r_ab[1] + r_ab[2] * r_ab[2];
    double r = sqrt(r2);
    double F = or_kernel_f(p->h, r);
    double vdr = v_ab[0] * r_ab[0] + v_ab[1] * r_ab[1] + v_ab[2] * r_ab[2];
    double eta2 = p->eta2_coef * p->h * p->h;
    double mu = p->h * vdr / (r2 + eta2);
    double Pi = 0.0;
    if (vdr < 0.0) {
        double cbar = 0.5 * (ca + cb);
        double rhobar = 0.5 * (rhoa + rhob);
        Pi = -p->alpha * cbar * mu / rhobar;
    }
    double T = 0.0;
    if (p->tensile_eps != 0.0 || p->tensile_pos != 0.0) {
        double f = or_kernel_w(p->h, r) / or_kernel_w(p->h, p->dp);
        T = tensile_r(p, Pa, rhoa, Pb, rhob) * pow(f, (double)p->tensile_n);
    }
    for (int d = 0; d < 3; ++d) o->acc[d] = 0.0;
    if (momentum) {
        double coef = -p->mass * (Pa / (rhoa * rhoa) + Pb / (rhob * rhob) + Pi + T);
        for (int d = 0; d < 3; ++d) o->acc[d] = coef * (F * r_ab[d]);
    }
    o->ar = p->mass * (vdr * F);
    o->visc = fabs(mu);
}

/* Neighbour lists of the fluid and of the boundary particles. */
typedef struct {
    int64_t dims[3], nc;
    int64_t nf, nb;
    int64_t *cell;    /* [nf + nb] cell of each particle (id order) */
    int64_t *ford, *fstart;   /* fluid list */
    int64_t *bord, *bstart;   /* boundary list (indices are nf + k) */
} or_lists;

static void lists_free(or_lists *L)
{
    free(L->cell); free(L->ford); free(L->fstart); free(L->bord); free(L->bstart);
    memset(L, 0, sizeof(*L));
}

static int lists_build(const or_params *p, int64_t nf, int64_t nb, const double *pos, or_lists *L)
{
    memset(L, 0, sizeof(*L));
    if (or_grid(p, L->dims)) return -1;
    L->nc = L->dims[0] * L->dims[1] * L->dims[2];
    L->nf = nf; L->nb = nb;
    L->cell = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nf + nb + 1));
    L->ford = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nf + 1));
    L->bord = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nb + 1));
    L->fstart = (int64_t *)malloc(sizeof(int64_t) * (size_t)(L->nc + 2));
    L->bstart = (int64_t *)malloc(sizeof(int64_t) * (size_t)(L->nc + 2));
    if (!L->cell || !L->ford || !L->bord || !L->fstart || !L->bstart) { lists_free(L); return -1; }
    or_cells(p, nf + nb, pos, L->cell);
    or_list(p, nf, L->cell, L->ford, L->fstart);
    or_list(p, nb, L->cell + nf, L->bord, L->bstart);
    for (int64_t k = 0; k < nb; ++k) L->bord[k] += nf;
    return 0;
}

/* Visit the members of the 27 cells around cell c of one list, in the order
 * dz, dy, dx = -1, 0, 1 and, inside a cell, list order. */
#define FOR_NEIGHBOURS(L, c, ord, start, j, BODY)                                   \
    do {                                                                            \
        int64_t cx_ = (c) % (L)->dims[0];                                           \
        int64_t cy_ = ((c) / (L)->dims[0]) % (L)->dims[1];                          \
        int64_t cz_ = (c) / ((L)->dims[0] * (L)->dims[1]);                          \
        for (int64_t dz_ = -1; dz_ <= 1; ++dz_) {                                   \
            int64_t z_ = cz_ + dz_;                                                 \
            if (z_ < 0 || z_ >= (L)->dims[2]) continue;                             \
            for (int64_t dy_ = -1; dy_ <= 1; ++dy_) {                               \
                int64_t y_ = cy_ + dy_;                                             \
                if (y_ < 0 || y_ >= (L)->dims[1]) continue;                         \
                for (int64_t dx_ = -1; dx_ <= 1; ++dx_) {                           \
                    int64_t x_ = cx_ + dx_;                                         \
                    if (x_ < 0 || x_ >= (L)->dims[0]) continue;                     \
                    int64_t cc_ = x_ + (L)->dims[0] * (y_ + (L)->dims[1] * z_);     \
                    for (int64_t k_ = (start)[cc_]; k_ < (start)[cc_ + 1]; ++k_) {  \
                        int64_t j = (ord)[k_];                                      \
                        BODY                                                        \
                    }                                                               \
                }                                                                   \
            }                                                                       \
        }                                                                           \
    } while (0)

/* Enumerate every ordered interacting pair (a, b): a != b, |x_a - x_b| < 2h,
 * type F-F, F-B or B-F (never B-B, Section 2).  Writes up to cap pairs and
 * the total count.  Used by the tests (brute-force pin) and the gradient oracle. */
int or_pairs(const or_params *p, int64_t nf, int64_t nb, const double *pos,
             int64_t *pa, int64_t *pb, int64_t cap, int64_t *npairs)
{
    or_lists L;
    if (lists_build(p, nf, nb, pos, &L)) return -1;
    double s2 = 4.0 * p->h * p->h;
    int64_t np = 0;
    for (int64_t a = 0; a < nf + nb; ++a) {
        int64_t c = L.cell[a];
        if (c >= L.nc) continue;
        const double *xa = pos + 3 * a;
#define OR_PAIR_BODY                                                               \
        if (j != a) {                                                              \
            const double *xb = pos + 3 * j;                                        \
            double dx = xa[0] - xb[0], dy = xa[1] - xb[1], dz = xa[2] - xb[2];     \
            if (dx * dx + dy * dy + dz * dz < s2) {                                \
                if (np < cap) { pa[np] = a; pb[np] = j; }                          \
                np++;                                                              \
            }                                                                      \
        }
        FOR_NEIGHBOURS(&L, c, L.ford, L.fstart, j, OR_PAIR_BODY);
        if (a < nf) FOR_NEIGHBOURS(&L, c, L.bord, L.bstart, j, OR_PAIR_BODY);
#undef OR_PAIR_BODY
    }
    *npairs = np;
    lists_free(&L);
    return 0;
}

/* PI for the targets a with a % stride == 0 (stride 1: all particles; a
 * larger stride times a uniform sample of the targets, the others get zero
 * outputs).  seconds (may be NULL) receives the wall time of the list build
 * and of the interaction loop.  Outputs (id order): ace[3*nf] (fluid acceleration
 * including gravity), ar[nf + nb] (density rate), the largest viscous term and
 * work counts: counts[0] candidates visited by fluid targets, counts[1] their
 * pairs, counts[2] candidates of boundary targets, counts[3] their pairs.
 * A candidate is a particle of the 27 cells (other than the target).
 * Returns the number of particles outside the cell grid. */
int64_t or_interact_sampled(const or_params *p, int64_t nf, int64_t nb,
                            const double *pos, const double *vel, const double *rho,
                            double *ace, double *ar, double *viscdt_max, int64_t *counts,
                            int nthreads, int64_t stride, double *seconds)
{
    or_lists L;
#ifdef _OPENMP
    double t0 = omp_get_wtime();
#endif
    if (lists_build(p, nf, nb, pos, &L)) return -1;
#ifdef _OPENMP
    double t1 = omp_get_wtime();
#endif
    if (stride < 1) stride = 1;
    int64_t n = nf + nb;
    double *P = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double *C = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    for (int64_t i = 0; i < n; ++i) { P[i] = or_pressure(p, rho[i]); C[i] = or_sound(p, rho[i]); }
    double s2 = 4.0 * p->h * p->h;
    double vmax = 0.0;
    int64_t cf = 0, pf = 0, cb = 0, pbn = 0, nout = 0;
    for (int64_t i = 0; i < n; ++i) if (L.cell[i] >= L.nc) nout++;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 256) reduction(max : vmax) reduction(+ : cf, pf, cb, pbn)
    for (int64_t a = 0; a < n; ++a) {
        int64_t c = L.cell[a];
        int fluid = a < nf;
        double acc[3] = {0.0, 0.0, 0.0}, dr = 0.0, vm = 0.0;
        int64_t ncand = 0, npair = 0;
        if (c < L.nc && a % stride == 0) {
            const double *xa = pos + 3 * a;
            const double *va = vel + 3 * a;
#define OR_PI_BODY                                                                  \
            if (j != a) {                                                           \
                const double *xb = pos + 3 * j;                                     \
                double dx = xa[0] - xb[0], dy = xa[1] - xb[1], dz = xa[2] - xb[2];  \
                ncand++;                                                            \
                if (dx * dx + dy * dy + dz * dz < s2) {                             \
                    pair_out o;                                                     \
                    pair_terms(p, fluid, xa, va, rho[a], P[a], C[a],                \
                               xb, vel + 3 * j, rho[j], P[j], C[j], &o);            \
                    acc[0] += o.acc[0]; acc[1] += o.acc[1]; acc[2] += o.acc[2];     \
                    dr += o.ar;                                                     \
                    if (o.visc > vm) vm = o.visc;                                   \
                    npair++;                                                        \
                }                                                                   \
            }
            /* fluid neighbours (F-F or B-F), then boundary neighbours (F-B only) */
            FOR_NEIGHBOURS(&L, c, L.ford, L.fstart, j, OR_PI_BODY);
            if (fluid) FOR_NEIGHBOURS(&L, c, L.bord, L.bstart, j, OR_PI_BODY);
#undef OR_PI_BODY
        }
        if (fluid) {
            if (c < L.nc) {
                for (int d = 0; d < 3; ++d) ace[3 * a + d] = acc[d] + p->g[d];
            } else {
                for (int d = 0; d < 3; ++d) ace[3 * a + d] = 0.0;
            }
            cf += ncand; pf += npair;
        } else {
            cb += ncand; pbn += npair;
        }
        ar[a] = dr;
        if (vm > vmax) vmax = vm;
    }
    *viscdt_max = vmax;
    if (counts) { counts[0] = cf; counts[1] = pf; counts[2] = cb; counts[3] = pbn; }
    free(P); free(C);
    lists_free(&L);
#ifdef _OPENMP
    if (seconds) { seconds[0] = t1 - t0; seconds[1] = omp_get_wtime() - t1; }
#else
    if (seconds) { seconds[0] = 0.0; seconds[1] = 0.0; }
#endif
    return nout;
}

/* PI for every target (see or_interact_sampled, stride 1). */
int64_t or_interact(const or_params *p, int64_t nf, int64_t nb,
                    const double *pos, const double *vel, const double *rho,
                    double *ace, double *ar, double *viscdt_max, int64_t *counts,
                    int nthreads)
{
    return or_interact_sampled(p, nf, nb, pos, vel, rho, ace, ar, viscdt_max, counts,
                               nthreads, 1, NULL);
}

/* Variable time step (Monaghan & Kos 1999; Table 1; the maxima of Section
 * 4.1):  dt = CFL * min( min_a sqrt(h / |f_a|),  h / (max_a c_a + max_ab |mu_ab|) ),
 * with f over the fluid particles (gravity included) and c over all particles
 * inside the grid. */
double or_dt(const or_params *p, int64_t nf, int64_t nb, const double *pos,
             const double *ace, const double *rho, double viscdt_max)
{
    if (p->fixed_dt > 0.0) return p->fixed_dt;
    int64_t dims[3];
    or_grid(p, dims);
    int64_t nc = dims[0] * dims[1] * dims[2];
    double dtf = INFINITY, cmax = 0.0;
    for (int64_t a = 0; a < nf + nb; ++a) {
        if (cell_of(p, dims, pos + 3 * a) >= nc) continue;
        if (a < nf) {
            double f = sqrt(ace[3 * a] * ace[3 * a] + ace[3 * a + 1] * ace[3 * a + 1] +
                            ace[3 * a + 2] * ace[3 * a + 2]);
            double t = sqrt(p->h / f);
            if (t < dtf) dtf = t;
        }
        double c = or_sound(p, rho[a]);
        if (c > cmax) cmax = c;
    }
    double dtcv = p->h / (cmax + viscdt_max);
    double m = dtf < dtcv ? dtf : dtcv;
    return p->cfl * m;
}

/* Verlet scheme (Verlet 1967, as in SPHysics; Table 1) for step index n
 * (0-based, counting completed steps):
 *   if (n + 1) % N_s != 0:  v^{n+1} = v^{n-1} + 2 dt F^n,  rho^{n+1} = rho^{n-1} + 2 dt D^n
 *   else (Euler):           v^{n+1} = v^n + dt F^n,        rho^{n+1} = rho^n + dt D^n
 *   always:                 x^{n+1} = x^n + dt v^n + 0.5 dt^2 F^n
 * Boundary particles keep x and v and update rho only, clamped at rho0 from
 * below.  Particles outside the grid are left unchanged. */
void or_update(const or_params *p, int64_t nf, int64_t nb, int64_t step, double dt,
               double *pos, double *vel, double *velm1, double *rho, double *rhom1,
               const double *ace, const double *ar)
{
    int64_t dims[3];
    or_grid(p, dims);
    int64_t nc = dims[0] * dims[1] * dims[2];
    int euler = ((step + 1) % p->verlet_euler_every) == 0;
    for (int64_t a = 0; a < nf + nb; ++a) {
        if (cell_of(p, dims, pos + 3 * a) >= nc) continue;
        double rnew = euler ? rho[a] + dt * ar[a] : rhom1[a] + 2.0 * dt * ar[a];
        if (a >= nf) {
            if (p->clamp_boundary_rho && rnew < p->rho0) rnew = p->rho0;
        } else {
            for (int d = 0; d < 3; ++d) {
                double x = pos[3 * a + d], v = vel[3 * a + d], f = ace[3 * a + d];
                double vnew = euler ? v + dt * f : velm1[3 * a + d] + 2.0 * dt * f;
                pos[3 * a + d] = x + dt * v + 0.5 * dt * dt * f;
                velm1[3 * a + d] = v;
                vel[3 * a + d] = vnew;
            }
        }
        rhom1[a] = rho[a];
        rho[a] = rnew;
    }
}

/* One full step NL -> PI -> SU.  Returns the number of particles outside the
 * grid (negative on allocation failure); dt_out receives the step used. */
int64_t or_step(const or_params *p, int64_t nf, int64_t nb, int64_t step,
                double *pos, double *vel, double *velm1, double *rho, double *rhom1,
                double *dt_out, int64_t *counts, int nthreads)
{
    int64_t n = nf + nb;
    double *ace = (double *)malloc(sizeof(double) * (size_t)(3 * nf + 3));
    double *ar = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    if (!ace || !ar) { free(ace); free(ar); return -1; }
    double vmax = 0.0;
    int64_t nout = or_interact(p, nf, nb, pos, vel, rho, ace, ar, &vmax, counts, nthreads);
    if (nout < 0) { free(ace); free(ar); return nout; }
    double dt = or_dt(p, nf, nb, pos, ace, rho, vmax);
    or_update(p, nf, nb, step, dt, pos, vel, velm1, rho, rhom1, ace, ar);
    if (dt_out) *dt_out = dt;
    free(ace); free(ar);
    return nout;
}

/* Pressure at sensor points by a Shepard-normalised kernel sum over the fluid
 * particles within 2h:  P_s = sum_b (m/rho_b) P_b W_sb / sum_b (m/rho_b) W_sb,
 * 0 where no fluid particle is in range.  A plain loop over all particles. */
void or_sensor_pressure(const or_params *p, int64_t nf, const double *pos, const double *rho,
                        int64_t ns, const double *spos, double *out)
{
    for (int64_t s = 0; s < ns; ++s) {
        double num = 0.0, den = 0.0;
        for (int64_t b = 0; b < nf; ++b) {
            double dx = spos[3 * s] - pos[3 * b], dy = spos[3 * s + 1] - pos[3 * b + 1],
                   dz = spos[3 * s + 2] - pos[3 * b + 2];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            if (r >= 2.0 * p->h) continue;
            double w = or_kernel_w(p->h, r) * p->mass / rho[b];
            num += w * or_pressure(p, rho[b]);
            den += w;
        }
        out[s] = den > 0.0 ? num / den : 0.0;
    }
}
