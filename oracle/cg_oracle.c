/*
 * cg_oracle.c -- plain FP64 CPU oracle of the particle <-> dual-grid
 * coupling step of arXiv 1807.11834 (see cg_oracle.h).
 *
 * TEST INFRASTRUCTURE ONLY: called by the tests, the smoke check and the
 * CPU baseline of the benchmark; never by the CUDA library.
 *
 * Compile with -ffp-contract=off: every product and sum below is rounded
 * on its own, as written.  The OpenMP pragmas mark loops whose iterations
 * are independent (one particle, one cell, one fine cell each); a build
 * with -fopenmp runs them on several threads with bit-identical results,
 * and a build without it ignores them.  Sorts and global sums stay
 * sequential.
 *
 * What the paper fixes and what is a reading of it:
 *  - Fig. 1 / Sec. 2.1: a coarse uniform "bulk" grid maps Lagrangian fields
 *    to Eulerian ones and solves the fluid-particle interaction; a fine grid
 *    carries the fluid.  Particle fields go bulk -> fine, the fluid solution
 *    fine -> bulk.
 *  - Table 1: porosity field from sum_i V_pi / V_cell over the n_pc particles
 *    of a cell; Sec. 2.4 defines porosity as fluid volume over cell volume.
 *    Reading: solid fraction phi = sum V_p / V_B, porosity eps = 1 - phi,
 *    deposit at the particle centre's cell.
 *  - Eq. (DragLaw): F_drag = beta (u_f - u_p), beta depending on slip,
 *    densities, diameter, area, viscosity and porosity.  The correlation
 *    itself is not printed; the readings are Di Felice and Ergun / Wen-Yu
 *    (Gidaspow), see or_drag_beta.
 *  - Sec. 1: the coupling takes the cell value or a value interpolated locally;
 *    reading: trilinear interpolation from bulk-cell centres with constant
 *    extrapolation in the outer half cell (or the cell value).
 *  - Eq. (UFP): F_fpi is the fluid-side reaction to F_drag; reading: the bulk source
 *    is S_B = -(1/V_B) sum_{p in B} F_p.
 *  - Eq. (DEM_EQUATIONS): m x'' = F_coll + F_drag + F_g; contacts are out of
 *    scope, the integrator is a reading (velocity first, then position).
 */
#include "cg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- */
/* Neumaier compensated sum                                          */
/* ---------------------------------------------------------------- */
typedef struct { double s, c; } ksum;

static void ks_add(ksum* k, double x)
{
    double t = k->s + x;
    if (fabs(k->s) >= fabs(x)) k->c += (k->s - t) + x;
    else                       k->c += (x - t) + k->s;
    k->s = t;
}

static double ks_get(const ksum* k) { return k->s + k->c; }

/* ---------------------------------------------------------------- */
/* Grid geometry                                                     */
/* ---------------------------------------------------------------- */
typedef struct {
    int32_t nb[3];
    double H[3], h[3];
    double VB, Vf;
    int64_t nbulk, nfine;
} geom;

static geom geometry(const or_grid* G)
{
    geom g;
    for (int a = 0; a < 3; ++a) {
        g.nb[a] = G->nf[a] / G->r;
        g.H[a] = G->L[a] / (double)g.nb[a];
        g.h[a] = G->L[a] / (double)G->nf[a];
    }
    g.VB = g.H[0] * g.H[1] * g.H[2];
    g.Vf = g.h[0] * g.h[1] * g.h[2];
    g.nbulk = (int64_t)g.nb[0] * g.nb[1] * g.nb[2];
    g.nfine = (int64_t)G->nf[0] * G->nf[1] * G->nf[2];
    return g;
}

static double sphere_volume(double d) { return M_PI * d * d * d / 6.0; }

/* ---------------------------------------------------------------- */
/* Bin index: i = clamp(floor((x - x0) / H), 0, nb - 1) per axis.    */
/* Half-open cells; x = x0 + L belongs to the last cell; a point     */
/* whose quotient lies outside [0, nb] (or is NaN) is outside.       */
/* ---------------------------------------------------------------- */
int32_t or_bin_cell(const or_grid* G, const double x[3], int* outside)
{
    geom g = geometry(G);
    int idx[3];
    int out = 0;
    for (int a = 0; a < 3; ++a) {
        double q = (x[a] - G->x0[a]) / g.H[a];
        int i;
        if (!(q >= 0.0)) i = 0;                 /* negative or NaN */
        else if (q >= (double)g.nb[a]) i = g.nb[a] - 1;
        else i = (int)floor(q);
        if (!(q >= 0.0 && q <= (double)g.nb[a])) out = 1;
        idx[a] = i;
    }
    if (outside) *outside = out;
    return idx[0] + g.nb[0] * (idx[1] + g.nb[1] * idx[2]);
}

/* Stable counting sort: particles of cell c are perm[cell_start[c] ..
 * cell_start[c+1]) in increasing original index (the per-step particle to
 * cell connectivity of Sec. 2.2). */
int64_t or_bin(const or_grid* G, int64_t n, const double* pos_d,
               int32_t* cell, int32_t* perm, int32_t* cell_start)
{
    geom g = geometry(G);
    int64_t outside = 0;
    int32_t* cursor = (int32_t*)calloc((size_t)g.nbulk + 1, sizeof(int32_t));
    for (int64_t c = 0; c <= g.nbulk; ++c) cell_start[c] = 0;
    for (int64_t p = 0; p < n; ++p) {
        int o = 0;
        cell[p] = or_bin_cell(G, &pos_d[4 * p], &o);
        outside += o;
        cell_start[cell[p] + 1] += 1;
    }
    for (int64_t c = 0; c < g.nbulk; ++c) cell_start[c + 1] += cell_start[c];
    for (int64_t c = 0; c < g.nbulk; ++c) cursor[c] = cell_start[c];
    for (int64_t p = 0; p < n; ++p) perm[cursor[cell[p]]++] = (int32_t)p;
    free(cursor);
    return outside;
}

/* Porosity (Table 1 and Sec. 2.4): phi_B = sum V_p / V_B, eps = 1 - phi. */
void or_deposit_volume(const or_grid* G, int64_t n, const double* pos_d,
                       const int32_t* cell_start, const int32_t* perm,
                       double* eps, double* phi)
{
    (void)n;
    geom g = geometry(G);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < g.nbulk; ++c) {
        ksum k = {0.0, 0.0};
        for (int32_t i = cell_start[c]; i < cell_start[c + 1]; ++i)
            ks_add(&k, sphere_volume(pos_d[4 * (int64_t)perm[i] + 3]));
        double ph = ks_get(&k) / g.VB;
        if (phi) phi[c] = ph;
        eps[c] = 1.0 - ph;
    }
}

/* Fine -> bulk transfer of the fluid solution (Fig. 1): for nested uniform
 * grids the volume-weighted average over the overlap is the plain mean of
 * the r^3 fine cells inside the bulk cell.  The variance is two-pass. */
void or_average(const or_grid* G, const double* u_fine, double* u_bulk, double* var_bulk)
{
    geom g = geometry(G);
    const int r = G->r;
    const int64_t nxf = G->nf[0], nyf = G->nf[1];
    const double cnt = (double)r * r * r;
#pragma omp parallel for schedule(static)
    for (int K = 0; K < g.nb[2]; ++K)
    for (int J = 0; J < g.nb[1]; ++J)
    for (int I = 0; I < g.nb[0]; ++I) {
        int64_t cb = I + (int64_t)g.nb[0] * (J + (int64_t)g.nb[1] * K);
        double mean[3];
        for (int comp = 0; comp < 3; ++comp) {
            ksum k = {0.0, 0.0};
            for (int dk = 0; dk < r; ++dk)
            for (int dj = 0; dj < r; ++dj)
            for (int di = 0; di < r; ++di) {
                int64_t f = (I * r + di) + nxf * ((J * r + dj) + nyf * (int64_t)(K * r + dk));
                ks_add(&k, u_fine[comp * g.nfine + f]);
            }
            mean[comp] = ks_get(&k) / cnt;
            u_bulk[comp * g.nbulk + cb] = mean[comp];
        }
        if (var_bulk) {
            ksum k = {0.0, 0.0};
            for (int dk = 0; dk < r; ++dk)
            for (int dj = 0; dj < r; ++dj)
            for (int di = 0; di < r; ++di) {
                int64_t f = (I * r + di) + nxf * ((J * r + dj) + nyf * (int64_t)(K * r + dk));
                for (int comp = 0; comp < 3; ++comp) {
                    double dv = u_fine[comp * g.nfine + f] - mean[comp];
                    ks_add(&k, dv * dv);
                }
            }
            var_bulk[cb] = ks_get(&k) / cnt;
        }
    }
}

/* Trilinear weights from bulk-cell centres: xi = (x - x0)/H - 1/2,
 * i0 = clamp(floor xi, 0, nb - 2), t = clamp(xi - i0, 0, 1). */
void or_weights(const or_grid* G, const double x[3], int32_t i0[3], double t[3], int clamped[3])
{
    geom g = geometry(G);
    for (int a = 0; a < 3; ++a) {
        double xi = (x[a] - G->x0[a]) / g.H[a] - 0.5;
        int i;
        if (!(xi >= 0.0)) i = 0;
        else if (xi >= (double)(g.nb[a] - 2)) i = g.nb[a] - 2;
        else i = (int)floor(xi);
        double tt = xi - (double)i;
        int cl = 0;
        if (!(tt >= 0.0)) { tt = 0.0; cl = 1; }
        else if (tt > 1.0) { tt = 1.0; cl = 1; }
        i0[a] = i;
        t[a] = tt;
        if (clamped) clamped[a] = cl;
    }
}

void or_gather(const or_grid* G, const double* bulk, int ncomp, const double x[3], double* out)
{
    geom g = geometry(G);
    if (G->interp == 1) {
        int32_t c = or_bin_cell(G, x, NULL);
        for (int comp = 0; comp < ncomp; ++comp) out[comp] = bulk[comp * g.nbulk + c];
        return;
    }
    int32_t i0[3];
    double t[3];
    or_weights(G, x, i0, t, NULL);
    for (int comp = 0; comp < ncomp; ++comp) {
        double acc = 0.0;
        for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
            double w = (dx ? t[0] : 1.0 - t[0]) * (dy ? t[1] : 1.0 - t[1]) * (dz ? t[2] : 1.0 - t[2]);
            int64_t c = (i0[0] + dx) + (int64_t)g.nb[0] * ((i0[1] + dy) + (int64_t)g.nb[1] * (i0[2] + dz));
            acc += w * bulk[comp * g.nbulk + c];
        }
        out[comp] = acc;
    }
}

void or_gather_grad(const or_grid* G, const double* bulk, const double x[3], double grad[3])
{
    geom g = geometry(G);
    int32_t i0[3];
    double t[3];
    int cl[3];
    or_weights(G, x, i0, t, cl);
    for (int a = 0; a < 3; ++a) {
        double acc = 0.0;
        if (!cl[a] && G->interp == 0) {
            for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                int d3[3] = {dx, dy, dz};
                double w = 1.0;
                for (int b = 0; b < 3; ++b) {
                    if (b == a) w *= d3[b] ? 1.0 : -1.0;
                    else w *= d3[b] ? t[b] : 1.0 - t[b];
                }
                int64_t c = (i0[0] + dx) + (int64_t)g.nb[0] * ((i0[1] + dy) + (int64_t)g.nb[1] * (i0[2] + dz));
                acc += w * bulk[c];
            }
            acc /= g.H[a];
        }
        grad[a] = acc;
    }
}

/* Per-particle drag factor of Eq. (DragLaw), F = beta_p (u_f - u_p).
 *
 * Di Felice (law 0):  Re = rho_f eps d |s| / mu_f,
 *   C_D0 = (0.63 + 4.8 / sqrt(Re))^2,
 *   chi  = 3.7 - 0.65 exp(-(1.5 - log10 Re)^2 / 2),
 *   F    = 1/2 C_D0 rho_f (pi d^2 / 4) eps^2 |s| s eps^(-chi),
 *   with C_D0 |s| written as (0.63 sqrt|s| + 4.8 sqrt(mu_f / (rho_f eps d)))^2
 *   so that zero slip gives zero force, and chi = 3.7 at Re = 0.
 *
 * Ergun / Wen-Yu (law 1, Gidaspow):  Re = rho_f d |s| / mu_f,
 *   eps <  eps_switch: beta = 150 (1-eps)^2 mu_f / (eps d^2) + 1.75 (1-eps) rho_f |s| / d
 *   eps >= eps_switch: C_D = 24 / (eps Re) (1 + 0.15 (eps Re)^0.687)  (eps Re < 1000), else 0.44
 *                      beta = 3/4 C_D eps (1-eps) rho_f |s| eps^(-2.65) / d
 *   and the force on one particle is beta V_p / (1 - eps) s; the factor
 *   (1 - eps) is cancelled algebraically (finite at eps = 1) and C_D |s| is
 *   expanded so that Re = 0 is finite.
 *
 * The porosity is raised to eps_min when smaller (over-packed cells). */
double or_drag_beta(const or_grid* G, double eps, double d, const double s[3], int* clamped)
{
    int cl = 0;
    if (eps < G->eps_min) { eps = G->eps_min; cl = 1; }
    if (clamped) *clamped = cl;
    const double rho = G->rho_f, mu = G->mu_f;
    const double smag = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    if (G->law == 0) {
        double Re = rho * eps * d * smag / mu;
        double cd_s = 0.63 * sqrt(smag) + 4.8 * sqrt(mu / (rho * eps * d));
        cd_s = cd_s * cd_s;                                  /* C_D0 |s| */
        double chi = 3.7;
        if (Re > 0.0) {
            double l = 1.5 - log10(Re);
            chi = 3.7 - 0.65 * exp(-l * l / 2.0);
        }
        return 0.5 * cd_s * rho * (M_PI * d * d / 4.0) * eps * eps * pow(eps, -chi);
    } else {
        double vp = sphere_volume(d);
        if (eps < G->eps_switch) {
            double phi = 1.0 - eps;
            /* beta * V_p / (1 - eps) with one factor (1 - eps) cancelled */
            return (150.0 * phi * mu / (eps * d * d) + 1.75 * rho * smag / d) * vp;
        } else {
            double Re = rho * d * smag / mu;
            double eRe = eps * Re;
            double cd_s;                                      /* C_D |s| */
            if (eRe < 1000.0) cd_s = 24.0 * mu / (eps * rho * d) * (1.0 + 0.15 * pow(eRe, 0.687));
            else cd_s = 0.44 * smag;
            return 0.75 * cd_s * eps * rho * pow(eps, -2.65) / d * vp;
        }
    }
}

int64_t or_drag(const or_grid* G, int64_t n, const double* pos_d, const double* vel,
                const double* eps_bulk, const double* u_bulk, double* force)
{
    int64_t nclamped = 0;
#pragma omp parallel for schedule(static) reduction(+ : nclamped)
    for (int64_t p = 0; p < n; ++p) {
        const double* x = &pos_d[4 * p];
        double eps_p, uf[3], s[3];
        or_gather(G, eps_bulk, 1, x, &eps_p);
        or_gather(G, u_bulk, 3, x, uf);
        for (int a = 0; a < 3; ++a) s[a] = uf[a] - vel[4 * p + a];
        int cl = 0;
        double beta = or_drag_beta(G, eps_p, x[3], s, &cl);
        nclamped += cl;
        for (int a = 0; a < 3; ++a) force[a * n + p] = beta * s[a];
    }
    return nclamped;
}

void or_particle_state(const or_grid* G, int64_t n, const double* pos_d, const double* vel,
                       const double* eps_bulk, const double* u_bulk, double* eps_p, double* slip)
{
    for (int64_t p = 0; p < n; ++p) {
        const double* x = &pos_d[4 * p];
        double uf[3];
        or_gather(G, eps_bulk, 1, x, &eps_p[p]);
        or_gather(G, u_bulk, 3, x, uf);
        double s2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            double s = uf[a] - vel[4 * p + a];
            s2 += s * s;
        }
        slip[p] = sqrt(s2);
    }
}

void or_mlp_features(const or_grid* G, int64_t n, const double* pos_d, const double* vel,
                     const double* eps_bulk, const double* u_stale, const double* var_stale,
                     const double* u_fresh, double* feat, double* target, double* F_stale)
{
    for (int64_t p = 0; p < n; ++p) {
        const double* x = &pos_d[4 * p];
        const double d = x[3];
        double eps, us[3], uf[3], var, grad[3], ss[3], sf[3];
        or_gather(G, eps_bulk, 1, x, &eps);
        or_gather(G, u_stale, 3, x, us);
        or_gather(G, u_fresh, 3, x, uf);
        or_gather(G, var_stale, 1, x, &var);
        or_gather_grad(G, eps_bulk, x, grad);
        for (int a = 0; a < 3; ++a) {
            ss[a] = us[a] - vel[4 * p + a];
            sf[a] = uf[a] - vel[4 * p + a];
        }
        const double epsc = eps < G->eps_min ? G->eps_min : eps;
        const double smag = sqrt(ss[0] * ss[0] + ss[1] * ss[1] + ss[2] * ss[2]);
        const double Re = G->rho_f * epsc * d * smag / G->mu_f;
        double* f = &feat[7 * p];
        f[0] = epsc;
        f[1] = log10(1.0 + Re);
        f[2] = smag;
        f[3] = grad[0];
        f[4] = grad[1];
        f[5] = grad[2];
        f[6] = var;
        const double bs = or_drag_beta(G, eps, d, ss, NULL);
        const double bf = or_drag_beta(G, eps, d, sf, NULL);
        double dot = 0.0, nn = 0.0;
        for (int a = 0; a < 3; ++a) {
            const double Fs = bs * ss[a], Ff = bf * sf[a];
            F_stale[a * n + p] = Fs;
            dot += Ff * Fs;
            nn += Fs * Fs;
        }
        target[p] = nn > 0.0 ? dot / nn : 1.0;
    }
}

void or_deposit_momentum(const or_grid* G, int64_t n, const double* force,
                         const int32_t* cell_start, const int32_t* perm, double* S_bulk)
{
    geom g = geometry(G);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < g.nbulk; ++c) {
        for (int comp = 0; comp < 3; ++comp) {
            ksum k = {0.0, 0.0};
            for (int32_t i = cell_start[c]; i < cell_start[c + 1]; ++i)
                ks_add(&k, force[comp * n + perm[i]]);
            S_bulk[comp * g.nbulk + c] = -ks_get(&k) / g.VB;
        }
    }
}

/* Semi-implicit exchange coefficients: the drag factor beta_p of each
 * particle (the same gather and correlation as or_drag), summed per cell in
 * the stable order and divided by the cell volume. */
void or_implicit(const or_grid* G, int64_t n, const double* pos_d, const double* vel,
                 const double* eps_bulk, const double* u_bulk, const int32_t* cell_start,
                 const int32_t* perm, double* coef)
{
    geom g = geometry(G);
    for (int64_t c = 0; c < g.nbulk; ++c) {
        ksum k[4];
        memset(k, 0, sizeof k);
        for (int32_t i = cell_start[c]; i < cell_start[c + 1]; ++i) {
            const int64_t p = perm[i];
            const double* x = &pos_d[4 * p];
            double eps_p, uf[3], s[3];
            or_gather(G, eps_bulk, 1, x, &eps_p);
            or_gather(G, u_bulk, 3, x, uf);
            for (int a = 0; a < 3; ++a) s[a] = uf[a] - vel[4 * p + a];
            const double beta = or_drag_beta(G, eps_p, x[3], s, NULL);
            ks_add(&k[0], beta);
            for (int a = 0; a < 3; ++a) ks_add(&k[1 + a], beta * vel[4 * p + a]);
        }
        for (int comp = 0; comp < 4; ++comp) coef[comp * g.nbulk + c] = ks_get(&k[comp]) / g.VB;
    }
}

/* ---------------------------------------------------------------- */
/* Non-nested grid maps                                               */
/* ---------------------------------------------------------------- */
static double box_lo(const or_box_grid* G, int a, int64_t i) { return G->x0[a] + (double)i * (G->L[a] / G->n[a]); }

/* Length of the overlap of [a0, a1) and [b0, b1). */
static double overlap(double a0, double a1, double b0, double b1)
{
    const double lo = a0 > b0 ? a0 : b0, hi = a1 < b1 ? a1 : b1;
    return hi > lo ? hi - lo : 0.0;
}

/* Cells of grid G along axis a that may overlap [lo, hi): [*i0, *i1]. */
static void index_range(const or_box_grid* G, int a, double lo, double hi, int64_t* i0, int64_t* i1)
{
    const double h = G->L[a] / G->n[a];
    int64_t a0 = (int64_t)floor((lo - G->x0[a]) / h) - 1, a1 = (int64_t)floor((hi - G->x0[a]) / h) + 1;
    if (a0 < 0) a0 = 0;
    if (a1 > G->n[a] - 1) a1 = G->n[a] - 1;
    *i0 = a0;
    *i1 = a1;
}

/* Intersection volume of cell (i, j, k) of A with cell (p, q, r) of B. */
static double cell_overlap(const or_box_grid* A, const int64_t ia[3], const or_box_grid* B, const int64_t ib[3])
{
    double v = 1.0;
    for (int a = 0; a < 3; ++a)
        v *= overlap(box_lo(A, a, ia[a]), box_lo(A, a, ia[a] + 1), box_lo(B, a, ib[a]), box_lo(B, a, ib[a] + 1));
    return v;
}

void or_map_average(const or_box_grid* bulk, const or_box_grid* fine, int ncomp, const double* u_fine,
                    double* u_bulk)
{
    const int64_t nbk = (int64_t)bulk->n[0] * bulk->n[1] * bulk->n[2];
    const int64_t nfn = (int64_t)fine->n[0] * fine->n[1] * fine->n[2];
    int64_t B[3];
    for (B[2] = 0; B[2] < bulk->n[2]; ++B[2])
    for (B[1] = 0; B[1] < bulk->n[1]; ++B[1])
    for (B[0] = 0; B[0] < bulk->n[0]; ++B[0]) {
        const int64_t cb = B[0] + (int64_t)bulk->n[0] * (B[1] + (int64_t)bulk->n[1] * B[2]);
        int64_t r0[3], r1[3];
        for (int a = 0; a < 3; ++a) index_range(fine, a, box_lo(bulk, a, B[a]), box_lo(bulk, a, B[a] + 1), &r0[a], &r1[a]);
        ksum w = {0.0, 0.0};
        ksum acc[8];
        memset(acc, 0, sizeof acc);
        int64_t f[3];
        for (f[2] = r0[2]; f[2] <= r1[2]; ++f[2])
        for (f[1] = r0[1]; f[1] <= r1[1]; ++f[1])
        for (f[0] = r0[0]; f[0] <= r1[0]; ++f[0]) {
            const double v = cell_overlap(bulk, B, fine, f);
            if (v == 0.0) continue;
            const int64_t cf = f[0] + (int64_t)fine->n[0] * (f[1] + (int64_t)fine->n[1] * f[2]);
            ks_add(&w, v);
            for (int c = 0; c < ncomp; ++c) ks_add(&acc[c], v * u_fine[c * nfn + cf]);
        }
        const double W = ks_get(&w);
        for (int c = 0; c < ncomp; ++c) u_bulk[c * nbk + cb] = W > 0.0 ? ks_get(&acc[c]) / W : 0.0;
    }
}

void or_map_project(const or_box_grid* bulk, const or_box_grid* fine, int ncomp, const double* s_bulk,
                    double* s_fine)
{
    const int64_t nbk = (int64_t)bulk->n[0] * bulk->n[1] * bulk->n[2];
    const int64_t nfn = (int64_t)fine->n[0] * fine->n[1] * fine->n[2];
    const double Vf = (fine->L[0] / fine->n[0]) * (fine->L[1] / fine->n[1]) * (fine->L[2] / fine->n[2]);
    int64_t f[3];
    for (f[2] = 0; f[2] < fine->n[2]; ++f[2])
    for (f[1] = 0; f[1] < fine->n[1]; ++f[1])
    for (f[0] = 0; f[0] < fine->n[0]; ++f[0]) {
        const int64_t cf = f[0] + (int64_t)fine->n[0] * (f[1] + (int64_t)fine->n[1] * f[2]);
        int64_t r0[3], r1[3];
        for (int a = 0; a < 3; ++a) index_range(bulk, a, box_lo(fine, a, f[a]), box_lo(fine, a, f[a] + 1), &r0[a], &r1[a]);
        ksum acc[8];
        memset(acc, 0, sizeof acc);
        int64_t B[3];
        for (B[2] = r0[2]; B[2] <= r1[2]; ++B[2])
        for (B[1] = r0[1]; B[1] <= r1[1]; ++B[1])
        for (B[0] = r0[0]; B[0] <= r1[0]; ++B[0]) {
            const double v = cell_overlap(bulk, B, fine, f);
            if (v == 0.0) continue;
            const int64_t cb = B[0] + (int64_t)bulk->n[0] * (B[1] + (int64_t)bulk->n[1] * B[2]);
            for (int c = 0; c < ncomp; ++c) ks_add(&acc[c], v * s_bulk[c * nbk + cb]);
        }
        for (int c = 0; c < ncomp; ++c) s_fine[c * nfn + cf] = ks_get(&acc[c]) / Vf;
    }
}

/* Bulk -> fine transfer of particle fields (Fig. 1): the bulk field is
 * interpolated at each fine cell centre with the particle stencil. */
void or_project(const or_grid* G, int ncomp, const double* bulk, double* fine)
{
    geom g = geometry(G);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < G->nf[2]; ++k)
    for (int j = 0; j < G->nf[1]; ++j)
    for (int i = 0; i < G->nf[0]; ++i) {
        double v[8];
        double x[3] = {G->x0[0] + (i + 0.5) * g.h[0],
                       G->x0[1] + (j + 0.5) * g.h[1],
                       G->x0[2] + (k + 0.5) * g.h[2]};
        or_gather(G, bulk, ncomp, x, v);
        int64_t f = i + (int64_t)G->nf[0] * (j + (int64_t)G->nf[1] * k);
        for (int comp = 0; comp < ncomp; ++comp) fine[comp * g.nfine + f] = v[comp];
    }
}

void or_euler(const or_grid* G, int64_t n, double* pos_d, double* vel,
              const double* force, double dt)
{
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < n; ++p) {
        double m = G->rho_p * sphere_volume(pos_d[4 * p + 3]);
        for (int a = 0; a < 3; ++a) {
            double u = vel[4 * p + a] + dt * (force[a * n + p] / m + G->g[a]);
            double x = pos_d[4 * p + a] + dt * u;
            double lo = G->x0[a], hi = G->x0[a] + G->L[a];
            if (x < lo) { x = 2.0 * lo - x; u = -u; }
            else if (x > hi) { x = 2.0 * hi - x; u = -u; }
            vel[4 * p + a] = u;
            pos_d[4 * p + a] = x;
        }
    }
}

int64_t or_step(const or_grid* G, int64_t n, double* pos_d, double* vel,
                const double* u_fine, double dt,
                int32_t* cell, int32_t* perm, int32_t* cell_start,
                double* eps_bulk, double* u_bulk, double* var_bulk,
                double* force, double* S_bulk, double* S_fine, double* eps_fine,
                double* sums)
{
    geom g = geometry(G);
    int64_t outside = or_bin(G, n, pos_d, cell, perm, cell_start);
    or_deposit_volume(G, n, pos_d, cell_start, perm, eps_bulk, NULL);
    or_average(G, u_fine, u_bulk, var_bulk);
    int64_t ncl = or_drag(G, n, pos_d, vel, eps_bulk, u_bulk, force);
    or_deposit_momentum(G, n, force, cell_start, perm, S_bulk);
    or_project(G, 3, S_bulk, S_fine);
    if (eps_fine) or_project(G, 1, eps_bulk, eps_fine);

    if (sums) {
        ksum k[OR_NSUMS];
        memset(k, 0, sizeof k);
        for (int64_t p = 0; p < n; ++p) {
            ks_add(&k[0], sphere_volume(pos_d[4 * p + 3]));
            double f2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                ks_add(&k[2 + a], force[a * n + p]);
                f2 += force[a * n + p] * force[a * n + p];
            }
            ks_add(&k[11], sqrt(f2));
        }
        for (int64_t c = 0; c < g.nbulk; ++c) {
            ks_add(&k[1], (1.0 - eps_bulk[c]) * g.VB);
            for (int a = 0; a < 3; ++a) ks_add(&k[5 + a], S_bulk[a * g.nbulk + c] * g.VB);
        }
        for (int64_t f = 0; f < g.nfine; ++f)
            for (int a = 0; a < 3; ++a) ks_add(&k[8 + a], S_fine[a * g.nfine + f] * g.Vf);
        if (dt > 0.0) or_euler(G, n, pos_d, vel, force, dt);
        for (int64_t p = 0; p < n; ++p) {
            double m = G->rho_p * sphere_volume(pos_d[4 * p + 3]);
            for (int a = 0; a < 3; ++a) ks_add(&k[12 + a], m * vel[4 * p + a]);
        }
        for (int i = 0; i < 15; ++i) sums[i] = ks_get(&k[i]);
        sums[15] = (double)ncl;
    } else if (dt > 0.0) {
        or_euler(G, n, pos_d, vel, force, dt);
    }
    return outside;
}
