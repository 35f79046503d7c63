/*
 * cg_oracle.h -- plain FP64 CPU oracle of the particle <-> dual-grid
 * coupling step (Pozzetti et al., "A parallel dual-grid multiscale approach
 * to CFD-DEM couplings", arXiv 1807.11834).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may call this code.  It shares no code,
 * header, table or constant with the CUDA library, and the library never
 * calls it.
 *
 * Everything is slow, sequential and in double precision: each function is
 * the definition it cites written out as loops.  Sums use Neumaier's
 * compensated summation (Neumaier 1974) so the oracle's own rounding error
 * stays far below the tolerances it is used to check.
 *
 * Layouts (x fastest everywhere):
 *   pos_d   [n][4]   x, y, z, diameter
 *   vel     [n][4]   u, v, w, (ignored)
 *   fine    [ncomp][nz_f][ny_f][nx_f]
 *   bulk    [ncomp][nz_b][ny_b][nx_b]
 *   force   [3][n]
 */
#ifndef CG_ORACLE_H
#define CG_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double x0[3];        /* domain origin                                  */
    double L[3];         /* domain extent                                  */
    int32_t nf[3];       /* fine cells per axis                            */
    int32_t r;           /* coarsening ratio: bulk cells = nf / r          */
    int32_t law;         /* 0 = Di Felice, 1 = Ergun / Wen-Yu              */
    int32_t interp;      /* 0 = trilinear, 1 = cell value (nearest cell)   */
    double rho_f, mu_f, rho_p;
    double eps_switch;   /* Ergun -> Wen-Yu switch porosity                */
    double eps_min;      /* lower clamp of the porosity seen by the drag   */
    double g[3];         /* gravity (Euler advance only)                   */
} or_grid;

enum { OR_NSUMS = 16 };

/* Bin index of one point (B1 rule); *outside set to 1 if clamped. */
int32_t or_bin_cell(const or_grid* G, const double x[3], int* outside);

/* Stable counting sort by bulk cell.  Returns the number of particles
 * outside the domain (clamped into the nearest cell). */
int64_t or_bin(const or_grid* G, int64_t n, const double* pos_d,
               int32_t* cell, int32_t* perm, int32_t* cell_start);

/* eps[c] = 1 - sum_{p in c} V_p / V_B ; phi[c] = sum V_p / V_B. */
void or_deposit_volume(const or_grid* G, int64_t n, const double* pos_d,
                       const int32_t* cell_start, const int32_t* perm,
                       double* eps, double* phi);

/* Mean of the r^3 nested fine cells per bulk cell, and the variance of
 * the velocity about that mean summed over the components (nullable). */
void or_average(const or_grid* G, const double* u_fine, double* u_bulk, double* var_bulk);

/* Clamped trilinear weights of point x on the bulk-cell-centre lattice. */
void or_weights(const or_grid* G, const double x[3], int32_t i0[3], double t[3], int clamped[3]);

/* Interpolate ncomp bulk fields at x (trilinear or cell value). */
void or_gather(const or_grid* G, const double* bulk, int ncomp, const double x[3], double* out);

/* Gradient of the trilinear interpolant of a scalar bulk field at x. */
void or_gather_grad(const or_grid* G, const double* bulk, const double x[3], double grad[3]);

/* Per-particle drag factor beta_p (force = beta_p * slip); *clamped set
 * to 1 when the porosity was raised to eps_min. */
double or_drag_beta(const or_grid* G, double eps, double d, const double s[3], int* clamped);

/* Drag force on every particle: F = beta_p (u_f(x_p) - u_p). Returns the
 * number of particles whose porosity was clamped. */
int64_t or_drag(const or_grid* G, int64_t n, const double* pos_d, const double* vel,
                const double* eps_bulk, const double* u_bulk, double* force);

/* Porosity and slip magnitude seen by each particle's drag law, before
 * the eps_min clamp (used by tests to locate correlation branch points). */
void or_particle_state(const or_grid* G, int64_t n, const double* pos_d, const double* vel,
                       const double* eps_bulk, const double* u_bulk, double* eps_p, double* slip);

/* Learned-closure inputs (not in the paper).  At each particle, with the
 * porosity of this step and the fluid velocity / variance of the last
 * refresh (stale) and of this step (fresh):
 *   feat[7p + 0..6] = eps_c, log10(1 + Re), |s|, d eps/dx, d eps/dy, d eps/dz, sigma^2
 *   with eps_c = max(eps, eps_min), s = u_stale - u_p, Re = rho_f eps_c d |s| / mu_f,
 *   target[p] = (F_fresh . F_stale) / |F_stale|^2  (1 when F_stale = 0),
 *   F_stale[3][n] the drag from the stale fields. */
void or_mlp_features(const or_grid* G, int64_t n, const double* pos_d, const double* vel,
                     const double* eps_bulk, const double* u_stale, const double* var_stale,
                     const double* u_fresh, double* feat, double* target, double* F_stale);

/* S_B = -(1/V_B) sum_{p in B} F_p  (per component). */
void or_deposit_momentum(const or_grid* G, int64_t n, const double* force,
                         const int32_t* cell_start, const int32_t* perm, double* S_bulk);

/* Semi-implicit exchange coefficients (Eq. UFP: F_fpi, the fluid-side reaction to
 * F_drag, is treated semi-implicitly).  With F_p = beta_p (u_f(x_p) - u_p):
 *   A_B = (1/V_B) sum_{p in B} beta_p,   b_B = (1/V_B) sum_{p in B} beta_p u_p,
 * so that the fluid solver takes F_fpi = -A u_f + b with A in its matrix.
 * coef[4][n_b] = (A, b_x, b_y, b_z); sums over each cell in the stable order.
 * PARITY: pinned by tests (uniform field: S_B = -(A u_f - b); sum A V_B =
 * sum beta_p; one particle; zero particle velocity). */
void or_implicit(const or_grid* G, int64_t n, const double* pos_d, const double* vel,
                 const double* eps_bulk, const double* u_bulk, const int32_t* cell_start,
                 const int32_t* perm, double* coef);

/* Non-nested grids (the grid-to-grid maps computed once per simulation,
 * Sec. 2.3): two uniform box grids, bulk and fine, in any relative
 * position and with any spacings.  V(B & f) is the volume of the
 * intersection of bulk cell B and fine cell f.
 *   average (fine -> bulk):  u_B = sum_f V(B & f) u_f / sum_f V(B & f)
 *                            (0 where no fine cell overlaps B);
 *   project (bulk -> fine):  S_f = sum_B V(B & f) S_B / V_f
 *                            (conservative: sum S_f V_f = sum S_B V_B
 *                            where the fine grid covers the bulk one).
 * Fields are [ncomp][cells], x fastest.
 * PARITY: pinned by tests (exact rational weights on tiny grids, nested
 * grids reduce to the plain mean and to cell injection, conservation,
 * the adjoint identity between the two maps). */
typedef struct {
    double x0[3];        /* origin        */
    double L[3];         /* extent        */
    int32_t n[3];        /* cells per axis */
} or_box_grid;

void or_map_average(const or_box_grid* bulk, const or_box_grid* fine, int ncomp, const double* u_fine,
                    double* u_bulk);
void or_map_project(const or_box_grid* bulk, const or_box_grid* fine, int ncomp, const double* s_bulk,
                    double* s_fine);

/* Interpolate ncomp bulk fields at every fine cell centre. */
void or_project(const or_grid* G, int ncomp, const double* bulk, double* fine);

/* Semi-implicit Euler: u += dt (F/m + g); x += dt u; specular walls. */
void or_euler(const or_grid* G, int64_t n, double* pos_d, double* vel,
              const double* force, double dt);

/* One whole coupling step.  eps_fine and var_bulk are nullable.
 * sums[OR_NSUMS]:  0 sum V_p, 1 sum phi_B V_B, 2-4 sum F_p, 5-7 sum S_B V_B,
 * 8-10 sum S_f V_f, 11 sum |F_p|, 12-14 sum m_p u_p (after the advance),
 * 15 particles with clamped porosity.  Returns particles outside the domain. */
int64_t or_step(const or_grid* G, int64_t n, double* pos_d, double* vel,
                const double* u_fine, double dt,
                int32_t* cell, int32_t* perm, int32_t* cell_start,
                double* eps_bulk, double* u_bulk, double* var_bulk,
                double* force, double* S_bulk, double* S_fine, double* eps_fine,
                double* sums);

#ifdef __cplusplus
}
#endif
#endif
