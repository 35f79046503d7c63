/*
 * cg.h -- C ABI of the GB300 (sm_103a) particle <-> dual-grid coupling
 * library: the per-step exchange between Lagrangian particles and the two
 * Eulerian grids of the dual-grid multiscale CFD-DEM coupling of
 * Pozzetti, Jasak, Besseron, Rousset, Peters, "A parallel dual-grid
 * multiscale approach to CFD-DEM couplings" (arXiv 1807.11834).
 *
 * Sec. 2.1 and Fig. 1 of the paper: a coarse uniform "bulk" grid maps the
 * Lagrangian particle fields to Eulerian ones and solves the fluid-particle
 * interaction; a fine grid carries the fluid.  Particle-related fields go
 * bulk -> fine, the fluid solution goes fine -> bulk.  One step is
 *   (a0) bin particles by bulk cell          cg_bin_particles
 *   (a1) deposit particle volume -> porosity cg_deposit(CG_DEP_VOLUME)
 *   (a2) average fine velocity onto bulk     cg_average_fine_to_bulk
 *   (a3) drag at the particles (+ reaction)  cg_drag / cg_deposit(CG_DEP_MOMENTUM)
 *   (a4) project the bulk source onto fine   cg_project_bulk_to_fine
 *   all fused in                              cg_step
 *
 * Conventions
 *   - Grids: origin x0[3], extent L[3], fine cells fine_n[3], integer
 *     coarsening ratio r, bulk cells n_b = fine_n / r, bulk spacing
 *     H = L / n_b.  Linear cell index i + n_x (j + n_y k), x fastest.
 *   - "T" below is float for CG_FP32 and double for CG_FP64.
 *   - Particle arrays are AoS of 4: pos_d[n] = (x, y, z, diameter),
 *     vel[n] = (u, v, w, unused).  Field arrays are SoA: [ncomp][cells].
 *     Per-particle outputs are in the caller's particle order.
 *   - Every pointer passed to a compute call is DEVICE memory owned by the
 *     caller (cg_step_host excepted), 16-byte aligned for either T (the
 *     kernels read particle records as 16-byte vectors: one float4, or two
 *     double2); misaligned particle and fine-field pointers are refused
 *     with CG_ERR_INVALID_ARG.  The library never frees them.
 *   - Every compute call is enqueued on the handle's CUDA stream and
 *     returns without synchronising.  Argument errors are reported
 *     synchronously by the return code and nothing is enqueued.
 *     Conditions found on the device (points outside the domain,
 *     non-finite inputs, porosity clamped for the drag law) are counted in
 *     a device status word read by cg_sync_status.
 *   - No call throws or aborts; no call allocates device memory once the
 *     handle's buffers fit the particle count (cg_step can then be captured
 *     in a CUDA graph).
 */
#ifndef CG_H
#define CG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CG_OK = 0,
    CG_ERR_INVALID_ARG = 1,   /* bad argument; nothing was enqueued          */
    CG_ERR_CUDA = 2,          /* a CUDA runtime call failed                  */
    CG_ERR_OOM = 3,           /* device allocation failed                    */
    CG_ERR_NOT_BINNED = 4,    /* needs cg_bin_particles with the same n first */
    CG_ERR_OUT_OF_RANGE = 5,  /* size beyond a documented limit              */
    CG_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up          */
    CG_ERR_NONFINITE = 7      /* non-finite input seen on the device         */
} cg_status;

typedef enum { CG_FP32 = 0, CG_FP64 = 1 } cg_precision;
typedef enum { CG_DRAG_DI_FELICE = 0, CG_DRAG_ERGUN_WEN_YU = 1 } cg_drag_law;
typedef enum { CG_INTERP_TRILINEAR = 0, CG_INTERP_CELL = 1 } cg_interp;
typedef enum { CG_DEP_VOLUME = 0, CG_DEP_MOMENTUM = 1 } cg_deposit_kind;

/* Status-word bits (cg_sync_status). */
enum {
    CG_FLAG_OUTSIDE = 1u,      /* a particle outside the domain was clamped  */
    CG_FLAG_NONFINITE = 2u,    /* a NaN/Inf position was seen                */
    CG_FLAG_EPS_CLAMPED = 4u,  /* porosity < eps_min was raised for the drag */
    CG_FLAG_TIMEOUT = 8u       /* a bounded device wait gave up              */
};

/* Binning sort choices (cg_grid_desc.sort_digits). */
#define CG_SORT_AUTO 0
#define CG_SORT_CELLS 1
#define CG_SORT_CELLS_AUTO_MAX 8388608   /* 2^23 particles */
#define CG_SORT_CELLS_AUTO_DENSITY 32   /* particles per bulk cell */

/* Stencil reads of the drag (cg_grid_desc.stencil). */
#define CG_STENCIL_GATHER 0   /* the eight records of each particle's stencil from global memory */
#define CG_STENCIL_WINDOW 1   /* in the sorted step, each warp's stencil window staged in shared memory */

/* Number of counters returned by cg_sync_status. */
#define CG_NCOUNTS 5

/* Number of entries of the conservation-sum vector written by cg_step. */
#define CG_NSUMS 16

/* Problem description.  Sec. 2.1 (two grids, the bulk one coarse and
 * uniform), Eq. (DragLaw) (beta depends on slip, rho_f, rho_p, d_p, A_p,
 * mu_f and porosity), Eq. (DEM_EQUATIONS) (gravity).
 *   eps_switch  Ergun -> Wen-Yu switch porosity (eps >= eps_switch is Wen-Yu), in (0, 1]
 *   eps_min     porosity seen by the drag law is max(eps, eps_min), in [0, 1)
 *   sort_digits the binning sort (every choice gives the same bins, and so
 *               the same results):
 *               CG_SORT_CELLS (1): per-cell sort (counts, arrival ranks,
 *                 placement, then each cell's ids sorted); fastest when its
 *                 particle-sized arrays fit in L2 or the particle order keeps
 *                 neighbours close, and cells hold at most a few hundred
 *                 particles (one warp sorts each larger cell);
 *               6..11: least-significant-digit sort with digits of at most
 *                 that many bits (one to three passes); fastest for large
 *                 particle sets in random order and for crowded cells;
 *               CG_SORT_AUTO (0): the per-cell sort for calls of at most
 *                 CG_SORT_CELLS_AUTO_MAX particles and at most
 *                 CG_SORT_CELLS_AUTO_DENSITY particles per bulk cell on
 *                 average, else the digit sort with digits of up to 10 bits
 *                 below 2^20 bulk cells, up to 8 from 2^20 on; an instance of
 *                 a batch (cg_batch_create) takes the digit sort unless its
 *                 descriptor asks for CG_SORT_CELLS
 *   stencil     how the drag reads the bulk records of each particle's
 *               trilinear stencil (both give the same bits):
 *               CG_STENCIL_GATHER (0): eight 16-byte loads per particle,
 *                 served by L1 and L2 (the bulk record of a 2^22-cell grid
 *                 is 64 MB, inside the 129 MB L2); the faster choice;
 *               CG_STENCIL_WINDOW (1): in cg_step_sorted on the FP32
 *                 trilinear path, each warp stages the bounding box of its
 *                 32 particles' stencils (with the +1 halo) in shared memory
 *                 and reads the corners there; a box of more than 64
 *                 records takes the global gather (measured slower, see
 *                 the design notes: the kernel is bound by instruction
 *                 issue, and the window costs instructions)
 * Limits: fine_n[a] % ratio == 0, bulk cells >= 2 per axis, at most 2^22
 * bulk cells and 2^31 - 1 fine cells. */
typedef struct {
    double origin[3];
    double extent[3];
    int32_t fine_n[3];
    int32_t ratio;
    int32_t prec;        /* cg_precision */
    int32_t law;         /* cg_drag_law  */
    int32_t interp;      /* cg_interp    */
    int32_t sort_digits; /* CG_SORT_AUTO, CG_SORT_CELLS or 6..11 */
    int32_t stencil;     /* CG_STENCIL_GATHER or CG_STENCIL_WINDOW */
    double rho_f, mu_f, rho_p;
    double eps_switch;
    double eps_min;
    double gravity[3];
} cg_grid_desc;

typedef struct cg_grids cg_grids;   /* opaque handle: bins, scratch, status */
typedef struct cg_mlp cg_mlp;       /* opaque learned drag closure          */

typedef struct {
    int64_t n;       /* number of particles, 0 <= n <= 2^31 - 1 */
    void* pos_d;     /* [n] T4: x, y, z, d (advanced in place when dt > 0) */
    void* vel;       /* [n] T4: u, v, w, -  (advanced in place when dt > 0) */
} cg_particles;

typedef struct {
    double* eps_bulk;      /* [n_b] porosity (always double)          required */
    void* u_bulk;          /* [3][n_b] T averaged fluid velocity        required */
    void* var_bulk;        /* [n_b] T sub-bulk velocity variance        nullable */
    void* S_bulk;          /* [3][n_b] T bulk momentum source           required */
    void* force;           /* [3][n] T drag force per particle          required */
    void* S_fine;          /* [3][n_f] T projected source               required */
    void* eps_fine;        /* [n_f] T projected porosity                nullable */
    double* sums;          /* [CG_NSUMS] device, conservation sums      nullable */
    int32_t* cell;         /* [n] bulk cell per particle                nullable */
    int32_t* perm;         /* [n] particles in cell order               nullable */
    int32_t* cell_start;   /* [n_b + 1] segment starts                  nullable */
    void* implicit_bulk;   /* [4][n_b] T semi-implicit coefficients     nullable */
    void* implicit_fine;   /* [4][n_f] T their projection (needs the bulk ones) nullable */
} cg_step_out;

/* Maps between two uniform grids that are not nested (any relative position
 * and spacings): the grid-to-grid transfers of Fig. 1 through a static
 * structure computed once (Sec. 2.3).  With V(B & f) the volume of the
 * intersection of bulk cell B and fine cell f:
 *   cg_map_average (fine -> bulk): u_B = sum_f V(B & f) u_f / sum_f V(B & f)
 *                                  (0 where no fine cell overlaps B);
 *   cg_map_project (bulk -> fine): S_f = sum_B V(B & f) S_B / V_f, which
 *                                  conserves sum S V where the fine grid
 *                                  covers the bulk one.
 * Fields are [ncomp][cells] T (x fastest), 1 <= ncomp <= 8, device memory
 * aligned to T; both grids take the same precision.  The map holds per-axis
 * compressed-row overlap tables on the device (a few arrays of the axis
 * sizes); calls are enqueued on its stream. */
typedef struct {
    double origin[3];
    double extent[3];
    int32_t n[3];        /* cells per axis, product < 2^31 */
    int32_t prec;        /* cg_precision */
} cg_box_grid;

typedef struct cg_map cg_map;

cg_status cg_map_create(const cg_box_grid* bulk, const cg_box_grid* fine, void* cuda_stream, cg_map** out);
cg_status cg_map_destroy(cg_map* m);   /* synchronises its stream; NULL is OK */
cg_status cg_map_average(cg_map* m, int32_t ncomp, const void* fine_in, void* bulk_out);
cg_status cg_map_project(cg_map* m, int32_t ncomp, const void* bulk_in, void* fine_out);

/* Human-readable name of a status code (static storage). */
const char* cg_status_string(cg_status s);

/* Create the coupling handle for one pair of nested grids (Sec. 2.1,
 * Fig. 1).  cuda_stream is a cudaStream_t (NULL = legacy default stream);
 * the handle allocates its bulk-sized buffers on the current device.
 * On error *out is set to NULL. */
cg_status cg_create_grids(const cg_grid_desc* desc, void* cuda_stream, cg_grids** out);

/* Free the handle and everything it owns (synchronises its stream). NULL is OK. */
cg_status cg_destroy_grids(cg_grids* g);

/* Host-side fault injection for the allocation failure paths (process-wide,
 * no device fault): the next k device allocations a coupling handle makes
 * for itself (its bulk buffers, particle scratch and host-entry staging)
 * succeed and the one after fails as if the device were out of memory, so
 * the call that made it returns CG_ERR_OOM; the injection then switches
 * itself off.  k = -1 switches it off at once; k < -1 is CG_ERR_INVALID_ARG.
 * A failed cg_create_grids frees everything and returns no handle; any
 * other call that fails this way enqueues no work, and its handle stays
 * valid and allocates again on its next call. */
cg_status cg_debug_fail_alloc_after(int64_t k);

/* Change the stream later calls are enqueued on. */
cg_status cg_set_stream(cg_grids* g, void* cuda_stream);

/* Bulk cells per axis and total bulk / fine cell counts (host values). */
cg_status cg_grid_dims(const cg_grids* g, int32_t bulk_n[3], int64_t* n_bulk, int64_t* n_fine);

/* (a0) Bin particles by bulk cell: the per-step particle-cell connectivity
 * of Sec. 2.2.  Cell of a point, per axis: clamp(floor((x - x0) / H), 0,
 * n_b - 1) with the quotient taken in IEEE double (subtraction, then
 * correctly rounded division); half-open cells, x = x0 + L in the last
 * cell; points with quotient outside [0, n_b] are clamped and counted.
 * Particles are sorted stably by cell: perm lists the particles of cell c
 * at perm[cell_start[c] .. cell_start[c+1]) in increasing index order.
 * pos_d: [n] T4.  Outputs (all nullable): cell_out[n], perm_out[n],
 * cell_start_out[n_b + 1].  The handle keeps the binning for later
 * cg_deposit / cg_drag calls with the same n.
 * Incremental rebinning: when the handle holds a binning of the same n (from
 * the last call of cg_bin_particles or of a step) and sort_digits is
 * CG_SORT_AUTO or CG_SORT_CELLS, the binning starts from it: only the
 * particles whose cell changed are re-sorted, with particle i taken to be
 * the particle i of that binning (or, for the sorted output of
 * cg_step_sorted, the particle at its slot i).  The result is the same
 * stable order whatever the particles did (moved, resized or permuted);
 * any share of them may change cell, and when a cell receives more than
 * 256 in one call the device falls back to the per-cell sort.  When none
 * changed cell the bins are kept and only the sorted diameters are read
 * afresh.  A descriptor with a digit width (6..11) always sorts from
 * scratch. */
cg_status cg_bin_particles(cg_grids* g, int64_t n, const void* pos_d,
                           int32_t* cell_out, int32_t* perm_out, int32_t* cell_start_out);

/* (a0, optional) Physical reorder of the particles into the binned order:
 * pos_out[s] = pos_d[perm[s]] and vel_out[s] = vel[perm[s]] (vel and
 * vel_out nullable together), for the binning of these n particles (made
 * by cg_bin_particles or cg_step with the same n; CG_ERR_NOT_BINNED
 * otherwise).  The output arrays are the caller's, [n] T4, 16-byte aligned,
 * and must not overlap the inputs.  Particles kept in cell order make the
 * later steps' memory access follow the grids: the per-cell sort
 * (CG_SORT_CELLS) then places and sorts in order, and the deposits and the
 * drag read neighbours together.  Rebinning the reordered positions gives
 * the identity permutation. */
cg_status cg_reorder_particles(cg_grids* g, int64_t n, const void* pos_d, const void* vel, void* pos_out,
                               void* vel_out);

/* Binning that allocates nothing, for callers that must not allocate
 * device memory (for example code running while another component
 * captures a CUDA graph, or plug-ins restricted to the memory their host
 * hands them).  The paper has no counterpart: this is a library facility.
 * Same cell rule, stable order and outputs as cg_bin_particles, but without
 * a handle: the grid comes from desc (the physics fields are not used) and
 * all scratch lives in one fixed device array inside the library (about
 * 12 MB per GPU that loads it, held until exit).
 *   n <= 262,144 particles (else CG_ERR_OUT_OF_RANGE), at most 2^22 cells.
 *   pos_d [n] T4 (16-byte aligned); perm_out [n] and cell_start_out
 *   [n_b + 1] required; cell_out [n] nullable.  Enqueued on cuda_stream.
 * The first call on a device looks up the array's address on that device;
 * make it before any stream capture.  All calls share the one array, so
 * calls that overlap on the GPU race: order them on one stream. */
cg_status cg_bin_particles_static(const cg_grid_desc* desc, int64_t n, const void* pos_d, int32_t* cell_out,
                                  int32_t* perm_out, int32_t* cell_start_out, void* cuda_stream);

/* (a1)/(a3) Deposit onto the bulk grid over the particles of each cell,
 * summed in the stable order of the last cg_bin_particles.
 *   CG_DEP_VOLUME:   per_particle = pos_d [n] T4 (diameter used);
 *                    bulk_out = eps double [n_b], eps = 1 - sum(pi d^3/6) / V_B
 *                    (Table 1 porosity field; Sec. 2.4 porosity definition).
 *   CG_DEP_MOMENTUM: per_particle = force [3][n] T;
 *                    bulk_out = S [3][n_b] T, S = -(1/V_B) sum F
 *                    (Eq. UFP: F_fpi is the fluid-side reaction to F_drag).
 * Returns CG_ERR_NOT_BINNED without a binning of this n. */
cg_status cg_deposit(cg_grids* g, int32_t kind, int64_t n, const void* per_particle, void* bulk_out);

/* (a2) Fine -> bulk transfer of the fluid solution (Fig. 1): mean of the
 * r^3 nested fine cells per bulk cell for each velocity component, and
 * optionally the variance of the velocity about that mean summed over the
 * three components.  u_fine [3][n_f] T -> u_bulk [3][n_b] T,
 * var_bulk [n_b] T (nullable). */
cg_status cg_average_fine_to_bulk(cg_grids* g, const void* u_fine, void* u_bulk, void* var_bulk);

/* (a3) Drag on every particle, Eq. (DragLaw): F = beta (u_f - u_p), with
 * porosity and fluid velocity interpolated at the particle from the bulk
 * cell centres (trilinear, constant extrapolation in the outer half cell;
 * or the cell value) and beta from the Di Felice or Ergun / Wen-Yu
 * correlation.  pos_d, vel: [n] T4; eps_bulk: double [n_b]; u_bulk: [3][n_b] T;
 * force_out: [3][n] T.  When S_bulk_out ([3][n_b] T) is not NULL the
 * reaction S = -(1/V_B) sum F is deposited in the same pass (needs the
 * binning of this n).  mlp NULL: the plain correlation.  mlp set (FP32
 * grids only; cg_mlp_bind first): u_bulk is the stale fluid record and the
 * learned closure of cg_step_learned below is applied with the bound age
 * (its fallback reads the bound fine field); the closure's parameters must
 * be ready on this handle's stream (same stream, or synchronised). */
cg_status cg_drag(cg_grids* g, int64_t n, const void* pos_d, const void* vel,
                  const double* eps_bulk, const void* u_bulk,
                  void* force_out, void* S_bulk_out, const cg_mlp* mlp);

/* (a4) Bulk -> fine transfer of particle-related fields (Fig. 1): each
 * fine cell centre takes the interpolant of the bulk field with the
 * particle stencil.  bulk [ncomp][n_b] T -> fine_out [ncomp][n_f] T,
 * 1 <= ncomp <= 4.  Conserves sum S V exactly in real arithmetic. */
cg_status cg_project_bulk_to_fine(cg_grids* g, int32_t ncomp, const void* bulk, void* fine_out);

/* One coupling step (a0..a4) on device memory: bin, porosity, fluid
 * average, drag with fused reaction deposit, projection of the source
 * (and of the porosity when out->eps_fine is set), conservation sums.
 * With dt > 0 the particles are then advanced by semi-implicit Euler
 * under drag and gravity, Eq. (DEM_EQUATIONS) without contacts:
 * u += dt (F/m + g), x += dt u, m = rho_p pi d^3 / 6, specular walls.
 * u_fine: [3][n_f] T.  sums (CG_NSUMS doubles): 0 sum V_p,
 * 1 sum (1 - eps_B) V_B, 2..4 sum F_p, 5..7 sum S_B V_B, 8..10 sum S_f V_f,
 * 11 sum |F_p|, 12..14 sum m_p u_p after the advance, 15 particles whose
 * porosity was clamped.
 * Semi-implicit exchange (Eq. UFP: F_fpi, the fluid-side reaction to F_drag, is
 * treated semi-implicitly): when out->implicit_bulk is set, it receives
 * A = (1/V_B) sum_p beta_p and b = (1/V_B) sum_p beta_p u_p per bulk cell
 * ([4][n_b] T: A, b_x, b_y, b_z; u_p before the advance), with which the
 * fluid solver takes F_fpi = -A u_f + b (A into its matrix); when
 * out->implicit_fine is also set, the four fields are projected onto the
 * fine grid like the source.  Device entries only: cg_step_learned, the
 * host-buffer entries and batched instances reject these fields
 * (CG_ERR_INVALID_ARG). */
cg_status cg_step(cg_grids* g, const cg_particles* p, const void* u_fine,
                  const cg_step_out* out, double dt);

/* One coupling step, as cg_step, that also leaves the particles in the order
 * of this step's binning (cell order): p_out->pos_d[s] and p_out->vel[s] are
 * the records of particle perm[s] of p, advanced when dt > 0 (unchanged when
 * dt == 0), and p's arrays are not written.  Per-particle outputs
 * (out->force, out->cell) are in p's order; out->perm (nullable) is the map
 * from p_out's slots to p's indices.  vel[.].w is carried unchanged, so a
 * particle id kept there travels with its particle.  p_out: the caller's
 * [n] T4 arrays, p_out->n == p->n, 16-byte aligned, overlapping neither
 * each other nor p's arrays (else CG_ERR_INVALID_ARG).
 * A DEM code keeps its particles in cell order this way (double-buffered
 * arrays, swapped every step): the next step's binning then starts from
 * this one with its particle i at slot i, and only the particles that
 * changed cell are re-sorted (the per-step connectivity rebuild of
 * Sec. 2.2); its memory accesses follow the grids.  The fields and forces
 * are those of cg_step on the same particles, each cell summing the same
 * particles in the same order. */
cg_status cg_step_sorted(cg_grids* g, const cg_particles* p, const cg_particles* p_out, const void* u_fine,
                         const cg_step_out* out, double dt);

/* Learned coupling step (closure below; not in the paper).  age == 0: a
 * refresh, exactly cg_step, which also writes the fresh u_bulk and var_bulk
 * that later steps use as their stale record.  age >= 1 (steps since that
 * refresh): the fine -> bulk average is skipped; out->u_bulk and
 * out->var_bulk are then INPUTS (the record of the last refresh, left
 * unchanged) and the drag is the learned closure F = (1 + age r) F_stale,
 * falling back per particle to the plain drag with the fluid velocity
 * averaged afresh from u_fine when its features lie outside the closure's
 * box (counted: cg_sync_status counts[4]).  The drag diagnostics of sums
 * (0, 2..4, 11..15) are NaN on such steps.  FP32 grids only;
 * out->var_bulk required. */
cg_status cg_step_learned(cg_grids* g, const cg_particles* p, const void* u_fine,
                          const cg_step_out* out, double dt, const cg_mlp* mlp, int32_t age);

/* cg_step on HOST buffers: copies the inputs to handle-owned device
 * buffers, runs cg_step, copies every requested output back and waits for
 * the stream.  Same layouts as cg_step with host pointers everywhere
 * (page-locked memory recommended); p->pos_d / p->vel are advanced in
 * place when dt > 0.  Allocates the device buffers on first use or growth. */
cg_status cg_step_host(cg_grids* g, const cg_particles* p, const void* u_fine,
                       const cg_step_out* out, double dt);

/* cg_step_host without the final wait: the call enqueues the copies in, the
 * step and the copies out, and returns.  Two staging sets are used in turn,
 * so the input copies of one call overlap the output copies of the
 * previous one.  Until cg_step_host_wait returns, the host inputs of a call
 * must stay unchanged and its host outputs are not yet valid.  One
 * exception: when a call advances its particles in place (dt > 0), a later
 * call given the same particle arrays (p->pos_d or p->vel) copies them in
 * only after the advanced particles have arrived there, so an advancing run
 * may enqueue its steps back to back on one pair of arrays. */
cg_status cg_step_host_async(cg_grids* g, const cg_particles* p, const void* u_fine,
                             const cg_step_out* out, double dt);
/* Wait for every host-buffer step enqueued on the handle. */
cg_status cg_step_host_wait(cg_grids* g);

/* ------------------------------------------------------------------------
 * Learned drag closure (not in the paper; the paper's drag law is the plain
 * correlation of Eq. DragLaw).  A multilayer perceptron c = f(features),
 * 16 (7 used) -> 64 -> 64 -> 1 with one activation in both hidden layers
 * (exact-erf GELU, the default, or ReLU), scales the drag computed from
 * stale bulk fields, F = c F_stale, in place of a fresh fine-to-bulk
 * average.  BF16 operands, FP32 accumulation on the tensor cores (the
 * biases b1, b2 enter the products exactly, as three BF16 terms each);
 * FP32 master weights; Adam.  Parameters (FP32, CG_MLP_NPARAM floats, in order):
 * W1 [16][64] (input, hidden), b1 [64], W2 [64][64] (in, out), b2 [64],
 * w3 [64], b3 [1].  Feature rows are 8 floats: eps, log10(1 + Re), |s|,
 * d eps/dx, d eps/dy, d eps/dz, sigma^2, unused; the network sees
 * (f - lo) / (hi - lo) per feature, and a row is in range when every
 * scaled feature lies in [0, 1].  The network output r is the drag
 * correction per step of record age: the learned drag is
 * F = (1 + age r) F_stale, age = steps since the record was refreshed.
 * ------------------------------------------------------------------------ */
#define CG_MLP_NPARAM 5313
#define CG_MLP_NFEAT 7
#define CG_MLP_GELU 0   /* x Phi(x), Phi the standard normal CDF */
#define CG_MLP_RELU 1   /* max(x, 0) */

/* Create a closure from host parameters and the feature box [lo, hi]
 * (host, CG_MLP_NFEAT each, hi > lo).  Allocates its device state. */
cg_status cg_mlp_create(const float* params, const float* feat_lo, const float* feat_hi, void* cuda_stream,
                        cg_mlp** out);
cg_status cg_mlp_destroy(cg_mlp* m);

/* The activation of both hidden layers (CG_MLP_GELU after create), used by
 * every later forward, gradient and learned drag of the closure.
 * CG_ERR_INVALID_ARG for another value. */
cg_status cg_mlp_set_activation(cg_mlp* m, int32_t activation);
cg_status cg_mlp_get_activation(const cg_mlp* m, int32_t* activation);

/* Copy the current parameters and / or the last reduced gradient to the
 * host (either nullable; waits for the stream). */
cg_status cg_mlp_get_params(cg_mlp* m, float* params, float* grads);
cg_status cg_mlp_set_params(cg_mlp* m, const float* params);

/* c for n feature rows: features [n][8] device (16-byte aligned),
 * c_out [n], in_range_out [n] (nullable, 1 when in range). */
cg_status cg_mlp_forward(cg_mlp* m, int64_t n, const float* features, float* c_out, int32_t* in_range_out);

/* Mean-square loss against targets [n] and its gradient (kept in the
 * handle, readable with cg_mlp_get_params); loss_out: device float, nullable. */
cg_status cg_mlp_grads(cg_mlp* m, int64_t n, const float* features, const float* targets, float* loss_out);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the batch. */
cg_status cg_mlp_train_step(cg_mlp* m, int64_t n, const float* features, const float* targets, float lr,
                            float* loss_out);

/* Closure inputs and training targets at every particle, in either
 * precision: features [n][8] float (layout above) from the porosity of
 * this step (eps_bulk, double [n_b]) and the stale record (u_stale [3][n_b]
 * T, var_stale [n_b] T), with the porosity gradient that of the trilinear
 * interpolant (zero along an axis where the particle is in the outer half
 * cell, and everywhere in cell-value mode); target [n] float
 * c* = (F_fresh . F_stale) / |F_stale|^2 (1 where F_stale = 0), F_fresh
 * the drag with u_fresh [3][n_b] T.  pos_d, vel, features 16-byte aligned.
 * Enqueued on the grids' stream. */
cg_status cg_mlp_features(cg_grids* g, int64_t n, const void* pos_d, const void* vel, const double* eps_bulk,
                          const void* u_stale, const void* var_stale, const void* u_fresh,
                          float* features_out, float* target_out);

/* Bind the stale variance field (var [n_b] float), the fine velocity
 * (u_fine [3][n_f] float, 16-byte aligned) and the record age (>= 1) used
 * by cg_drag with this closure; both pointers NULL unbinds.  The pointers
 * are kept, not copied. */
cg_status cg_mlp_bind(cg_mlp* m, const void* var_stale, const void* u_fine, int32_t age);

/* Checkpoints of a trained closure (the same files closure.save_checkpoint
 * and closure.load_checkpoint of the Python binding read and write), two
 * files beside each other:
 *   <path>.f32   the CG_MLP_NPARAM parameters, little-endian float32, in the
 *                order above;
 *   <path>.json  a JSON object with "format": "dual-grid drag closure",
 *                "version": 1, "nparam", "nfeat", "hidden" (64), "k0" (16),
 *                "params_file" (the .f32 file's name, no directory),
 *                "params_sha256" (SHA-256 of that file, FIPS 180-4, lower-case
 *                hex), "feature_lo" / "feature_hi" (the feature box),
 *                "activation" ("gelu" or "relu"; a head without it is
 *                read as "gelu") and "meta" (a JSON object the caller
 *                chooses).
 * cg_mlp_save writes the closure's current parameters, feature box and
 * activation (waits for its stream); meta_json is a JSON object text or
 * NULL ({}).  cg_mlp_load reads a checkpoint and creates a closure from it
 * on the current device, as cg_mlp_create followed by
 * cg_mlp_set_activation.  The host-only pair underneath works on host
 * arrays (no device needed): cg_mlp_checkpoint_write(params [NPARAM],
 * feat_lo / feat_hi [NFEAT], activation CG_MLP_*) and
 * cg_mlp_checkpoint_read (outputs nullable).
 * CG_ERR_INVALID_ARG: a file cannot be written or read, or does not hold a
 * checkpoint of this network (format, version or sizes differ, the
 * checksum does not match, a value is not finite, the feature box is
 * empty), or meta_json is not a JSON object; nothing is created then. */
cg_status cg_mlp_save(cg_mlp* m, const char* path, const char* meta_json);
cg_status cg_mlp_load(const char* path, void* cuda_stream, cg_mlp** out);
cg_status cg_mlp_checkpoint_write(const char* path, const float* params, const float* feat_lo, const float* feat_hi,
                                  int32_t activation, const char* meta_json);
cg_status cg_mlp_checkpoint_read(const char* path, float* params, float* feat_lo, float* feat_hi,
                                 int32_t* activation);

/* Wait for the closure's stream; CG_ERR_TIMEOUT if a bounded wait of its
 * kernels expired (flags: CG_FLAG_*).  Reading the status clears it. */
cg_status cg_mlp_sync_status(cg_mlp* m, uint32_t* flags);

/* Check of the failure path of the bounded device waits (no GPU fault, no
 * hang): enqueues on the closure's stream one warp that waits, with the
 * tensor-core kernels' bounded mbarrier wait, on a barrier that nothing
 * arrives at, for at most `polls` polls (1 .. 2^22), and records the expiry
 * in the closure's status word as a stalled tensor-core kernel would.  The
 * next cg_mlp_sync_status returns CG_ERR_TIMEOUT with CG_FLAG_TIMEOUT set;
 * the context and the handle stay usable.  CG_ERR_INVALID_ARG for a NULL
 * handle or polls outside the range. */
cg_status cg_mlp_wait_selftest(cg_mlp* m, uint32_t polls);

/* ------------------------------------------------------------------------
 * Batched coupling (not in the paper): many independent FP32 instances of
 * uneven grids and particle counts stepped together.  Each phase of the
 * step (zeroing, binning passes, porosity, fine -> bulk average, pack, drag,
 * reaction, projections, sums) is one persistent launch over every
 * instance, so a batched step is about 16 launches whatever the number of
 * instances; cg_batch_use_graph replays them as one CUDA graph.  Every
 * field of an instance is bit-identical to cg_step of that instance (and
 * across configurations); the FP64 sums may differ in their last bits.
 * ------------------------------------------------------------------------ */
typedef struct cg_batch cg_batch;

/* One instance: grids (prec CG_FP32, ratio 2, 4 or 8), device particles
 * (n >= 1, 16-byte aligned), device u_fine [3][n_f], device outputs as for
 * cg_step (var_bulk, eps_fine, sums nullable; cell, perm, cell_start must
 * be NULL).  The pointers are kept for the life of the batch. */
typedef struct {
    cg_grid_desc desc;
    cg_particles particles;
    const void* u_fine;
    cg_step_out out;
} cg_batch_item;

/* Work decomposition (results do not depend on it). */
typedef struct {
    int32_t digit_bits;  /* widest radix digit of a binning pass, 8..11      */
    int32_t drag_items;  /* particles per thread of a drag block, 1..64      */
    int32_t avg_items;   /* bulk cells per thread of an average block, 1..64 */
    int32_t seg_chunks;  /* 256-slot chunks per warp of the deposits, 1..64  */
    int32_t grid_mult;   /* persistent CTAs = grid_mult x resident per SM x SMs, 1..8 */
} cg_batch_config;

cg_status cg_batch_default_config(cg_batch_config* c);
/* Creates one grids handle per instance (its scratch) plus the batch's own
 * stream and buffers; cuda_stream is the caller's stream, joined before
 * and after every step.  CG_ERR_INVALID_ARG for a bad item. */
cg_status cg_batch_create(const cg_batch_item* items, int32_t count, void* cuda_stream, cg_batch** out);
cg_status cg_batch_destroy(cg_batch* b);
/* Re-plan under a configuration (waits for the batch stream; CG_ERR_OUT_OF_RANGE
 * when digit_bits cannot bin an instance in two passes). */
cg_status cg_batch_set_config(cg_batch* b, const cg_batch_config* c);
cg_status cg_batch_get_config(const cg_batch* b, cg_batch_config* c);
/* on != 0: cg_batch_step captures its launches once per dt and replays the graph. */
cg_status cg_batch_use_graph(cg_batch* b, int32_t on);
/* One coupling step of every instance (dt as for cg_step, same for all). */
cg_status cg_batch_step(cg_batch* b, double dt);
/* The same step as cg_step of each instance in turn (each on its own
 * handle with its own launch shapes): the one-by-one reference; replayed
 * as one graph when graphs are on. */
cg_status cg_batch_step_each(cg_batch* b, double dt);
/* Autotune the configuration: coordinate search over the knobs, each
 * candidate timed as the median of reps batched steps with dt = 0.
 * cache_path (nullable) maps the batch's signature to its choice and is
 * read before / appended after a search.  chosen, best_ms nullable
 * (best_ms = -1 on a cache hit). */
cg_status cg_batch_tune(cg_batch* b, int32_t reps, const char* cache_path, cg_batch_config* chosen,
                        double* best_ms);
/* Status over all instances, as cg_sync_status (counts summed). */
cg_status cg_batch_sync_status(cg_batch* b, uint32_t* flags, int64_t* counts);
/* The grids handle of instance i (for stepping it alone), NULL if out of range. */
cg_grids* cg_batch_instance(cg_batch* b, int32_t i);
int64_t cg_batch_launch_count(const cg_batch* b);
int64_t cg_batch_launches_per_step(const cg_batch* b);

/* Wait for the handle's stream and read-and-clear the device status word.
 * flags (nullable) gets CG_FLAG_* bits; counts (nullable, CG_NCOUNTS
 * entries) gets particles outside, non-finite positions, clamped
 * porosities, timeouts, learned-drag fallbacks.
 * Returns CG_ERR_NONFINITE / CG_ERR_TIMEOUT when those bits are set,
 * CG_ERR_CUDA if the stream holds an error, else CG_OK. */
cg_status cg_sync_status(cg_grids* g, uint32_t* flags, int64_t* counts);

/* Number of CUDA kernels this handle has launched so far. */
int64_t cg_launch_count(const cg_grids* g);

/* Per-kernel device timing.  When enabled, every kernel launch of the
 * handle is bracketed by CUDA events on its stream; cg_profile_read waits
 * for the stream and returns, for kernel slot k (0 <= k < count), its name,
 * launches and total milliseconds since the last reset.  Returns the
 * number of slots in *count. */
cg_status cg_profile_enable(cg_grids* g, int32_t on);
cg_status cg_profile_reset(cg_grids* g);
cg_status cg_profile_read(cg_grids* g, int32_t k, const char** name,
                          int64_t* launches, double* total_ms, int32_t* count);

#ifdef __cplusplus
}
#endif
#endif
