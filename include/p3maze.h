/*
 * p3maze.h -- C ABI of the P3MaZe long-range electrostatics library (one GPU).
 *
 * P3MaZe (Mass-Zero particle-particle particle-mesh electrostatics) splits the
 * periodic Coulomb energy into a short-range erfc pair sum, a smooth long-range
 * mesh part and a Gaussian self term (Eqs. 3-6).  The long-range mesh potential
 * phi is a zero-inertia auxiliary field: each MD step predicts it by Verlet
 * (phi_p = 2 phi^k - phi^{k-1}) and enforces the discrete Poisson equation
 * (h/4pi) M phi + q^s = 0 (Eq. 13) as a holonomic constraint by solving the
 * correction problem M y = sigma_p (Eqs. 16-17) with multigrid V-cycles until
 * max|M y - sigma_p| <= tol (Eq. 20), then phi^{k+1} = phi_p - (4pi/h) y
 * (supporting information Sec. 1, "Numerical integration").
 *
 * One step of the library, all on the device:
 *   kick/drift/wrap (velocity Verlet) -> cell list -> cubic B-spline charge
 *   assignment q -> K diffusion steps q^s = (I + cM)^K q -> predicted residual
 *   sigma_p and multiplier guess y0 -> multigrid correction solve -> field
 *   update -> erfc + Born-Mayer / Lennard-Jones pair forces -> force
 *   interpolation F = -Q W . D phi (Eq. 21) -> (SPC/Fw bonded terms) -> kick.
 *
 * Units: A, fs, g/mol, e, kcal/mol.  Positions are wrapped into [0, L).
 *
 * Conventions for every entry point:
 *   - Return 0 (P3MAZE_OK) or a negative P3MAZE_ERR_* code; the message is
 *     available from p3maze_last_error(ctx) (or p3maze_last_error(NULL) when
 *     no context was created).
 *   - Host pointers are read (or written) during the call only; the caller
 *     keeps ownership.  The context owns all device memory it allocates.
 *   - A context is bound to the device current at init and to the CUDA stream
 *     given there: every call is ordered after the work already queued on
 *     that stream, and the stream is ordered after the call's work.  The
 *     context runs its kernels on two internal streams (the mesh pipeline at
 *     the highest priority, the short-range pair branch at the lowest).  A
 *     context is not thread safe; use one context per thread.
 *   - Chained mesh kernels (the diffusion steps, the V-cycle, the fused
 *     residual update) are launched with programmatic dependent launch, so a
 *     grid is scheduled while its predecessor drains; each waits for its
 *     predecessor's completion before touching memory.  The environment
 *     variable P3MAZE_PDL=0, read when a context is created, launches them
 *     plainly (the same arithmetic).
 */
#ifndef P3MAZE_H
#define P3MAZE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------- */
#define P3MAZE_OK                  0
#define P3MAZE_ERR_INVALID        -1  /* bad argument or parameter                      */
#define P3MAZE_ERR_OOM            -2  /* device allocation failed                       */
#define P3MAZE_ERR_CUDA           -3  /* a CUDA call failed (message has the CUDA text) */
#define P3MAZE_ERR_NOT_CONVERGED  -4  /* multigrid reached max_mg_iters above tol       */
#define P3MAZE_ERR_NONFINITE      -5  /* NaN/Inf in the constraint residual             */

/* ---- enumerations ------------------------------------------------------------ */
#define P3MAZE_FP64   0   /* every mesh and particle array in FP64                        */
#define P3MAZE_MIXED  1   /* FP32 assignment, smoothing, multigrid hierarchy and pair math;
                             FP64 positions, fields phi and y, constraint residual, coarse
                             solve, neutrality sum and all energy/force accumulation      */

#define P3MAZE_METHOD_MAZE 0  /* P3MaZe: Verlet-predicted field corrected by the multiplier y,
                                 convergence on max|M y - sigma_p| (Eq. 20)              */
#define P3MAZE_METHOD_P3M  1  /* real-space P3M baseline (Sec. 3.3): the same splitting,
                                 smoothing and Verlet-predicted initial field, the Poisson
                                 equation solved directly by multigrid with no multiplier
                                 predictor, convergence on max|M phi + (4pi/h) q^s| (the P3M
                                 residual of Sec. 3.3) <= tol                               */
#define P3MAZE_METHOD_PMAZE 2 /* PMaZe, the comparison method of Secs. 1-2: the whole Coulomb
                                 problem on the mesh.  The assigned charge q itself is the
                                 source (no smoothing, K = 0), the same Mass-Zero constraint
                                 (h/4pi) M phi + q = 0 is enforced by the same prediction and
                                 correction, the mesh force of Eq. 21 is the whole
                                 electrostatic force, and pairs carry only the non-Coulomb
                                 term (no erfc term, no Gaussian self term; alpha is not
                                 used).  v_lr = 1/2 ke phi^T q then contains the grid
                                 self-energy of every charge (Sec. 2, "electrostatic
                                 energy"); the work-based energy the paper uses for PMaZe is
                                 not formed.  Molecular topologies are rejected (their
                                 intramolecular exclusions would need the mesh pair
                                 interaction), and so is P3MAZE_LR_FORCE_ANALYTIC (with the
                                 whole charge on the mesh the exact gradient is dominated by
                                 the gradient of the grid self-energy).  The mesh must resolve the charges: the
                                 paper's NaCl comparison uses twice the P3MaZe mesh per axis */

/* Long-range force interpolation */
#define P3MAZE_LR_FORCE_FD       0  /* F = -ke Q W . D phi, central differences (Eq. 21; default):
                                       momentum conserving, not the exact energy gradient   */
#define P3MAZE_LR_FORCE_ANALYTIC 1  /* F = -ke Q grad W . phi: the exact gradient of
                                       V_LR = 1/2 ke phi^T q (energy conserving), not the
                                       paper's force; momentum conserved to discretisation error */

/* Short-range truncation at r_cut (reading A13 leaves the cutoff unshifted) */
#define P3MAZE_SR_TRUNCATE    0  /* pair forces and energies cut off at r_cut, unshifted (default) */
#define P3MAZE_SR_SHIFT_FORCE 1  /* shifted force: every pair term (erfc Coulomb and non-Coulomb)
                                    becomes U(r) - U(r_cut) + (r - r_cut) F(r_cut) with force
                                    F(r) - F(r_cut), so energy and force are continuous at r_cut;
                                    an option for energy-conservation studies, not the paper's */

#define P3MAZE_SR_NONE 0  /* Coulomb only                                               */
#define P3MAZE_SR_BMH  1  /* Born-Huggins-Mayer: A exp((s-r)/rho) - C/r^6 - D/r^8         */
#define P3MAZE_SR_LJ   2  /* Lennard-Jones: 4 eps ((s/r)^12 - (s/r)^6), pairs with eps=0 skipped */

#define P3MAZE_MAX_TYPES 4

/* Mesh arrays readable with p3maze_get_mesh (N^3 doubles, x fastest:
 * index (iz*N + iy)*N + ix). */
#define P3MAZE_MESH_Q      0  /* assigned charge q = A(r)Q at the current positions        */
#define P3MAZE_MESH_QS     1  /* smoothed charge q^s with its mean removed                 */
#define P3MAZE_MESH_PHI    2  /* constrained mesh potential phi^k (e/A)                    */
#define P3MAZE_MESH_Y      3  /* converged correction y* of the last solve                 */
#define P3MAZE_MESH_SIGMA  4  /* predicted constraint residual sigma_p of the last solve
                                 (after at least one step)                                  */

/* Force parts readable with p3maze_get_forces (n*3 doubles, particle-major). */
#define P3MAZE_F_TOTAL 0
#define P3MAZE_F_SR    1  /* erfc Coulomb + non-Coulomb pair terms (Eq. 19 + V-bar)        */
#define P3MAZE_F_LR    2  /* mesh force -Q W . D phi (Eq. 21)                              */
#define P3MAZE_F_BOND  3  /* SPC/Fw bonds, angles and intramolecular exclusion             */

/* ---- parameter structs ------------------------------------------------------- */
typedef struct {
    int32_t kind;                       /* P3MAZE_SR_*                                    */
    int32_t n_types;                    /* 1..P3MAZE_MAX_TYPES                            */
    /* Row-major [n_types][n_types] symmetric tables.
     * BMH: p[0]=A (kcal/mol), p[1]=rho (A), p[2]=s (A), p[3]=C (kcal/mol A^6),
     *      p[4]=D (kcal/mol A^8).   LJ: p[0]=eps (kcal/mol), p[1]=sigma (A).        */
    double p[5][P3MAZE_MAX_TYPES * P3MAZE_MAX_TYPES];
} p3maze_sr_table;

typedef struct {
    /* Rigid-topology water-like molecules (SPC/Fw, Table S1): each molecule is a
     * triple (h1, o, h2) of particle indices, every particle in at most one
     * triple.  Bonds o-h1, o-h2: (kb/2)(r-r0)^2; angle h1-o-h2: (ka/2)(t-t0)^2.
     * The three intramolecular pairs are left out of the short-range Coulomb sum
     * and their mesh part ke Q Q erf(r/(sqrt2 sigma))/r is subtracted.            */
    int32_t n_molecules;
    const int32_t *triples;             /* host, [n_molecules][3]                        */
    double kb, r0, ka, theta0;          /* kcal/mol/A^2, A, kcal/mol/rad^2, rad          */
} p3maze_topology;

typedef struct {
    double box[3];          /* cubic: |box[i]-box[0]| <= 1e-12 box[0], else INVALID       */
    int32_t n_particles;    /* >= 1                                                        */
    const double *charges;  /* host [n] e; total charge |sum Q| <= 1e-9 sum|Q| else INVALID */
    const double *masses;   /* host [n] g/mol, > 0                                         */
    const int32_t *types;   /* host [n] species index < sr->n_types (may be NULL if no sr) */
    double alpha;           /* Ewald splitting, 1/A; sigma = 1/(sqrt(2) alpha) (Eq. 5);
                               not used (may be 0) with P3MAZE_METHOD_PMAZE                */
    double r_cut;           /* real-space cutoff, A; need r_cut <= L                        */
    int32_t mesh;           /* N points per axis, N >= 4, N = m 2^l with m <= 64: the
                               multigrid levels N, N/2, ... are halved while even and
                               above 16, and the deepest must be <= 64                    */
    int32_t order;          /* assignment order; 4 (cubic B-spline) is the only one         */
    double tol;             /* max-norm tolerance of M y - sigma_p, e per mesh point (> 0)  */
    double dt;              /* time step, fs                                                */
    int32_t predictor;      /* multiplier guess y0: 1 -> y^k, 2 -> 2y^k - y^{k-1},
                               3 -> 3y^k - 3y^{k-1} + y^{k-2} (Sec. 3.3); 0 -> 3           */
    int32_t precision;      /* P3MAZE_FP64 or P3MAZE_MIXED                                  */
    int32_t max_mg_iters;   /* V-cycle cap per step; 0 -> 50                                */
    int32_t pre_sweeps;     /* red-black Gauss-Seidel sweeps before restriction; 0 -> 2    */
    int32_t post_sweeps;    /* sweeps after prolongation; 0 -> 2                            */
    double coulomb_k;       /* kcal A/(mol e^2); 0 -> 332.0637                              */
    const p3maze_sr_table *sr;      /* may be NULL: Coulomb only                           */
    const p3maze_topology *topology;/* may be NULL                                         */
    int32_t method;         /* P3MAZE_METHOD_MAZE (0), P3MAZE_METHOD_P3M or
                               P3MAZE_METHOD_PMAZE                                         */
    int32_t coarse_max;     /* the first level with n <= coarse_max is solved exactly
                               (separable Hartley transforms: by FFT in mixed precision
                               at n = 32 and 64, dense otherwise); 0 -> 64 (mixed),
                               16 (FP64)                                                   */
    int32_t lr_force;       /* P3MAZE_LR_FORCE_FD (0, the paper's Eq. 21) or
                               P3MAZE_LR_FORCE_ANALYTIC                                    */
    int32_t sr_shift;       /* P3MAZE_SR_TRUNCATE (0) or P3MAZE_SR_SHIFT_FORCE               */
} p3maze_params;

typedef struct {
    double v_sr;        /* erfc pair energy (Eq. 5)                                        */
    double v_lr;        /* 1/2 phi^T q with q the assigned (unsmoothed) charge             */
    double v_self;      /* -(1/(sqrt(2 pi) sigma)) sum Q^2 (Eq. 6)                          */
    double v_excl;      /* minus the mesh part of intramolecular pairs                     */
    double v_vdw;       /* non-Coulomb pair energy                                         */
    double v_bond;      /* bonds + angles                                                  */
    double kinetic;
    double total;
    double w_sr;        /* short-range pair virial sum_{i<j} r_ij . F_ij of the erfc and
                           non-Coulomb pair terms (kcal/mol; not part of total)          */
} p3maze_energies;

typedef struct {
    int32_t last_iters;         /* V-cycles of the last constraint solve                  */
    double last_residual;       /* max|M y - sigma_p| after it (P3M: max|M phi + 4pi q^s/h|) */
    int64_t steps;              /* MD steps taken since init                               */
    int64_t total_iters;        /* V-cycles summed over those steps                        */
    int32_t init_iters;         /* V-cycles of the initial full solve                      */
    int32_t smooth_steps;       /* K                                                       */
    double smooth_coeff;        /* c                                                       */
    int32_t mg_levels;          /* multigrid levels in use, the last solved exactly        */
    int32_t coarse_n;           /* points per axis of that coarse level                    */
    int32_t cells_per_axis;     /* cell-list grid                                          */
    double sigma;               /* Gaussian width, A                                       */
    int64_t device_bytes;       /* device memory the context allocated                     */
} p3maze_stats;

/* Pipeline stages timed by p3maze_set_timing / p3maze_get_timing. */
#define P3MAZE_ST_INTEGRATE 0  /* kick + drift + wrap, final kick                          */
#define P3MAZE_ST_CELLS     1  /* cell list and cell-ordered copies                        */
#define P3MAZE_ST_SPREAD    2  /* B-spline charge assignment                               */
#define P3MAZE_ST_SMOOTH    3  /* K diffusion steps                                        */
#define P3MAZE_ST_PREDICT   4  /* neutrality sum, sigma_p and y0                           */
#define P3MAZE_ST_SOLVE     5  /* residual tests and V-cycles (includes the host waits of
                                  the convergence test)                                    */
#define P3MAZE_ST_UPDATE    6  /* phi update                                               */
#define P3MAZE_ST_PAIR      7  /* short-range pair forces                                  */
#define P3MAZE_ST_GATHER    8  /* force interpolation and bonded terms                     */
#define P3MAZE_NSTAGES      9

typedef struct {
    double ms[P3MAZE_NSTAGES];        /* summed device time per stage (timing enabled)   */
    int64_t launches[P3MAZE_NSTAGES]; /* kernels launched per stage (always counted)     */
    int64_t timed_steps;              /* steps covered by ms                             */
    int64_t total_launches;           /* all kernels launched since init or reset        */
} p3maze_timing;

typedef struct {
    int32_t predictor;          /* chosen multiplier predictor (0 for P3M)              */
    int32_t pre_sweeps;         /* chosen red-black Gauss-Seidel sweeps before / after  */
    int32_t post_sweeps;
    int32_t diffusion_zc;       /* z planes per thread (modes 1, 2) or per block (3, 4) of the
                                   diffusion kernel                                        */
    int32_t diffusion_fuse;     /* diffusion steps per launch: 1; 2 (two steps as one 25-point
                                   stencil, FP32, N % 4 == 0); 3 or 4 (temporal blocking in
                                   shared memory, the input planes copied asynchronously;
                                   FP32 quads when N % 4 == 0);
                                   5: all K steps in one launch, the mesh resident in the
                                   shared memory of a thread-block cluster (FP32,
                                   16 <= N <= 64, N % 4 == 0); 6: all K steps at once in
                                   the Hartley basis, where (I + cM)^K is the diagonal
                                   (1 + c lambda_k)^K -- the same operator, rounded
                                   differently (FP32, N <= 64 or N in {128, 192, 256,
                                   320, 384}; each 1D transform by FFT for N = 32, 64,
                                   128 (three launches) and 192, 256, 320, 384 (five
                                   passes over global memory; radix 3 or 5 times a power
                                   of two at 192, 320, 384), dense transforms otherwise;
                                   the default at those sizes)                             */
    int32_t pair_fork;          /* short-range forces start after: 0 smoothing, 1 the cell list */
    int32_t coarse_max;         /* chosen coarse-level limit (16, 32 or 64)                */
    int32_t pair_blocks;        /* pair-kernel grid: 0 one block per home box, else that many
                                   persistent blocks (one or two per SM)                      */
    int32_t cluster_ctas;       /* mode 5: CTAs per cluster, 1, 2, 4, 8 or 16, at least the
                                   fewest whose two slab buffers (2 x 4 ceil(N/ctas) N^2 bytes)
                                   fit 200 KiB of shared memory; 0 = automatic: 16 for a
                                   context stepped alone, and in a per-member batch the
                                   largest that keeps the batch's launch within one CTA
                                   per SM.  Ignored by the other modes.                      */
    int32_t sweep_fuse;         /* 1 (default): on FP32 levels of at most 64^3 with N % 4 == 0
                                   every red-black sweep after the first is one out-of-place
                                   launch (the correction alternates between two buffers;
                                   larger levels, where it is slower, keep the half sweeps);
                                   0: two in-place half sweeps per sweep everywhere.  The
                                   same bits either way.                                     */
    double ms_per_step;         /* measured with the chosen setting (confirmation round) */
    double initial_ms_per_step; /* measured with the setting in use before tuning (the
                                   same round)                                          */
    int32_t trials;             /* settings timed                                      */
    int32_t steps;              /* MD steps advanced while tuning                      */
} p3maze_tuning;

typedef struct p3maze_ctx p3maze_ctx;

/* ---- lifecycle ------------------------------------------------------------- */

/* Validate parameters, allocate device state on the current device, upload
 * pos/vel (host [n][3] A and A/fs; vel may be NULL for zero), wrap positions
 * into the box, and initialise the field by a full constraint solve from
 * phi = 0 (phi^{-1} = phi^0, empty multiplier history), then compute F^0.
 * `cuda_stream` is a cudaStream_t (NULL = legacy default stream).
 * Errors: INVALID (parameters), OOM, CUDA, NOT_CONVERGED (initial solve).      */
int p3maze_init(const p3maze_params *params, const double *pos, const double *vel,
                void *cuda_stream, p3maze_ctx **out);

/* As p3maze_init, but positions and velocities live in caller-owned device
 * arrays d_pos/d_vel ([n][3] FP64, 8-byte aligned, on the current device):
 * the context borrows them as its own r and v -- every step updates them in
 * place, positions are wrapped into the box in place at init -- and never
 * frees them; they must outlive the context.  NaN/Inf in them is reported as
 * INVALID.  Other errors as p3maze_init.                                        */
int p3maze_init_device(const p3maze_params *params, double *d_pos, double *d_vel, void *cuda_stream,
                       p3maze_ctx **out);

/* Advance nsteps velocity-Verlet steps (Sec. 2; supporting information Sec. 1)
 * and wait for them.  The first steps after (re)initialisation, before the
 * multiplier history is full, test convergence on the host after every
 * V-cycle; later steps replay a captured CUDA graph whose multigrid loop is a
 * device-side while node, so the host waits once per call.  On
 * NOT_CONVERGED or NONFINITE (recorded on the device, first failure kept)
 * the steps are left applied and the error returned; re-initialise with
 * p3maze_reinit.                                                               */
int p3maze_step(p3maze_ctx *ctx, int32_t nsteps);

/* As p3maze_step, but return once the steps are queued (graph steps do not
 * wait for the GPU); the caller's stream is ordered after them.  Convergence
 * failures are reported by the next p3maze_wait.                               */
int p3maze_step_async(p3maze_ctx *ctx, int32_t nsteps);

/* Wait for queued steps and report a recorded solver failure.                  */
int p3maze_wait(p3maze_ctx *ctx);

/* Rollback of failed steps (SURVEY-style recovery; off by default).
 * enable = 1: the context keeps a device copy of its state (the segments of
 * p3maze_save_state and the solver state; p3maze_state_bytes of extra device
 * memory, not part of p3maze_device_bytes), taken by the first p3maze_step,
 * p3maze_step_async or p3maze_step_host after the last wait.  When the steps
 * of that call (or of the p3maze_step_async calls up to the p3maze_wait) end
 * in NOT_CONVERGED, NONFINITE or INVALID (non-finite state copied in), the
 * copy is put back before the error is returned: positions, velocities,
 * forces, fields, multiplier history and step count are those before the
 * failed steps, and the context can step again (e.g. after
 * p3maze_set_solver).  p3maze_equilibrate and batch steps are not covered.
 * enable = 0 frees the copy.  Errors: INVALID (NULL), OOM.                    */
int p3maze_set_rollback(p3maze_ctx *ctx, int32_t enable);

/* Change the constraint tolerance (e per mesh point, as params.tol) and the
 * V-cycle limit of every later solve; recorded step graphs are dropped.
 * Errors: INVALID (tol <= 0 or non-finite, max_mg_iters < 1).                 */
int p3maze_set_solver(p3maze_ctx *ctx, double tol, int32_t max_mg_iters);

/* One host round trip in one call, for drivers that keep the state on the
 * host: copy pos_in/vel_in (host [n][3], A and A/fs; either may be NULL to
 * keep the device copy) in as the continuing state (as p3maze_set_state:
 * forces and field histories kept, positions wrapped), advance nsteps steps,
 * copy positions/velocities out to pos_out/vel_out (either may be NULL), and
 * wait once.  Pinned host buffers make the copies asynchronous; pageable ones
 * work too.  pos_in may equal pos_out (and vel_in vel_out).  Inputs are
 * checked for NaN/Inf on the device: a non-finite input returns INVALID after
 * the call, with the steps applied to garbage (re-initialise with
 * p3maze_set_state + p3maze_reinit).  Solver failures as p3maze_step.          */
int p3maze_step_host(p3maze_ctx *ctx, const double *pos_in, const double *vel_in, int32_t nsteps,
                     double *pos_out, double *vel_out);

/* Full constraint solve from phi = 0 at the current positions and new forces:
 * the same initialisation as p3maze_init (after an external state change).   */
int p3maze_reinit(p3maze_ctx *ctx);

/* Relaxation before measurements that need a settled melt (the energy-drift
 * reading of the random d_min = 2 A starts, whose close like-charge pairs
 * heat the system): nsteps MD steps as p3maze_step, each followed by a
 * rescaling of all velocities on the device so that sum m v^2 equals
 * (3n - 3) k_B temperature_K (kinetic temperature with the net momentum
 * removed).  Not part of the paper's NVE method; it changes the state like
 * any steps.  Waits at the end.  Errors: INVALID (nsteps < 0 or
 * temperature_K <= 0), and as p3maze_step.                                     */
int p3maze_equilibrate(p3maze_ctx *ctx, int32_t nsteps, double temperature_K);

/* Device memory (bytes requested from cudaMalloc) that p3maze_init would
 * allocate for these parameters; host-only, no CUDA call.  For admission
 * control by memory (the allocator rounds each array up, add a margin).      */
int p3maze_device_bytes(const p3maze_params *params, size_t *out);

/* Free everything the context owns.  NULL is ignored.                          */
void p3maze_destroy(p3maze_ctx *ctx);

/* ---- observables (synchronise the context's stream) ------------------------- */

/* Energy terms of Eq. 4 at the current state (kcal/mol).                        */
int p3maze_energy(p3maze_ctx *ctx, p3maze_energies *out);

/* Statistics of the solver.                                                   */
int p3maze_get_stats(p3maze_ctx *ctx, p3maze_stats *out);

/* Copy particle arrays to host [n][3] (original particle order).              */
int p3maze_get_positions(p3maze_ctx *ctx, double *out);
int p3maze_get_velocities(p3maze_ctx *ctx, double *out);
/* which = P3MAZE_F_*                                                           */
int p3maze_get_forces(p3maze_ctx *ctx, int32_t which, double *out);

/* Copy positions and velocities in from host [n][3] as the continuing state:
 * forces and field histories are kept (use after a host round trip of the
 * same state, or call p3maze_reinit after an arbitrary change).  Positions
 * are wrapped into the box.                                                    */
int p3maze_set_state(p3maze_ctx *ctx, const double *pos, const double *vel);

/* Checkpoint and resume.  p3maze_save_state writes into a host buffer of
 * p3maze_state_bytes bytes everything the next step reads -- positions,
 * velocities, forces and their parts, per-particle energies, the assigned
 * charge, phi^k and phi^{k-1}, (h/4pi) M phi (or M phi in fixed point), the
 * correction history, the last residual, the step count and the solver
 * tallies -- and p3maze_load_state restores it into a context created with
 * the same parameters (INVALID otherwise), so that stepping continues from
 * exactly the saved state: later steps repeat an uninterrupted run bit for
 * bit (every kernel of a step is deterministic).  Both wait for
 * the context's stream.                                                        */
int p3maze_state_bytes(p3maze_ctx *ctx, size_t *out);
int p3maze_save_state(p3maze_ctx *ctx, void *buf, size_t bytes);
int p3maze_load_state(p3maze_ctx *ctx, const void *buf, size_t bytes);

/* Copy a mesh array (P3MAZE_MESH_*) to host, N^3 doubles.                      */
int p3maze_get_mesh(p3maze_ctx *ctx, int32_t which, double *out);

/* The cell list of the last force evaluation: cell index of every particle
 * ((cz*nc + cy)*nc + cx, x fastest, c = min(floor(r nc/L), nc-1)), start
 * offsets [nc^3 + 1] and the particle order sorted by (cell, index).  Any
 * pointer may be NULL.  nc = floor(L / (r_cut/2)).                            */
int p3maze_get_cells(p3maze_ctx *ctx, int32_t *cell_of, int32_t *cell_start, int32_t *order);

/* Enable (1) or disable (0) per-stage CUDA-event timing of p3maze_step and
 * reset the timing and launch counters.  Timing adds two event records per
 * stage per step on the context's stream.                                     */
int p3maze_set_timing(p3maze_ctx *ctx, int32_t enable);

/* Per-stage device time and kernel-launch counts since the last reset.       */
int p3maze_get_timing(p3maze_ctx *ctx, p3maze_timing *out);

/* Steady-state steps (full multiplier history) replay captured CUDA graphs by
 * default (enable = 1): one graph launch per step with the multigrid loop as
 * a device-side while node.  enable = 0 issues every kernel individually (same
 * kernels and launch shapes), e.g. for profilers that do not list kernels of
 * conditional graph nodes.                                                    */
/* Apply a setting (as p3maze_autotune returns it) without timing anything:
 * predictor (1..3; ignored for P3M), pre_sweeps >= 1, post_sweeps >= 0,
 * diffusion_zc >= 1, diffusion_fuse 1..6, pair_fork 0 or 1, coarse_max >= 1,
 * pair_blocks >= 0, cluster_ctas 0 or a power of two up to 16, sweep_fuse 0 or
 * 1; the timing fields are ignored.  Captured step graphs are
 * dropped.  Errors: INVALID (out-of-range field, nothing changed).            */
int p3maze_set_tuning(p3maze_ctx *ctx, const p3maze_tuning *setting);

/* The setting in use (timing fields zero).                                     */
int p3maze_get_tuning(p3maze_ctx *ctx, p3maze_tuning *out);

int p3maze_set_graphs(p3maze_ctx *ctx, int32_t enable);

/* Diffusion smoothing of a caller-owned mesh that allocates nothing.
 * The paper has no counterpart: this call exists for callers that cannot
 * allocate device memory when they need the smoothing -- code running under a
 * fixed device-memory budget owned by a host framework that makes every
 * allocation itself, or long-running services that reserve their memory at
 * start-up and must not grow their footprint afterwards.
 *   q     device, [mesh^3] FP64 input (x fastest), read only
 *   qs    device, [mesh^3] FP64 output: (I + coeff M)^steps q with its mean
 *         removed -- the same q^s the context computes (P3MAZE_MESH_QS) for
 *         steps = K, coeff = c of p3maze_get_stats; must not overlap q
 *   mesh  4..64 points per axis; larger meshes are rejected (INVALID)
 *   steps >= 0; coeff in (0, 1/6] when steps > 0
 *   cuda_stream  cudaStream_t the work is queued on (NULL = legacy stream)
 * Scratch: one file-scope device array of 2 MiB + 32 KiB (a 64^3 FP64
 * ping-pong mesh and the block sums of the mean), present on every GPU that
 * loads this library until the process exits.  No cudaMalloc, cudaFree or
 * allocating library routine is called.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device current
 * and keeps it for the life of the process, so calls must not span a
 * cudaDeviceReset of the device.  q and qs must not overlap each other or the scratch array
 * (INVALID).  All calls on a device share the array and keep nothing from
 * earlier calls: calls that overlap on the GPU (different streams, or host
 * threads queueing concurrently) race on it and must be ordered by the
 * caller.  Returns 0 or INVALID/CUDA; the
 * message is p3maze_last_error(NULL).  Asynchronous: outputs are ready when
 * the stream reaches this point.                                              */
int p3maze_smooth_noalloc(const double *q, double *qs, int32_t mesh, int32_t steps, double coeff,
                          void *cuda_stream);

/* Autotuner: time real MD steps under candidate settings and keep the
 * fastest, in greedy passes:
 *  - multiplier predictor 1..3 (P3MaZe only) x smoothing sweeps (pre, post)
 *    in {(1,1), (2,1), (1,2), (2,2), (3,3)};
 *  - the smoothing kernel (diffusion_fuse 1..6 where the mesh and precision
 *    allow it) with its z planes per thread or block;
 *  - the size of the exactly solved coarse level (coarse_max 16, 32, 64);
 *  - where the short-range pair kernel is forked onto its low-priority
 *    stream (after smoothing, or right after the cell list) and its grid
 *    (one block per home box, or a persistent grid of one block per two
 *    SMs, one or two blocks per SM); the smoothing candidates are timed
 *    again if that placement changed, since the fastest kernel depends on
 *    what runs beside it;
 *  - a confirmation round: the starting setting and the three fastest other
 *    settings timed again with 2 x steps_per_trial steps each, in two rounds
 *    of opposite order; the fastest of these is kept, and out->ms_per_step
 *    and out->initial_ms_per_step are these re-measurements.
 * None of the settings changes the converged field beyond tol (they change
 * iteration counts and speed only).  Every trial runs 2 warm-up steps (graph
 * capture) and its timed steps (CUDA events); the system advances by all of
 * them (out->steps).  Errors as p3maze_step.                                  */
int p3maze_autotune(p3maze_ctx *ctx, int32_t steps_per_trial, p3maze_tuning *out);

/* ---- batches: many systems advanced by shared launches ---------------------- */

/* A batch advances several contexts (independent systems of any size on the
 * current device) together: each batch step is ONE CUDA graph launch holding
 * one MD step of every member as a parallel branch -- each member with its
 * own device-side multigrid loop -- so their kernels overlap on the GPU.
 * Members keep all their state resident.  The batch records a graph per
 * pointer phase of its members (four at most) until the membership changes.
 * Stepping a member by itself (p3maze_step) while it is in a batch is
 * allowed between batch steps.                                                */
typedef struct p3maze_batch p3maze_batch;

/* cuda_stream: the caller's stream; each p3maze_batch_step is ordered after
 * the work queued on it, and the stream after the step.                        */
int p3maze_batch_create(void *cuda_stream, p3maze_batch **out);

/* Add a context (same device).  A context whose multiplier history is not yet
 * full is first advanced by the missing steps on its own (those steps test
 * convergence on the host).  Invalidates the recorded graphs.                  */
int p3maze_batch_add(p3maze_batch *batch, p3maze_ctx *ctx);

/* Remove a member (waits for queued batch steps).  The context stays valid.    */
int p3maze_batch_remove(p3maze_batch *batch, p3maze_ctx *ctx);

/* Queue nsteps batch steps (one graph launch each); does not wait.             */
int p3maze_batch_step(p3maze_batch *batch, int32_t nsteps);

/* Wait for queued batch steps; report the first member with a solver failure. */
int p3maze_batch_wait(p3maze_batch *batch);

int p3maze_batch_size(const p3maze_batch *batch);

/* P3MAZE_BATCH_SHARED_GRAPH (default): one graph launch per batch step, the
 * graph recorded again after every membership change.  P3MAZE_BATCH_PER_MEMBER:
 * each member replays its own cached step graphs on its own stream (forked
 * from and joined to the batch stream), with no re-recording when members
 * come and go; used by the serving loop.  The members whose smoothing runs
 * as a cluster launch (diffusion_fuse 5) can be smoothed together
 * (p3maze_batch_set_fused_smoothing): every member's step head (kick/drift, cell list, assignment),
 * then ONE launch per cluster size with one cluster per such member doing
 * all their diffusion steps, then the step tails (solve, interpolation,
 * kick); the results are those of each member stepped alone, bit for bit.
 * The batch allocates a small device table of those members (its only
 * device allocation).  A member's setting changed while it is in the batch
 * (p3maze_set_tuning, p3maze_autotune, p3maze_set_timing, p3maze_set_graphs)
 * is picked up at the next batch step.                                      */
#define P3MAZE_BATCH_SHARED_GRAPH 0
#define P3MAZE_BATCH_PER_MEMBER   1
int p3maze_batch_set_mode(p3maze_batch *batch, int32_t mode);

/* enable = 1: the members whose smoothing is a cluster launch are smoothed
 * together, as described above; 0: each member's cluster launch stays inside
 * its own step (no split of the step, no join across members); -1 (default):
 * together in P3MAZE_BATCH_PER_MEMBER, each in its own step in
 * P3MAZE_BATCH_SHARED_GRAPH (where the join costs more than the launches it
 * saves).  Results are the same bit for bit either way.
 * Errors: INVALID (NULL).                                                    */
int p3maze_batch_set_fused_smoothing(p3maze_batch *batch, int32_t enable);
void p3maze_batch_destroy(p3maze_batch *batch);
const char *p3maze_batch_last_error(const p3maze_batch *batch);

/* Message of the last failing call on ctx (or of the last failing init when
 * ctx is NULL).  Never NULL.                                                   */
const char *p3maze_last_error(const p3maze_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* P3MAZE_H */
