/*
 * sbm.h — C ABI of the GB300 (sm_103a) multigrid solver for smooth-boundary-
 * method (SBM) linear elasticity (Agrawal & Runnels, arXiv 2212.02362).
 *
 * The solved problem is the diffuse-boundary equilibrium equation of Sec. 2.1
 * (eq. SBMLinearElasticity):   div(psi sigma) = source,  sigma = C grad u,
 * with the displacement u stored at grid nodes and the indicator psi stored in
 * cells (Sec. 2.3), psi floored at psi_min so that the operator stays definite.
 * It is discretised as the cell-flux operator
 *     (K u)_n = h^-d  sum_{cells c containing n}  psi_c  int_c B_n^T C B u_c,
 * which reduces in 1D to minus C times the cell-placed-psi stencil of Sec. 2.3,
 * and solved with a geometric multigrid V-cycle (Sec. 2.2) whose smoother is
 * damped Jacobi or 2^d-colour Gauss-Seidel (Sec. 2.3); coarse psi is the mean of
 * the fine cells (Sec. 2.4).  The equation solved is K u = f on free dofs, with
 * f = -(psi b + t |grad psi|) in the paper's notation.
 *
 * Conventions shared by every entry point
 *  - Arrays are packed, component-major ("SoA"):
 *        node (i,j,k), component p  ->  p*nnodes + i + nx*(j + ny*k)
 *        cell (i,j,k)               ->  i + (nx-1)*(j + (ny-1)*k)
 *    (cell (i,j,k) has lower corner node (i,j,k); 2D grids have nz = 1 and
 *    (nx-1)*(ny-1) cells).  Faces: 0:-x 1:+x 2:-y 3:+y 4:-z 5:+z.
 *  - Pointers documented as "device" must be CUDA device (or managed) memory of
 *    the grid's device; the library checks this with cudaPointerGetAttributes and
 *    returns SBM_ERR_ARG otherwise.  Pointers documented as "host" are plain host
 *    memory.  The caller owns every buffer it passes; sbm_set_* copy what they
 *    need into library-owned device storage, so inputs may be freed afterwards.
 *  - All work is ordered on the stream given in sbm_grid_desc.  Entry points
 *    that return results to the host (sbm_solve, sbm_adjoint, norms) synchronise
 *    that stream before returning.
 *  - No entry point aborts or throws.  Each returns a status; on failure
 *    sbm_last_error() gives a one-line description.  A handle is not thread-safe.
 */
#ifndef SBM_H
#define SBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sbm_grid_s *sbm_grid;          /* opaque; created and freed by the library */

typedef enum {
    SBM_OK = 0,
    SBM_ERR_ARG = 1,       /* bad argument: null/host pointer, size, index, value */
    SBM_ERR_STATE = 2,     /* call out of order (e.g. solve before sbm_set_psi) */
    SBM_ERR_CUDA = 3,      /* a CUDA runtime call failed */
    SBM_ERR_OOM = 4,       /* device allocation failed */
    SBM_ERR_NOCONV = 5,    /* max_cycles reached before the tolerance */
    SBM_ERR_DIVERGED = 6   /* relative residual not finite or above 1e10 */
} sbm_status;

enum { SBM_FP64 = 0, SBM_MIXED = 1 };                  /* precision of the V-cycle */
enum { SBM_JACOBI = 0, SBM_MCGS = 1 };                  /* smoother */
enum { SBM_CUBIC = 0, SBM_ISO_LAME = 1, SBM_ISO_ENU = 2 };  /* moduli kinds */
enum { SBM_FREE = 0, SBM_DIRICHLET = 1, SBM_DIRICHLET_FROM_U = 2 };  /* face conditions */

typedef struct {
    int dim;               /* 2 (plane strain) or 3 */
    int n[3];              /* nodes per axis; n[2] = 1 when dim == 2; every n >= 2 */
    double h;              /* node spacing (equal on every axis), > 0 */
    int precision;         /* SBM_FP64: every level in FP64.  SBM_MIXED: FP32 V-cycle
                              inside an FP64 defect correction (FP64 fine residual,
                              update and norms) */
    void *stream;          /* cudaStream_t to order all work on; NULL: the library creates
                              its own blocking stream (ordered after legacy-stream work) */
    int device;            /* CUDA device ordinal the grid lives on */
} sbm_grid_desc;

typedef struct {
    double tol;            /* stop when ||f - K u||_2 / ||f - K u_0||_2 <= tol (free dofs) */
    int max_cycles;        /* outer iterations (V-cycles in FP64 mode) */
    int nu1, nu2;          /* pre / post smoothing sweeps */
    double omega;          /* Jacobi damping (ignored by SBM_MCGS) */
    int smoother;          /* SBM_JACOBI or SBM_MCGS */
    int inner_cycles;      /* SBM_MIXED: FP32 V-cycles per FP64 defect (>= 1).  SBM_FP64: V-cycles
                              enqueued per host read of the residual (>= 1): each V-cycle is
                              followed by its FP64 residual and a device-side check that records
                              relres and stops the rest of the batch once the tolerance is met
                              or the iteration diverges (same iterates and counts as 1) */
    int use_graph;         /* 1: replay the cycle as a CUDA graph; 0: launch eagerly */
    double inner_rtol;     /* SBM_MIXED, > 0: inner_cycles is a maximum; the FP32 V-cycles of an outer
                              iteration stop (on the device) once the FP32 residual after a V-cycle's
                              pre-smoothing is <= max(inner_rtol * |r64|, tol/2 * |r0|); 0: fixed count */
} sbm_opts;

typedef struct {
    int status;            /* the sbm_status the call returned */
    int cycles;            /* outer iterations performed */
    int vcycles;           /* V-cycles performed (cycles * inner_cycles in mixed mode) */
    int levels;            /* multigrid levels */
    double r0;             /* ||f - K u_0||_2 */
    double relres;         /* final relative residual */
    double *history;       /* host, optional: relres after each outer iteration, [0] = 1 */
    int history_capacity;  /* entries available in history */
    double setup_ms;       /* device time of psi/bottom set-up triggered by this call */
    double solve_ms;       /* device time of the solve (CUDA events on the grid stream) */
    long long launches;    /* library kernels launched by the call (graph nodes included) */
} sbm_info;

/* Fill opts with the defaults tol 1e-10, max_cycles 500, V(2,2), omega 2/3,
 * Jacobi, inner_cycles 1, use_graph 1. */
void sbm_default_opts(sbm_opts *opts);

const char *sbm_status_string(int status);
/* Last error message of a handle (or of the library when grid is NULL). */
const char *sbm_last_error(sbm_grid grid);

/* Create a grid and its multigrid hierarchy: levels are coarsened by 2 while
 * every (n-1) is even and stays >= 4 after halving (Sec. 2.2 level sequence).
 * Allocates all level storage on desc->device.  Returns SBM_ERR_ARG for a bad
 * descriptor, SBM_ERR_OOM / SBM_ERR_CUDA on allocation failure. */
sbm_status sbm_grid_create(const sbm_grid_desc *desc, sbm_grid *out);
sbm_status sbm_grid_destroy(sbm_grid grid);
/* Number of multigrid levels and the node counts of level l (0 = coarsest). */
sbm_status sbm_grid_levels(sbm_grid grid, int *nlevels);
sbm_status sbm_grid_level_shape(sbm_grid grid, int level, int n[3], double *h);

/* psi in cells (Sec. 2.3), device, FP64, packed cell layout of the finest
 * level.  psi <- max(psi, psi_min), psi_min > 0; coarse levels get the mean of
 * their 2^d fine cells (Sec. 2.4).  NaN or Inf in psi gives SBM_ERR_ARG.
 * `level` must be the finest level index (nlevels-1). */
sbm_status sbm_set_psi(sbm_grid grid, int level, const double *psi_cells, double psi_min);
/* SIMP stiffness map for topology optimisation (Sec. 3.3 uses a power of the
 * order parameter as the stiffness factor): psi = psi_min + (1 - psi_min) rho^q,
 * rho in cells (device, FP64).  The density is kept so that sbm_adjoint can
 * also return dJ/drho. */
sbm_status sbm_set_density(sbm_grid grid, int level, const double *rho_cells,
                           double psi_min, double q);
/* Uniform moduli (Sec. 2.4 vector-space parameters): SBM_CUBIC p = (C11, C12, C44)
 * axis-aligned; SBM_ISO_LAME p = (lambda, mu, -); SBM_ISO_ENU p = (E, nu, -). */
sbm_status sbm_set_moduli(sbm_grid grid, int kind, const double p[3]);
/* Face condition for one component.  SBM_DIRICHLET writes `value` into u on that
 * face before each solve (faces written in order 0..5, so a later face wins on
 * shared edges); SBM_DIRICHLET_FROM_U keeps the values the caller put in u;
 * SBM_FREE is the traction-free (natural) condition of the cell-flux form. */
sbm_status sbm_set_bc(sbm_grid grid, int face, int comp, int type, double value);
/* Right-hand side f (device, FP64, packed node layout, finest level), K u = f. */
sbm_status sbm_set_source(sbm_grid grid, int level, const double *f_nodes);

/* Load f of K u = f from the source terms of eq. SBMLinearElasticity (Sec. 2.1),
 *     div(psi C (grad u - eps0)) - psi b = t |grad psi|
 * with the cell-flux discretisation of the operator:
 *     f_n = h^-d sum_{cells c of n} psi_c int_c B_n^T C eps0_c - w_n (psi_n b_n + t_n |grad psi|_n).
 * psi: device, packed cells of `level` (used as given, no floor).  eps0 (may be NULL):
 * device, per-cell eigenstrain, Voigt slots 2D (xx, yy, xy), 3D (xx, yy, zz, yz, xz, xy)
 * holding tensor (not engineering) shear, slot-major over the packed cells.  b, t (each
 * may be NULL): device, packed nodes; b the body force, t the diffuse traction
 * (Sec. 2.1: the traction of the closest point of the boundary).  psi_n is the mean of
 * the 2^d cells around node n, grad psi_n the mean difference of the cells facing each
 * other across it, cells beyond a face of the box mirrored inside; w_n is the node's
 * share of the volume ((cells of the grid around n) / 2^d).  By Theorem 1 the traction
 * term integrates to the boundary load as the interface width goes to 0.  f: device,
 * packed nodes of `level`, overwritten (Dirichlet dofs included; the solve replaces
 * their rows).  Uses the grid's moduli; FP64; synchronises the grid stream.  Pass f on
 * to sbm_set_source.  SBM_ERR_ARG for a level out of range or host pointers,
 * SBM_ERR_STATE before sbm_set_moduli. */
sbm_status sbm_source_terms(sbm_grid grid, int level, const double *psi, const double *eps0, const double *b,
                            const double *t, double *f);

/* Solve K u = f.  u (device, FP64, packed) holds the initial guess on entry and
 * the solution on return; Dirichlet dofs are set from the face conditions and
 * never changed by the iteration.  opts may be NULL (defaults); info may be NULL.
 * Synchronises the grid stream.  Returns SBM_OK, SBM_ERR_NOCONV or
 * SBM_ERR_DIVERGED (info is filled in all three cases). */
sbm_status sbm_solve(sbm_grid grid, double *u, const sbm_opts *opts, sbm_info *info);

/* Adjoint of a solve: lambda solves K lambda = dJdu with homogeneous Dirichlet
 * conditions (the same multigrid), then for every cell
 *     dJdpsi_c = -lambda_c^T S_c u_c      (S_c: unit-psi cell matrix),
 * the sensitivity of J(u(psi)) to psi_c.  u: the solution (device, packed);
 * dJdu, lambda: device, packed nodes; dJdpsi: device, packed cells; dJdrho
 * (optional, may be NULL) receives dJdpsi * dpsi/drho when the stiffness was set
 * by sbm_set_density, and is zeroed where the psi_min floor is active otherwise.
 * Status as for sbm_solve. */
sbm_status sbm_adjoint(sbm_grid grid, const double *u, const double *dJdu, double *lambda,
                       double *dJdpsi, double *dJdrho, const sbm_opts *opts, sbm_info *info);

/* ---- single steps of the hot path, for parity tests and custom drivers ---- */
/* All step calls take packed device arrays of the given level and run the same
 * kernels as the solve.  `fp32` selects the FP32 kernels (inputs and outputs
 * are still FP64 arrays; values are rounded to FP32 on entry). */

/* Ku over all dofs, no Dirichlet masking (Sec. 2.1 operator). */
sbm_status sbm_apply(sbm_grid grid, int level, int fp32, const double *u, double *Ku);
/* r = f - K u on free dofs, 0 on Dirichlet dofs; *norm (host, may be NULL)
 * receives ||r||_2 over free dofs (deterministic two-pass reduction). */
sbm_status sbm_residual(sbm_grid grid, int level, int fp32, const double *f, const double *u,
                        double *r, double *norm);
/* One smoothing sweep in place on u (damped Jacobi with omega, or one 2^d-colour
 * Gauss-Seidel sweep, colours ascending or descending), Sec. 2.3. */
sbm_status sbm_smooth(sbm_grid grid, int level, int fp32, int smoother, double omega,
                      int descending, const double *f, double *u);
/* r_c = P^T r_f / 2^d (full weighting), zero on coarse Dirichlet dofs; level is the
 * fine level (>= 1), r_c has the layout of level-1. */
sbm_status sbm_restrict(sbm_grid grid, int level, int fp32, const double *r_f, double *r_c);
/* u_f += P e_c (bi/trilinear) on free fine dofs; level is the fine level (>= 1). */
sbm_status sbm_prolong_add(sbm_grid grid, int level, int fp32, const double *e_c, double *u_f);
/* Copy of the psi the library holds for a level (after flooring / coarsening). */
sbm_status sbm_get_psi(sbm_grid grid, int level, double *psi_cells);
/* Bottom solve on the coarsest level: u_F += K_FF^-1 (f - K u)_F (device arrays). */
sbm_status sbm_bottom_correct(sbm_grid grid, int fp32, const double *f, double *u);
/* dJdpsi_c = -lambda_c^T S_c u_c for every cell of the finest level. */
sbm_status sbm_dJdpsi(sbm_grid grid, const double *u, const double *lambda, double *dJdpsi);

/* ---- phase-field topology optimisation (Sec. 3.3): an outer staggered loop ----
 * The order parameter eta lives in the cells of the finest level and sets the
 * stiffness psi = (eta + zeta)^2 (eq. topop_objective).  One explicit Euler step of
 * eq. topop_evolution is
 *   eta' = eta - dt L [2 alpha eta (1-eta)(1-2eta) - beta Lap(eta) - (eta+zeta) e_c
 *                      + lambda(t) (V(eta) - V0)],
 * with e_c = u_c^T S_c u_c the unit-psi strain energy of cell c at the equilibrium u of
 * psi (the eta-derivative of half the compliance is -(eta+zeta) e_c), Lap the (2d+1)-
 * point cell Laplacian with eta's Neumann condition (a missing neighbour takes the
 * cell's own value), V(eta) = h^d sum_c eta_c (eq. topop_volume_constraint) and
 * lambda(t) = lambda + lambda_rate t, t = step dt.  The step is explicit: it is stable
 * for dt L (2 alpha + 4 d beta / h^2 + lambda |Omega| + max_c e_c) below about 1.  eta is
 * not clipped; psi is floored at psi_min for the solve. */
typedef struct {
    double alpha, beta;    /* double-well height and gradient-energy coefficient */
    double zeta;           /* stiffness regularisation: psi = (eta + zeta)^2 */
    double lambda;         /* volume-constraint multiplier at t = 0 ... */
    double lambda_rate;    /* ... and its linear growth rate */
    double V0;             /* target volume int eta dx */
    double mobility, dt;   /* L of eq. topop_evolution and the time step */
    double psi_min;        /* floor of psi for the solve (as sbm_set_psi) */
} sbm_topopt_params;
typedef struct {
    int steps;             /* steps completed */
    int capacity;          /* entries available in each history array below */
    double *compliance;    /* host, optional: h^d u^T K(psi) u of step s's solve (= h^d f.u for
                            * homogeneous Dirichlet data) */
    double *volume;        /* host, optional: V(eta) after step s */
    int *cycles;           /* host, optional: outer iterations of step s's solve */
    double ms;             /* wall time of the loop */
} sbm_topopt_info;
/* One step: eta_out (device, packed cells of the finest level) from eta (device,
 * packed cells; not modified) at the displacement u (device, packed nodes; the caller's
 * equilibrium for psi(eta)); `step` sets lambda(t).  volume (host, may be NULL)
 * receives V(eta_out); compliance (host, may be NULL) h^d sum_c psi_c e_c with the psi the
 * grid holds (0 before any psi is set).  Finest level of a single-level grid; needs the
 * moduli.  Synchronises the grid stream. */
sbm_status sbm_topopt_step(sbm_grid grid, const sbm_topopt_params *p, int step, const double *eta, const double *u,
                           double *eta_out, double *volume, double *compliance);
/* The staggered loop: `steps` times { psi <- max((eta+zeta)^2, psi_min) (as sbm_set_psi);
 * solve K(psi) u = f from the current u (warm start; f of sbm_set_source, opts as
 * sbm_solve); eta <- one step }.  eta and u (device, packed) are updated in place.  The
 * grid keeps the psi of the last solve.  Single-level grids only (SBM_ERR_STATE with
 * refinement patches).  A solve that ends in SBM_ERR_NOCONV / SBM_ERR_DIVERGED stops the
 * loop with that status (info->steps counts the completed steps).  opts->tol is
 * relative to each solve's initial residual, that of its warm start. */
sbm_status sbm_topopt_run(sbm_grid grid, const sbm_topopt_params *p, int steps, double *eta, double *u,
                          const sbm_opts *opts, sbm_topopt_info *info);

/* ---- the operator variants of Sec. 2.3 (for comparison with the cell-flux form) ----
 * The literal product-rule discretisation of the strong form
 *     div(psi C grad u) = psi C : grad grad u + grad psi . C grad u
 * at interior nodes by centred differences (3-point second differences, 4-point
 * mixed differences; Sec. 2.3 prints its 1D form), K u = -(that), with psi either
 *   SBM_OP_PRODUCT_NODE: at nodes (psi packed over the nodes of the finest level;
 *     grad psi by centred differences) -- the node-placed operator whose Jacobi
 *     update Sec. 2.3 shows to diverge next to a region where psi vanishes, or
 *   SBM_OP_PRODUCT_CELL: in cells (packed over the cells) and averaged to the node
 *     (psi_n = mean of the 2^d cells, grad psi from the cells facing each other
 *     across the node) -- the cell-placed update of Sec. 2.3 (in 1D the flux form).
 * Both are defined at interior nodes only: K u is 0 on the box faces.  psi is used
 * as given (no floor), so a psi of 0 is allowed.  Finest-level grid, the grid's
 * moduli; FP64.  Not part of the solve: the solver's operator is the cell-flux form. */
enum { SBM_OP_PRODUCT_NODE = 1, SBM_OP_PRODUCT_CELL = 2 };
/* Ku = K u for the chosen variant (device, packed). */
sbm_status sbm_apply_product(sbm_grid grid, int variant, const double *psi, const double *u, double *Ku);
/* `sweeps` damped Jacobi sweeps u += omega (f - K u) / diag(K) on the interior dofs
 * that carry no Dirichlet condition (diag(K) = psi_n sum_a 2 C_papa / h^2); u (device,
 * packed) in place; f device, packed.  A vanishing diagonal gives Inf/NaN entries,
 * not an error (that is the divergence the comparison exhibits). */
sbm_status sbm_jacobi_product(sbm_grid grid, int variant, const double *psi, const double *f, double *u,
                              double omega, int sweeps);

/* ---- failure-path hooks (not part of the paper's method) ----
 * For tests of the error paths without a GPU fault or real memory pressure.
 * sbm_set_alloc_limit: from now on, a grid creation (or patch addition) whose
 * device allocations would exceed `bytes` in total fails with SBM_ERR_OOM, as if
 * cudaMalloc had run out of memory; a failed creation frees what it allocated and
 * reports through sbm_last_error(NULL).  0 removes the cap.  Process-wide.
 * sbm_set_wait_limit: polls each block makes at one grid barrier of the
 * bottom-level inversion (one cooperative launch, run by the first solve after
 * psi or the moduli change) before it gives up; on a timeout every block leaves
 * the launch and the solve returns SBM_ERR_CUDA with the GPU context intact.  0
 * restores the default bound.  Forces the next solve to invert again. */
void sbm_set_alloc_limit(size_t bytes);
sbm_status sbm_set_wait_limit(sbm_grid grid, long long spins);

/* ---- measurement ---- */
enum { SBM_K_RESIDUAL64 = 0, SBM_K_JACOBI = 1, SBM_K_RESIDUAL = 2, SBM_K_SOURCE = 3, SBM_K_TOPOPT = 4,
       SBM_K_FMA64 = 5, SBM_K_FMA32 = 6, SBM_K_GS = 7 };
/* Launch one hot-path kernel of the finest level `reps` times back to back on
 * the grid stream between two CUDA events (after one untimed launch) and report
 * the mean duration per launch (host, ms), together with the algorithmic DRAM
 * bytes and floating-point operations of one launch (host, may be NULL):
 *   SBM_K_RESIDUAL64  the FP64 defect residual (FP32 output on SBM_MIXED grids)
 *   SBM_K_JACOBI      one damped-Jacobi sweep in the V-cycle precision
 *   SBM_K_RESIDUAL    the V-cycle residual in the V-cycle precision
 *   SBM_K_SOURCE      sbm_source_terms with eigenstrain, body force and traction
 *                     (FP64; bytes: psi, the d(d+1)/2 eigenstrain slots per cell and b,
 *                     t, f per node, each once)
 *   SBM_K_TOPOPT      the step of sbm_topopt_step (FP64; bytes: eta, psi, eta' and the
 *                     next psi per cell and u per node, each once)
 *   SBM_K_FMA64/32    a register-only multiply-add probe on every SM (8 independent
 *                     chains per thread, 8 blocks of 256 threads per SM): the measured
 *                     FP64 / FP32 rate that ALU-bound kernels are compared with (bytes 0)
 *   SBM_K_GS          one 2^d-colour Gauss-Seidel sweep (all colours, one launch) in the
 *                     V-cycle precision; 2D grids only (SBM_ERR_ARG otherwise); flops 190
 *                     per node (the row of K formed from the unit-psi cell matrix)
 * Bytes count one read of u, f and psi and one write of the output per node;
 * flops count the sum-factorised cell arithmetic per cell plus the per-node
 * gather and update.  flush_l2 != 0: before every launch a 256 MB scratch buffer
 * (allocated for the call) is written and a second 256 MB buffer read, so that the
 * launch reads its inputs from HBM and finds no dirty lines of other data in L2
 * (their write-back would be charged to it); each launch is timed by its own pair
 * of events.  Uses the level's work buffers (overwrites them); SBM_K_SOURCE and
 * SBM_K_TOPOPT run on scratch arrays allocated for the call. */
sbm_status sbm_time_kernel(sbm_grid grid, int which, int reps, int flush_l2, double *ms_per_launch,
                           double *bytes_per_launch, double *flops_per_launch);

/* ---- block-structured refinement (Sec. 2.2) ----
 * A grid may carry up to 64 refinement patches.  A patch of level L refines one
 * patch of level L-1 (its parent; the base grid for L = 1) by 2 on one node box; a
 * level may hold several patches (at most 8 children per parent), whose boxes are
 * at least two parent cells apart.  Patches are numbered 1, 2, ... in the order they
 * are added, every parent before its children.  The composite problem: a patch node
 * inside the box (or on a box face lying on the domain boundary) obeys the fine
 * equation; the parent node under it is covered (it takes the injected fine value);
 * the patch's other nodes (its faces inside the domain, and one layer of padding
 * nodes around the box) are ghosts interpolated from the parent; parent cells under
 * the patch hold the mean of their fine cells (Sec. 2.4).  Every fine stencil of an
 * owned node and every full-weighting stencil of a covered node is complete, so no
 * coarse/fine flux correction ("reflux") is applied.  Patch arrays cover the box
 * grown by one padding node per side: nodes [lo-1, hi+1], cells [lo-1, hi], packed x
 * fastest, component-major; values at padding nodes are outputs only.  Below, a
 * "patch a" argument is that numbering (a = 0: the base grid). */
typedef struct {
    int lo[3], hi[3];      /* node box in the new level's indices; even corners; 2D: lo[2] = hi[2] = 0 */
} sbm_box;

/* Add a patch of refinement level `level` (1 .. deepest existing level + 1) on `box`
 * (node indices of that level).  Its parent is the one patch of level-1 (the base
 * grid for level 1) that contains the box with at least one parent cell to spare on
 * every side not on the domain boundary; the box must be at least two parent cells
 * (four nodes) apart from every other patch of its level.  *index (may be NULL)
 * receives the new patch number.  Allocates the patch storage.  SBM_ERR_ARG on a bad
 * box (odd corners, outside the level, thinner than 2, no unique parent, too close to
 * a sibling, a ninth child, a 65th patch), SBM_ERR_OOM when the storage cannot
 * be allocated (nothing is kept). */
sbm_status sbm_amr_add_box(sbm_grid grid, int level, const sbm_box *box, int *index);
/* Remove every patch of refinement level >= `level` (>= 1) and free its storage; the
 * remaining patches are renumbered 1, 2, ... in their previous order.  The psi of the
 * base grid and of the kept patches is restored to what was set (their cells under
 * removed patches lose the fine means), so a later sbm_amr_regrid / sbm_amr_add_box
 * starts from the psi of the callers.  level = 1 leaves the base grid alone.  Together
 * with sbm_amr_regrid: regridding of an evolving psi. */
sbm_status sbm_amr_remove_levels(sbm_grid grid, int level);
/* Box, refinement level and parent (0: the base grid) of patch a >= 1; any output
 * pointer (host) may be NULL. */
sbm_status sbm_amr_get_box(sbm_grid grid, int a, sbm_box *box, int *level, int *parent);
/* sbm_amr_add_box at one level deeper than the deepest patch so far (level 1 on a
 * grid without patches): the one-patch-per-level hierarchy, patch a at level a. */
sbm_status sbm_amr_add_level(sbm_grid grid, const sbm_box *box);
/* Regridding (Sec. 2.2: refine where the indicator varies): build refinement level
 * `level` (= deepest existing level + 1) from the psi the grid holds (the base grid's
 * after sbm_set_psi, each patch's after sbm_amr_set_psi; floored at psi_min).  For each
 * patch of level-1 (the base grid for level 1), in patch order:
 *   - on the device, its cells in the allowed region (one parent cell inside its box,
 *     the whole level on the domain boundary) are tagged where h |grad psi| >
 *     threshold (centred differences of the cell values, no gradient across the
 *     domain boundary);
 *   - on the host: the tags are dilated by `grow` cells (Chebyshev distance) and
 *     restricted to the allowed region; connected components (cells sharing a face,
 *     edge or corner), in the order of their first cell, give boxes (child nodes
 *     [2 c_min, 2 (c_max + 1)], clipped to the allowed region, dropped if thinner than
 *     2); boxes closer than two parent cells are merged into their union and, while
 *     more than 8 remain, the pair whose union adds the least volume; the boxes are
 *     sorted by (lo, hi), x first.
 * The boxes are added as patches (sbm_amr_add_box, parents in patch order); their psi
 * is 0 until sbm_amr_set_psi.  *nadded (host, may be NULL) receives the number added.
 * SBM_ERR_ARG for another level or bad parameters, SBM_ERR_STATE before sbm_set_psi. */
sbm_status sbm_amr_regrid(sbm_grid grid, int level, double threshold, int grow, int *nadded);
/* psi of patch a (device, FP64) on the cells of the padded box, floored at psi_min.
 * Covered parent cells are replaced by fine means at the next solve. */
sbm_status sbm_amr_set_psi(sbm_grid grid, int a, const double *psi_cells, double psi_min);
/* Right-hand side of patch a (device, FP64, padded-box nodes). */
sbm_status sbm_amr_set_source(sbm_grid grid, int a, const double *f_nodes);
/* Composite solve.  u[0]: base grid nodes (packed, device); u[a], a >= 1: padded
 * box nodes of patch a (device).  In: initial guess with the Dirichlet values (the
 * face values of sbm_set_bc are written on the base level; patch Dirichlet values
 * are taken from u[a]).  Out: the composite solution with ghosts filled.  Each
 * cycle: FP64 composite residual; patches finest first (smoothing of the
 * correction, full-weighting of its residual onto the parent nodes it covers); the
 * base multigrid V-cycle; patches coarsest first (parent correction prolongated and
 * ghosts filled, smoothing); u += e on owned dofs.  SBM_MIXED runs the cycle in FP32, and
 * opts->inner_cycles of them per FP64 residual: between two of them the FP32
 * right-hand side becomes r - A e (the correction injected into covered parents,
 * every level's residual of it, owned free rows kept); opts->inner_rtol is ignored
 * (the count is fixed).  info->cycles counts FP64 residuals, info->vcycles
 * correction cycles.  Status as for sbm_solve. */
sbm_status sbm_amr_solve(sbm_grid grid, double *const *u, const sbm_opts *opts, sbm_info *info);
/* Adjoint of the composite problem of sbm_amr_solve (Sec. 2.2 levels, Sec. 2.4 psi
 * averaging; the adjoint reading D10 applied to every level).  u: the composite
 * solution (layouts as sbm_amr_solve).  dJdu[a]: dJ/du on level a, packed like u[a];
 * only its owned free dofs count.  Out: lambda[a] (packed like u[a]), the solution of
 * A^T lambda = dJ/du for the composite operator A (0 off the owned free dofs), by the
 * transposed correction iteration lambda += B^T (dJ/du - A^T lambda), B^T the
 * transpose of one correction cycle with damped-Jacobi patch sweeps (weight
 * opts->omega; on SBM_MIXED grids its stencil products and base V-cycle run in FP32,
 * A^T lambda and the vector updates in FP64), to relative residual opts->tol within
 * opts->max_cycles transposed cycles (the iteration converges at the rate of the forward
 * one).  On SBM_MIXED grids with opts->inner_cycles = k > 1, each FP64 residual is
 * followed by k transposed cycles on the correction equation A^T d = r whose residual
 * updates take FP32 stencil products, then lambda += d (as sbm_amr_solve runs k FP32
 * cycles per FP64 residual); k = 1: one cycle per FP64 residual.
 * With opts->smoother = SBM_MCGS the patch sweeps of B^T stay damped Jacobi (the
 * transpose of a colour sweep is not a colour sweep) and the base V-cycle uses the
 * colour smoother; B^T only preconditions, the fixed point A^T lambda = dJ/du is the
 * same; dJdpsi[a] (the
 * array or all of dJdpsi may be null): dJ/dpsi of level a's cells, packed like the
 * psi of sbm_set_psi (a = 0) / sbm_amr_set_psi (a >= 1): -lambda_c^T S_c u_c, where a
 * coarse cell under a patch passes its gradient to its 2^d fine cells and keeps
 * none (its psi is the fine mean), and 0 where psi sits at psi_min.  All pointers
 * are device pointers.  info: cycles = FP64 residuals (outer iterations), vcycles =
 * transposed cycles, relres, history (one entry per FP64 residual).
 * SBM_ERR_STATE without patch levels (use sbm_adjoint); status otherwise as for
 * sbm_solve. */
sbm_status sbm_amr_adjoint(sbm_grid grid, double *const *u, double *const *dJdu, double *const *lambda,
                           double *const *dJdpsi, const sbm_opts *opts, sbm_info *info);
/* Composite residual of u (layouts as sbm_amr_solve): r[a] = f_a - K_a u_a on the
 * owned free dofs of level a, 0 on ghost, covered and Dirichlet dofs; *norm (host)
 * = its 2-norm over all levels.  u is not modified.  SBM_ERR_STATE when no patch
 * level has been added (use sbm_residual). */
sbm_status sbm_amr_residual(sbm_grid grid, double *const *u, double *const *r, double *norm);

/* ---- allocation-free entry point ---- */

/* Stencil blocks whose partial sums fit the fixed scratch array of
 * sbm_residual_noalloc: 16384 doubles (128 KiB) plus 8 result slots. */
#define SBM_NOALLOC_MAX_BLOCKS 16384

/* r = f - K u on free dofs (0 on Dirichlet dofs) and ||r||_2 over free dofs, in
 * FP64, on buffers the caller owns: no grid handle and no device allocation.
 * The paper has no counterpart to this call.  It is for callers that cannot call
 * cudaMalloc: an application whose device memory belongs to its own pool allocator,
 * code that must not trigger the implicit device synchronisation of cudaMalloc and
 * cudaFree, or a process too close to its memory limit to build the level
 * hierarchy that sbm_grid_create allocates.
 * Scratch: the per-block partial sums and the result live in one fixed device array
 * of SBM_NOALLOC_MAX_BLOCKS + 8 doubles inside the library, which every GPU that
 * loads the library holds until the process exits.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress, with the device
 * current); make this first call before any stream capture.  All calls share the
 * array and it keeps the last call's contents, so calls that overlap on the GPU
 * (other streams or host threads) race: the caller must serialise them.
 * dim: 2 or 3.  n: nodes per axis (n[2] = 1 in 2D).  h: spacing.  moduli: (C11, C12,
 * C44) of an axis-aligned cubic material (isotropic: lambda + 2 mu, lambda, mu).
 * dirichlet_faces[p]: bit f set => face f (0:-x 1:+x 2:-y 3:+y 4:-z 5:+z) is
 * Dirichlet for component p.  psi (device, FP64): the floored cell values in
 * node-indexed layout, cell (i,j,k) at i + nx*(j + ny*k), the last x, y (and z)
 * slot unused.  f, u (device, FP64, packed nodes) in; r (device, packed nodes) out;
 * norm (host) out.  stream: cudaStream_t, NULL = legacy default; the call
 * synchronises it.  A grid that needs more than SBM_NOALLOC_MAX_BLOCKS stencil
 * blocks is rejected with SBM_ERR_ARG before any device work; sbm_last_error(NULL)
 * describes every failure. */
sbm_status sbm_residual_noalloc(int dim, const int n[3], double h, const double moduli[3],
                                const unsigned dirichlet_faces[3], const double *psi, const double *f,
                                const double *u, double *r, double *norm, void *stream);

#ifdef __cplusplus
}
#endif
#endif
