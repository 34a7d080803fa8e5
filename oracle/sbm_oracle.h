/*
 * sbm_oracle.h — plain, slow, FP64 CPU oracle for the smooth-boundary-method
 * (SBM) elasticity multigrid solve of Agrawal & Runnels (arXiv 2212.02362).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this code.  It is used by tests/, by __graft_entry__.smoke() (to check one
 * small GPU solve) and by bench.py's CPU-baseline leg.  It shares no source with
 * the CUDA library: every formula here is written from the paper's equations
 * and from textbook finite-element definitions.
 *
 * What is computed (paper section and equation in brackets):
 *   - The strong form div(psi C grad u) = source  [Sec. 2.1, eq. SBMLinearElasticity]
 *     with u at nodes and psi in cells [Sec. 2.3], discretised as the cell-flux
 *     (Q1, 2^d-point Gauss) operator
 *        (K u)_n = h^-d sum_{cells c containing n} psi_c  int_c B_n^T C B u_c .
 *     In 1D this is exactly minus C times the cell-placed-psi stencil of Sec. 2.3.
 *   - Damped Jacobi  u <- u + omega D^-1 (f - K u)            [Sec. 2.3, Jacobi eq.]
 *   - 2^d-colour Gauss-Seidel (colour = index parity)          [Sec. 2.3: "Gauss-Seidel"]
 *   - Coarse psi = mean of the 2^d fine cells                  [Sec. 2.4: model averaging]
 *   - Full-weighting restriction R = P^T / 2^d, (bi/tri)linear prolongation P,
 *     V(nu1,nu2) cycle, dense Cholesky bottom solve            [Sec. 2.2 level sequence]
 *   - Dense direct solve, adjoint solve and dJ/dpsi_c = -lambda_c^T S_c u_c.
 *   - Source terms of eq. SBMLinearElasticity: eigenstrain load, body force psi b
 *     and the diffuse traction t |grad psi| (Theorem 1)      [Sec. 2.1]
 *   - Phase-field topology optimisation: one explicit Allen-Cahn step with the
 *     volume constraint, psi = (eta + zeta)^2                 [Sec. 3.3]
 *
 * Layout (the same packed layout as the C ABI of the CUDA library):
 *   node (i,j,k)  -> i + nx*(j + ny*k);     component p at offset p*nnodes
 *   cell (i,j,k)  -> i + (nx-1)*(j + (ny-1)*k)   (cell with lower corner node (i,j,k))
 *   2D problems have nz = 1 and cells (nx-1)*(ny-1).
 * Faces: 0:-x 1:+x 2:-y 3:+y 4:-z 5:+z.
 */
#ifndef SBM_ORACLE_H
#define SBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int dim;               /* 2 (plane strain) or 3 */
    int n[3];              /* nodes per axis; n[2] == 1 when dim == 2 */
    double h;              /* node spacing, equal on all axes */
    double c11, c12, c44;  /* axis-aligned cubic moduli (isotropic: lambda+2mu, lambda, mu) */
    unsigned dirichlet[3]; /* per component p: bit f set => face f is Dirichlet for p */
} orc_problem;

typedef struct {
    int nu1, nu2;          /* pre / post smoothing sweeps */
    double omega;          /* Jacobi damping */
    int smoother;          /* 0 = damped Jacobi, 1 = 2^d-colour Gauss-Seidel */
    double tol;            /* stop when ||f - K u|| / ||f - K u0|| <= tol */
    int max_cycles;
} orc_mg_opts;

long orc_nnodes(const orc_problem *P);
long orc_ncells(const orc_problem *P);
int  orc_is_dirichlet(const orc_problem *P, int i, int j, int k, int p);

/* Element matrix of one cell with unit psi, FD scaled (h^-d), (2^d d) x (2^d d),
 * row index = corner*d + component.  Corner bit a gives the offset on axis a. */
void orc_element_matrix(const orc_problem *P, double *Ke);

/* Ku over all dofs (no Dirichlet masking). */
void orc_apply(const orc_problem *P, const double *psi, const double *u, double *Ku);
/* r = f - K u on free dofs, 0 on Dirichlet dofs. */
void orc_residual(const orc_problem *P, const double *psi, const double *f,
                  const double *u, double *r);
/* D_{n,p} = K_{(n,p),(n,p)} */
void orc_diagonal(const orc_problem *P, const double *psi, double *D);
/* Euclidean norm over free dofs, summed in index order. */
double orc_norm_free(const orc_problem *P, const double *r);

void orc_jacobi_sweep(const orc_problem *P, const double *psi, const double *f,
                      double *u, double omega);
/* one sweep over all 2^d colours, ascending (descending != 0: descending) */
void orc_gs_sweep(const orc_problem *P, const double *psi, const double *f,
                  double *u, int descending);

int  orc_can_coarsen(const orc_problem *P);
void orc_coarse_problem(const orc_problem *fine, orc_problem *coarse);
void orc_coarsen_psi(const orc_problem *fine, const double *psi_f, double *psi_c);
void orc_restrict(const orc_problem *fine, const double *r_f, double *r_c);
void orc_prolong_add(const orc_problem *fine, const double *e_c, double *u_f);
int  orc_num_levels(const orc_problem *P);

/* Dense (ndof x ndof) row-major assembly of K over all dofs. */
void orc_assemble_dense(const orc_problem *P, const double *psi, double *K);
/* Solve K_FF u_F = f_F - K_FD u_D by dense Cholesky; u holds Dirichlet values
 * on entry.  Returns 0, or 3 if the free-dof matrix is not positive definite. */
int  orc_direct_solve(const orc_problem *P, const double *psi, const double *f, double *u);

/* Multigrid solve.  u holds the initial guess and Dirichlet values on entry.
 * hist (max_cycles+1 entries, may be NULL) receives relres after each cycle.
 * Returns 0 converged, 1 not converged in max_cycles, 2 diverged, 3 bottom failed. */
int  orc_mg_solve(const orc_problem *P, const double *psi, const double *f, double *u,
                  const orc_mg_opts *o, double *hist, int *cycles);

/* Product-rule strong form (Sec. 2.3): the literal discretisation of
 *     div(psi C grad u) = psi C : grad grad u + grad psi . C grad u
 * at interior nodes by centred differences (3-point second differences, 4-point
 * mixed differences), with psi either at nodes (ORC_NODE_PSI, psi packed over nodes;
 * grad psi by centred differences: the node-placed operator of Sec. 2.3) or in
 * cells averaged to the node (ORC_CELL_PSI, psi packed over cells; psi_n = mean of
 * the 2^d cells, grad psi from the cells facing each other across the node: the
 * cell-placed update of Sec. 2.3, which in 1D is the flux form).  K u = -A u at the
 * interior nodes, 0 on the box faces (the form is defined at interior nodes only). */
enum { ORC_NODE_PSI = 1, ORC_CELL_PSI = 2 };
void orc_apply_product(const orc_problem *P, int variant, const double *psi, const double *u, double *Ku);
/* Diagonal of K for the product-rule form: psi_n * sum_a 2 C_papa / h^2 (interior). */
void orc_diagonal_product(const orc_problem *P, int variant, const double *psi, double *D);
/* One damped Jacobi sweep u += omega (f - K u) / D on the interior free dofs. */
void orc_jacobi_product(const orc_problem *P, int variant, const double *psi, const double *f, double *u,
                        double omega);

/* Right-hand side of eq. SBMLinearElasticity (Sec. 2.1),
 *     div(psi C (grad u - eps0)) - psi b = t |grad psi|,
 * in the form K u = f of orc_apply:
 *     f = h^-d sum_c psi_c int_c B^T C eps0_c  -  w_n (psi_n b_n + t_n |grad psi|_n).
 * eps0: per cell, Voigt components (2D xx, yy, xy; 3D xx, yy, zz, yz, xz, xy; tensor,
 * not engineering, shear), component-major over the packed cells; b, t: per node,
 * component-major; any of the three may be NULL.  psi_n, |grad psi|_n from the cells
 * around the node (cells beyond the box mirrored inside: no normal gradient at the
 * box faces), w_n = (cells of the grid around n) / 2^d (the node's share of the
 * volume).  The diffuse traction t is the value at the node (Sec. 2.1: the traction
 * of the closest point of the boundary). */
void orc_source_terms(const orc_problem *P, const double *psi, const double *eps0, const double *b, const double *t,
                      double *f);
/* psi_n, |grad psi|_n and w_n of orc_source_terms at every node. */
void orc_node_psi(const orc_problem *P, const double *psi, double *pn, double *gn, double *w);

/* Phase-field topology optimisation (Sec. 3.3, eqs. topop_objective,
 * topop_volume_constraint, topop_evolution).  eta in cells, stiffness psi = (eta+zeta)^2. */
typedef struct {
    double alpha, beta;    /* double-well height and gradient-energy coefficient */
    double zeta;           /* stiffness regularisation: psi = (eta + zeta)^2 */
    double lambda;         /* Lagrange multiplier of the volume constraint at t = 0 ... */
    double lambda_rate;    /* ... growing linearly: lambda(t) = lambda + lambda_rate t, t = step dt */
    double V0;             /* target volume */
    double mobility, dt;   /* L of eq. topop_evolution and the explicit time step */
} orc_topopt_params;
/* One explicit Euler step of eq. topop_evolution:
 *   eta_out = eta - dt L [2 alpha eta (1-eta)(1-2eta) - beta Lap(eta) - (eta+zeta) e_c
 *                         + lambda(t) (V(eta) - V0)],
 * e_c = u_c^T S_c u_c the unit-psi strain energy of cell c at the equilibrium u of psi,
 * Lap the (2d+1)-point cell Laplacian with eta's Neumann condition (a missing
 * neighbour takes the cell's own value), V(eta) = h^d sum_c eta_c. */
void orc_topopt_step(const orc_problem *P, const orc_topopt_params *T, int step, const double *eta, const double *u,
                     double *eta_out);
/* The non-elastic parts of the discrete energy whose eta-gradient the step follows:
 * out[0] = h^d sum alpha eta^2 (1-eta)^2, out[1] = h^d sum over interior faces
 * beta/2 (difference / h)^2, out[2] = lambda(t)/2 (V - V0)^2.  (The elastic part is
 * half the compliance h^d f.u of the equilibrium solve.) */
void orc_topopt_energy(const orc_problem *P, const orc_topopt_params *T, int step, const double *eta, double out[3]);

/* g_c = -lambda_c^T S_c u_c for every cell (S_c = unit-psi element matrix). */
void orc_dJdpsi(const orc_problem *P, const double *u, const double *lam, double *g);

/* ------------------------------------------------------------ BSAMR composite
 * Block-structured refinement (Sec. 2.2): patch 0 is the whole box (the base
 * level); patch a >= 1 refines its parent patch (parent[a] < a) by 2 on one node
 * box [lo, hi] given in the node indices of its level (level[a] = level of the
 * parent + 1; even corners, nested one parent cell inside the parent's box unless
 * on the domain boundary).  A level may hold several patches; patches of one
 * level are disjoint with their padded boxes apart (at least two coarse cells
 * between them), so no node of one is a ghost or padding node of another.  Patch a
 * is stored on its box grown by one padding node on every side: nodes [lo-1, hi+1],
 * cells [lo-1, hi]; arrays are packed over that padded box (x fastest,
 * component-major).  Patch 0 arrays are the ordinary full-grid arrays.
 *
 * Composite problem (reflux-free reading of Sec. 2.2):
 *  - a patch node is OWNED by its patch when on every axis it is inside the box or
 *    on a box face that lies on the domain boundary; owned nodes obey the fine
 *    equation (K_a u_a)_n = f_a(n);
 *  - the other box nodes (interface) and the padding nodes are GHOSTS, filled from
 *    the parent by (bi/tri)linear interpolation (coincident nodes copy);
 *  - a parent node coinciding with a node of a child's box region (owned there or
 *    itself covered by a grandchild) is COVERED: its value is the injected value of
 *    the finest patch whose region contains the point, and it carries no equation;
 *    so every point is owned by exactly one patch.  The other parent nodes obey the
 *    coarse equation with covered neighbours injected;
 *  - coarse cells inside a child's box hold the mean of their 2^d fine cells;
 *    padding cells beyond a domain face are not part of the body (psi ignored).
 * The padding layer gives every interface node a complete fine stencil, which
 * the multigrid restriction uses so that it is the same full weighting everywhere.
 * Functions taking "level a" below take a patch index.
 */
typedef struct {
    orc_problem base;
    int nlev;                   /* number of patches including the base (<= 65) */
    int lo[65][3], hi[65][3];   /* [a] for a >= 1, in level[a] node indices */
    int level[65];              /* refinement level of patch a (0 for a = 0) */
    int parent[65];             /* parent patch of a >= 1 (< a); -1 for a = 0 */
} orc_amr;

/* Problem (grid, h, moduli, Dirichlet faces) of the padded patch grid of level a. */
void orc_amr_level_problem(const orc_amr *A, int a, orc_problem *P);
/* 1 if level-a node (global level-a indices) is owned by level a (in its box
 * region and not covered by a finer level). */
int  orc_amr_owned(const orc_amr *A, int a, int i, int j, int k);
/* Coarse cells under each patch <- mean of the fine cells (finest first). */
void orc_amr_coarsen_psi(const orc_amr *A, double *const *psi);
/* Injection (covered coarse <- fine, finest first) then ghost fill (coarsest first). */
void orc_amr_fill(const orc_amr *A, double *const *u);
/* Composite residual: r_a = f_a - K_a u_a on owned free dofs of every level, 0 on
 * ghost, covered and Dirichlet dofs.  u is filled (injection + ghosts) in place. */
void orc_amr_residual(const orc_amr *A, double *const *psi, double *const *f, double *const *u,
                      double *const *r);
/* The composite residual at n sampled dofs (level lev[s], global level indices
 * node[3s..3s+2], component comp[s]) without filling or touching the arrays:
 * ghost and covered values are evaluated on the fly.  Equals orc_amr_residual at
 * those dofs; for checking hierarchies too large to fill and sweep whole. */
/* Gradient of J(psi) for the composite problem (Sec. 2.4 averaging of psi under
 * patches, reading D10 on every level): u = the filled composite solution, lam = the
 * adjoint solution of A^T lam = dJ/dx scattered to the owned free dofs (0
 * elsewhere).  g[a] (level-a storage cells) = -lam_c^T S_c u_c for cells inside the
 * domain; then each coarse cell under a patch passes g / 2^d to its fine cells
 * (coarse to fine) and is set to 0 (its psi is the fine mean, not a parameter). */
void orc_amr_dJdpsi(const orc_amr *A, double *const *u, double *const *lam, double *const *g);
void orc_amr_residual_at(const orc_amr *A, double *const *psi, double *const *f, double *const *u, long n,
                         const int *lev, const int *node, const int *comp, double *r);

typedef struct {
    int nu1, nu2;          /* pre / post smoothing sweeps (every level) */
    double omega;          /* damped-Jacobi factor on the patch levels */
    double omega_base;     /* damping of the base-level V-cycle's smoother */
    int smoother_base;     /* 0 = damped Jacobi, 1 = 2^d-colour Gauss-Seidel on the base level */
    double tol;            /* stop when ||r|| / ||r0|| <= tol (composite residual, owned free dofs) */
    int max_cycles;
} orc_amr_opts;

/* Composite solve by the correction iteration u += B (f - A u), A the composite
 * operator above, B one correction cycle in the level order of Sec. 2.2:
 *   - patches from the finest down: the correction e_a of level a starts at 0 and
 *     gets nu1 damped-Jacobi sweeps on K_a e_a = rhs_a over the free dofs of the
 *     level's solve region (owned and covered nodes; ghosts held at 0), where rhs_a
 *     is the composite residual on the owned dofs and, on the covered nodes, the
 *     full-weighting restriction R = P^T / 2^d of the next finer level's residual
 *     rhs - K e after its smoothing;
 *   - the base level: one V-cycle of orc_mg_solve on its correction equation;
 *   - patches from the coarsest up: e_a += the (bi/tri)linear interpolation of e_{a-1}
 *     at every patch node, then nu2 sweeps as above;
 *   - u_a += e_a on the owned free dofs.
 * psi must hold the coarse means under the patches (orc_amr_coarsen_psi).  The
 * fixed point is A u = f whatever B is; B only sets the rate.  u is filled on
 * return.  hist (max_cycles + 1 entries, may be NULL) receives relres per cycle.
 * Returns 0 converged, 1 not converged in max_cycles, 2 diverged, 3 bottom failed. */
int orc_amr_solve(const orc_amr *A, double *const *psi, double *const *f, double *const *u,
                  const orc_amr_opts *o, double *hist, int *cycles);

#ifdef __cplusplus
}
#endif
#endif
