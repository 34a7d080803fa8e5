/*
 * sbm_oracle.c — plain FP64 CPU oracle.  TEST INFRASTRUCTURE ONLY (see the
 * header for who may use it and for the layout).  Every loop follows the
 * definition it names, in the order the definition states it; nothing is
 * blocked, fused or reordered for speed.
 */
#include "sbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ grid */

long orc_nnodes(const orc_problem *P) { return (long)P->n[0] * P->n[1] * P->n[2]; }

static int ncell_axis(const orc_problem *P, int a)
{
    if (a == 2 && P->dim == 2) return 1;
    return P->n[a] - 1;
}

long orc_ncells(const orc_problem *P)
{
    return (long)ncell_axis(P, 0) * ncell_axis(P, 1) * ncell_axis(P, 2);
}

static long nid(const orc_problem *P, int i, int j, int k)
{
    return i + (long)P->n[0] * (j + (long)P->n[1] * k);
}

static long cid(const orc_problem *P, int i, int j, int k)
{
    return i + (long)(P->n[0] - 1) * (j + (long)(P->n[1] - 1) * k);
}

/* Dirichlet dofs sit only on the faces of the box (Sec. 2.1: essential
 * conditions are not imposed on the diffuse boundary).  A dof on an edge or
 * corner is Dirichlet if any face it lies on is Dirichlet for that component. */
int orc_is_dirichlet(const orc_problem *P, int i, int j, int k, int p)
{
    unsigned m = P->dirichlet[p];
    if ((m & 1u) && i == 0) return 1;
    if ((m & 2u) && i == P->n[0] - 1) return 1;
    if ((m & 4u) && j == 0) return 1;
    if ((m & 8u) && j == P->n[1] - 1) return 1;
    if (P->dim == 3) {
        if ((m & 16u) && k == 0) return 1;
        if ((m & 32u) && k == P->n[2] - 1) return 1;
    }
    return 0;
}

/* ------------------------------------------------------- element matrix */

/* Fourth-order stiffness of an axis-aligned cubic crystal:
 *   C_iiii = c11, C_iijj = c12 (i != j), C_ijij = C_ijji = c44 (i != j). */
static double cubic_C(const orc_problem *P, int i, int j, int k, int l)
{
    if (i == j && k == l) return (i == k) ? P->c11 : P->c12;
    if (i != j && ((i == k && j == l) || (i == l && j == k))) return P->c44;
    return 0.0;
}

/* Q1 shape function of a corner along one axis and its derivative (unit cell). */
static double shape1(int bit, double xi) { return bit ? xi : 1.0 - xi; }
static double dshape1(int bit) { return bit ? 1.0 : -1.0; }

void orc_element_matrix(const orc_problem *P, double *Ke)
{
    const int d = P->dim, nc = 1 << d, nd = nc * d;
    const double h = P->h;
    const double gp[2] = {0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)};
    const double w = pow(h, d) / nc;           /* Gauss weight, 2 points per axis */
    double eps[8][3][3][3];                    /* eps[corner][comp][i][j] at one Gauss point */
    double sig[8][3][3][3];
    memset(Ke, 0, sizeof(double) * nd * nd);
    for (int g = 0; g < nc; ++g) {
        double xi[3];
        for (int a = 0; a < d; ++a) xi[a] = gp[(g >> a) & 1];
        for (int c = 0; c < nc; ++c) {
            double dN[3];                     /* physical gradient of N_c */
            for (int a = 0; a < d; ++a) {
                double v = dshape1((c >> a) & 1) / h;
                for (int b = 0; b < d; ++b)
                    if (b != a) v *= shape1((c >> b) & 1, xi[b]);
                dN[a] = v;
            }
            for (int p = 0; p < d; ++p) {
                /* strain of the displacement field N_c e_p:  eps_ij = (d_ip dN_j + d_jp dN_i)/2 */
                for (int i = 0; i < d; ++i)
                    for (int j = 0; j < d; ++j)
                        eps[c][p][i][j] = 0.5 * ((i == p ? dN[j] : 0.0) + (j == p ? dN[i] : 0.0));
                for (int i = 0; i < d; ++i)
                    for (int j = 0; j < d; ++j) {
                        double s = 0.0;
                        for (int k = 0; k < d; ++k)
                            for (int l = 0; l < d; ++l) s += cubic_C(P, i, j, k, l) * eps[c][p][k][l];
                        sig[c][p][i][j] = s;
                    }
            }
        }
        for (int a = 0; a < nc; ++a)
            for (int p = 0; p < d; ++p)
                for (int b = 0; b < nc; ++b)
                    for (int q = 0; q < d; ++q) {
                        double s = 0.0;
                        for (int i = 0; i < d; ++i)
                            for (int j = 0; j < d; ++j) s += eps[a][p][i][j] * sig[b][q][i][j];
                        Ke[(a * d + p) * nd + (b * d + q)] += w * s;
                    }
    }
    const double scale = pow(h, -d);            /* FD scaling: (Ku)_n ~ -div(psi C grad u)(x_n) */
    for (int e = 0; e < nd * nd; ++e) Ke[e] *= scale;
}

/* ------------------------------------------------------------- operator */

static void cell_corner(const orc_problem *P, int ci, int cj, int ck, int a, int *i, int *j, int *k)
{
    *i = ci + (a & 1);
    *j = cj + ((a >> 1) & 1);
    *k = (P->dim == 3) ? ck + ((a >> 2) & 1) : 0;
}

void orc_apply(const orc_problem *P, const double *psi, const double *u, double *Ku)
{
    const int d = P->dim, nc = 1 << d, nd = nc * d;
    const long N = orc_nnodes(P);
    double Ke[24 * 24], ue[24], fe[24];
    orc_element_matrix(P, Ke);
    memset(Ku, 0, sizeof(double) * d * N);
    for (int ck = 0; ck < ncell_axis(P, 2); ++ck)
        for (int cj = 0; cj < ncell_axis(P, 1); ++cj)
            for (int ci = 0; ci < ncell_axis(P, 0); ++ci) {
                const double pc = psi[cid(P, ci, cj, ck)];
                long node[8];
                for (int a = 0; a < nc; ++a) {
                    int i, j, k;
                    cell_corner(P, ci, cj, ck, a, &i, &j, &k);
                    node[a] = nid(P, i, j, k);
                    for (int q = 0; q < d; ++q) ue[a * d + q] = u[q * N + node[a]];
                }
                for (int r = 0; r < nd; ++r) {
                    double s = 0.0;
                    for (int c = 0; c < nd; ++c) s += Ke[r * nd + c] * ue[c];
                    fe[r] = s;
                }
                for (int a = 0; a < nc; ++a)
                    for (int p = 0; p < d; ++p) Ku[p * N + node[a]] += pc * fe[a * d + p];
            }
}

void orc_residual(const orc_problem *P, const double *psi, const double *f,
                  const double *u, double *r)
{
    const int d = P->dim;
    const long N = orc_nnodes(P);
    orc_apply(P, psi, u, r);
    for (int k = 0; k < P->n[2]; ++k)
        for (int j = 0; j < P->n[1]; ++j)
            for (int i = 0; i < P->n[0]; ++i)
                for (int p = 0; p < d; ++p) {
                    long e = p * N + nid(P, i, j, k);
                    r[e] = orc_is_dirichlet(P, i, j, k, p) ? 0.0 : f[e] - r[e];
                }
}

void orc_diagonal(const orc_problem *P, const double *psi, double *D)
{
    const int d = P->dim, nc = 1 << d, nd = nc * d;
    const long N = orc_nnodes(P);
    double Ke[24 * 24];
    orc_element_matrix(P, Ke);
    memset(D, 0, sizeof(double) * d * N);
    for (int ck = 0; ck < ncell_axis(P, 2); ++ck)
        for (int cj = 0; cj < ncell_axis(P, 1); ++cj)
            for (int ci = 0; ci < ncell_axis(P, 0); ++ci) {
                const double pc = psi[cid(P, ci, cj, ck)];
                for (int a = 0; a < nc; ++a) {
                    int i, j, k;
                    cell_corner(P, ci, cj, ck, a, &i, &j, &k);
                    for (int p = 0; p < d; ++p)
                        D[p * N + nid(P, i, j, k)] += pc * Ke[(a * d + p) * nd + (a * d + p)];
                }
            }
}

double orc_norm_free(const orc_problem *P, const double *r)
{
    const long N = orc_nnodes(P);
    double s = 0.0;
    for (int p = 0; p < P->dim; ++p)
        for (int k = 0; k < P->n[2]; ++k)
            for (int j = 0; j < P->n[1]; ++j)
                for (int i = 0; i < P->n[0]; ++i)
                    if (!orc_is_dirichlet(P, i, j, k, p)) {
                        double v = r[p * N + nid(P, i, j, k)];
                        s += v * v;
                    }
    return sqrt(s);
}

/* -------------------------------------------------------------- smoothers */

/* Jacobi (Sec. 2.3): u^{n+1} = D^-1 (b - (A - D) u^n), damped:
 * u <- u + omega D^-1 (f - K u) on free dofs. */
void orc_jacobi_sweep(const orc_problem *P, const double *psi, const double *f,
                      double *u, double omega)
{
    const int d = P->dim;
    const long N = orc_nnodes(P);
    double *r = malloc(sizeof(double) * d * N);
    double *D = malloc(sizeof(double) * d * N);
    orc_residual(P, psi, f, u, r);
    orc_diagonal(P, psi, D);
    for (int p = 0; p < d; ++p)
        for (int k = 0; k < P->n[2]; ++k)
            for (int j = 0; j < P->n[1]; ++j)
                for (int i = 0; i < P->n[0]; ++i)
                    if (!orc_is_dirichlet(P, i, j, k, p)) {
                        long e = p * N + nid(P, i, j, k);
                        u[e] += omega * r[e] / D[e];
                    }
    free(r);
    free(D);
}

/* Row (n,p) of K u, gathered from the cells around node n. */
static double apply_row(const orc_problem *P, const double *Ke, const double *psi,
                        const double *u, int i, int j, int k, int p)
{
    const int d = P->dim, nc = 1 << d, nd = nc * d;
    const long N = orc_nnodes(P);
    double s = 0.0;
    for (int a = 0; a < nc; ++a) {          /* n is corner a of cell (i,j,k) - offset(a) */
        int ci = i - (a & 1), cj = j - ((a >> 1) & 1), ck = (d == 3) ? k - ((a >> 2) & 1) : 0;
        if (ci < 0 || cj < 0 || ck < 0) continue;
        if (ci >= ncell_axis(P, 0) || cj >= ncell_axis(P, 1) || ck >= ncell_axis(P, 2)) continue;
        const double pc = psi[cid(P, ci, cj, ck)];
        for (int b = 0; b < nc; ++b) {
            int bi, bj, bk;
            cell_corner(P, ci, cj, ck, b, &bi, &bj, &bk);
            for (int q = 0; q < d; ++q)
                s += pc * Ke[(a * d + p) * nd + (b * d + q)] * u[q * N + nid(P, bi, bj, bk)];
        }
    }
    return s;
}

/* 2^d-colour Gauss-Seidel: colour = (i&1) + 2(j&1) [+ 4(k&1)].  Nodes of one
 * colour do not couple through the 3^d stencil; within a node the components
 * are relaxed in order x, y[, z] using the latest values. */
void orc_gs_sweep(const orc_problem *P, const double *psi, const double *f,
                  double *u, int descending)
{
    const int d = P->dim, ncol = 1 << d, nc = 1 << d, nd = nc * d;
    const long N = orc_nnodes(P);
    double Ke[24 * 24];
    orc_element_matrix(P, Ke);
    double *D = malloc(sizeof(double) * d * N);
    orc_diagonal(P, psi, D);
    for (int s = 0; s < ncol; ++s) {
        const int col = descending ? ncol - 1 - s : s;
        for (int k = 0; k < P->n[2]; ++k)
            for (int j = 0; j < P->n[1]; ++j)
                for (int i = 0; i < P->n[0]; ++i) {
                    int c = (i & 1) + 2 * (j & 1) + (d == 3 ? 4 * (k & 1) : 0);
                    if (c != col) continue;
                    for (int p = 0; p < d; ++p) {
                        if (orc_is_dirichlet(P, i, j, k, p)) continue;
                        long e = p * N + nid(P, i, j, k);
                        double r = f[e] - apply_row(P, Ke, psi, u, i, j, k, p);
                        u[e] += r / D[e];
                    }
                }
    }
    free(D);
}

/* ------------------------------------------------------ level transfers */

/* Coarsen while every active N-1 is even and every coarse N-1 stays >= 4. */
int orc_can_coarsen(const orc_problem *P)
{
    for (int a = 0; a < P->dim; ++a) {
        int m = P->n[a] - 1;
        if (m % 2 != 0 || m / 2 < 4) return 0;
    }
    return 1;
}

void orc_coarse_problem(const orc_problem *fine, orc_problem *coarse)
{
    *coarse = *fine;
    for (int a = 0; a < fine->dim; ++a) coarse->n[a] = (fine->n[a] - 1) / 2 + 1;
    coarse->h = 2.0 * fine->h;
}

int orc_num_levels(const orc_problem *P)
{
    orc_problem a = *P, b;
    int L = 1;
    while (orc_can_coarsen(&a)) {
        orc_coarse_problem(&a, &b);
        a = b;
        ++L;
    }
    return L;
}

/* Coarse material = average of the 2^d fine cells it covers (Sec. 2.4: the
 * material model is a vector space, so averaging is well defined). */
void orc_coarsen_psi(const orc_problem *fine, const double *psi_f, double *psi_c)
{
    orc_problem C;
    orc_coarse_problem(fine, &C);
    const int d = fine->dim, nc = 1 << d;
    for (int K = 0; K < ncell_axis(&C, 2); ++K)
        for (int J = 0; J < ncell_axis(&C, 1); ++J)
            for (int I = 0; I < ncell_axis(&C, 0); ++I) {
                double s = 0.0;
                for (int a = 0; a < nc; ++a) {
                    int i = 2 * I + (a & 1), j = 2 * J + ((a >> 1) & 1), k = (d == 3) ? 2 * K + ((a >> 2) & 1) : 0;
                    s += psi_f[cid(fine, i, j, k)];
                }
                psi_c[cid(&C, I, J, K)] = s / nc;
            }
}

/* Linear interpolation weight between fine offset m and coarse node 2I. */
static double pw(int off)
{
    if (off == 0) return 1.0;
    if (off == 1 || off == -1) return 0.5;
    return 0.0;
}

/* r_c = P^T r_f / 2^d, zero at coarse Dirichlet dofs. */
void orc_restrict(const orc_problem *fine, const double *r_f, double *r_c)
{
    orc_problem C;
    orc_coarse_problem(fine, &C);
    const int d = fine->dim;
    const long Nf = orc_nnodes(fine), Nc = orc_nnodes(&C);
    const double scale = 1.0 / (1 << d);
    for (int p = 0; p < d; ++p)
        for (int K = 0; K < C.n[2]; ++K)
            for (int J = 0; J < C.n[1]; ++J)
                for (int I = 0; I < C.n[0]; ++I) {
                    double s = 0.0;
                    if (!orc_is_dirichlet(&C, I, J, K, p)) {
                        int k0 = (d == 3) ? -1 : 0, k1 = (d == 3) ? 1 : 0;
                        for (int dk = k0; dk <= k1; ++dk)
                            for (int dj = -1; dj <= 1; ++dj)
                                for (int di = -1; di <= 1; ++di) {
                                    int i = 2 * I + di, j = 2 * J + dj, k = (d == 3) ? 2 * K + dk : 0;
                                    if (i < 0 || j < 0 || k < 0) continue;
                                    if (i >= fine->n[0] || j >= fine->n[1] || k >= fine->n[2]) continue;
                                    s += pw(di) * pw(dj) * (d == 3 ? pw(dk) : 1.0) * r_f[p * Nf + nid(fine, i, j, k)];
                                }
                        s *= scale;
                    }
                    r_c[p * Nc + nid(&C, I, J, K)] = s;
                }
}

/* u_f += P e_c on free fine dofs. */
void orc_prolong_add(const orc_problem *fine, const double *e_c, double *u_f)
{
    orc_problem C;
    orc_coarse_problem(fine, &C);
    const int d = fine->dim;
    const long Nf = orc_nnodes(fine), Nc = orc_nnodes(&C);
    for (int p = 0; p < d; ++p)
        for (int k = 0; k < fine->n[2]; ++k)
            for (int j = 0; j < fine->n[1]; ++j)
                for (int i = 0; i < fine->n[0]; ++i) {
                    if (orc_is_dirichlet(fine, i, j, k, p)) continue;
                    double s = 0.0;
                    for (int K = k / 2; K <= (k + 1) / 2 && K < C.n[2]; ++K)
                        for (int J = j / 2; J <= (j + 1) / 2 && J < C.n[1]; ++J)
                            for (int I = i / 2; I <= (i + 1) / 2 && I < C.n[0]; ++I)
                                s += pw(i - 2 * I) * pw(j - 2 * J) * (d == 3 ? pw(k - 2 * K) : 1.0) *
                                     e_c[p * Nc + nid(&C, I, J, K)];
                    u_f[p * Nf + nid(fine, i, j, k)] += s;
                }
}

/* ------------------------------------------------------------ dense solve */

void orc_assemble_dense(const orc_problem *P, const double *psi, double *K)
{
    const int d = P->dim;
    const long N = orc_nnodes(P), n = d * N;
    double *e = calloc(n, sizeof(double));
    double *col = malloc(sizeof(double) * n);
    for (long c = 0; c < n; ++c) {           /* column c = K e_c */
        e[c] = 1.0;
        orc_apply(P, psi, e, col);
        for (long r = 0; r < n; ++r) K[r * n + c] = col[r];
        e[c] = 0.0;
    }
    free(e);
    free(col);
}

/* In-place Cholesky A = L L^T (lower triangle), m x m row-major. */
static int cholesky(double *A, long m)
{
    for (long j = 0; j < m; ++j) {
        double s = A[j * m + j];
        for (long k = 0; k < j; ++k) s -= A[j * m + k] * A[j * m + k];
        if (!(s > 0.0)) return 3;
        double ljj = sqrt(s);
        A[j * m + j] = ljj;
        for (long i = j + 1; i < m; ++i) {
            double t = A[i * m + j];
            for (long k = 0; k < j; ++k) t -= A[i * m + k] * A[j * m + k];
            A[i * m + j] = t / ljj;
        }
    }
    return 0;
}

static void cholesky_solve(const double *L, long m, double *b)
{
    for (long i = 0; i < m; ++i) {
        double s = b[i];
        for (long k = 0; k < i; ++k) s -= L[i * m + k] * b[k];
        b[i] = s / L[i * m + i];
    }
    for (long i = m - 1; i >= 0; --i) {
        double s = b[i];
        for (long k = i + 1; k < m; ++k) s -= L[k * m + i] * b[k];
        b[i] = s / L[i * m + i];
    }
}

/* free-dof index list (dof = p*N + node) */
static long free_dofs(const orc_problem *P, long *list)
{
    const long N = orc_nnodes(P);
    long m = 0;
    for (int p = 0; p < P->dim; ++p)
        for (int k = 0; k < P->n[2]; ++k)
            for (int j = 0; j < P->n[1]; ++j)
                for (int i = 0; i < P->n[0]; ++i)
                    if (!orc_is_dirichlet(P, i, j, k, p)) list[m++] = p * N + nid(P, i, j, k);
    return m;
}

typedef struct {
    long m;
    long *dofs;
    double *L;
} orc_chol;

static int chol_factor(const orc_problem *P, const double *psi, orc_chol *c)
{
    const long n = P->dim * orc_nnodes(P);
    double *K = malloc(sizeof(double) * n * n);
    orc_assemble_dense(P, psi, K);
    c->dofs = malloc(sizeof(long) * n);
    c->m = free_dofs(P, c->dofs);
    c->L = malloc(sizeof(double) * c->m * c->m);
    for (long a = 0; a < c->m; ++a)
        for (long b = 0; b < c->m; ++b) c->L[a * c->m + b] = K[c->dofs[a] * n + c->dofs[b]];
    free(K);
    return cholesky(c->L, c->m);
}

static void chol_free(orc_chol *c)
{
    free(c->dofs);
    free(c->L);
}

/* u_F += K_FF^-1 (f - K u)_F : exact solve in correction form. */
static void chol_correct(const orc_problem *P, const double *psi, const orc_chol *c,
                         const double *f, double *u)
{
    const long n = P->dim * orc_nnodes(P);
    double *r = malloc(sizeof(double) * n);
    double *b = malloc(sizeof(double) * c->m);
    orc_residual(P, psi, f, u, r);
    for (long a = 0; a < c->m; ++a) b[a] = r[c->dofs[a]];
    cholesky_solve(c->L, c->m, b);
    for (long a = 0; a < c->m; ++a) u[c->dofs[a]] += b[a];
    free(r);
    free(b);
}

int orc_direct_solve(const orc_problem *P, const double *psi, const double *f, double *u)
{
    orc_chol c;
    int st = chol_factor(P, psi, &c);
    if (st == 0) chol_correct(P, psi, &c, f, u);
    chol_free(&c);
    return st;
}

/* -------------------------------------------------------------- V-cycle */

typedef struct {
    orc_problem P;
    double *psi, *u, *f, *r;
} orc_level;

static void smooth(orc_level *L, const orc_mg_opts *o, int nsweeps, int descending)
{
    for (int s = 0; s < nsweeps; ++s) {
        if (o->smoother == 1) orc_gs_sweep(&L->P, L->psi, L->f, L->u, descending);
        else orc_jacobi_sweep(&L->P, L->psi, L->f, L->u, o->omega);
    }
}

/* V(nu1, nu2): smooth, restrict the residual, recurse from a zero guess,
 * prolongate the correction, smooth (Sec. 2.2: refined levels extend the
 * multigrid coarse/fine sequence; here every level covers the whole box). */
static void vcycle(orc_level *lev, int l, const orc_mg_opts *o, const orc_chol *bottom)
{
    orc_level *L = &lev[l];
    if (l == 0) {
        chol_correct(&L->P, L->psi, bottom, L->f, L->u);
        return;
    }
    orc_level *C = &lev[l - 1];
    smooth(L, o, o->nu1, 0);
    orc_residual(&L->P, L->psi, L->f, L->u, L->r);
    orc_restrict(&L->P, L->r, C->f);
    memset(C->u, 0, sizeof(double) * C->P.dim * orc_nnodes(&C->P));
    vcycle(lev, l - 1, o, bottom);
    orc_prolong_add(&L->P, C->u, L->u);
    smooth(L, o, o->nu2, 1);
}

int orc_mg_solve(const orc_problem *P, const double *psi, const double *f, double *u,
                 const orc_mg_opts *o, double *hist, int *cycles)
{
    const int nl = orc_num_levels(P);
    orc_level *lev = calloc(nl, sizeof(orc_level));
    /* finest level = index nl-1 */
    lev[nl - 1].P = *P;
    for (int l = nl - 2; l >= 0; --l) orc_coarse_problem(&lev[l + 1].P, &lev[l].P);
    for (int l = 0; l < nl; ++l) {
        const long N = orc_nnodes(&lev[l].P), NC = orc_ncells(&lev[l].P);
        const int d = P->dim;
        lev[l].psi = malloc(sizeof(double) * NC);
        lev[l].r = malloc(sizeof(double) * d * N);
        if (l < nl - 1) {
            lev[l].u = calloc(d * N, sizeof(double));
            lev[l].f = calloc(d * N, sizeof(double));
        }
    }
    memcpy(lev[nl - 1].psi, psi, sizeof(double) * orc_ncells(P));
    lev[nl - 1].u = u;
    lev[nl - 1].f = (double *)f;
    for (int l = nl - 1; l > 0; --l) orc_coarsen_psi(&lev[l].P, lev[l].psi, lev[l - 1].psi);

    orc_chol bottom;
    int status = chol_factor(&lev[0].P, lev[0].psi, &bottom);
    int ncyc = 0;
    if (status == 0) {
        double *r = lev[nl - 1].r;
        orc_residual(P, psi, f, u, r);
        const double r0 = orc_norm_free(P, r);
        double rel = 1.0;
        if (hist) hist[0] = 1.0;
        status = 1;
        if (r0 == 0.0) status = 0;
        while (status == 1 && ncyc < o->max_cycles) {
            vcycle(lev, nl - 1, o, &bottom);
            ++ncyc;
            orc_residual(P, psi, f, u, r);
            rel = orc_norm_free(P, r) / r0;
            if (hist) hist[ncyc] = rel;
            if (!isfinite(rel) || rel > 1e10) status = 2;
            else if (rel <= o->tol) status = 0;
        }
    }
    chol_free(&bottom);
    for (int l = 0; l < nl; ++l) {
        free(lev[l].psi);
        free(lev[l].r);
        if (l < nl - 1) {
            free(lev[l].u);
            free(lev[l].f);
        }
    }
    free(lev);
    if (cycles) *cycles = ncyc;
    return status;
}

/* ------------------------------------------------------------- gradient */

/* For J with adjoint lambda (K lambda = dJ/du, lambda = 0 on Dirichlet dofs):
 * dJ/dpsi_c = -lambda_c^T S_c u_c, S_c the unit-psi element matrix. */
void orc_dJdpsi(const orc_problem *P, const double *u, const double *lam, double *g)
{
    const int d = P->dim, nc = 1 << d, nd = nc * d;
    const long N = orc_nnodes(P);
    double Ke[24 * 24], ue[24], le[24];
    orc_element_matrix(P, Ke);
    for (int ck = 0; ck < ncell_axis(P, 2); ++ck)
        for (int cj = 0; cj < ncell_axis(P, 1); ++cj)
            for (int ci = 0; ci < ncell_axis(P, 0); ++ci) {
                for (int a = 0; a < nc; ++a) {
                    int i, j, k;
                    cell_corner(P, ci, cj, ck, a, &i, &j, &k);
                    for (int q = 0; q < d; ++q) {
                        ue[a * d + q] = u[q * N + nid(P, i, j, k)];
                        le[a * d + q] = lam[q * N + nid(P, i, j, k)];
                    }
                }
                double s = 0.0;
                for (int r = 0; r < nd; ++r)
                    for (int c = 0; c < nd; ++c) s += le[r] * Ke[r * nd + c] * ue[c];
                g[cid(P, ci, cj, ck)] = -s;
            }
}

/* ------------------------------------------------------------------- BSAMR */

static int amr_N(const orc_amr *A, int a, int axis)
{
    if (axis >= A->base.dim) return 1;
    return (A->base.n[axis] - 1) * (1 << A->level[a]) + 1;
}

void orc_amr_level_problem(const orc_amr *A, int a, orc_problem *P)
{
    *P = A->base;
    if (a == 0) return;
    for (int ax = 0; ax < 3; ++ax)
        P->n[ax] = (ax < A->base.dim) ? A->hi[a][ax] - A->lo[a][ax] + 3 : 1;
    P->h = A->base.h / (double)(1 << A->level[a]);
    P->dirichlet[0] = P->dirichlet[1] = P->dirichlet[2] = 0u;
}

/* global level-a node -> local index in the level's storage, or -1 if outside it */
static long amr_local(const orc_amr *A, int a, int g[3])
{
    orc_problem P;
    orc_amr_level_problem(A, a, &P);
    int l[3];
    for (int ax = 0; ax < 3; ++ax) {
        l[ax] = (a == 0 || ax >= A->base.dim) ? g[ax] : g[ax] - A->lo[a][ax] + 1;
        if (l[ax] < 0 || l[ax] >= P.n[ax]) return -1;
    }
    return l[0] + (long)P.n[0] * (l[1] + (long)P.n[1] * l[2]);
}

/* Level-a node g is inside level a's solve region: inside the domain for the base
 * level; for a patch, inside its box on every axis or on a box face that lies on
 * the domain boundary. */
static int amr_box_owned(const orc_amr *A, int a, const int g[3])
{
    for (int ax = 0; ax < A->base.dim; ++ax) {
        const int N = amr_N(A, a, ax);
        if (a == 0) {
            if (g[ax] < 0 || g[ax] > N - 1) return 0;
        } else {
            const int lo = A->lo[a][ax], hi = A->hi[a][ax];
            const int inside = (g[ax] > lo && g[ax] < hi) || (g[ax] == lo && lo == 0) || (g[ax] == hi && hi == N - 1);
            if (!inside) return 0;
        }
    }
    return 1;
}

/* The child of patch a whose solve region contains the node coincident with g,
 * or -1.  That node is either owned by the child or itself covered, so by
 * induction the finest patch whose region contains the point owns it. */
static int amr_cover_child(const orc_amr *A, int a, const int g[3])
{
    const int g2[3] = {2 * g[0], 2 * g[1], A->base.dim == 3 ? 2 * g[2] : 0};
    for (int c = a + 1; c < A->nlev; ++c)
        if (A->parent[c] == a && amr_box_owned(A, c, g2)) return c;
    return -1;
}

/* Covered: the node coincides with a node of a child's solve region. */
static int amr_covered(const orc_amr *A, int a, const int g[3]) { return amr_cover_child(A, a, g) >= 0; }

int orc_amr_owned(const orc_amr *A, int a, int i, int j, int k)
{
    const int g[3] = {i, j, k};
    return amr_box_owned(A, a, g) && !amr_covered(A, a, g);
}

static int amr_dirichlet(const orc_amr *A, int a, int g[3], int p)
{
    const unsigned m = A->base.dirichlet[p];
    for (int ax = 0; ax < A->base.dim; ++ax) {
        if ((m & (1u << (2 * ax))) && g[ax] == 0) return 1;
        if ((m & (1u << (2 * ax + 1))) && g[ax] == amr_N(A, a, ax) - 1) return 1;
    }
    return 0;
}

/* loop over the storage nodes of level a, giving global coordinates and local index */
#define AMR_FOR_NODES(A, a, P, g, loc)                                                  \
    for (int l2_ = 0; l2_ < (P).n[2]; ++l2_)                                            \
        for (int l1_ = 0; l1_ < (P).n[1]; ++l1_)                                        \
            for (int l0_ = 0; l0_ < (P).n[0]; ++l0_)                                    \
                for (int once_ = 1; once_; once_ = 0)                                   \
                    for (long loc = l0_ + (long)(P).n[0] * (l1_ + (long)(P).n[1] * l2_); once_; once_ = 0) \
                        for (int g[3] = {(a) ? l0_ + (A)->lo[a][0] - 1 : l0_,           \
                                         (a) ? l1_ + (A)->lo[a][1] - 1 : l1_,           \
                                         ((a) && (A)->base.dim == 3) ? l2_ + (A)->lo[a][2] - 1 : l2_}; \
                             once_; once_ = 0)

void orc_amr_coarsen_psi(const orc_amr *A, double *const *psi)
{
    const int d = A->base.dim, nc = 1 << d;
    for (int a = A->nlev - 1; a >= 1; --a) {
        const int pa = A->parent[a];
        orc_problem Pf, Pc;
        orc_amr_level_problem(A, a, &Pf);
        orc_amr_level_problem(A, pa, &Pc);
        /* parent cell C covers fine cells 2C .. 2C+1; it is inside box a when
         * 2C >= lo and 2C + 2 <= hi on every axis */
        const int ncx = Pc.n[0] - 1, ncy = Pc.n[1] - 1, ncz = (d == 3) ? Pc.n[2] - 1 : 1;
        for (int lk = 0; lk < ncz; ++lk)
            for (int lj = 0; lj < ncy; ++lj)
                for (int li = 0; li < ncx; ++li) {
                    int C[3] = {li, lj, lk};
                    if (pa > 0)
                        for (int ax = 0; ax < d; ++ax) C[ax] += A->lo[pa][ax] - 1;
                    int in = 1;
                    for (int ax = 0; ax < d; ++ax)
                        if (2 * C[ax] < A->lo[a][ax] || 2 * C[ax] + 2 > A->hi[a][ax]) in = 0;
                    if (!in) continue;
                    double s = 0.0;
                    for (int c = 0; c < nc; ++c) {
                        int fl[3] = {0, 0, 0};
                        for (int ax = 0; ax < d; ++ax) fl[ax] = 2 * C[ax] + ((c >> ax) & 1) - A->lo[a][ax] + 1;
                        s += psi[a][fl[0] + (long)(Pf.n[0] - 1) * (fl[1] + (long)(Pf.n[1] - 1) * fl[2])];
                    }
                    psi[pa][li + (long)ncx * (lj + (long)ncy * lk)] = s / nc;
                }
    }
}

void orc_amr_fill(const orc_amr *A, double *const *u)
{
    const int d = A->base.dim;
    /* injection, finest first (children have larger indices than their parents) */
    for (int a = A->nlev - 1; a >= 1; --a) {
        const int pa = A->parent[a];
        orc_problem Pf, Pc;
        orc_amr_level_problem(A, a, &Pf);
        orc_amr_level_problem(A, pa, &Pc);
        const long Nf = orc_nnodes(&Pf), Nc = orc_nnodes(&Pc);
        AMR_FOR_NODES(A, a, Pf, g, loc) {
            int even = 1;
            for (int ax = 0; ax < d; ++ax) even &= (g[ax] % 2 == 0);
            if (!even || !amr_box_owned(A, a, g)) continue;
            int gc[3] = {g[0] / 2, g[1] / 2, d == 3 ? g[2] / 2 : 0};
            const long lc = amr_local(A, pa, gc);
            for (int p = 0; p < d; ++p) u[pa][p * Nc + lc] = u[a][p * Nf + loc];
        }
    }
    /* ghosts, coarsest first: (bi/tri)linear interpolation of the parent */
    for (int a = 1; a < A->nlev; ++a) {
        const int pa = A->parent[a];
        orc_problem Pf, Pc;
        orc_amr_level_problem(A, a, &Pf);
        orc_amr_level_problem(A, pa, &Pc);
        const long Nf = orc_nnodes(&Pf), Nc = orc_nnodes(&Pc);
        AMR_FOR_NODES(A, a, Pf, g, loc) {
            if (amr_box_owned(A, a, g)) continue;      /* owned, or covered (injected) */
            int outside = 0;
            for (int ax = 0; ax < d; ++ax)
                if (g[ax] < 0 || g[ax] > amr_N(A, a, ax) - 1) outside = 1;
            for (int p = 0; p < d; ++p) {
                double s = 0.0;
                if (!outside) {
                    /* average over the 2^(odd axes) coarse nodes around g/2 */
                    int nodd = 0;
                    for (int ax = 0; ax < d; ++ax) nodd += g[ax] & 1;
                    for (int c = 0; c < (1 << d); ++c) {
                        int gc[3] = {0, 0, 0}, skip = 0;
                        for (int ax = 0; ax < d; ++ax) {
                            const int bit = (c >> ax) & 1;
                            if (!(g[ax] & 1) && bit) skip = 1;
                            gc[ax] = (g[ax] >> 1) + ((g[ax] & 1) ? bit : 0);
                        }
                        if (skip) continue;
                        s += u[pa][p * Nc + amr_local(A, pa, gc)];
                    }
                    s /= (double)(1 << nodd);
                }
                u[a][p * Nf + loc] = s;
            }
        }
    }
}

void orc_amr_residual(const orc_amr *A, double *const *psi, double *const *f, double *const *u,
                      double *const *r)
{
    const int d = A->base.dim;
    orc_amr_fill(A, u);
    for (int a = 0; a < A->nlev; ++a) {
        orc_problem P;
        orc_amr_level_problem(A, a, &P);
        const long N = orc_nnodes(&P);
        double *Ku = malloc(sizeof(double) * d * N);
        /* padding cells beyond a domain face are not part of the body */
        const long nc = orc_ncells(&P);
        double *pa = malloc(sizeof(double) * nc);
        const int ncx = P.n[0] - 1, ncy = P.n[1] - 1;
        for (long c = 0; c < nc; ++c) {
            int C[3] = {(int)(c % ncx), (int)((c / ncx) % ncy), (int)(c / ((long)ncx * ncy))};
            int in = 1;
            for (int ax = 0; ax < d; ++ax) {
                const int gc = a ? C[ax] + A->lo[a][ax] - 1 : C[ax];
                if (gc < 0 || gc > amr_N(A, a, ax) - 2) in = 0;
            }
            pa[c] = in ? psi[a][c] : 0.0;
        }
        orc_apply(&P, pa, u[a], Ku);
        free(pa);
        AMR_FOR_NODES(A, a, P, g, loc) {
            const int own = orc_amr_owned(A, a, g[0], g[1], g[2]);
            for (int p = 0; p < d; ++p) {
                const long e = p * N + loc;
                r[a][e] = (own && !amr_dirichlet(A, a, g, p)) ? f[a][e] - Ku[e] : 0.0;
            }
        }
        free(Ku);
    }
}

/* Filled value of component p at level-a node g (global level-a indices): the
 * stored value on the level's own solve region (owned nodes), the value of the
 * next finer level at the coincident node on covered nodes (recursively, so the
 * finest owner's value), the (bi/tri)linear interpolation of the parent's filled
 * values on ghosts, and 0 outside the domain.  This is what orc_amr_fill leaves
 * in the arrays, evaluated at one node. */
static double amr_value(const orc_amr *A, double *const *u, int a, const int g[3], int p)
{
    const int d = A->base.dim;
    for (int ax = 0; ax < d; ++ax)
        if (g[ax] < 0 || g[ax] > amr_N(A, a, ax) - 1) return 0.0;
    if (amr_box_owned(A, a, g)) {
        const int c = amr_cover_child(A, a, g);
        if (c >= 0) {
            const int g2[3] = {2 * g[0], 2 * g[1], d == 3 ? 2 * g[2] : 0};
            return amr_value(A, u, c, g2, p);
        }
        orc_problem P;
        orc_amr_level_problem(A, a, &P);
        return u[a][p * orc_nnodes(&P) + amr_local(A, a, (int *)g)];
    }
    int nodd = 0;
    for (int ax = 0; ax < d; ++ax) nodd += g[ax] & 1;
    double s = 0.0;
    for (int c = 0; c < (1 << d); ++c) {
        int gc[3] = {0, 0, 0}, skip = 0;
        for (int ax = 0; ax < d; ++ax) {
            const int bit = (c >> ax) & 1;
            if (!(g[ax] & 1) && bit) skip = 1;
            gc[ax] = (g[ax] >> 1) + ((g[ax] & 1) ? bit : 0);
        }
        if (skip) continue;
        s += amr_value(A, u, A->parent[a], gc, p);
    }
    return s / (double)(1 << nodd);
}

void orc_amr_residual_at(const orc_amr *A, double *const *psi, double *const *f, double *const *u, long n,
                         const int *lev, const int *node, const int *comp, double *r)
{
    const int d = A->base.dim, nc = 1 << d, nd = nc * d;
    double Ke[24 * 24];
    for (long s = 0; s < n; ++s) {
        const int a = lev[s], p = comp[s];
        const int g[3] = {node[3 * s], node[3 * s + 1], d == 3 ? node[3 * s + 2] : 0};
        if (!orc_amr_owned(A, a, g[0], g[1], g[2]) || amr_dirichlet(A, a, (int *)g, p)) {
            r[s] = 0.0;
            continue;
        }
        orc_problem P;
        orc_amr_level_problem(A, a, &P);
        orc_element_matrix(&P, Ke);
        const int ncx = P.n[0] - 1, ncy = P.n[1] - 1;
        double Ku = 0.0;
        for (int b = 0; b < nc; ++b) {        /* g is corner b of cell g - offset(b) */
            int C[3] = {g[0] - (b & 1), g[1] - ((b >> 1) & 1), d == 3 ? g[2] - ((b >> 2) & 1) : 0};
            int inside = 1, lc[3] = {0, 0, 0};
            for (int ax = 0; ax < d; ++ax) {
                if (C[ax] < 0 || C[ax] > amr_N(A, a, ax) - 2) inside = 0;
                lc[ax] = a ? C[ax] - A->lo[a][ax] + 1 : C[ax];
            }
            if (!inside) continue;
            const double pc = psi[a][lc[0] + (long)ncx * (lc[1] + (long)ncy * lc[2])];
            for (int e = 0; e < nc; ++e) {
                const int ge[3] = {C[0] + (e & 1), C[1] + ((e >> 1) & 1), d == 3 ? C[2] + ((e >> 2) & 1) : 0};
                for (int q = 0; q < d; ++q)
                    Ku += pc * Ke[(b * d + p) * nd + e * d + q] * amr_value(A, u, a, ge, q);
            }
        }
        r[s] = f[a][p * orc_nnodes(&P) + amr_local(A, a, (int *)g)] - Ku;
    }
}

void orc_amr_dJdpsi(const orc_amr *A, double *const *u, double *const *lam, double *const *g)
{
    const int d = A->base.dim, nc = 1 << d, nd = nc * d;
    double Ke[24 * 24], ue[24], le[24];
    for (int a = 0; a < A->nlev; ++a) {
        orc_problem P;
        orc_amr_level_problem(A, a, &P);
        orc_element_matrix(&P, Ke);
        const long N = orc_nnodes(&P);
        const int ncx = P.n[0] - 1, ncy = P.n[1] - 1, ncz = d == 3 ? P.n[2] - 1 : 1;
        for (int ck = 0; ck < ncz; ++ck)
            for (int cj = 0; cj < ncy; ++cj)
                for (int ci = 0; ci < ncx; ++ci) {
                    const long cidx = ci + (long)ncx * (cj + (long)ncy * ck);
                    const int C[3] = {a ? ci + A->lo[a][0] - 1 : ci, a ? cj + A->lo[a][1] - 1 : cj,
                                      (a && d == 3) ? ck + A->lo[a][2] - 1 : ck};
                    int inside = 1;
                    for (int ax = 0; ax < d; ++ax)
                        if (C[ax] < 0 || C[ax] > amr_N(A, a, ax) - 2) inside = 0;
                    if (!inside) {
                        g[a][cidx] = 0.0;
                        continue;
                    }
                    for (int b = 0; b < nc; ++b) {
                        const long n = (ci + (b & 1)) + (long)P.n[0] * ((cj + ((b >> 1) & 1)) +
                                       (long)P.n[1] * (d == 3 ? ck + ((b >> 2) & 1) : 0));
                        for (int q = 0; q < d; ++q) {
                            ue[b * d + q] = u[a][q * N + n];
                            le[b * d + q] = lam[a][q * N + n];
                        }
                    }
                    double s = 0.0;
                    for (int r = 0; r < nd; ++r)
                        for (int c = 0; c < nd; ++c) s += le[r] * Ke[r * nd + c] * ue[c];
                    g[a][cidx] = -s;
                }
    }
    /* coarse cells under a patch hold the mean of their fine cells: their gradient
     * passes to those cells (coarse to fine: a parent before its children) and they
     * keep none of their own */
    for (int b = 1; b < A->nlev; ++b) {
        const int a = A->parent[b];
        orc_problem Pc, Pf;
        orc_amr_level_problem(A, a, &Pc);
        orc_amr_level_problem(A, b, &Pf);
        const int ncx = Pc.n[0] - 1, ncy = Pc.n[1] - 1, ncz = d == 3 ? Pc.n[2] - 1 : 1;
        for (int ck = 0; ck < ncz; ++ck)
            for (int cj = 0; cj < ncy; ++cj)
                for (int ci = 0; ci < ncx; ++ci) {
                    int C[3] = {ci, cj, ck};
                    if (a > 0)
                        for (int ax = 0; ax < d; ++ax) C[ax] += A->lo[a][ax] - 1;
                    int in = 1;
                    for (int ax = 0; ax < d; ++ax)
                        if (2 * C[ax] < A->lo[b][ax] || 2 * C[ax] + 2 > A->hi[b][ax]) in = 0;
                    if (!in) continue;
                    const long cidx = ci + (long)ncx * (cj + (long)ncy * ck);
                    const double share = g[a][cidx] / nc;
                    for (int c = 0; c < nc; ++c) {
                        int fl[3] = {0, 0, 0};
                        for (int ax = 0; ax < d; ++ax) fl[ax] = 2 * C[ax] + ((c >> ax) & 1) - A->lo[b][ax] + 1;
                        g[b][fl[0] + (long)(Pf.n[0] - 1) * (fl[1] + (long)(Pf.n[1] - 1) * fl[2])] += share;
                    }
                    g[a][cidx] = 0.0;
                }
    }
}


/* ------------------------------------------------- composite correction iteration */

/* Level a's storage psi with the padding cells beyond the domain zeroed (they are
 * not part of the body), as orc_amr_residual uses it. */
static double *amr_body_psi(const orc_amr *A, int a, const double *psi_a)
{
    orc_problem P;
    orc_amr_level_problem(A, a, &P);
    const int d = A->base.dim;
    const long nc = orc_ncells(&P);
    const int ncx = P.n[0] - 1, ncy = P.n[1] - 1;
    double *pa = malloc(sizeof(double) * nc);
    for (long c = 0; c < nc; ++c) {
        const int C[3] = {(int)(c % ncx), (int)((c / ncx) % ncy), (int)(c / ((long)ncx * ncy))};
        int in = 1;
        for (int ax = 0; ax < d; ++ax) {
            const int gc = a ? C[ax] + A->lo[a][ax] - 1 : C[ax];
            if (gc < 0 || gc > amr_N(A, a, ax) - 2) in = 0;
        }
        pa[c] = in ? psi_a[c] : 0.0;
    }
    return pa;
}

/* Damped Jacobi sweeps on K_a e = rhs over the free dofs of level a's solve region
 * (owned and covered nodes); every other value of e is held fixed. */
static void amr_masked_jacobi(const orc_amr *A, int a, const double *pa, const double *rhs, double *e,
                              double omega, int nsweeps)
{
    orc_problem P;
    orc_amr_level_problem(A, a, &P);
    const int d = A->base.dim;
    const long N = orc_nnodes(&P);
    double *Ke = malloc(sizeof(double) * d * N), *D = malloc(sizeof(double) * d * N);
    orc_diagonal(&P, pa, D);
    for (int s = 0; s < nsweeps; ++s) {
        orc_apply(&P, pa, e, Ke);
        AMR_FOR_NODES(A, a, P, g, loc) {
            if (!amr_box_owned(A, a, g)) continue;
            for (int p = 0; p < d; ++p) {
                if (amr_dirichlet(A, a, g, p)) continue;
                const long q = p * N + loc;
                e[q] += omega * (rhs[q] - Ke[q]) / D[q];
            }
        }
    }
    free(Ke);
    free(D);
}

/* res = rhs - K_a e on the free dofs of level a's solve region, 0 elsewhere. */
static void amr_region_residual(const orc_amr *A, int a, const double *pa, const double *rhs, const double *e,
                                double *res)
{
    orc_problem P;
    orc_amr_level_problem(A, a, &P);
    const int d = A->base.dim;
    const long N = orc_nnodes(&P);
    orc_apply(&P, pa, e, res);
    AMR_FOR_NODES(A, a, P, g, loc) {
        const int in = amr_box_owned(A, a, g);
        for (int p = 0; p < d; ++p) {
            const long q = p * N + loc;
            res[q] = (in && !amr_dirichlet(A, a, g, p)) ? rhs[q] - res[q] : 0.0;
        }
    }
}

/* rhs_c at the parent nodes covered by patch a += R res_a, R = P^T / 2^d (full
 * weighting about the coincident fine node); Dirichlet dofs are left alone. */
static void amr_restrict_covered(const orc_amr *A, int a, const double *res, double *rhs_c)
{
    const int pa = A->parent[a];
    orc_problem Pf, Pc;
    orc_amr_level_problem(A, a, &Pf);
    orc_amr_level_problem(A, pa, &Pc);
    const int d = A->base.dim;
    const long Nf = orc_nnodes(&Pf), Nc = orc_nnodes(&Pc);
    AMR_FOR_NODES(A, pa, Pc, gc, locc) {
        if (amr_cover_child(A, pa, gc) != a) continue;
        for (int p = 0; p < d; ++p) {
            if (amr_dirichlet(A, pa, gc, p)) continue;
            double s = 0.0;
            for (int dk = (d == 3 ? -1 : 0); dk <= (d == 3 ? 1 : 0); ++dk)
                for (int dj = -1; dj <= 1; ++dj)
                    for (int di = -1; di <= 1; ++di) {
                        int gf[3] = {2 * gc[0] + di, 2 * gc[1] + dj, d == 3 ? 2 * gc[2] + dk : 0};
                        const long lf = amr_local(A, a, gf);
                        if (lf < 0) continue;
                        s += pw(di) * pw(dj) * (d == 3 ? pw(dk) : 1.0) * res[p * Nf + lf];
                    }
            rhs_c[p * Nc + locc] += s / (double)(1 << d);
        }
    }
}

/* e_a += P e_{a-1} at every storage node of level a inside the domain
 * ((bi/tri)linear interpolation, coincident nodes copy). */
static void amr_interpolate_add(const orc_amr *A, int a, const double *ec, double *ef)
{
    const int pa = A->parent[a];
    orc_problem Pf, Pc;
    orc_amr_level_problem(A, a, &Pf);
    orc_amr_level_problem(A, pa, &Pc);
    const int d = A->base.dim;
    const long Nf = orc_nnodes(&Pf), Nc = orc_nnodes(&Pc);
    AMR_FOR_NODES(A, a, Pf, g, loc) {
        int outside = 0, nodd = 0;
        for (int ax = 0; ax < d; ++ax) {
            if (g[ax] < 0 || g[ax] > amr_N(A, a, ax) - 1) outside = 1;
            nodd += g[ax] & 1;
        }
        if (outside) continue;
        for (int p = 0; p < d; ++p) {
            double s = 0.0;
            for (int c = 0; c < (1 << d); ++c) {
                int gcn[3] = {0, 0, 0}, skip = 0;
                for (int ax = 0; ax < d; ++ax) {
                    const int bit = (c >> ax) & 1;
                    if (!(g[ax] & 1) && bit) skip = 1;
                    gcn[ax] = (g[ax] >> 1) + ((g[ax] & 1) ? bit : 0);
                }
                if (skip) continue;
                s += ec[p * Nc + amr_local(A, pa, gcn)];
            }
            ef[p * Nf + loc] += s / (double)(1 << nodd);
        }
    }
}

int orc_amr_solve(const orc_amr *A, double *const *psi, double *const *f, double *const *u,
                  const orc_amr_opts *o, double *hist, int *cycles)
{
    const int L = A->nlev, d = A->base.dim;
    double *r[65], *e[65], *rhs[65], *res[65], *pa[65];
    long N[65];
    for (int a = 0; a < L; ++a) {
        orc_problem P;
        orc_amr_level_problem(A, a, &P);
        N[a] = orc_nnodes(&P);
        r[a] = calloc(d * N[a], sizeof(double));
        e[a] = calloc(d * N[a], sizeof(double));
        rhs[a] = calloc(d * N[a], sizeof(double));
        res[a] = calloc(d * N[a], sizeof(double));
        pa[a] = amr_body_psi(A, a, psi[a]);
    }
    orc_mg_opts base = {o->nu1, o->nu2, o->omega_base, o->smoother_base, 0.0, 1};
    double r0 = 0.0, rel = 1.0;
    int status = 1, ncyc = 0;
    for (;;) {
        orc_amr_residual(A, psi, f, u, r);
        double s = 0.0;
        for (int a = 0; a < L; ++a)
            for (long q = 0; q < d * N[a]; ++q) s += r[a][q] * r[a][q];
        s = sqrt(s);
        if (ncyc == 0) {
            r0 = s;
            if (hist) hist[0] = 1.0;
            if (r0 == 0.0) {
                status = 0;
                break;
            }
        } else {
            rel = s / r0;
            if (hist) hist[ncyc] = rel;
            if (!isfinite(rel) || rel > 1e10) {
                status = 2;
                break;
            }
        }
        if (rel <= o->tol) {
            status = 0;
            break;
        }
        if (ncyc >= o->max_cycles) break;
        /* patches, finest first: smooth the correction, residual of its equation,
         * full weighting onto the covered parent nodes */
        for (int a = L - 1; a >= 0; --a) {
            memcpy(rhs[a], r[a], sizeof(double) * d * N[a]);
            for (int c = a + 1; c < L; ++c)
                if (A->parent[c] == a) amr_restrict_covered(A, c, res[c], rhs[a]);
            memset(e[a], 0, sizeof(double) * d * N[a]);
            if (a == 0) break;
            amr_masked_jacobi(A, a, pa[a], rhs[a], e[a], o->omega, o->nu1);
            amr_region_residual(A, a, pa[a], rhs[a], e[a], res[a]);
        }
        /* the base level: one multigrid V-cycle on its correction equation */
        {
            int c1 = 0;
            const int st = orc_mg_solve(&A->base, pa[0], rhs[0], e[0], &base, NULL, &c1);
            if (st == 3) {
                status = 3;
                break;
            }
        }
        /* patches, coarsest first: the parent's correction interpolated onto every
         * node of the patch, then smoothing */
        for (int a = 1; a < L; ++a) {
            amr_interpolate_add(A, a, e[A->parent[a]], e[a]);
            amr_masked_jacobi(A, a, pa[a], rhs[a], e[a], o->omega, o->nu2);
        }
        /* u += e on the owned free dofs; ghosts and covered nodes follow at the next fill */
        for (int a = 0; a < L; ++a) {
            orc_problem P;
            orc_amr_level_problem(A, a, &P);
            AMR_FOR_NODES(A, a, P, g, loc) {
                if (!orc_amr_owned(A, a, g[0], g[1], g[2])) continue;
                for (int p = 0; p < d; ++p)
                    if (!amr_dirichlet(A, a, g, p)) u[a][p * N[a] + loc] += e[a][p * N[a] + loc];
            }
        }
        ++ncyc;
    }
    orc_amr_fill(A, u);
    for (int a = 0; a < L; ++a) {
        free(r[a]);
        free(e[a]);
        free(rhs[a]);
        free(res[a]);
        free(pa[a]);
    }
    if (cycles) *cycles = ncyc;
    return status;
}

/* ---------------------------------------- product-rule strong form (Sec. 2.3) */

/* Nodal value of psi and its gradient g at interior node (i,j,k).
 * variant ORC_NODE_PSI: psi is nodal, g_a = (psi(n + e_a) - psi(n - e_a)) / (2h);
 * variant ORC_CELL_PSI: psi is in cells, psi_n = mean of the 2^d cells around n and
 *   g_a = mean over the 2^(d-1) cell pairs facing each other across n along a of
 *   (psi_+ - psi_-) / h  (in 1D: the cell-placed update of Sec. 2.3). */
static void product_psi(const orc_problem *P, int variant, const double *psi, int i, int j, int k, double *pn,
                        double g[3])
{
    const int d = P->dim, nc = 1 << d;
    const int n3[3] = {i, j, k};
    g[0] = g[1] = g[2] = 0.0;
    if (variant == ORC_NODE_PSI) {
        *pn = psi[nid(P, i, j, k)];
        for (int a = 0; a < d; ++a) {
            int up[3] = {i, j, k}, dn[3] = {i, j, k};
            up[a] += 1;
            dn[a] -= 1;
            g[a] = (psi[nid(P, up[0], up[1], up[2])] - psi[nid(P, dn[0], dn[1], dn[2])]) / (2.0 * P->h);
        }
        return;
    }
    double s = 0.0;
    for (int c = 0; c < nc; ++c) {           /* cell with lower corner n - 1 + bits of c */
        int cc[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) cc[a] = n3[a] - 1 + ((c >> a) & 1);
        const double v = psi[cid(P, cc[0], cc[1], cc[2])];
        s += v;
        for (int a = 0; a < d; ++a) g[a] += (((c >> a) & 1) ? v : -v);
    }
    *pn = s / nc;
    for (int a = 0; a < d; ++a) g[a] /= (double)(nc / 2) * P->h;
}

void orc_apply_product(const orc_problem *P, int variant, const double *psi, const double *u, double *Ku)
{
    const int d = P->dim;
    const long N = orc_nnodes(P);
    const double h = P->h;
    memset(Ku, 0, sizeof(double) * d * N);
    for (int k = (d == 3 ? 1 : 0); k < (d == 3 ? P->n[2] - 1 : 1); ++k)
        for (int j = 1; j < P->n[1] - 1; ++j)
            for (int i = 1; i < P->n[0] - 1; ++i) {
                const int n3[3] = {i, j, k};
                double pn, g[3];
                product_psi(P, variant, psi, i, j, k, &pn, g);
                /* centred first differences D[l][q] = d_l u_q and second differences
                 * H[a][b][q] = d_a d_b u_q of u at the node */
                double D[3][3] = {{0}}, H[3][3][3] = {{{0}}};
                for (int q = 0; q < d; ++q) {
                    const double *uq = u + q * N;
                    const double c = uq[nid(P, i, j, k)];
                    for (int a = 0; a < d; ++a) {
                        int up[3] = {i, j, k}, dn[3] = {i, j, k};
                        up[a] += 1;
                        dn[a] -= 1;
                        const double vu = uq[nid(P, up[0], up[1], up[2])], vd = uq[nid(P, dn[0], dn[1], dn[2])];
                        D[a][q] = (vu - vd) / (2.0 * h);
                        H[a][a][q] = (vu - 2.0 * c + vd) / (h * h);
                        for (int b = a + 1; b < d; ++b) {
                            int pp[3] = {n3[0], n3[1], n3[2]}, pm[3] = {n3[0], n3[1], n3[2]};
                            int mp[3] = {n3[0], n3[1], n3[2]}, mm[3] = {n3[0], n3[1], n3[2]};
                            pp[a] += 1; pp[b] += 1;
                            pm[a] += 1; pm[b] -= 1;
                            mp[a] -= 1; mp[b] += 1;
                            mm[a] -= 1; mm[b] -= 1;
                            const double x = (uq[nid(P, pp[0], pp[1], pp[2])] - uq[nid(P, pm[0], pm[1], pm[2])] -
                                              uq[nid(P, mp[0], mp[1], mp[2])] + uq[nid(P, mm[0], mm[1], mm[2])]) /
                                             (4.0 * h * h);
                            H[a][b][q] = x;
                            H[b][a][q] = x;
                        }
                    }
                }
                /* (A u)_p = sum_{a,q,b} C_{p a q b} (psi_n d_a d_b u_q + g_a d_b u_q);  K = -A */
                for (int p = 0; p < d; ++p) {
                    double s = 0.0;
                    for (int a = 0; a < d; ++a)
                        for (int q = 0; q < d; ++q)
                            for (int b = 0; b < d; ++b) {
                                const double C = cubic_C(P, p, a, q, b);
                                if (C == 0.0) continue;
                                s += C * (pn * H[a][b][q] + g[a] * D[b][q]);
                            }
                    Ku[p * N + nid(P, i, j, k)] = -s;
                }
            }
}

void orc_diagonal_product(const orc_problem *P, int variant, const double *psi, double *D)
{
    const int d = P->dim;
    const long N = orc_nnodes(P);
    memset(D, 0, sizeof(double) * d * N);
    for (int k = (d == 3 ? 1 : 0); k < (d == 3 ? P->n[2] - 1 : 1); ++k)
        for (int j = 1; j < P->n[1] - 1; ++j)
            for (int i = 1; i < P->n[0] - 1; ++i) {
                double pn, g[3];
                product_psi(P, variant, psi, i, j, k, &pn, g);
                /* only the second differences d_a d_a u_p touch u_p at the node itself
                 * (coefficient -2/h^2); K = -A */
                for (int p = 0; p < d; ++p) {
                    double s = 0.0;
                    for (int a = 0; a < d; ++a) s += cubic_C(P, p, a, p, a) * 2.0 / (P->h * P->h);
                    D[p * N + nid(P, i, j, k)] = pn * s;
                }
            }
}

void orc_jacobi_product(const orc_problem *P, int variant, const double *psi, const double *f, double *u,
                        double omega)
{
    const int d = P->dim;
    const long N = orc_nnodes(P);
    double *Ku = malloc(sizeof(double) * d * N), *D = malloc(sizeof(double) * d * N);
    orc_apply_product(P, variant, psi, u, Ku);
    orc_diagonal_product(P, variant, psi, D);
    for (int p = 0; p < d; ++p)
        for (int k = (d == 3 ? 1 : 0); k < (d == 3 ? P->n[2] - 1 : 1); ++k)
            for (int j = 1; j < P->n[1] - 1; ++j)
                for (int i = 1; i < P->n[0] - 1; ++i) {
                    if (orc_is_dirichlet(P, i, j, k, p)) continue;
                    const long e = p * N + nid(P, i, j, k);
                    u[e] += omega * (f[e] - Ku[e]) / D[e];
                }
    free(Ku);
    free(D);
}

/* ------------------------------------- source terms of eq. SBMLinearElasticity */

/* Voigt index of the symmetric pair (i, j): 2D (xx, yy, xy), 3D (xx, yy, zz, yz, xz, xy). */
static int voigt(int d, int i, int j)
{
    if (i == j) return i;
    if (d == 2) return 2;
    const int s = i + j;                      /* (1,2) -> 3, (0,2) -> 4, (0,1) -> 5 */
    return s == 3 ? 3 : (s == 2 ? 4 : 5);
}

/* psi, grad psi and the lumping weight at node (i,j,k) from the cells around it:
 * cells beyond a face of the box take the value of their mirror image inside (no
 * gradient of psi normal to the box), psi_n is the mean of the 2^d cells, the
 * gradient along a is the mean over the 2^(d-1) cell pairs facing each other
 * across the node of (psi_+ - psi_-) / h, and w_n = (cells of the grid around n) / 2^d. */
static void node_psi(const orc_problem *P, const double *psi, int i, int j, int k, double *pn, double g[3], double *w)
{
    const int d = P->dim, nc = 1 << d;
    const int n3[3] = {i, j, k};
    double s = 0.0;
    int inside = 0;
    g[0] = g[1] = g[2] = 0.0;
    for (int c = 0; c < nc; ++c) {
        int cc[3] = {0, 0, 0}, in = 1;
        for (int a = 0; a < d; ++a) {
            int v = n3[a] - 1 + ((c >> a) & 1);
            const int m = ncell_axis(P, a);
            if (v < 0) { v = 0; in = 0; }
            if (v > m - 1) { v = m - 1; in = 0; }
            cc[a] = v;
        }
        inside += in;
        const double v = psi[cid(P, cc[0], cc[1], cc[2])];
        s += v;
        for (int a = 0; a < d; ++a) g[a] += ((c >> a) & 1) ? v : -v;
    }
    *pn = s / nc;
    for (int a = 0; a < d; ++a) g[a] /= (double)(nc / 2) * P->h;
    *w = (double)inside / nc;
}

void orc_source_terms(const orc_problem *P, const double *psi, const double *eps0, const double *b, const double *t,
                      double *f)
{
    const int d = P->dim, nc = 1 << d, nv = d == 3 ? 6 : 3;
    const long N = orc_nnodes(P), NC = orc_ncells(P);
    const double h = P->h;
    memset(f, 0, sizeof(double) * d * N);
    if (eps0) {
        /* K u = f_eps is the weak form of div(psi C (grad u - eps0)) = 0:
         * f_eps(n) = h^-d sum_c psi_c int_c B_n^T C eps0_c, by 2-point Gauss quadrature */
        const double gp[2] = {0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)};
        const double wq = pow(h, d) / nc;
        for (int ck = 0; ck < ncell_axis(P, 2); ++ck)
            for (int cj = 0; cj < ncell_axis(P, 1); ++cj)
                for (int ci = 0; ci < ncell_axis(P, 0); ++ci) {
                    const long c = cid(P, ci, cj, ck);
                    double sig[3][3];
                    for (int p = 0; p < d; ++p)
                        for (int q = 0; q < d; ++q) {
                            double s = 0.0;
                            for (int r = 0; r < d; ++r)
                                for (int l = 0; l < d; ++l) s += cubic_C(P, p, q, r, l) * eps0[voigt(d, r, l) * NC + c];
                            sig[p][q] = psi[c] * s;
                        }
                    for (int gq = 0; gq < nc; ++gq) {
                        double xi[3];
                        for (int a = 0; a < d; ++a) xi[a] = gp[(gq >> a) & 1];
                        for (int a = 0; a < nc; ++a) {
                            double dN[3];
                            for (int ax = 0; ax < d; ++ax) {
                                double v = dshape1((a >> ax) & 1) / h;
                                for (int bx = 0; bx < d; ++bx)
                                    if (bx != ax) v *= shape1((a >> bx) & 1, xi[bx]);
                                dN[ax] = v;
                            }
                            int i, j, k;
                            cell_corner(P, ci, cj, ck, a, &i, &j, &k);
                            for (int p = 0; p < d; ++p) {
                                double s = 0.0;
                                for (int q = 0; q < d; ++q) s += sig[p][q] * dN[q];
                                f[p * N + nid(P, i, j, k)] += wq * s * pow(h, -d);
                            }
                        }
                    }
                }
    }
    (void)nv;
    /* body force and diffuse traction:  -w_n (psi_n b_n + t_n |grad psi|_n) */
    for (int k = 0; k < P->n[2]; ++k)
        for (int j = 0; j < P->n[1]; ++j)
            for (int i = 0; i < P->n[0]; ++i) {
                double pn, g[3], w;
                node_psi(P, psi, i, j, k, &pn, g, &w);
                const double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
                const long n = nid(P, i, j, k);
                for (int p = 0; p < d; ++p) {
                    double s = 0.0;
                    if (b) s += pn * b[p * N + n];
                    if (t) s += t[p * N + n] * gn;
                    f[p * N + n] -= w * s;
                }
            }
}

void orc_node_psi(const orc_problem *P, const double *psi, double *pn, double *gn, double *w)
{
    for (int k = 0; k < P->n[2]; ++k)
        for (int j = 0; j < P->n[1]; ++j)
            for (int i = 0; i < P->n[0]; ++i) {
                double g[3];
                const long n = nid(P, i, j, k);
                node_psi(P, psi, i, j, k, &pn[n], g, &w[n]);
                gn[n] = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
            }
}

/* ------------------------------------- phase-field topology optimisation (Sec. 3.3) */

/* eta of the cell (ci,cj,ck) with the cell's own value beyond a face of the box
 * (the order parameter's Neumann condition). */
static double eta_at(const orc_problem *P, const double *eta, int ci, int cj, int ck, int axis, int side,
                     double self)
{
    int c[3] = {ci, cj, ck};
    c[axis] += side;
    if (c[axis] < 0 || c[axis] >= ncell_axis(P, axis)) return self;
    return eta[cid(P, c[0], c[1], c[2])];
}

void orc_topopt_step(const orc_problem *P, const orc_topopt_params *T, int step, const double *eta, const double *u,
                     double *eta_out)
{
    const int d = P->dim;
    const long NC = orc_ncells(P);
    const double hd = pow(P->h, d);
    /* the volume int eta dx of eq. topop_volume_constraint, cell-centred rule */
    double V = 0.0;
    for (long c = 0; c < NC; ++c) V += hd * eta[c];
    /* lambda(t): grows linearly from lambda at t = 0 at the rate lambda_rate */
    const double lam = T->lambda + T->lambda_rate * step * T->dt;
    /* unit-psi cell strain energy e_c = u_c^T S_c u_c = -dJ/dpsi_c of the compliance (lambda = u) */
    double *e = malloc(sizeof(double) * NC);
    orc_dJdpsi(P, u, u, e);
    for (long c = 0; c < NC; ++c) e[c] = -e[c];
    for (int ck = 0; ck < ncell_axis(P, 2); ++ck)
        for (int cj = 0; cj < ncell_axis(P, 1); ++cj)
            for (int ci = 0; ci < ncell_axis(P, 0); ++ci) {
                const long c = cid(P, ci, cj, ck);
                const double n = eta[c];
                /* variational derivative of eq. topop_objective:
                 *   d/deta [alpha eta^2 (1-eta)^2]      = 2 alpha eta (1-eta)(1-2 eta)
                 *   d/deta [beta/2 |grad eta|^2]        = -beta Laplacian(eta)
                 *   d/deta [compliance / 2], psi = (eta+zeta)^2 = -(eta+zeta) e_c      */
                double lap = 0.0;
                for (int a = 0; a < d; ++a)
                    lap += (eta_at(P, eta, ci, cj, ck, a, +1, n) - 2.0 * n + eta_at(P, eta, ci, cj, ck, a, -1, n)) /
                           (P->h * P->h);
                const double dW = 2.0 * T->alpha * n * (1.0 - n) * (1.0 - 2.0 * n) - T->beta * lap -
                                  (n + T->zeta) * e[c];
                /* eq. topop_evolution, one explicit Euler step */
                eta_out[c] = n - T->dt * T->mobility * (dW + lam * (V - T->V0));
            }
    free(e);
}

void orc_topopt_energy(const orc_problem *P, const orc_topopt_params *T, int step, const double *eta, double out[3])
{
    const int d = P->dim;
    const double hd = pow(P->h, d);
    double well = 0.0, grad = 0.0, V = 0.0;
    for (int ck = 0; ck < ncell_axis(P, 2); ++ck)
        for (int cj = 0; cj < ncell_axis(P, 1); ++cj)
            for (int ci = 0; ci < ncell_axis(P, 0); ++ci) {
                const double n = eta[cid(P, ci, cj, ck)];
                well += hd * T->alpha * n * n * (1.0 - n) * (1.0 - n);
                V += hd * n;
                /* |grad eta|^2 from the differences across the interior faces (each once) */
                for (int a = 0; a < d; ++a) {
                    const int cc[3] = {ci, cj, ck};
                    if (cc[a] + 1 >= ncell_axis(P, a)) continue;
                    const double m = eta_at(P, eta, ci, cj, ck, a, +1, n);
                    grad += hd * 0.5 * T->beta * (m - n) * (m - n) / (P->h * P->h);
                }
            }
    const double lam = T->lambda + T->lambda_rate * step * T->dt;
    out[0] = well;
    out[1] = grad;
    out[2] = 0.5 * lam * (V - T->V0) * (V - T->V0);
}
