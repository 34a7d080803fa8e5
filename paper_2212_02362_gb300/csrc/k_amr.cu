// k_amr.cu — kernels of the block-structured refinement (Sec. 2.2): ownership
// masks of the composite problem, injection of fine values into covered coarse
// nodes, ghost fill of a patch's interface and padding nodes from its parent
// level (coarse-to-fine interpolation), full-weighting restriction of a patch's
// residual onto the covered parent nodes, prolongation of a parent correction
// into a patch, the owned-dof update and the composite norm.
//
// A patch refines its parent (the base level or a patch one level coarser) by 2 on
// one node box [lo, hi] (indices of its level); a level may hold several patches,
// disjoint and apart.  A patch's storage is the box grown by one padding node per
// side; `AmrInfo` carries the global extents, the box, the storage origin, the
// boxes of the patch's children and the domain Dirichlet faces, from which every
// node's role follows:
//   owned   - inside the box on every axis, or on a box face lying on the domain
//             boundary, and not covered by a child;
//   covered - coincident with a node of a child's box region: carries the injected
//             fine value and no equation of its own;
//   ghost   - the other storage nodes: interpolated from the parent.
// Kernels that move data between one child and its parent take both infos and
// test membership in that child's own box.
#include "sbm_common.cuh"

namespace sbm {

namespace {

__host__ __device__ __forceinline__ bool axes_owned(const AmrInfo &L, const int g[3])
{
    for (int ax = 0; ax < L.dim; ++ax) {
        if (L.is_base) {
            if (g[ax] < 0 || g[ax] > L.N[ax] - 1) return false;
        } else {
            const bool in = (g[ax] > L.lo[ax] && g[ax] < L.hi[ax]) || (g[ax] == L.lo[ax] && L.lo[ax] == 0) ||
                            (g[ax] == L.hi[ax] && L.hi[ax] == L.N[ax] - 1);
            if (!in) return false;
        }
    }
    return true;
}

// child-level coordinates g2 in the box region of child c (the child's axes rule)
__host__ __device__ __forceinline__ bool child_axes_owned(const AmrInfo &L, int c, const int g2[3])
{
    for (int ax = 0; ax < L.dim; ++ax) {
        const int Nc = 2 * (L.N[ax] - 1) + 1;
        const int lo = L.clo[c][ax], hi = L.chi[c][ax];
        const bool in = (g2[ax] > lo && g2[ax] < hi) || (g2[ax] == lo && lo == 0) || (g2[ax] == hi && hi == Nc - 1);
        if (!in) return false;
    }
    return true;
}

__host__ __device__ __forceinline__ bool covered(const AmrInfo &L, const int g[3])
{
    const int g2[3] = {2 * g[0], 2 * g[1], L.dim == 3 ? 2 * g[2] : 0};
    for (int c = 0; c < L.nchild; ++c)
        if (child_axes_owned(L, c, g2)) return true;
    return false;
}

// parent node G coincides with a node of the box region of the child described by Lc
__host__ __device__ __forceinline__ bool covered_by(const AmrInfo &Lc, const int G[3])
{
    const int g2[3] = {2 * G[0], 2 * G[1], Lc.dim == 3 ? 2 * G[2] : 0};
    return axes_owned(Lc, g2);
}

__host__ __device__ __forceinline__ bool owned(const AmrInfo &L, const int g[3])
{
    return axes_owned(L, g) && !covered(L, g);
}

__host__ __device__ __forceinline__ bool domain_dirichlet(const AmrInfo &L, const int g[3], int p)
{
    const unsigned m = L.dm[p];
    for (int ax = 0; ax < L.dim; ++ax) {
        if ((m >> (2 * ax)) & 1u && g[ax] == 0) return true;
        if ((m >> (2 * ax + 1)) & 1u && g[ax] == L.N[ax] - 1) return true;
    }
    return false;
}

__device__ __forceinline__ bool inside_domain(const AmrInfo &L, const int g[3])
{
    for (int ax = 0; ax < L.dim; ++ax)
        if (g[ax] < 0 || g[ax] > L.N[ax] - 1) return false;
    return true;
}

// Storage node of the current thread: (i,j,k) local, g global.
__device__ __forceinline__ bool thread_node(const Geom &s, const AmrInfo &L, int &i, int &j, int &k, int g[3])
{
    i = blockIdx.x * blockDim.x + threadIdx.x;
    j = blockIdx.y * blockDim.y + threadIdx.y;
    k = blockIdx.z * blockDim.z + threadIdx.z;
    if (i >= s.nx || j >= s.ny || k >= s.nz) return false;
    g[0] = i + L.org[0];
    g[1] = j + L.org[1];
    g[2] = k + L.org[2];
    return true;
}

// Value of a parent-level field at child global coordinates g (linear
// interpolation; coincident nodes copy); 0 outside the parent's storage.
template <typename T>
__device__ __forceinline__ T parent_interp(const Geom &sp, const AmrInfo &Lp, const T *up, int p, const int g[3])
{
    T s = T(0);
    int nodd = 0;
    for (int ax = 0; ax < Lp.dim; ++ax) nodd += g[ax] & 1;
    for (int c = 0; c < (1 << Lp.dim); ++c) {
        int l[3] = {0, 0, 0};
        bool skip = false;
        for (int ax = 0; ax < Lp.dim; ++ax) {
            const int bit = (c >> ax) & 1;
            if (!(g[ax] & 1) && bit) skip = true;
            l[ax] = (g[ax] >> 1) + ((g[ax] & 1) ? bit : 0) - Lp.org[ax];
        }
        if (skip) continue;
        if (l[0] < 0 || l[1] < 0 || l[2] < 0 || l[0] >= sp.nx || l[1] >= sp.ny || l[2] >= sp.nz) continue;
        s += up[p * sp.cs + gidx(sp, l[0], l[1], l[2])];
    }
    return s * (T(1) / T(1 << nodd));
}

__global__ void k_amr_mask(const Geom s, const AmrInfo L, double *r)
{
    int i, j, k, g[3];
    if (!thread_node(s, L, i, j, k, g)) return;
    const bool own = owned(L, g);
    const long long o = gidx(s, i, j, k);
    for (int p = 0; p < L.dim; ++p)
        if (!own || domain_dirichlet(L, g, p)) r[p * s.cs + o] = 0.0;
}

template <typename T>
__global__ void k_amr_inject(const Geom sc, const AmrInfo Lc, const Geom sp, const AmrInfo Lp, const T *uc, T *up)
{
    int i, j, k, g[3];
    if (!thread_node(sc, Lc, i, j, k, g)) return;
    for (int ax = 0; ax < Lc.dim; ++ax)
        if (g[ax] & 1) return;
    if (!axes_owned(Lc, g)) return;
    const int lp[3] = {g[0] / 2 - Lp.org[0], g[1] / 2 - Lp.org[1], Lc.dim == 3 ? g[2] / 2 - Lp.org[2] : 0};
    if (lp[0] < 0 || lp[1] < 0 || lp[2] < 0 || lp[0] >= sp.nx || lp[1] >= sp.ny || lp[2] >= sp.nz) return;
    const long long oc = gidx(sc, i, j, k), op = gidx(sp, lp[0], lp[1], lp[2]);
    for (int p = 0; p < Lc.dim; ++p) up[p * sp.cs + op] = uc[p * sc.cs + oc];
}

// out <- r on the owned rows that are not on a Dirichlet face of the domain, 0 on
// every other storage node (the residual of the correction equation in the
// layout of the cycle's right-hand side).
template <typename T>
__global__ void k_amr_mask_to(const Geom s, const AmrInfo L, const T *r, T *out)
{
    int i, j, k, g[3];
    if (!thread_node(s, L, i, j, k, g)) return;
    const bool own = owned(L, g);
    const long long o = gidx(s, i, j, k);
    for (int p = 0; p < L.dim; ++p) out[p * s.cs + o] = (own && !domain_dirichlet(L, g, p)) ? r[p * s.cs + o] : T(0);
}

// psi of the cells of a patch's view (storage cells 1 .. n-3 per axis, the view
// starting at storage node 1), 0 on the padding cells and the unused last index:
// the cell field the TMA sweep of the view stages.
__global__ void k_amr_view_cells(const Geom s, const float *src, float *dst)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    if (i >= s.nx || j >= s.ny || k >= s.nz) return;
    const bool in = i >= 1 && i <= s.nx - 3 && j >= 1 && j <= s.ny - 3 && (s.dim == 2 || (k >= 1 && k <= s.nz - 3));
    const long long o = gidx(s, i, j, k);
    dst[o] = in ? src[o] : 0.f;
}

// mode 0: ghosts <- interpolated parent values (owned/active nodes untouched).
// mode 1: correction prolongation: nodes solved on this level (inside the box or
//         on a domain face) += interpolated parent correction; ghosts <- it.
template <typename T>
__global__ void k_amr_ghost(const Geom sc, const AmrInfo Lc, const Geom sp, const AmrInfo Lp, T *uc, const T *up,
                            int mode)
{
    int i, j, k, g[3];
    if (!thread_node(sc, Lc, i, j, k, g)) return;
    const long long o = gidx(sc, i, j, k);
    const bool solved = axes_owned(Lc, g);
    const bool in = inside_domain(Lc, g);
    for (int p = 0; p < Lc.dim; ++p) {
        const T v = in ? parent_interp<T>(sp, Lp, up, p, g) : T(0);
        if (!solved) uc[p * sc.cs + o] = v;
        else if (mode == 1 && !domain_dirichlet(Lc, g, p)) uc[p * sc.cs + o] += v;
    }
}

// rhs_parent at the parent nodes covered by this child <- full weighting of the
// child residual (the child nodes of the stencil are all inside the child box).
template <typename T>
__global__ void k_amr_restrict(const Geom sc, const AmrInfo Lc, const Geom sp, const AmrInfo Lp, const T *rc, T *rhsp)
{
    int i, j, k, g[3];
    if (!thread_node(sp, Lp, i, j, k, g)) return;
    if (!covered_by(Lc, g)) return;
    const bool d3 = Lp.dim == 3;
    const T w[3] = {T(0.5), T(1), T(0.5)};
    const T scale = d3 ? T(0.125) : T(0.25);
    const long long op = gidx(sp, i, j, k);
    for (int p = 0; p < Lp.dim; ++p) {
        T s = T(0);
        if (!domain_dirichlet(Lp, g, p)) {
            for (int dk = (d3 ? -1 : 0); dk <= (d3 ? 1 : 0); ++dk)
                for (int dj = -1; dj <= 1; ++dj)
                    for (int di = -1; di <= 1; ++di) {
                        const int li = 2 * g[0] + di - Lc.org[0], lj = 2 * g[1] + dj - Lc.org[1];
                        const int lk = d3 ? 2 * g[2] + dk - Lc.org[2] : 0;
                        if (li < 0 || lj < 0 || lk < 0 || li >= sc.nx || lj >= sc.ny || lk >= sc.nz) continue;
                        s += w[di + 1] * w[dj + 1] * (d3 ? w[dk + 1] : T(1)) * rc[p * sc.cs + gidx(sc, li, lj, lk)];
                    }
            s *= scale;
        }
        rhsp[p * sp.cs + op] = s;
    }
}

// u += e on owned free dofs.
template <typename T>
__global__ void k_amr_update(const Geom s, const AmrInfo L, const T *e, double *u)
{
    int i, j, k, g[3];
    if (!thread_node(s, L, i, j, k, g)) return;
    if (!owned(L, g)) return;
    const long long o = gidx(s, i, j, k);
    for (int p = 0; p < L.dim; ++p)
        if (!domain_dirichlet(L, g, p)) u[p * s.cs + o] += double(e[p * s.cs + o]);
}

// per-block sums of squares of a masked residual (fixed order), then rounded to T
template <typename TO>
__global__ void k_amr_sumsq_round(const Geom s, const AmrInfo L, const double *r, TO *out, double *part)
{
    __shared__ double red[256];
    int i, j, k, g[3];
    double acc = 0.0;
    if (thread_node(s, L, i, j, k, g)) {
        const long long o = gidx(s, i, j, k);
        for (int p = 0; p < L.dim; ++p) {
            const double v = r[p * s.cs + o];
            acc += v * v;
            if (out) out[p * s.cs + o] = TO(v);
        }
    }
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    red[tid] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (tid < w) red[tid] += red[tid + w];
        __syncthreads();
    }
    if (tid == 0) part[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = red[0];
}

// Parent cells inside the child box <- mean of their 2^d child cells.
__global__ void k_amr_coarsen_psi(const Geom sc, const AmrInfo Lc, const Geom sp, const AmrInfo Lp,
                                  const double *psic, double *psip)
{
    int i, j, k, g[3];
    if (!thread_node(sp, Lp, i, j, k, g)) return;     // g = global index of the parent cell
    if (i >= sp.nx - 1 || j >= sp.ny - 1 || (Lp.dim == 3 && k >= sp.nz - 1)) return;
    for (int ax = 0; ax < Lp.dim; ++ax)
        if (2 * g[ax] < Lc.lo[ax] || 2 * g[ax] + 2 > Lc.hi[ax]) return;
    double s = 0.0;
    const int nc = 1 << Lp.dim;
    for (int c = 0; c < nc; ++c) {
        const int li = 2 * g[0] + (c & 1) - Lc.org[0], lj = 2 * g[1] + ((c >> 1) & 1) - Lc.org[1];
        const int lk = Lp.dim == 3 ? 2 * g[2] + ((c >> 2) & 1) - Lc.org[2] : 0;
        s += psic[gidx(sc, li, lj, lk)];
    }
    psip[gidx(sp, i, j, k)] = s / nc;
}

// cells of a padded box: packed (i + (nx-1)*(j + (ny-1)*k)) -> node-indexed storage
__global__ void k_amr_set_cells(const Geom s, const double *packed, double psi_min, double *lev, int *bad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    const int ncx = s.nx - 1, ncy = s.ny - 1, ncz = s.dim == 3 ? s.nz - 1 : 1;
    if (i >= ncx || j >= ncy || k >= ncz) return;
    const double v = packed[i + (long long)ncx * (j + (long long)ncy * k)];
    if (!isfinite(v)) atomicAdd(bad, 1);
    lev[gidx(s, i, j, k)] = fmax(v, psi_min);
}

// ------------------------------------------------ adjoint of the composite problem

// Transpose of the ghost fill: parent node G collects w from the child ghosts that
// interpolate it (child nodes 2G + {-1, 0, 1} per axis that are not in the child's
// box region, inside the domain), with the interpolation weights (1 on coincident
// axes, 1/2 on odd ones), and adds the sum to wp.
// with_solved != 0: also the child's solved free nodes (the correction
// prolongation adds the interpolated parent value there).
__global__ void k_amr_ghostT(const Geom sc, const AmrInfo Lc, const Geom sp, const AmrInfo Lp, const double *wc,
                             double *wp, int with_solved)
{
    int i, j, k, G[3];
    if (!thread_node(sp, Lp, i, j, k, G)) return;
    const bool d3 = Lp.dim == 3;
    const long long op = gidx(sp, i, j, k);
    for (int p = 0; p < Lp.dim; ++p) {
        double s = 0.0;
        for (int dk = (d3 ? -1 : 0); dk <= (d3 ? 1 : 0); ++dk)
            for (int dj = -1; dj <= 1; ++dj)
                for (int di = -1; di <= 1; ++di) {
                    const int g[3] = {2 * G[0] + di, 2 * G[1] + dj, d3 ? 2 * G[2] + dk : 0};
                    const int l[3] = {g[0] - Lc.org[0], g[1] - Lc.org[1], g[2] - Lc.org[2]};
                    if (l[0] < 0 || l[1] < 0 || l[2] < 0 || l[0] >= sc.nx || l[1] >= sc.ny || l[2] >= sc.nz) continue;
                    if (!inside_domain(Lc, g)) continue;
                    if (axes_owned(Lc, g) && (!with_solved || domain_dirichlet(Lc, g, p))) continue;
                    const double w = (di ? 0.5 : 1.0) * (dj ? 0.5 : 1.0) * (dk ? 0.5 : 1.0);
                    s += w * wc[p * sc.cs + gidx(sc, l[0], l[1], l[2])];
                }
        wp[p * sp.cs + op] += s;
    }
}

// Zero everything but the solved free dofs (box region, not on a Dirichlet face):
// the dofs a patch's smoother updates.
__global__ void k_amr_mask_solved(const Geom s, const AmrInfo L, double *x)
{
    int i, j, k, g[3];
    if (!thread_node(s, L, i, j, k, g)) return;
    const bool solved = axes_owned(L, g);
    const long long o = gidx(s, i, j, k);
    for (int p = 0; p < L.dim; ++p)
        if (!solved || domain_dirichlet(L, g, p)) x[p * s.cs + o] = 0.0;
}

// out = W x on the solved free dofs (W = omega / (kdiag_p * sum of the psi of the
// node's cells), the damped-Jacobi scaling), 0 elsewhere.
__global__ void k_amr_scaleW(const Geom s, const AmrInfo L, const double *psi, double omega, double k0, double k1,
                             double k2, const double *x, double *out)
{
    int i, j, k, g[3];
    if (!thread_node(s, L, i, j, k, g)) return;
    const long long o = gidx(s, i, j, k);
    const bool solved = axes_owned(L, g);
    double ps = 0.0;
    if (solved) {
        const bool d3 = L.dim == 3;
        for (int c = 0; c < (1 << L.dim); ++c) {
            const int ci = i - (c & 1), cj = j - ((c >> 1) & 1), ck = d3 ? k - ((c >> 2) & 1) : 0;
            if (ci < 0 || cj < 0 || ck < 0 || ci >= s.nx - 1 || cj >= s.ny - 1 || (d3 && ck >= s.nz - 1)) continue;
            const int C[3] = {ci + L.org[0], cj + L.org[1], ck + L.org[2]};
            bool in = true;
            for (int ax = 0; ax < L.dim; ++ax)
                if (C[ax] < 0 || C[ax] > L.N[ax] - 2) in = false;
            if (in) ps += psi[gidx(s, ci, cj, ck)];
        }
    }
    const double kd[3] = {k0, k1, k2};
    for (int p = 0; p < L.dim; ++p) {
        const bool free = solved && !domain_dirichlet(L, g, p) && ps > 0.0 && kd[p] != 0.0;
        out[p * s.cs + o] = free ? omega / (kd[p] * ps) * x[p * s.cs + o] : 0.0;
    }
}

// Transpose of the full-weighting restriction onto the covered parent nodes:
// child node g collects scale * w(g - 2G) * rp(G) from the parents G covered by
// this child with
// |g - 2G| <= 1 (parents on a Dirichlet face of the component contribute 0).
__global__ void k_amr_restrictT(const Geom sc, const AmrInfo Lc, const Geom sp, const AmrInfo Lp, const double *rp,
                                double *rc)
{
    int i, j, k, g[3];
    if (!thread_node(sc, Lc, i, j, k, g)) return;
    const bool d3 = Lc.dim == 3;
    const double scale = d3 ? 0.125 : 0.25;
    const long long oc = gidx(sc, i, j, k);
    for (int p = 0; p < Lc.dim; ++p) {
        double s = 0.0;
        // parents G with 2G in {g-1, g, g+1} per axis
        for (int dk = (d3 ? -1 : 0); dk <= (d3 ? 1 : 0); ++dk)
            for (int dj = -1; dj <= 1; ++dj)
                for (int di = -1; di <= 1; ++di) {
                    const int t[3] = {g[0] + di, g[1] + dj, d3 ? g[2] + dk : 0};
                    if ((t[0] & 1) || (t[1] & 1) || (t[2] & 1)) continue;
                    const int G[3] = {t[0] / 2, t[1] / 2, t[2] / 2};
                    if (!covered_by(Lc, G) || domain_dirichlet(Lp, G, p)) continue;
                    const int l[3] = {G[0] - Lp.org[0], G[1] - Lp.org[1], G[2] - Lp.org[2]};
                    if (l[0] < 0 || l[1] < 0 || l[2] < 0 || l[0] >= sp.nx || l[1] >= sp.ny || l[2] >= sp.nz) continue;
                    const double w = (di ? 0.5 : 1.0) * (dj ? 0.5 : 1.0) * (dk ? 0.5 : 1.0);
                    s += scale * w * rp[p * sp.cs + gidx(sp, l[0], l[1], l[2])];
                }
        rc[p * sc.cs + oc] = s;
    }
}

// Transpose of the injection: a child node of the box region with even
// coordinates receives w of the coincident (covered) parent node.
__global__ void k_amr_injectT(const Geom sc, const AmrInfo Lc, const Geom sp, const AmrInfo Lp, const double *wp,
                              double *wc)
{
    int i, j, k, g[3];
    if (!thread_node(sc, Lc, i, j, k, g)) return;
    for (int ax = 0; ax < Lc.dim; ++ax)
        if (g[ax] & 1) return;
    if (!axes_owned(Lc, g)) return;
    const int lp[3] = {g[0] / 2 - Lp.org[0], g[1] / 2 - Lp.org[1], Lc.dim == 3 ? g[2] / 2 - Lp.org[2] : 0};
    if (lp[0] < 0 || lp[1] < 0 || lp[2] < 0 || lp[0] >= sp.nx || lp[1] >= sp.ny || lp[2] >= sp.nz) return;
    const long long oc = gidx(sc, i, j, k), op = gidx(sp, lp[0], lp[1], lp[2]);
    for (int p = 0; p < Lc.dim; ++p) wc[p * sc.cs + oc] += wp[p * sp.cs + op];
}

// Per-block sums of x.y over the owned free dofs (fixed order).
__global__ void k_amr_dot(const Geom s, const AmrInfo L, const double *x, const double *y, double *part)
{
    __shared__ double red[256];
    int i, j, k, g[3];
    double acc = 0.0;
    if (thread_node(s, L, i, j, k, g) && owned(L, g)) {
        const long long o = gidx(s, i, j, k);
        for (int p = 0; p < L.dim; ++p)
            if (!domain_dirichlet(L, g, p)) acc += x[p * s.cs + o] * y[p * s.cs + o];
    }
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    red[tid] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (tid < w) red[tid] += red[tid + w];
        __syncthreads();
    }
    if (tid == 0) part[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = red[0];
}

// dJ/dpsi of every storage cell: -lam_c^T S_c u_c (unit-psi cell matrix of the
// level, via the cell routine), 0 for cells outside the domain.
__global__ void k_amr_dJdpsi(const Geom s, const AmrInfo L, const Coef<double> c, const double *u, const double *lam,
                             double *g)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    const bool d3 = L.dim == 3;
    if (i >= s.nx - 1 || j >= s.ny - 1 || (d3 ? k >= s.nz - 1 : k > 0)) return;
    const int C[3] = {i + L.org[0], j + L.org[1], k + L.org[2]};
    bool in = true;
    for (int ax = 0; ax < L.dim; ++ax)
        if (C[ax] < 0 || C[ax] > L.N[ax] - 2) in = false;
    double acc = 0.0;
    if (in) {
        if (d3) {
            double U[3][8], Lm[3][8];
            for (int b = 0; b < 8; ++b) {
                const long long o = gidx(s, i + (b & 1), j + ((b >> 1) & 1), k + ((b >> 2) & 1));
                for (int p = 0; p < 3; ++p) {
                    U[p][b] = u[p * s.cs + o];
                    Lm[p][b] = lam[p * s.cs + o];
                }
            }
            cell_forces3<double>(U, 1.0, c);
            for (int b = 0; b < 8; ++b)
                for (int p = 0; p < 3; ++p) acc += Lm[p][b] * U[p][b];
        } else {
            double U[2][4], Lm[2][4];
            for (int b = 0; b < 4; ++b) {
                const long long o = gidx(s, i + (b & 1), j + ((b >> 1) & 1), 0);
                for (int p = 0; p < 2; ++p) {
                    U[p][b] = u[p * s.cs + o];
                    Lm[p][b] = lam[p * s.cs + o];
                }
            }
            cell_forces2<double>(U, 1.0, c);
            for (int b = 0; b < 4; ++b)
                for (int p = 0; p < 2; ++p) acc += Lm[p][b] * U[p][b];
        }
    }
    g[gidx(s, i, j, k)] = -acc;
}

// Coarse cells under the child box hold the fine mean: their gradient passes to
// their 2^d fine cells and they keep none.
__global__ void k_amr_grad_chain(const Geom sc, const AmrInfo Lc, const Geom sp, const AmrInfo Lp, double *gp,
                                 double *gc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    const bool d3 = Lp.dim == 3;
    if (i >= sp.nx - 1 || j >= sp.ny - 1 || (d3 ? k >= sp.nz - 1 : k > 0)) return;
    const int C[3] = {i + Lp.org[0], j + Lp.org[1], k + Lp.org[2]};
    for (int ax = 0; ax < Lp.dim; ++ax)
        if (2 * C[ax] < Lc.lo[ax] || 2 * C[ax] + 2 > Lc.hi[ax]) return;
    const long long op = gidx(sp, i, j, k);
    const int nc = 1 << Lp.dim;
    const double share = gp[op] / nc;
    for (int c = 0; c < nc; ++c) {
        const int li = 2 * C[0] + (c & 1) - Lc.org[0], lj = 2 * C[1] + ((c >> 1) & 1) - Lc.org[1];
        const int lk = d3 ? 2 * C[2] + ((c >> 2) & 1) - Lc.org[2] : 0;
        gc[gidx(sc, li, lj, lk)] += share;
    }
    gp[op] = 0.0;
}

// node-indexed cells of a padded box -> packed (i + (nx-1)*(j + (ny-1)*k)); cells
// whose psi sits at the floor get 0 (psi = max(raw, psi_min) is flat there).
__global__ void k_amr_get_cells(const Geom s, const double *lev, const double *psi, double psi_min, double *packed)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    const int ncx = s.nx - 1, ncy = s.ny - 1, ncz = s.dim == 3 ? s.nz - 1 : 1;
    if (i >= ncx || j >= ncy || k >= ncz) return;
    const long long o = gidx(s, i, j, k);
    packed[i + (long long)ncx * (j + (long long)ncy * k)] = psi[o] > psi_min ? lev[o] : 0.0;
}

// Regridding tags: storage cell (i,j,k) of a patch (or of the base level) gets 1
// when its global cell index lies in [cmin, cmax] on every axis and h |grad psi|
// > thr, grad psi by centred differences of the cell values, a neighbour beyond the
// domain replaced by the cell itself.  Output packed over the storage cells
// (x fastest).
__global__ void k_amr_tag(const Geom s, const AmrInfo L, const double *psi, double thr, int3 cmin, int3 cmax,
                          unsigned char *tags)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    const bool d3 = L.dim == 3;
    const int ncx = s.nx - 1, ncy = s.ny - 1, ncz = d3 ? s.nz - 1 : 1;
    if (i >= ncx || j >= ncy || k >= ncz) return;
    const int C[3] = {i + L.org[0], j + L.org[1], k + L.org[2]};
    const int lo[3] = {cmin.x, cmin.y, cmin.z}, hi[3] = {cmax.x, cmax.y, cmax.z};
    bool in = true;
    for (int ax = 0; ax < L.dim; ++ax)
        if (C[ax] < lo[ax] || C[ax] > hi[ax]) in = false;
    unsigned char t = 0;
    if (in) {
        const int l[3] = {i, j, k};
        double g2 = 0.0;
        for (int ax = 0; ax < L.dim; ++ax) {
            int up[3] = {l[0], l[1], l[2]}, dn[3] = {l[0], l[1], l[2]};
            if (C[ax] + 1 <= L.N[ax] - 2) ++up[ax];
            if (C[ax] - 1 >= 0) --dn[ax];
            const double d = 0.5 * (psi[gidx(s, up[0], up[1], up[2])] - psi[gidx(s, dn[0], dn[1], dn[2])]);
            g2 += d * d;
        }
        t = sqrt(g2) > thr ? 1 : 0;
    }
    tags[i + (long long)ncx * (j + (long long)ncy * k)] = t;
}

const dim3 kAmrBlock(32, 4, 2);
inline dim3 amr_grid(const Geom &s) { return dim3((s.nx + 31) / 32, (s.ny + 3) / 4, (s.nz + 1) / 2); }

}  // namespace

long long amr_blocks(const Geom &s)
{
    const dim3 g = amr_grid(s);
    return (long long)g.x * g.y * g.z;
}

bool amr_owned_host(const AmrInfo &L, int i, int j, int k)
{
    const int g[3] = {i, j, k};
    return owned(L, g);
}

cudaError_t launch_amr_mask(const Geom &s, const AmrInfo &L, double *r, cudaStream_t st)
{
    k_amr_mask<<<amr_grid(s), kAmrBlock, 0, st>>>(s, L, r);
    ++g_launches;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_amr_inject(const Geom &sc, const AmrInfo &Lc, const Geom &sp, const AmrInfo &Lp, const T *uc, T *up,
                              cudaStream_t st)
{
    k_amr_inject<T><<<amr_grid(sc), kAmrBlock, 0, st>>>(sc, Lc, sp, Lp, uc, up);
    ++g_launches;
    return cudaGetLastError();
}
template cudaError_t launch_amr_inject<double>(const Geom &, const AmrInfo &, const Geom &, const AmrInfo &,
                                               const double *, double *, cudaStream_t);
template cudaError_t launch_amr_inject<float>(const Geom &, const AmrInfo &, const Geom &, const AmrInfo &,
                                              const float *, float *, cudaStream_t);

cudaError_t launch_amr_view_cells(const Geom &s, const float *src, float *dst, cudaStream_t st)
{
    k_amr_view_cells<<<amr_grid(s), kAmrBlock, 0, st>>>(s, src, dst);
    ++g_launches;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_amr_mask_to(const Geom &s, const AmrInfo &L, const T *r, T *out, cudaStream_t st)
{
    k_amr_mask_to<T><<<amr_grid(s), kAmrBlock, 0, st>>>(s, L, r, out);
    ++g_launches;
    return cudaGetLastError();
}
template cudaError_t launch_amr_mask_to<float>(const Geom &, const AmrInfo &, const float *, float *, cudaStream_t);

template <typename T>
cudaError_t launch_amr_ghost(const Geom &sc, const AmrInfo &Lc, const Geom &sp, const AmrInfo &Lp, T *uc, const T *up,
                             int mode, cudaStream_t st)
{
    k_amr_ghost<T><<<amr_grid(sc), kAmrBlock, 0, st>>>(sc, Lc, sp, Lp, uc, up, mode);
    ++g_launches;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_amr_restrict(const Geom &sc, const AmrInfo &Lc, const Geom &sp, const AmrInfo &Lp, const T *rc,
                                T *rhsp, cudaStream_t st)
{
    k_amr_restrict<T><<<amr_grid(sp), kAmrBlock, 0, st>>>(sc, Lc, sp, Lp, rc, rhsp);
    ++g_launches;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_amr_update(const Geom &s, const AmrInfo &L, const T *e, double *u, cudaStream_t st)
{
    k_amr_update<T><<<amr_grid(s), kAmrBlock, 0, st>>>(s, L, e, u);
    ++g_launches;
    return cudaGetLastError();
}

template <typename TO>
cudaError_t launch_amr_sumsq_round(const Geom &s, const AmrInfo &L, const double *r, TO *out, double *part,
                                   cudaStream_t st)
{
    k_amr_sumsq_round<TO><<<amr_grid(s), kAmrBlock, 0, st>>>(s, L, r, out, part);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_amr_coarsen_psi(const Geom &sc, const AmrInfo &Lc, const Geom &sp, const AmrInfo &Lp,
                                   const double *psic, double *psip, cudaStream_t st)
{
    k_amr_coarsen_psi<<<amr_grid(sp), kAmrBlock, 0, st>>>(sc, Lc, sp, Lp, psic, psip);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_amr_set_cells(const Geom &s, const double *packed, double psi_min, double *lev, int *bad,
                                 cudaStream_t st)
{
    k_amr_set_cells<<<amr_grid(s), kAmrBlock, 0, st>>>(s, packed, psi_min, lev, bad);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_amr_ghostT(const Geom &sc, const AmrInfo &Lc, const Geom &sp, const AmrInfo &Lp, const double *wc,
                              double *wp, int with_solved, cudaStream_t st)
{
    k_amr_ghostT<<<amr_grid(sp), kAmrBlock, 0, st>>>(sc, Lc, sp, Lp, wc, wp, with_solved);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_amr_mask_solved(const Geom &s, const AmrInfo &L, double *x, cudaStream_t st)
{
    k_amr_mask_solved<<<amr_grid(s), kAmrBlock, 0, st>>>(s, L, x);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_amr_scaleW(const Geom &s, const AmrInfo &L, const double *psi, double omega, const double kdiag[3],
                              const double *x, double *out, cudaStream_t st)
{
    k_amr_scaleW<<<amr_grid(s), kAmrBlock, 0, st>>>(s, L, psi, omega, kdiag[0], kdiag[1], kdiag[2], x, out);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_amr_restrictT(const Geom &sc, const AmrInfo &Lc, const Geom &sp, const AmrInfo &Lp,
                                 const double *rp, double *rc, cudaStream_t st)
{
    k_amr_restrictT<<<amr_grid(sc), kAmrBlock, 0, st>>>(sc, Lc, sp, Lp, rp, rc);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_amr_injectT(const Geom &sc, const AmrInfo &Lc, const Geom &sp, const AmrInfo &Lp, const double *wp,
                               double *wc, cudaStream_t st)
{
    k_amr_injectT<<<amr_grid(sc), kAmrBlock, 0, st>>>(sc, Lc, sp, Lp, wp, wc);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_amr_dot(const Geom &s, const AmrInfo &L, const double *x, const double *y, double *part,
                           cudaStream_t st)
{
    k_amr_dot<<<amr_grid(s), kAmrBlock, 0, st>>>(s, L, x, y, part);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_amr_dJdpsi(const Geom &s, const AmrInfo &L, const Coef<double> &c, const double *u,
                              const double *lam, double *g, cudaStream_t st)
{
    k_amr_dJdpsi<<<amr_grid(s), kAmrBlock, 0, st>>>(s, L, c, u, lam, g);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_amr_grad_chain(const Geom &sc, const AmrInfo &Lc, const Geom &sp, const AmrInfo &Lp, double *gp,
                                  double *gc, cudaStream_t st)
{
    k_amr_grad_chain<<<amr_grid(sp), kAmrBlock, 0, st>>>(sc, Lc, sp, Lp, gp, gc);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_amr_tag(const Geom &s, const AmrInfo &L, const double *psi, double thr, const int cmin[3],
                           const int cmax[3], unsigned char *tags, cudaStream_t st)
{
    k_amr_tag<<<amr_grid(s), kAmrBlock, 0, st>>>(s, L, psi, thr, make_int3(cmin[0], cmin[1], cmin[2]),
                                                 make_int3(cmax[0], cmax[1], cmax[2]), tags);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_amr_get_cells(const Geom &s, const double *lev, const double *psi, double psi_min, double *packed,
                                 cudaStream_t st)
{
    k_amr_get_cells<<<amr_grid(s), kAmrBlock, 0, st>>>(s, lev, psi, psi_min, packed);
    ++g_launches;
    return cudaGetLastError();
}

template cudaError_t launch_amr_ghost<double>(const Geom &, const AmrInfo &, const Geom &, const AmrInfo &, double *,
                                              const double *, int, cudaStream_t);
template cudaError_t launch_amr_ghost<float>(const Geom &, const AmrInfo &, const Geom &, const AmrInfo &, float *,
                                             const float *, int, cudaStream_t);
template cudaError_t launch_amr_restrict<double>(const Geom &, const AmrInfo &, const Geom &, const AmrInfo &,
                                                 const double *, double *, cudaStream_t);
template cudaError_t launch_amr_restrict<float>(const Geom &, const AmrInfo &, const Geom &, const AmrInfo &,
                                                const float *, float *, cudaStream_t);
template cudaError_t launch_amr_update<double>(const Geom &, const AmrInfo &, const double *, double *, cudaStream_t);
template cudaError_t launch_amr_update<float>(const Geom &, const AmrInfo &, const float *, double *, cudaStream_t);
template cudaError_t launch_amr_sumsq_round<double>(const Geom &, const AmrInfo &, const double *, double *, double *,
                                                    cudaStream_t);
template cudaError_t launch_amr_sumsq_round<float>(const Geom &, const AmrInfo &, const double *, float *, double *,
                                                   cudaStream_t);

}  // namespace sbm
