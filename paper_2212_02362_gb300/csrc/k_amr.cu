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
// One thread per parent cell B (global parent coordinates): the 2^d corners B + c
// are loaded once (0 outside the parent's storage) and the child nodes 2B + delta,
// delta in {0,1}^d, of the child's storage are written; a child node's value is the
// sum of its corners (corner 0 on even axes, both on odd ones, ascending order)
// times 2^-(odd axes).  In mode 0 a block whose child nodes are all solved returns
// before loading.
template <typename T, int D>
__global__ void k_amr_ghost(const Geom sc, const AmrInfo Lc, const Geom sp, const AmrInfo Lp, T *uc, const T *up,
                            int mode, int3 b0, int3 nb)
{
    const int bx = blockIdx.x * blockDim.x + threadIdx.x, by = blockIdx.y * blockDim.y + threadIdx.y,
              bz = blockIdx.z * blockDim.z + threadIdx.z;
    if (bx >= nb.x || by >= nb.y || bz >= nb.z) return;
    const int B[3] = {b0.x + bx, b0.y + by, b0.z + bz};
    const int sn[3] = {sp.nx, sp.ny, sp.nz}, cn[3] = {sc.nx, sc.ny, sc.nz};
    if (mode != 1) {
        bool all_solved = true;
#pragma unroll
        for (int d = 0; d < (1 << D); ++d) {
            const int g[3] = {2 * B[0] + (d & 1), 2 * B[1] + ((d >> 1) & 1), D == 3 ? 2 * B[2] + (d >> 2) : 0};
            if (!axes_owned(Lc, g)) all_solved = false;
        }
        if (all_solved) return;
    }
    T v[1 << D][D];
#pragma unroll
    for (int c = 0; c < (1 << D); ++c) {
        const int l[3] = {B[0] + (c & 1) - Lp.org[0], B[1] + ((c >> 1) & 1) - Lp.org[1],
                          D == 3 ? B[2] + (c >> 2) - Lp.org[2] : 0};
        bool in = true;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax)
            if (l[ax] < 0 || l[ax] >= sn[ax]) in = false;
        const long long o = in ? gidx(sp, l[0], l[1], l[2]) : 0;
#pragma unroll
        for (int p = 0; p < D; ++p) v[c][p] = in ? up[p * sp.cs + o] : T(0);
    }
#pragma unroll
    for (int d = 0; d < (1 << D); ++d) {
        const int dl[3] = {d & 1, (d >> 1) & 1, D == 3 ? d >> 2 : 0};
        const int g[3] = {2 * B[0] + dl[0], 2 * B[1] + dl[1], 2 * B[2] + dl[2]};
        int l[3];
        bool in = true;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            l[ax] = g[ax] - Lc.org[ax];
            if (l[ax] < 0 || l[ax] >= cn[ax]) in = false;
        }
        if (!in) continue;
        const bool solved = axes_owned(Lc, g);
        if (solved && mode != 1) continue;
        T val[D];
#pragma unroll
        for (int p = 0; p < D; ++p) val[p] = T(0);
        if (inside_domain(Lc, g)) {
            int nodd = 0;
#pragma unroll
            for (int c = 0; c < (1 << D); ++c) {
                bool use = true;
#pragma unroll
                for (int ax = 0; ax < D; ++ax)
                    if (!dl[ax] && ((c >> ax) & 1)) use = false;
                if (!use) continue;
#pragma unroll
                for (int p = 0; p < D; ++p) val[p] += v[c][p];
            }
#pragma unroll
            for (int ax = 0; ax < D; ++ax) nodd += dl[ax];
            const T sc_ = T(1) / T(1 << nodd);
#pragma unroll
            for (int p = 0; p < D; ++p) val[p] *= sc_;
        }
        const long long o = gidx(sc, l[0], l[1], l[2]);
#pragma unroll
        for (int p = 0; p < D; ++p) {
            if (!solved) uc[p * sc.cs + o] = val[p];
            else if (!domain_dirichlet(Lc, g, p)) uc[p * sc.cs + o] += val[p];
        }
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
    T s[3] = {T(0), T(0), T(0)};
    for (int dk = (d3 ? -1 : 0); dk <= (d3 ? 1 : 0); ++dk)
        for (int dj = -1; dj <= 1; ++dj)
            for (int di = -1; di <= 1; ++di) {
                const int li = 2 * g[0] + di - Lc.org[0], lj = 2 * g[1] + dj - Lc.org[1];
                const int lk = d3 ? 2 * g[2] + dk - Lc.org[2] : 0;
                if (li < 0 || lj < 0 || lk < 0 || li >= sc.nx || lj >= sc.ny || lk >= sc.nz) continue;
                const T wt = w[di + 1] * w[dj + 1] * (d3 ? w[dk + 1] : T(1));
                const long long oc = gidx(sc, li, lj, lk);
                for (int p = 0; p < Lp.dim; ++p) s[p] += wt * rc[p * sc.cs + oc];
            }
    for (int p = 0; p < Lp.dim; ++p) rhsp[p * sp.cs + op] = domain_dirichlet(Lp, g, p) ? T(0) : s[p] * scale;
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
// prolongation adds the interpolated parent value there).  The child nodes around
// parent node G are enumerated directly (clipped to the child's storage and the
// domain); a parent whose whole neighbourhood lies strictly inside the child's box
// has no ghost child and is skipped when only ghosts count.
__global__ void k_amr_ghostT(const Geom sc, const AmrInfo Lc, const Geom sp, const AmrInfo Lp, const double *wc,
                             double *wp, int with_solved)
{
    int i, j, k, G[3];
    if (!thread_node(sp, Lp, i, j, k, G)) return;
    const int D = Lp.dim;
    const int sn[3] = {sc.nx, sc.ny, sc.nz};
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    bool interior = true;
    for (int ax = 0; ax < D; ++ax) {
        const int c = 2 * G[ax];
        lo[ax] = max(max(c - 1, Lc.org[ax]), 0);
        hi[ax] = min(min(c + 1, Lc.org[ax] + sn[ax] - 1), Lc.N[ax] - 1);
        if (lo[ax] > hi[ax]) return;
        if (!(c - 1 > Lc.lo[ax] && c + 1 < Lc.hi[ax])) interior = false;
    }
    if (interior && !with_solved) return;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int gz = lo[2]; gz <= hi[2]; ++gz)
        for (int gy = lo[1]; gy <= hi[1]; ++gy)
            for (int gx = lo[0]; gx <= hi[0]; ++gx) {
                const int g[3] = {gx, gy, gz};
                const bool own = axes_owned(Lc, g);
                if (own && !with_solved) continue;
                const double w = (gx != 2 * G[0] ? 0.5 : 1.0) * (gy != 2 * G[1] ? 0.5 : 1.0) *
                                 (D == 3 && gz != 2 * G[2] ? 0.5 : 1.0);
                const long long o = gidx(sc, gx - Lc.org[0], gy - Lc.org[1], gz - Lc.org[2]);
                for (int p = 0; p < D; ++p) {
                    if (own && domain_dirichlet(Lc, g, p)) continue;
                    acc[p] += w * wc[p * sc.cs + o];
                }
            }
    const long long op = gidx(sp, i, j, k);
    for (int p = 0; p < D; ++p) wp[p * sp.cs + op] += acc[p];
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
        out[p * s.cs + o] = free ? omega / (kd[p] * ps) * (x ? x[p * s.cs + o] : 1.0) : 0.0;
    }
}

// One transposed damped-Jacobi sweep, first half: t = W eb (W from k_amr_scaleW with
// x = null: 0 off the solved free dofs), rb += t, and t written in the precision of
// the stencil product that follows (every storage node).
template <typename TS>
__global__ void k_amr_jacT_scale(long long n, const double *__restrict__ W, const double *__restrict__ eb,
                                 double *__restrict__ rb, TS *__restrict__ t)
{
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= n) return;
    const double v = W[q] * eb[q];
    rb[q] += v;
    t[q] = TS(v);
}

// eb += alpha y on the nodes of a patch view (extents of v, storage strides; both
// arrays start at the storage origin, the view at element offset voff).
template <typename TS>
__global__ void k_axpy_view(const Geom v, long long voff, double alpha, const TS *__restrict__ y,
                            double *__restrict__ eb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    if (i >= v.nx || j >= v.ny || k >= v.nz) return;
    const long long o = voff + gidx(v, i, j, k);
    for (int p = 0; p < v.dim; ++p) eb[p * v.cs + o] += alpha * double(y[p * v.cs + o]);
}

// Transpose of the full-weighting restriction onto the covered parent nodes:
// child node g collects scale * w(g - 2G) * rp(G) from the parents G covered by
// this child with |g - 2G| <= 1 (parents on a Dirichlet face of the component
// contribute 0).  One thread per parent cell B (global parent coordinates): it
// loads the 2^d corners B + c once (0 where not covered, outside the parent's
// storage or Dirichlet) and writes the child nodes 2B + delta, delta in {0,1}^d,
// that lie in the child's storage: even axes take corner 0 with weight 1, odd axes
// corners 0 and 1 with weight 1/2, summed in ascending parent order.
template <int D>
__global__ void k_amr_restrictT(const Geom sc, const AmrInfo Lc, const Geom sp, const AmrInfo Lp, const double *rp,
                                double *rc, int3 b0, int3 nb)
{
    const int bx = blockIdx.x * blockDim.x + threadIdx.x, by = blockIdx.y * blockDim.y + threadIdx.y,
              bz = blockIdx.z * blockDim.z + threadIdx.z;
    if (bx >= nb.x || by >= nb.y || bz >= nb.z) return;
    const int B[3] = {b0.x + bx, b0.y + by, b0.z + bz};
    const int sn[3] = {sp.nx, sp.ny, sp.nz}, cn[3] = {sc.nx, sc.ny, sc.nz};
    const double scale = D == 3 ? 0.125 : 0.25;
    double v[1 << D][D];
#pragma unroll
    for (int c = 0; c < (1 << D); ++c) {
        const int G[3] = {B[0] + (c & 1), B[1] + ((c >> 1) & 1), D == 3 ? B[2] + (c >> 2) : 0};
        bool in = covered_by(Lc, G);
        int l[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            l[ax] = G[ax] - Lp.org[ax];
            if (l[ax] < 0 || l[ax] >= sn[ax]) in = false;
        }
        const long long o = in ? gidx(sp, l[0], l[1], l[2]) : 0;
#pragma unroll
        for (int p = 0; p < D; ++p) v[c][p] = (in && !domain_dirichlet(Lp, G, p)) ? rp[p * sp.cs + o] : 0.0;
    }
#pragma unroll
    for (int d = 0; d < (1 << D); ++d) {
        const int dl[3] = {d & 1, (d >> 1) & 1, D == 3 ? d >> 2 : 0};
        int l[3];
        bool in = true;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            l[ax] = 2 * B[ax] + dl[ax] - Lc.org[ax];
            if (l[ax] < 0 || l[ax] >= cn[ax]) in = false;
        }
        if (!in) continue;
        double acc[D];
#pragma unroll
        for (int p = 0; p < D; ++p) acc[p] = 0.0;
#pragma unroll
        for (int c = 0; c < (1 << D); ++c) {
            const int cb[3] = {c & 1, (c >> 1) & 1, c >> 2};
            bool use = true;
            double w = 1.0;
#pragma unroll
            for (int ax = 0; ax < D; ++ax) {
                if (!dl[ax] && cb[ax]) use = false;
                if (dl[ax]) w *= 0.5;
            }
            if (!use) continue;
#pragma unroll
            for (int p = 0; p < D; ++p) acc[p] += scale * w * v[c][p];
        }
        const long long oc = gidx(sc, l[0], l[1], l[2]);
#pragma unroll
        for (int p = 0; p < D; ++p) rc[p * sc.cs + oc] = acc[p];
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

// Parent cells B (global parent coordinates, first b0, counts nb) whose child
// blocks 2B + {0,1}^d cover the child's storage, and the launch grid over them.
dim3 child_blocks(const Geom &sc, const AmrInfo &Lc, int3 &b0, int3 &nb)
{
    int lo[3] = {0, 0, 0}, n[3] = {1, 1, 1};
    const int cn[3] = {sc.nx, sc.ny, sc.nz};
    for (int ax = 0; ax < sc.dim; ++ax) {
        const int g0 = Lc.org[ax], g1 = Lc.org[ax] + cn[ax] - 1;
        lo[ax] = (g0 >= 0 ? g0 : g0 - 1) / 2;        // floor(g0 / 2)
        n[ax] = (g1 >= 0 ? g1 : g1 - 1) / 2 - lo[ax] + 1;
    }
    b0 = make_int3(lo[0], lo[1], lo[2]);
    nb = make_int3(n[0], n[1], n[2]);
    Geom gb = sc;
    gb.nx = n[0];
    gb.ny = n[1];
    gb.nz = n[2];
    return amr_grid(gb);
}

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
    int3 b0, nb;
    const dim3 gr = child_blocks(sc, Lc, b0, nb);
    if (sc.dim == 3) k_amr_ghost<T, 3><<<gr, kAmrBlock, 0, st>>>(sc, Lc, sp, Lp, uc, up, mode, b0, nb);
    else k_amr_ghost<T, 2><<<gr, kAmrBlock, 0, st>>>(sc, Lc, sp, Lp, uc, up, mode, b0, nb);
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

template <typename TS>
cudaError_t launch_amr_jacT_scale(long long n, const double *W, const double *eb, double *rb, TS *t, cudaStream_t st)
{
    k_amr_jacT_scale<TS><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, W, eb, rb, t);
    ++g_launches;
    return cudaGetLastError();
}
template cudaError_t launch_amr_jacT_scale<float>(long long, const double *, const double *, double *, float *,
                                                  cudaStream_t);
template cudaError_t launch_amr_jacT_scale<double>(long long, const double *, const double *, double *, double *,
                                                   cudaStream_t);

template <typename TS>
cudaError_t launch_axpy_view(const Geom &v, long long voff, double alpha, const TS *y, double *eb, cudaStream_t st)
{
    k_axpy_view<TS><<<amr_grid(v), kAmrBlock, 0, st>>>(v, voff, alpha, y, eb);
    ++g_launches;
    return cudaGetLastError();
}
template cudaError_t launch_axpy_view<float>(const Geom &, long long, double, const float *, double *, cudaStream_t);
template cudaError_t launch_axpy_view<double>(const Geom &, long long, double, const double *, double *,
                                              cudaStream_t);

cudaError_t launch_amr_restrictT(const Geom &sc, const AmrInfo &Lc, const Geom &sp, const AmrInfo &Lp,
                                 const double *rp, double *rc, cudaStream_t st)
{
    int3 b0, nb;
    const dim3 gr = child_blocks(sc, Lc, b0, nb);
    if (sc.dim == 3) k_amr_restrictT<3><<<gr, kAmrBlock, 0, st>>>(sc, Lc, sp, Lp, rp, rc, b0, nb);
    else k_amr_restrictT<2><<<gr, kAmrBlock, 0, st>>>(sc, Lc, sp, Lp, rp, rc, b0, nb);
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
