// k_misc.cu — level transfers (full-weighting restriction, linear prolongation,
// psi coarsening), packed <-> level copies, the deterministic norm reduction,
// the coarsest-level dense solve (assembly, Gauss-Jordan inverse, matvec), the
// FP64 defect update and the dJ/dpsi gradient kernel.
#include "sbm_common.cuh"

namespace sbm {

long long g_launches = 0;

namespace {

constexpr int kThreads = 256;

inline int nblk(long long n, int t = kThreads) { return (int)((n + t - 1) / t); }

__device__ __forceinline__ void node_of(const Geom &g, long long t, int &i, int &j, int &k)
{
    i = (int)(t % g.nx);
    long long r = t / g.nx;
    j = (int)(r % g.ny);
    k = (int)(r / g.ny);
}

// ---------------------------------------------------------------- transfers

// Launch geometry of the node-wise kernels: a 3D grid of (32, 4, 2) blocks covers
// (nx, ny, nz) directly, so no index decoding by division is needed.
const dim3 kNodeBlock(32, 4, 2);
inline dim3 node_grid(const Geom &g)
{
    return dim3((g.nx + 31) / 32, (g.ny + 3) / 4, (g.nz + 1) / 2);
}

// r_c = P^T r_f / 2^d on free coarse dofs (Sec. 2.2 level transfers); coarse
// node (I,J,K) sits on fine node (2I,2J,2K), the linear weights are 1, 1/2.
template <typename T>
__global__ void k_restrict(const Geom gf, const Geom gc, const T *__restrict__ rf, T *__restrict__ fc)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int K = blockIdx.z * blockDim.z + threadIdx.z;
    if (I >= gc.nx || J >= gc.ny || K >= gc.nz) return;
    const bool d3 = gf.dim == 3;
    const T w[3] = {T(0.5), T(1), T(0.5)};
    const T scale = d3 ? T(0.125) : T(0.25);
    const long long oc = gidx(gc, I, J, K);
    for (int p = 0; p < gf.dim; ++p) {
        T s = T(0);
        if (!is_dir(gc, p, I, J, K)) {
            for (int dk = (d3 ? -1 : 0); dk <= (d3 ? 1 : 0); ++dk) {
                const int k = 2 * K + dk;
                if (k < 0 || k >= gf.nz) continue;
                for (int dj = -1; dj <= 1; ++dj) {
                    const int j = 2 * J + dj;
                    if (j < 0 || j >= gf.ny) continue;
                    T sr = T(0);
                    for (int di = -1; di <= 1; ++di) {
                        const int i = 2 * I + di;
                        if (i < 0 || i >= gf.nx) continue;
                        sr += w[di + 1] * rf[p * gf.cs + gidx(gf, i, j, k)];
                    }
                    s += (d3 ? w[dk + 1] : T(1)) * w[dj + 1] * sr;
                }
            }
            s *= scale;
        }
        fc[p * gc.cs + oc] = s;
    }
}

// u_f += P e_c on free fine dofs.
template <typename T>
__global__ void k_prolong_add(const Geom gf, const Geom gc, const T *__restrict__ ec, T *__restrict__ uf)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    if (i >= gf.nx || j >= gf.ny || k >= gf.nz) return;
    const int I0 = i >> 1, I1 = (i + 1) >> 1, J0 = j >> 1, J1 = (j + 1) >> 1;
    const int K0 = k >> 1, K1 = (gf.dim == 3) ? (k + 1) >> 1 : K0;
    const T wi = (I0 == I1) ? T(1) : T(0.5), wj = (J0 == J1) ? T(1) : T(0.5), wk = (K0 == K1) ? T(1) : T(0.5);
    const long long of = gidx(gf, i, j, k);
    for (int p = 0; p < gf.dim; ++p) {
        if (is_dir(gf, p, i, j, k)) continue;
        const T *e = ec + p * gc.cs;
        T s = wi * wj * e[gidx(gc, I0, J0, K0)];
        if (I1 != I0) s += wi * wj * e[gidx(gc, I1, J0, K0)];
        if (J1 != J0) s += wi * wj * e[gidx(gc, I0, J1, K0)];
        if (I1 != I0 && J1 != J0) s += wi * wj * e[gidx(gc, I1, J1, K0)];
        if (K1 != K0) {
            T s2 = e[gidx(gc, I0, J0, K1)];
            if (I1 != I0) s2 += e[gidx(gc, I1, J0, K1)];
            if (J1 != J0) s2 += e[gidx(gc, I0, J1, K1)];
            if (I1 != I0 && J1 != J0) s2 += e[gidx(gc, I1, J1, K1)];
            s = wk * (s + wi * wj * s2);
        }
        uf[p * gf.cs + of] += s;
    }
}

// Coarse psi = mean of the 2^d fine cells (Sec. 2.4 material averaging).
__global__ void k_coarsen_psi(const Geom gf, const Geom gc, const double *__restrict__ pf, double *__restrict__ pc)
{
    const int ncx = gc.nx - 1, ncy = gc.ny - 1, ncz = gc.dim == 3 ? gc.nz - 1 : 1;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)ncx * ncy * ncz) return;
    const int I = (int)(t % ncx), J = (int)((t / ncx) % ncy), K = (int)(t / ((long long)ncx * ncy));
    double s = 0.0;
    if (gf.dim == 3) {
        for (int a = 0; a < 8; ++a) s += pf[gidx(gf, 2 * I + (a & 1), 2 * J + ((a >> 1) & 1), 2 * K + ((a >> 2) & 1))];
        s *= 0.125;
    } else {
        for (int a = 0; a < 4; ++a) s += pf[gidx(gf, 2 * I + (a & 1), 2 * J + ((a >> 1) & 1), 0)];
        s *= 0.25;
    }
    pc[gidx(gc, I, J, K)] = s;
}

// ------------------------------------------------------------------ copies

template <typename TS, typename TD>
__global__ void k_pack(const Geom g, int ncomp, const TS *__restrict__ packed, TD *__restrict__ lev)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    if (i >= g.nx || j >= g.ny || k >= g.nz) return;
    const long long N = (long long)g.nx * g.ny * g.nz;
    const long long t = i + (long long)g.nx * (j + (long long)g.ny * k), o = gidx(g, i, j, k);
    for (int p = 0; p < ncomp; ++p) lev[p * g.cs + o] = TD(packed[p * N + t]);
}

template <typename TS, typename TD>
__global__ void k_unpack(const Geom g, int ncomp, const TS *__restrict__ lev, TD *__restrict__ packed)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    if (i >= g.nx || j >= g.ny || k >= g.nz) return;
    const long long N = (long long)g.nx * g.ny * g.nz;
    const long long t = i + (long long)g.nx * (j + (long long)g.ny * k), o = gidx(g, i, j, k);
    for (int p = 0; p < ncomp; ++p) packed[p * N + t] = TD(lev[p * g.cs + o]);
}

__device__ __forceinline__ void cell_of(const Geom &g, long long t, int &i, int &j, int &k)
{
    const int ncx = g.nx - 1, ncy = g.ny - 1;
    i = (int)(t % ncx);
    j = (int)((t / ncx) % ncy);
    k = (int)(t / ((long long)ncx * ncy));
}

__host__ __device__ inline long long ncells(const Geom &g)
{
    return (long long)(g.nx - 1) * (g.ny - 1) * (g.dim == 3 ? g.nz - 1 : 1);
}

// psi <- max(psi, psi_min); non-finite inputs are counted in *bad.
__global__ void k_set_psi(const Geom g, const double *__restrict__ in, double psi_min, double *__restrict__ lev,
                          int *bad)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= ncells(g)) return;
    int i, j, k;
    cell_of(g, t, i, j, k);
    const double v = in[t];
    if (!isfinite(v)) atomicAdd(bad, 1);
    lev[gidx(g, i, j, k)] = fmax(v, psi_min);
}

// SIMP map psi = psi_min + (1 - psi_min) rho^q.
__global__ void k_set_density(const Geom g, const double *__restrict__ rho, double psi_min, double q,
                              double *__restrict__ lev, int *bad)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= ncells(g)) return;
    int i, j, k;
    cell_of(g, t, i, j, k);
    const double r = rho[t];
    if (!isfinite(r) || r < 0.0) atomicAdd(bad, 1);
    const double rq = (q == 3.0) ? r * r * r : pow(r, q);
    lev[gidx(g, i, j, k)] = psi_min + (1.0 - psi_min) * rq;
}

__global__ void k_get_cells(const Geom g, const double *__restrict__ lev, double *__restrict__ out)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= ncells(g)) return;
    int i, j, k;
    cell_of(g, t, i, j, k);
    out[t] = lev[gidx(g, i, j, k)];
}

__global__ void k_round_cells(const Geom g, const double *__restrict__ src, float *__restrict__ dst)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= ncells(g)) return;
    int i, j, k;
    cell_of(g, t, i, j, k);
    const long long o = gidx(g, i, j, k);
    dst[o] = float(src[o]);
}

__global__ void k_set_face(const Geom g, int face, int comp, double value, double *u)
{
    const int axis = face >> 1;
    const int n0 = axis == 0 ? g.ny : g.nx;
    const int n1 = axis == 2 ? g.ny : g.nz;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)n0 * n1) return;
    const int a = (int)(t % n0), b = (int)(t / n0);
    int i, j, k;
    if (axis == 0) { i = (face & 1) ? g.nx - 1 : 0; j = a; k = b; }
    else if (axis == 1) { j = (face & 1) ? g.ny - 1 : 0; i = a; k = b; }
    else { k = (face & 1) ? g.nz - 1 : 0; i = a; j = b; }
    u[comp * g.cs + gidx(g, i, j, k)] = value;
}

template <typename TE>
__global__ void k_add(long long n, const TE *__restrict__ e, double *__restrict__ u)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < n) u[t] += double(e[t]);
}

__global__ void k_round(long long n, const double *__restrict__ src, float *__restrict__ dst)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < n) dst[t] = float(src[t]);
}

// ------------------------------------------------------------------- norms

// scal[which] = sum of part[0..n) in a fixed order (one block, 256 threads);
// scal[which+1] = sqrt(scal[which]); when which == 2 also scal[4] = relres =
// sqrt(scal[2]) / scal[1] (scal[1] holds ||r0||).
__global__ void k_norm_final(const double *__restrict__ part, int n, double *scal, int which)
{
    __shared__ double red[kThreads];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += kThreads) s += part[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double ss = red[0];
        scal[which] = ss;
        scal[which + 1] = sqrt(ss);
        if (which == 2) scal[4] = (scal[1] > 0.0) ? sqrt(ss) / scal[1] : 0.0;
    }
}

// -------------------------------------------------------------- bottom solve

// Dense K of the coarsest level over packed dofs (p*N + node).  One thread per
// column (q, node m): it applies the cell routine to the unit vector e_(m,q) in
// each of the 2^d cells around m and writes that column in a fixed order, so the
// assembly is deterministic (no atomics).
__global__ void k_bottom_assemble(const Geom g, const double *__restrict__ psi, const Coef<double> c,
                                  double *A)
{
    const int d = g.dim, nc = 1 << d;
    const long long N = (long long)g.nx * g.ny * g.nz, n = N * d;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int q = (int)(t / N);
    int mi, mj, mk;
    node_of(g, t % N, mi, mj, mk);
    for (int b = 0; b < nc; ++b) {          // node m is corner b of cell m - offset(b)
        const int ci = mi - (b & 1), cj = mj - ((b >> 1) & 1), ck = (d == 3) ? mk - ((b >> 2) & 1) : 0;
        if (ci < 0 || cj < 0 || ck < 0 || ci >= g.nx - 1 || cj >= g.ny - 1 || (d == 3 && ck >= g.nz - 1)) continue;
        const double pc = psi[gidx(g, ci, cj, ck)];
        auto pidx = [&](int a) -> long long {
            return (ci + (a & 1)) + (long long)g.nx * ((cj + ((a >> 1) & 1)) + (long long)g.ny * (d == 3 ? ck + ((a >> 2) & 1) : 0));
        };
        if (d == 3) {
            double U[3][8] = {};
            U[q][b] = 1.0;
            cell_forces3<double>(U, pc, c);
            for (int a = 0; a < 8; ++a)
                for (int p = 0; p < 3; ++p) A[(p * N + pidx(a)) * n + t] += U[p][a];
        } else {
            double U[2][4] = {};
            U[q][b] = 1.0;
            cell_forces2<double>(U, pc, c);
            for (int a = 0; a < 4; ++a)
                for (int p = 0; p < 2; ++p) A[(p * N + pidx(a)) * n + t] += U[p][a];
        }
    }
}

// Dirichlet dofs: identity rows and columns (their correction is zero).
__global__ void k_bottom_dirichlet(const Geom g, double *A)
{
    const long long N = (long long)g.nx * g.ny * g.nz, n = N * g.dim;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int p = (int)(t / N);
    int i, j, k;
    node_of(g, t % N, i, j, k);
    if (!is_dir(g, p, i, j, k)) return;
    for (long long m = 0; m < n; ++m) {
        A[t * n + m] = (m == t) ? 1.0 : 0.0;
        A[m * n + t] = (m == t) ? 1.0 : 0.0;
    }
}

// Gauss-Jordan inversion without pivoting (SPD matrix), pivot k:
//   stage 1: tmp[0..n) = row k / a_kk with the pivot entry replaced by 1/a_kk,
//            tmp[n..2n) = column k (the multipliers);
//   stage 2: every row i != k subtracts multiplier_i * tmp; row k becomes tmp.
__global__ void k_gj_stage1(int n, int k, const double *A, double *tmp)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double ip = 1.0 / A[(long long)k * n + k];
    tmp[t] = (t == k) ? ip : A[(long long)k * n + t] * ip;
    tmp[n + t] = A[(long long)t * n + k];
}

__global__ void k_gj_stage2(int n, int k, double *A, const double *tmp)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)n * n) return;
    const int i = (int)(t / n), j = (int)(t % n);
    if (i == k) {
        A[t] = tmp[j];
    } else {
        const double m = tmp[n + i];
        const double akj = (j == k) ? 0.0 : A[t];
        A[t] = ((j == k) ? 0.0 : akj) - m * tmp[j];
    }
}

// u[gather[r]] (+)= sum_c Ainv[r][c] b[gather[c]]: one warp per row.
template <typename T>
__global__ void k_bottom_apply(int n, const T *__restrict__ Ainv, const int *__restrict__ gather,
                               const T *__restrict__ b, T *__restrict__ u, int accumulate)
{
    const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    T s = T(0);
    for (int c = lane; c < n; c += 32) s += Ainv[(long long)row * n + c] * b[gather[c]];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) {
        if (accumulate) u[gather[row]] += s;
        else u[gather[row]] = s;
    }
}

// ----------------------------------------------------------------- gradient

// dJ/dpsi_c = -lambda_c^T S_c u_c, u and lambda packed; optional chain rule:
// density != 0: dJ/drho = dJ/dpsi (1 - psi_min) q rho^(q-1);  density == 0 and
// grho != null: dJ/dpsi_raw = dJ/dpsi where psi_raw > psi_min, else 0.
__global__ void k_dJdpsi(const Geom g, const Coef<double> c, const double *__restrict__ u,
                         const double *__restrict__ lam, double *__restrict__ gout, double *__restrict__ grho,
                         const double *__restrict__ rho, const double *__restrict__ praw, double psi_min,
                         double q, int density)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= ncells(g)) return;
    int ci, cj, ck;
    cell_of(g, t, ci, cj, ck);
    const long long N = (long long)g.nx * g.ny * g.nz;
    double s = 0.0;
    if (g.dim == 3) {
        double U[3][8], L[3][8];
        for (int a = 0; a < 8; ++a) {
            const long long o = (ci + (a & 1)) + (long long)g.nx * ((cj + ((a >> 1) & 1)) + (long long)g.ny * (ck + ((a >> 2) & 1)));
            for (int p = 0; p < 3; ++p) { U[p][a] = u[p * N + o]; L[p][a] = lam[p * N + o]; }
        }
        cell_forces3<double>(U, 1.0, c);
        for (int a = 0; a < 8; ++a)
            for (int p = 0; p < 3; ++p) s += L[p][a] * U[p][a];
    } else {
        double U[2][4], L[2][4];
        for (int a = 0; a < 4; ++a) {
            const long long o = (ci + (a & 1)) + (long long)g.nx * (cj + ((a >> 1) & 1));
            for (int p = 0; p < 2; ++p) { U[p][a] = u[p * N + o]; L[p][a] = lam[p * N + o]; }
        }
        cell_forces2<double>(U, 1.0, c);
        for (int a = 0; a < 4; ++a)
            for (int p = 0; p < 2; ++p) s += L[p][a] * U[p][a];
    }
    const double gv = -s;
    gout[t] = gv;
    if (grho) {
        if (density) {
            const double r = rho[t];
            const double dr = (q == 3.0) ? 3.0 * r * r : q * pow(r, q - 1.0);
            grho[t] = gv * (1.0 - psi_min) * dr;
        } else {
            grho[t] = (praw[t] > psi_min) ? gv : 0.0;
        }
    }
}

}  // namespace

// ------------------------------------------------------------------ launchers

template <typename T>
cudaError_t launch_restrict(const Geom &gf, const Geom &gc, const T *rf, T *fc, cudaStream_t s)
{
    k_restrict<T><<<node_grid(gc), kNodeBlock, 0, s>>>(gf, gc, rf, fc);
    ++g_launches;
    return cudaGetLastError();
}
template cudaError_t launch_restrict<double>(const Geom &, const Geom &, const double *, double *, cudaStream_t);
template cudaError_t launch_restrict<float>(const Geom &, const Geom &, const float *, float *, cudaStream_t);

template <typename T>
cudaError_t launch_prolong_add(const Geom &gf, const Geom &gc, const T *ec, T *uf, cudaStream_t s)
{
    k_prolong_add<T><<<node_grid(gf), kNodeBlock, 0, s>>>(gf, gc, ec, uf);
    ++g_launches;
    return cudaGetLastError();
}
template cudaError_t launch_prolong_add<double>(const Geom &, const Geom &, const double *, double *, cudaStream_t);
template cudaError_t launch_prolong_add<float>(const Geom &, const Geom &, const float *, float *, cudaStream_t);

cudaError_t launch_coarsen_psi(const Geom &gf, const Geom &gc, const double *pf, double *pc, cudaStream_t s)
{
    k_coarsen_psi<<<nblk(ncells(gc)), kThreads, 0, s>>>(gf, gc, pf, pc);
    ++g_launches;
    return cudaGetLastError();
}

template <typename TS, typename TD>
cudaError_t launch_pack(const Geom &g, int ncomp, const TS *packed, TD *lev, cudaStream_t s)
{
    k_pack<TS, TD><<<node_grid(g), kNodeBlock, 0, s>>>(g, ncomp, packed, lev);
    ++g_launches;
    return cudaGetLastError();
}
template cudaError_t launch_pack<double, double>(const Geom &, int, const double *, double *, cudaStream_t);
template cudaError_t launch_pack<double, float>(const Geom &, int, const double *, float *, cudaStream_t);

template <typename TS, typename TD>
cudaError_t launch_unpack(const Geom &g, int ncomp, const TS *lev, TD *packed, cudaStream_t s)
{
    k_unpack<TS, TD><<<node_grid(g), kNodeBlock, 0, s>>>(g, ncomp, lev, packed);
    ++g_launches;
    return cudaGetLastError();
}
template cudaError_t launch_unpack<double, double>(const Geom &, int, const double *, double *, cudaStream_t);
template cudaError_t launch_unpack<float, double>(const Geom &, int, const float *, double *, cudaStream_t);

cudaError_t launch_set_psi(const Geom &g, const double *packed, double psi_min, double *lev, int *bad, cudaStream_t s)
{
    k_set_psi<<<nblk(ncells(g)), kThreads, 0, s>>>(g, packed, psi_min, lev, bad);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_set_density(const Geom &g, const double *rho, double psi_min, double q, double *lev, int *bad,
                               cudaStream_t s)
{
    k_set_density<<<nblk(ncells(g)), kThreads, 0, s>>>(g, rho, psi_min, q, lev, bad);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_get_cells(const Geom &g, const double *lev, double *packed, cudaStream_t s)
{
    k_get_cells<<<nblk(ncells(g)), kThreads, 0, s>>>(g, lev, packed);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_round_cells(const Geom &g, const double *src, float *dst, cudaStream_t s)
{
    k_round_cells<<<nblk(ncells(g)), kThreads, 0, s>>>(g, src, dst);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_set_face(const Geom &g, int face, int comp, double value, double *u, cudaStream_t s)
{
    const int axis = face >> 1;
    const long long n = (long long)(axis == 0 ? g.ny : g.nx) * (axis == 2 ? g.ny : g.nz);
    k_set_face<<<nblk(n), kThreads, 0, s>>>(g, face, comp, value, u);
    ++g_launches;
    return cudaGetLastError();
}

template <typename TE>
cudaError_t launch_add(long long n, const TE *e, double *u, cudaStream_t s)
{
    k_add<TE><<<nblk(n), kThreads, 0, s>>>(n, e, u);
    ++g_launches;
    return cudaGetLastError();
}
template cudaError_t launch_add<float>(long long, const float *, double *, cudaStream_t);
template cudaError_t launch_add<double>(long long, const double *, double *, cudaStream_t);

cudaError_t launch_norm_final(const double *part, int nparts, double *scal, int which, cudaStream_t s)
{
    k_norm_final<<<1, kThreads, 0, s>>>(part, nparts, scal, which);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_bottom_assemble(const Geom &g, const double *psi, const Coef<double> &c, double *A, cudaStream_t s)
{
    const long long n = (long long)g.nx * g.ny * g.nz * g.dim;
    k_bottom_assemble<<<nblk(n, 128), 128, 0, s>>>(g, psi, c, A);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_bottom_dirichlet(const Geom &g, double *A, cudaStream_t s)
{
    const long long n = (long long)g.nx * g.ny * g.nz * g.dim;
    k_bottom_dirichlet<<<nblk(n), kThreads, 0, s>>>(g, A);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_gauss_jordan(int n, double *A, double *tmp, cudaStream_t s)
{
    for (int k = 0; k < n; ++k) {
        k_gj_stage1<<<nblk(n), kThreads, 0, s>>>(n, k, A, tmp);
        k_gj_stage2<<<nblk((long long)n * n), kThreads, 0, s>>>(n, k, A, tmp);
    }
    g_launches += 2LL * n - 1;
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_round(long long n, const double *src, float *dst, cudaStream_t s)
{
    k_round<<<nblk(n), kThreads, 0, s>>>(n, src, dst);
    ++g_launches;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bottom_apply(int n, const T *Ainv, const int *gather, const T *b, T *u, int accumulate,
                                cudaStream_t s)
{
    const int rows_per_block = 8;
    k_bottom_apply<T><<<(n + rows_per_block - 1) / rows_per_block, 32 * rows_per_block, 0, s>>>(n, Ainv, gather, b, u,
                                                                                                accumulate);
    ++g_launches;
    return cudaGetLastError();
}
template cudaError_t launch_bottom_apply<double>(int, const double *, const int *, const double *, double *, int, cudaStream_t);
template cudaError_t launch_bottom_apply<float>(int, const float *, const int *, const float *, float *, int, cudaStream_t);

cudaError_t launch_dJdpsi(const Geom &g, const Coef<double> &c, const double *u, const double *lam, double *g_out,
                          double *grho_out, const double *rho, const double *psi_raw, double psi_min, double q,
                          int density, cudaStream_t s)
{
    k_dJdpsi<<<nblk(ncells(g), 128), 128, 0, s>>>(g, c, u, lam, g_out, grho_out, rho, psi_raw, psi_min, q, density);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace sbm
