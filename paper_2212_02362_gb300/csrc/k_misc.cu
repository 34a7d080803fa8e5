// k_misc.cu — level transfers (full-weighting restriction, linear prolongation,
// psi coarsening), packed <-> level copies, the deterministic norm reduction,
// the coarsest-level dense solve (assembly, Gauss-Jordan inverse, matvec), the
// FP64 defect update and the dJ/dpsi gradient kernel.
#include <algorithm>

#include "sbm_common.cuh"
#include "sbm_bodies.cuh"

namespace sbm {

thread_local long long g_launches = 0;

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

// zero_uc (may be null): the coarse correction, zeroed at each coarse node (the
// start of the coarse level's cycle).
template <typename T, int D>
__global__ void k_restrict(const Geom gf, const Geom gc, const T *__restrict__ rf, T *__restrict__ fc, const int *gate,
                           T *__restrict__ zero_uc)
{
    pdl_begin();
    if (gate && *gate) return;
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int K = blockIdx.z * blockDim.z + threadIdx.z;
    if (I >= gc.nx || J >= gc.ny || K >= gc.nz) return;
    body::restrict_node<T, D>(gf, gc, rf, fc, I, J, K);
    if (zero_uc) {
        const long long o = gidx(gc, I, J, K);
        for (int p = 0; p < D; ++p) zero_uc[p * gc.cs + o] = T(0);
    }
}

template <typename T, int D>
__global__ void k_prolong_add(const Geom gf, const Geom gc, const T *__restrict__ ec, T *__restrict__ uf,
                              const int *gate)
{
    pdl_begin();
    if (gate && *gate) return;
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int K = blockIdx.z * blockDim.z + threadIdx.z;
    if (I >= gc.nx || J >= gc.ny || K >= gc.nz) return;
    body::prolong_node<T, D>(gf, gc, ec, uf, I, J, K);
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
    pdl_begin();
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < n) u[t] += double(e[t]);
}

// out = a x + b y (+ c z): the vector updates of the adjoint Krylov solver.
__global__ void k_lincomb(long long n, double a, const double *x, double b, const double *y, double c,
                          const double *z, double *out)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= n) return;
    double v = a * x[t] + b * y[t];
    if (z) v += c * z[t];
    out[t] = v;
}

// out[0] = sum of part[0..n) in a fixed order (one block).
__global__ void k_sum_parts(const double *part, int n, double *out)
{
    __shared__ double red[kThreads];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
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
__global__ void k_norm_final(const double *__restrict__ part, int n, double *scal, int which, const int *gate)
{
    pdl_begin();
    if (gate && *gate) return;
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
        if (which == 0 || which == 2) scal[7] = sqrt(ss);     // latest FP64 residual norm
    }
}

__global__ void k_inner_gate(const double *__restrict__ part, int n, const double *scal, double rtol,
                             double tol_frac, int *gate, int *count)
{
    pdl_begin();
    if (*gate) return;
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
        const double rn = sqrt(red[0]);
        const double thr = fmax(rtol * scal[7], tol_frac * scal[1]);
        *count += 1;
        if (rn <= thr) *gate = 1;
    }
}

// Batched FP64 V-cycles: after each V-cycle's residual norm (scal[4] = relres),
// record it in hist[count], count the cycle and set the done flag once relres <=
// tol, relres is not finite or above 1e10, or max_cycles cycles have run; every
// later kernel of the batch sees the flag and returns at once.  state = {done, count}.
__global__ void k_outer_gate(const double *scal, double tol, int max_cycles, double *hist, int *state)
{
    pdl_begin();
    if (state[0]) return;
    const double rel = scal[4];
    const int c = state[1] + 1;
    state[1] = c;
    hist[c] = rel;
    if (!(rel == rel) || rel > 1e10 || rel <= tol || c >= max_cycles) state[0] = 1;
}

// dst <- src (n elements) unless the gate is set.
template <typename T>
__global__ void k_copy_gated(long long n, const T *__restrict__ src, T *__restrict__ dst, const int *gate)
{
    pdl_begin();
    if (gate && *gate) return;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = src[i];
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

// Dirichlet dofs: identity rows and columns (their correction is zero).  One thread
// per matrix entry (t, m): it clears entry (t, m) and (m, t) when dof t is Dirichlet.
__global__ void k_bottom_dirichlet(const Geom g, double *A)
{
    const long long N = (long long)g.nx * g.ny * g.nz, n = N * g.dim;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    const long long t = e / n, m = e % n;
    const int p = (int)(t / N);
    int i, j, k;
    node_of(g, t % N, i, j, k);
    if (!is_dir(g, p, i, j, k)) return;
    A[t * n + m] = (m == t) ? 1.0 : 0.0;
    A[m * n + t] = (m == t) ? 1.0 : 0.0;
}

// Grid barriers of the bottom-level inversion: every wait is bounded (on timeout
// bar[2] is set and the kernel ends).
constexpr long long kGridSpinLimit = 1LL << 22;

// Grid barrier number `phase` (1, 2, ...): every block adds 1 to a counter that is
// never reset during the launch and waits until it reaches nblocks * phase.  One
// atomic per block and plain polling; the wait is bounded (bar[2] set on timeout).
__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned nblocks, unsigned phase, long long limit)
{
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        const unsigned target = nblocks * phase;
        volatile unsigned *cnt = bar;
        long long it = 0;
        while (*cnt < target) {
            if (++it > limit || *(volatile unsigned *)(bar + 2)) {
                atomicExch(bar + 2, 1u);
                ok = 0;
                break;
            }
        }
        __threadfence();
    }
    return __syncthreads_and(ok) != 0;
}

// In-place inversion of the dense bottom matrix (SPD, Dirichlet rows and columns
// replaced by the identity) by block Gauss-Jordan: pivot blocks P of kGJB consecutive
// indices, each pass
//     A_PP <- A_PP^-1,  A_PQ <- A_PP^-1 A_PQ,  A_QP <- -A_QP A_PP^-1,
//     A_QQ <- A_QQ - A_QP A_PP^-1 A_PQ          (Q = the other indices),
// after the last pass A holds the inverse.  The principal blocks of an SPD matrix are
// SPD, so no pivoting is needed.  One cooperative launch; each block owns rows
// i = blockIdx.x + m gridDim.x; the pivot rows and columns of the next pass are
// written to a double-buffered exchange area during the current pass, so one grid
// barrier per pass (ceil(n / kGJB) of them) orders the passes.
constexpr int kGJB = 16;

__global__ void k_gauss_jordan(const Geom g, int n, double *A, double *tmp, unsigned *bar, int in_smem,
                               long long limit)
{
    (void)g;
    // dynamic shared memory: the kGJB pivot rows of the current pass (rs; in_smem bit 1,
    // else they are read from the exchange buffer in L2), then, when in_smem bit 0, the
    // block's rows (blockIdx.x + m gridDim.x)
    extern __shared__ double smem_gj[];
    const bool piv_smem = (in_smem & 2) != 0;
    in_smem &= 1;
    double *srow = smem_gj + (piv_smem ? (long long)kGJB * n : 0);
    __shared__ double Pinv[kGJB][kGJB + 1];
    __shared__ double mrow[kGJB];
    const unsigned nb = gridDim.x;
    const long long xb = 2LL * kGJB * n;          // one exchange buffer: kGJB rows + kGJB columns
    if (in_smem)
        for (int i = blockIdx.x, m = 0; i < n; i += gridDim.x, ++m)
            for (int j = threadIdx.x; j < n; j += blockDim.x) srow[(long long)m * n + j] = A[(long long)i * n + j];
    // buffer 0 <- pivot rows R[r][j] = A[r][j] and columns C[i][r] = A[i][r] of block 0
    {
        const int b0 = min(kGJB, n);
        for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)b0 * n;
             t += (long long)gridDim.x * blockDim.x) {
            const int r = (int)(t / n), j = (int)(t % n);
            tmp[(long long)r * n + j] = A[(long long)r * n + j];
            tmp[(long long)kGJB * n + (long long)j * kGJB + r] = A[(long long)j * n + r];
        }
    }
    unsigned phase = 1;
    if (!grid_barrier(bar, nb, phase++, limit)) return;
    int cur = 0;
    for (int k0 = 0; k0 < n; k0 += kGJB) {
        const int b = min(kGJB, n - k0);
        const int k1 = k0 + kGJB, bn = min(kGJB, n - k1);      // the next pivot block (bn <= 0: none)
        const double *R = tmp + cur * xb, *Cc = R + (long long)kGJB * n;
        double *Rn = tmp + (1 - cur) * xb, *Cn = Rn + (long long)kGJB * n;
        // Pinv = inverse of the pivot block (Gauss-Jordan on kGJB x kGJB in shared memory,
        // one element per thread); the pivot rows were written by other blocks: read them
        // from L2 into shared memory once per pass
        for (int t = threadIdx.x; t < kGJB * kGJB; t += blockDim.x) {
            const int r = t / kGJB, c = t % kGJB;
            Pinv[r][c] = (r < b && c < b) ? __ldcg(R + (long long)r * n + k0 + c) : (r == c ? 1.0 : 0.0);
        }
        if (piv_smem)
            for (int t = threadIdx.x; t < b * n; t += blockDim.x) smem_gj[t] = __ldcg(R + t);
        // the exchange buffers alternate between passes: reads of them bypass L1
        auto rget = [&](long long idx) -> double { return piv_smem ? smem_gj[idx] : __ldcg(R + idx); };
        __syncthreads();
        for (int q = 0; q < kGJB; ++q) {
            double v = 0.0;
            const int t = threadIdx.x, r = t / kGJB, c = t % kGJB;
            if (t < kGJB * kGJB) {
                const double ip = 1.0 / Pinv[q][q];
                const double pqc = (c == q) ? ip : Pinv[q][c] * ip;
                v = (r == q) ? pqc : ((c == q) ? 0.0 : Pinv[r][c]) - Pinv[r][q] * pqc;
            }
            __syncthreads();
            if (t < kGJB * kGJB) Pinv[r][c] = v;
            __syncthreads();
        }
        for (int i = blockIdx.x, ri = 0; i < n; i += gridDim.x, ++ri) {
            double *row = in_smem ? srow + (long long)ri * n : A + (long long)i * n;
            const bool inP = i >= k0 && i < k0 + b;
            // m_i = A_iP Pinv (rows outside P), or the row of Pinv (rows inside P)
            if (threadIdx.x < kGJB) {
                const int c = threadIdx.x;
                double acc = 0.0;
                if (inP) {
                    acc = Pinv[i - k0][c];
                } else {
                    for (int r = 0; r < b; ++r) acc += __ldcg(Cc + (long long)i * kGJB + r) * Pinv[r][c];
                }
                mrow[c] = (c < b) ? acc : 0.0;
            }
            __syncthreads();
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                const bool jP = j >= k0 && j < k0 + b;
                double v;
                if (inP) {
                    if (jP) {
                        v = Pinv[i - k0][j - k0];
                    } else {
                        v = 0.0;
                        for (int c = 0; c < b; ++c) v += mrow[c] * rget((long long)c * n + j);
                    }
                } else {
                    if (jP) {
                        v = -mrow[j - k0];
                    } else {
                        v = row[j];
                        for (int c = 0; c < b; ++c) v -= mrow[c] * rget((long long)c * n + j);
                    }
                }
                row[j] = v;
                if (bn > 0 && i >= k1 && i < k1 + bn) Rn[(long long)(i - k1) * n + j] = v;
                if (bn > 0 && j >= k1 && j < k1 + bn) Cn[(long long)i * kGJB + (j - k1)] = v;
            }
            __syncthreads();
        }
        if (!grid_barrier(bar, nb, phase++, limit)) return;
        cur ^= 1;
    }
    if (in_smem)
        for (int i = blockIdx.x, m = 0; i < n; i += gridDim.x, ++m)
            for (int j = threadIdx.x; j < n; j += blockDim.x) A[(long long)i * n + j] = srow[(long long)m * n + j];
}

// u[gather[r]] (+)= sum_c Ainv[r][c] b[gather[c]]: one warp per row.
template <typename T>
__global__ void k_bottom_apply(int n, const T *__restrict__ Ainv, const int *__restrict__ gather,
                               const T *__restrict__ b, T *__restrict__ u, int accumulate, const int *gate)
{
    pdl_begin();
    if (gate && *gate) return;
    const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (row >= n) return;
    body::bottom_row<T>(n, Ainv, gather, b, u, accumulate, row, threadIdx.x & 31);
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
cudaError_t launch_restrict(const Geom &gf, const Geom &gc, const T *rf, T *fc, cudaStream_t s, const int *gate,
                            T *zero_uc)
{
    cudaError_t e = gf.dim == 3 ? launch_pdl(k_restrict<T, 3>, node_grid(gc), kNodeBlock, 0, s, gf, gc, rf, fc, gate, zero_uc)
                                : launch_pdl(k_restrict<T, 2>, node_grid(gc), kNodeBlock, 0, s, gf, gc, rf, fc, gate, zero_uc);
    if (e != cudaSuccess) return e;
    ++g_launches;
    return cudaGetLastError();
}
template cudaError_t launch_restrict<double>(const Geom &, const Geom &, const double *, double *, cudaStream_t,
                                             const int *, double *);
template cudaError_t launch_restrict<float>(const Geom &, const Geom &, const float *, float *, cudaStream_t, const int *,
                                            float *);

template <typename T>
cudaError_t launch_prolong_add(const Geom &gf, const Geom &gc, const T *ec, T *uf, cudaStream_t s, const int *gate)
{
    cudaError_t e = gf.dim == 3 ? launch_pdl(k_prolong_add<T, 3>, node_grid(gc), kNodeBlock, 0, s, gf, gc, ec, uf, gate)
                                : launch_pdl(k_prolong_add<T, 2>, node_grid(gc), kNodeBlock, 0, s, gf, gc, ec, uf, gate);
    if (e != cudaSuccess) return e;
    ++g_launches;
    return cudaGetLastError();
}
template cudaError_t launch_prolong_add<double>(const Geom &, const Geom &, const double *, double *, cudaStream_t,
                                                const int *);
template cudaError_t launch_prolong_add<float>(const Geom &, const Geom &, const float *, float *, cudaStream_t,
                                               const int *);

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
    cudaError_t err = launch_pdl(k_add<TE>, dim3(nblk(n)), dim3(kThreads), 0, s, n, e, u);
    if (err != cudaSuccess) return err;
    ++g_launches;
    return cudaGetLastError();
}
template cudaError_t launch_add<float>(long long, const float *, double *, cudaStream_t);
template cudaError_t launch_add<double>(long long, const double *, double *, cudaStream_t);

cudaError_t launch_norm_final(const double *part, int nparts, double *scal, int which, cudaStream_t s,
                              const int *gate)
{
    cudaError_t e = launch_pdl(k_norm_final, dim3(1), dim3(kThreads), 0, s, part, nparts, scal, which, gate);
    if (e != cudaSuccess) return e;
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_outer_gate(const double *scal, double tol, int max_cycles, double *hist, int *state, cudaStream_t s)
{
    cudaError_t e = launch_pdl(k_outer_gate, dim3(1), dim3(1), 0, s, scal, tol, max_cycles, hist, state);
    if (e != cudaSuccess) return e;
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_copy_gated(long long n, const double *src, double *dst, const int *gate, cudaStream_t s)
{
    cudaError_t e = launch_pdl(k_copy_gated<double>, dim3((unsigned)std::min<long long>(nblk(n), 152 * 8)), dim3(kThreads),
                               0, s, n, src, dst, gate);
    if (e != cudaSuccess) return e;
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_inner_gate(const double *part, int nparts, const double *scal, double rtol, double tol_frac,
                              int *gate, int *count, cudaStream_t s)
{
    cudaError_t e = launch_pdl(k_inner_gate, dim3(1), dim3(kThreads), 0, s, part, nparts, scal, rtol, tol_frac, gate, count);
    if (e != cudaSuccess) return e;
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_bottom_assemble(const Geom &g, const double *psi, const Coef<double> &c, double *A, cudaStream_t s)
{
    const long long n = (long long)g.nx * g.ny * g.nz * g.dim;
    k_bottom_assemble<<<nblk(n, 32), 32, 0, s>>>(g, psi, c, A);      // a column per thread, spread over SMs
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_bottom_dirichlet(const Geom &g, double *A, cudaStream_t s)
{
    const long long n = (long long)g.nx * g.ny * g.nz * g.dim;
    k_bottom_dirichlet<<<nblk((long long)n * n), kThreads, 0, s>>>(g, A);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_gauss_jordan(const Geom &g, int n, double *A, double *tmp, unsigned *bar, long long spins,
                                cudaStream_t s)
{
    int dev = 0, nsm = 0, per_sm = 0, coop = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e != cudaSuccess) return e;
    int nblocks = nsm;                      // one block per SM, all co-resident
    if (nblocks > n) nblocks = n;
    // the rows of each block in shared memory when they fit
    const size_t rows_bytes = (size_t)((n + nblocks - 1) / nblocks) * n * sizeof(double);
    const size_t pivot_bytes = (size_t)kGJB * n * sizeof(double);
    const bool piv = pivot_bytes <= 160 * 1024;                 // the pivot rows in shared memory
    const bool rows = (piv ? pivot_bytes : 0) + rows_bytes <= 200 * 1024;
    int in_smem = (rows ? 1 : 0) | (piv ? 2 : 0);
    const size_t smem = (piv ? pivot_bytes : 0) + (rows ? rows_bytes : 0);
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(k_gauss_jordan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gauss_jordan, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (!coop || per_sm < 1) return cudaErrorNotSupported;
    e = cudaMemsetAsync(bar, 0, 4 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    Geom gg = g;
    long long limit = spins > 0 ? spins : kGridSpinLimit;
    void *args[] = {&gg, &n, &A, &tmp, &bar, &in_smem, &limit};
    e = cudaLaunchCooperativeKernel((const void *)k_gauss_jordan, dim3(nblocks), dim3(kThreads), args, smem, s);
    ++g_launches;
    return e;
}

cudaError_t launch_lincomb(long long n, double a, const double *x, double b, const double *y, double c,
                           const double *z, double *out, cudaStream_t s)
{
    k_lincomb<<<nblk(n), kThreads, 0, s>>>(n, a, x, b, y, c, z, out);
    ++g_launches;
    return cudaGetLastError();
}

// Measurement helper: read n4 float4 of a buffer larger than L2 (nothing is
// written unless the impossible sum appears), so that L2 ends up holding clean
// lines of that buffer.
__global__ void k_l2_read(const float4 *__restrict__ a, long long n4, float *sink)
{
    float acc = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
        const float4 v = a[i];
        acc += (v.x + v.y) + (v.z + v.w);
    }
    if (acc == 1234567.f) sink[0] = acc;
}

// FMA throughput probe: every thread runs 8 independent multiply-add chains of
// `iters` steps (2 flops each); the result is stored only under a condition the
// values never meet, so nothing is optimised away.
template <typename T>
__global__ void k_fma_rate(int iters, T a, T b, T *sink)
{
    T x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = T(threadIdx.x + j) * T(1e-3);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = x[j] * a + b;
    T s = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    if (s == T(-1234567)) sink[0] = s;
}

cudaError_t launch_fma_rate(int fp64, int blocks, int threads, int iters, void *sink, cudaStream_t s)
{
    if (fp64) k_fma_rate<double><<<blocks, threads, 0, s>>>(iters, 0.999999, 1e-7, static_cast<double *>(sink));
    else k_fma_rate<float><<<blocks, threads, 0, s>>>(iters, 0.9999f, 1e-4f, static_cast<float *>(sink));
    return cudaGetLastError();
}

cudaError_t launch_l2_read(const void *buf, size_t bytes, float *sink, cudaStream_t s)
{
    k_l2_read<<<152 * 8, 256, 0, s>>>(static_cast<const float4 *>(buf), (long long)(bytes / 16), sink);
    return cudaGetLastError();
}

cudaError_t launch_sum_parts(const double *part, int n, double *out, cudaStream_t s)
{
    k_sum_parts<<<1, kThreads, 0, s>>>(part, n, out);
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
                                cudaStream_t s, const int *gate)
{
    const int rows_per_block = 8;
    cudaError_t e = launch_pdl(k_bottom_apply<T>, dim3((n + rows_per_block - 1) / rows_per_block),
                               dim3(32 * rows_per_block), 0, s, n, Ainv, gather, b, u, accumulate, gate);
    if (e != cudaSuccess) return e;
    ++g_launches;
    return cudaGetLastError();
}
template cudaError_t launch_bottom_apply<double>(int, const double *, const int *, const double *, double *, int, cudaStream_t,
                                                 const int *);
template cudaError_t launch_bottom_apply<float>(int, const float *, const int *, const float *, float *, int, cudaStream_t,
                                                const int *);

cudaError_t launch_dJdpsi(const Geom &g, const Coef<double> &c, const double *u, const double *lam, double *g_out,
                          double *grho_out, const double *rho, const double *psi_raw, double psi_min, double q,
                          int density, cudaStream_t s)
{
    k_dJdpsi<<<nblk(ncells(g), 128), 128, 0, s>>>(g, c, u, lam, g_out, grho_out, rho, psi_raw, psi_min, q, density);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace sbm
