// k_source.cu — the source terms of eq. SBMLinearElasticity (Sec. 2.1),
//     div(psi C (grad u - eps0)) - psi b = t |grad psi|,
// brought to the form K u = f of the cell-flux operator:
//     f_n = h^-d sum_{cells c of n} psi_c int_c B_n^T C eps0_c  -  w_n (psi_n b_n + t_n |grad psi|_n).
// For an eigenstrain that is constant in each cell the cell integral is closed form:
// int_c dN_n/dx_q = s_q h^(d-1) / 2^(d-1), s_q = +1 when the cell lies below the node
// along q, -1 above, so the eigenstrain load is sum_c sum_q s_q (psi_c C eps0_c)_pq /
// (2^(d-1) h).  psi_n is the mean of the 2^d cells around the node, the gradient along
// a the mean of (psi_+ - psi_-) / h over the cell pairs facing each other across the
// node; cells beyond a face of the box take the value of their mirror image (no
// normal gradient at the box), and w_n = (cells of the grid around n) / 2^d is the
// node's share of the volume.  The diffuse traction t is given at the nodes (the
// traction of the closest point of the boundary).  FP64, packed arrays; a cell pass
// forms each cell's eigenstrain stress once, then one thread per node gathers from
// its cells (no atomics).  This is setup work, run once per load: not part of the
// V-cycle.
#include "sbm_common.cuh"

namespace sbm {

namespace {

constexpr int kThr = 256;

struct SourceArgs {
    int nx, ny, nz;
    double inv;            // 1 / (2^(d-1) h)
    double c11, c12, c44;
};

// Voigt slot of the symmetric pair (a, b): 2D (xx, yy, xy), 3D (xx, yy, zz, yz, xz, xy).
template <int D>
__device__ __forceinline__ int vslot(int a, int b)
{
    if (a == b) return a;
    if (D == 2) return 2;
    return 6 - a - b;        // (1,2) -> 3, (0,2) -> 4, (0,1) -> 5
}

// Pass 1: the eigenstrain stress of every cell, sig_c = psi_c C eps0_c (Voigt slots,
// slot-major like eps0).
template <int D>
__global__ void __launch_bounds__(kThr) k_cell_stress(const SourceArgs A, const double *__restrict__ psi,
                                                      const double *__restrict__ eps0, double *__restrict__ sig)
{
    const int NC = (A.nx - 1) * (A.ny - 1) * (D == 3 ? A.nz - 1 : 1);
    const int c = blockIdx.x * kThr + threadIdx.x;
    if (c >= NC) return;
    double e[D == 3 ? 6 : 3];
#pragma unroll
    for (int v = 0; v < (D == 3 ? 6 : 3); ++v) e[v] = eps0[v * NC + c];
    double tr = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) tr += e[a];
    const double pc = psi[c];
    // cubic C: sigma_pp = c11 e_pp + c12 (tr - e_pp), sigma_pq = 2 c44 e_pq (tensor shear)
#pragma unroll
    for (int a = 0; a < D; ++a) sig[a * NC + c] = pc * (A.c11 * e[a] + A.c12 * (tr - e[a]));
#pragma unroll
    for (int v = D; v < (D == 3 ? 6 : 3); ++v) sig[v * NC + c] = pc * (2.0 * A.c44 * e[v]);
}

// Pass 2 (or the only pass without eigenstrain): one thread per node gathering its
// 2^d cells: the eigenstrain load sum_c sum_q s_q sig_pq(c) / (2^(d-1) h) from the
// cell stresses, psi_n, |grad psi|_n and the volume share for the body force and
// the traction.
template <int D>
__global__ void __launch_bounds__(kThr) k_source_terms(const SourceArgs A, const double *__restrict__ psi,
                                                       const double *__restrict__ sig, const double *__restrict__ b,
                                                       const double *__restrict__ t, double *__restrict__ f)
{
    const int N = A.nx * A.ny * A.nz;          // < 2^31 (checked by the launcher)
    const int n = blockIdx.x * kThr + threadIdx.x;
    if (n >= N) return;
    const int nxy = A.nx * A.ny;
    const int nd[3] = {n % A.nx, (n % nxy) / A.nx, n / nxy};
    const int mc[3] = {A.nx - 1, A.ny - 1, D == 3 ? A.nz - 1 : 1};
    const int NC = mc[0] * mc[1] * mc[2];
    double acc[3] = {0.0, 0.0, 0.0};
    double ps = 0.0, g[3] = {0.0, 0.0, 0.0};
    int inside = 0;
#pragma unroll
    for (int c = 0; c < (1 << D); ++c) {
        int cc[3] = {0, 0, 0};
        bool in = true;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            int v = nd[a] - 1 + ((c >> a) & 1);
            if (v < 0 || v >= mc[a]) in = false;
            cc[a] = min(max(v, 0), mc[a] - 1);
        }
        const int cid = cc[0] + mc[0] * (cc[1] + mc[1] * cc[2]);
        const double pc = psi[cid];
        ps += pc;
#pragma unroll
        for (int a = 0; a < D; ++a) g[a] += ((c >> a) & 1) ? pc : -pc;
        if (!in) continue;
        ++inside;
        if (sig) {
            // s_q = +1 when the cell lies below the node along q (bit clear), -1 above
#pragma unroll
            for (int p = 0; p < D; ++p)
#pragma unroll
                for (int q = 0; q < D; ++q) {
                    const double v = sig[vslot<D>(p, q) * NC + cid];
                    acc[p] += ((c >> q) & 1) ? -v : v;
                }
        }
    }
    const double inv = A.inv;
    const double pn = ps * (1.0 / (1 << D));
    double gg = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) gg += (g[a] * inv) * (g[a] * inv);
    const double gn = sqrt(gg);
    const double w = (double)inside * (1.0 / (1 << D));
#pragma unroll
    for (int p = 0; p < D; ++p) {
        double s = 0.0;
        if (b) s += pn * b[p * N + n];
        if (t) s += t[p * N + n] * gn;
        f[p * N + n] = acc[p] * inv - w * s;
    }
}

}  // namespace

cudaError_t launch_source_terms(int dim, const int n[3], double h, const double mod[3], const double *psi,
                                const double *eps0, const double *b, const double *t, double *f, double *sig,
                                cudaStream_t s)
{
    SourceArgs A;
    A.nx = n[0];
    A.ny = n[1];
    A.nz = dim == 3 ? n[2] : 1;
    A.inv = 1.0 / ((dim == 3 ? 4.0 : 2.0) * h);
    A.c11 = mod[0];
    A.c12 = mod[1];
    A.c44 = mod[2];
    const long long N = (long long)A.nx * A.ny * A.nz;
    if (N * (dim == 3 ? 6 : 3) >= (1ll << 31)) return cudaErrorInvalidValue;   // 32-bit indexing
    const long long NC = (long long)(A.nx - 1) * (A.ny - 1) * (dim == 3 ? A.nz - 1 : 1);
    if (eps0) {
        if (!sig) return cudaErrorInvalidValue;
        const dim3 cgrid((unsigned)((NC + kThr - 1) / kThr));
        if (dim == 3) k_cell_stress<3><<<cgrid, kThr, 0, s>>>(A, psi, eps0, sig);
        else k_cell_stress<2><<<cgrid, kThr, 0, s>>>(A, psi, eps0, sig);
        ++g_launches;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const dim3 grid((unsigned)((N + kThr - 1) / kThr));
    if (dim == 3) k_source_terms<3><<<grid, kThr, 0, s>>>(A, psi, eps0 ? sig : nullptr, b, t, f);
    else k_source_terms<2><<<grid, kThr, 0, s>>>(A, psi, eps0 ? sig : nullptr, b, t, f);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace sbm
