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
// traction of the closest point of the boundary).  FP64, packed arrays, one thread
// per node gathering from its cells (no atomics).  This is setup work, run once per
// load: not part of the V-cycle.
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

template <int D>
__global__ void __launch_bounds__(kThr) k_source_terms(const SourceArgs A, const double *__restrict__ psi,
                                                       const double *__restrict__ eps0, const double *__restrict__ b,
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
        if (eps0) {
            double e[D][D];
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
                for (int q = 0; q < D; ++q) e[a][q] = eps0[vslot<D>(a, q) * NC + cid];
            double tr = 0.0;
#pragma unroll
            for (int a = 0; a < D; ++a) tr += e[a][a];
#pragma unroll
            for (int p = 0; p < D; ++p) {
                double s = 0.0;
#pragma unroll
                for (int q = 0; q < D; ++q) {
                    // cubic C: sigma_pp = c11 e_pp + c12 (tr - e_pp), sigma_pq = 2 c44 e_pq
                    const double sig = p == q ? A.c11 * e[p][p] + A.c12 * (tr - e[p][p]) : 2.0 * A.c44 * e[p][q];
                    s += ((c >> q) & 1) ? -sig : sig;
                }
                acc[p] += pc * s;
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
                                const double *eps0, const double *b, const double *t, double *f, cudaStream_t s)
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
    const dim3 grid((unsigned)((N + kThr - 1) / kThr));
    if (dim == 3) k_source_terms<3><<<grid, kThr, 0, s>>>(A, psi, eps0, b, t, f);
    else k_source_terms<2><<<grid, kThr, 0, s>>>(A, psi, eps0, b, t, f);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace sbm
