// k_variant.cu — the product-rule strong form of Sec. 2.3 on the GPU: the
// literal discretisation of
//     div(psi C grad u) = psi C : grad grad u + grad psi . C grad u
// at interior nodes by centred differences (3-point second differences, 4-point
// mixed differences), with psi either at nodes (the node-placed operator whose
// Jacobi update Sec. 2.3 shows to diverge where psi vanishes) or in cells averaged
// to the node (the cell-placed update, which in 1D is the conservative flux form).
// These are the paper's operator variants, used to compare with the cell-flux
// operator of the solver; they are defined at interior nodes only (rows on the box
// faces are 0 and a Jacobi sweep leaves face values unchanged).  FP64, packed
// arrays (node (i,j,k), component p at p*N + i + nx*(j + ny*k)), one thread per node.
#include "sbm_common.cuh"

namespace sbm {

namespace {

constexpr int kThr = 256;

struct ProductArgs {
    int nx, ny, nz;
    double h;
    double c11, c12, c44;
    unsigned dm[3];        // Dirichlet faces per component (Jacobi leaves those dofs alone)
    int variant;           // 1 = psi at nodes, 2 = psi in cells
    double omega;
};

// Axis-aligned cubic stiffness C_{p a q b}.
__device__ __forceinline__ double cubic(const ProductArgs &A, int p, int a, int q, int b)
{
    if (p == a && q == b) return p == q ? A.c11 : A.c12;
    if (p != a && ((p == q && a == b) || (p == b && a == q))) return A.c44;
    return 0.0;
}

template <int D>
__device__ __forceinline__ void psi_at(const ProductArgs &A, const double *psi, int i, int j, int k, double &pn,
                                       double (&g)[3])
{
    const long long N = (long long)A.nx * A.ny * A.nz;
    (void)N;
    g[0] = g[1] = g[2] = 0.0;
    if (A.variant == 1) {
        const long long n = i + (long long)A.nx * (j + (long long)A.ny * k);
        pn = psi[n];
        g[0] = (psi[n + 1] - psi[n - 1]) / (2.0 * A.h);
        g[1] = (psi[n + A.nx] - psi[n - A.nx]) / (2.0 * A.h);
        if (D == 3) g[2] = (psi[n + (long long)A.nx * A.ny] - psi[n - (long long)A.nx * A.ny]) / (2.0 * A.h);
        return;
    }
    // cells: (nx-1)(ny-1)(nz-1) packed; the 2^D cells around node (i,j,k) have lower
    // corners (i-1+bx, j-1+by, k-1+bz)
    const int cx = A.nx - 1, cy = A.ny - 1;
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < (1 << D); ++c) {
        const int ci = i - 1 + (c & 1), cj = j - 1 + ((c >> 1) & 1), ck = D == 3 ? k - 1 + ((c >> 2) & 1) : 0;
        const double v = psi[ci + (long long)cx * (cj + (long long)cy * ck)];
        s += v;
        g[0] += (c & 1) ? v : -v;
        g[1] += ((c >> 1) & 1) ? v : -v;
        if (D == 3) g[2] += ((c >> 2) & 1) ? v : -v;
    }
    pn = s / (1 << D);
    const double sc = 1.0 / ((1 << (D - 1)) * A.h);
    g[0] *= sc;
    g[1] *= sc;
    g[2] *= sc;
}

// MODE 0: out = K u (interior rows; 0 on the faces).  MODE 1: one damped Jacobi
// sweep, out = u + omega (f - K u) / diag(K) on interior free dofs, u elsewhere.
template <int D, int MODE>
__global__ void __launch_bounds__(kThr) k_product(const ProductArgs A, const double *__restrict__ psi,
                                                  const double *__restrict__ u, const double *__restrict__ f,
                                                  double *__restrict__ out)
{
    const long long N = (long long)A.nx * A.ny * A.nz;
    const long long n = (long long)blockIdx.x * kThr + threadIdx.x;
    if (n >= N) return;
    const int i = (int)(n % A.nx);
    const int j = (int)((n / A.nx) % A.ny);
    const int k = (int)(n / ((long long)A.nx * A.ny));
    const bool interior = i > 0 && i < A.nx - 1 && j > 0 && j < A.ny - 1 && (D == 2 || (k > 0 && k < A.nz - 1));
    if (!interior) {
#pragma unroll
        for (int p = 0; p < D; ++p) out[p * N + n] = MODE == 0 ? 0.0 : u[p * N + n];
        return;
    }
    double pn, g[3];
    psi_at<D>(A, psi, i, j, k, pn, g);
    const long long st[3] = {1, A.nx, (long long)A.nx * A.ny};
    const double h = A.h, i2h = 1.0 / (2.0 * h), ih2 = 1.0 / (h * h), i4h2 = 1.0 / (4.0 * h * h);
    double Dq[3][3], H[3][3][3];
#pragma unroll
    for (int q = 0; q < D; ++q) {
        const double *uq = u + q * N;
        const double c = uq[n];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const double vu = uq[n + st[a]], vd = uq[n - st[a]];
            Dq[a][q] = (vu - vd) * i2h;
            H[a][a][q] = (vu - 2.0 * c + vd) * ih2;
#pragma unroll
            for (int b = a + 1; b < D; ++b) {
                const double x = (uq[n + st[a] + st[b]] - uq[n + st[a] - st[b]] - uq[n - st[a] + st[b]] +
                                  uq[n - st[a] - st[b]]) * i4h2;
                H[a][b][q] = x;
                H[b][a][q] = x;
            }
        }
    }
#pragma unroll
    for (int p = 0; p < D; ++p) {
        double s = 0.0, dg = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
#pragma unroll
            for (int q = 0; q < D; ++q)
#pragma unroll
                for (int b = 0; b < D; ++b) {
                    const double Cv = cubic(A, p, a, q, b);
                    s += Cv * (pn * H[a][b][q] + g[a] * Dq[b][q]);
                }
            dg += cubic(A, p, a, p, a) * 2.0 * ih2;
        }
        const double Ku = -s;
        if (MODE == 0) {
            out[p * N + n] = Ku;
        } else {
            const unsigned m = A.dm[p];
            const bool dir = ((m & 1u) && i == 0) || ((m & 2u) && i == A.nx - 1) || ((m & 4u) && j == 0) ||
                             ((m & 8u) && j == A.ny - 1) || ((m & 16u) && k == 0) || ((m & 32u) && k == A.nz - 1);
            const double uv = u[p * N + n];
            out[p * N + n] = dir ? uv : uv + A.omega * (f[p * N + n] - Ku) / (pn * dg);
        }
    }
}

template <int MODE>
cudaError_t launch_product_mode(const ProductArgs &A, int dim, const double *psi, const double *u, const double *f,
                                double *out, cudaStream_t s)
{
    const long long N = (long long)A.nx * A.ny * A.nz;
    const dim3 grid((unsigned)((N + kThr - 1) / kThr));
    if (dim == 3) k_product<3, MODE><<<grid, kThr, 0, s>>>(A, psi, u, f, out);
    else k_product<2, MODE><<<grid, kThr, 0, s>>>(A, psi, u, f, out);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_product(int mode, int dim, const int n[3], double h, const double mod[3], const unsigned dm[3],
                           int variant, double omega, const double *psi, const double *u, const double *f, double *out,
                           cudaStream_t s)
{
    ProductArgs A;
    A.nx = n[0];
    A.ny = n[1];
    A.nz = dim == 3 ? n[2] : 1;
    A.h = h;
    A.c11 = mod[0];
    A.c12 = mod[1];
    A.c44 = mod[2];
    for (int p = 0; p < 3; ++p) A.dm[p] = dm[p];
    A.variant = variant;
    A.omega = omega;
    if (variant != 1 && variant != 2) return cudaErrorInvalidValue;
    return mode == 0 ? launch_product_mode<0>(A, dim, psi, u, f, out, s)
                     : launch_product_mode<1>(A, dim, psi, u, f, out, s);
}

}  // namespace sbm
