// k_topopt.cu — the phase-field topology optimisation step of Sec. 3.3 on the GPU.
// The order parameter eta lives in cells, the stiffness is psi = (eta + zeta)^2, and
// one explicit Euler step of eq. topop_evolution is
//     eta' = eta - dt L [ 2 alpha eta (1-eta)(1-2eta) - beta Lap(eta) - (eta+zeta) e_c
//                         + lambda (V(eta) - V0) ],
// the variational derivative of eq. topop_objective with the elastic part read as
// half the compliance (its eta-derivative at the equilibrium u is -(eta+zeta) e_c,
// e_c = u_c^T S_c u_c the unit-psi strain energy of the cell) and the volume
// constraint of eq. topop_volume_constraint as a penalty.  Lap is the (2d+1)-point
// cell Laplacian with eta's Neumann condition (a missing neighbour takes the cell's
// own value), V = h^d sum_c eta_c.
//
// One thread per cell: eta and its 2d face neighbours, u at the 2^d corner nodes
// (d components, packed), the cell's force vector S_c u_c from the sum-factorised
// cell routine of the operator, and the update.  The kernel also writes the next
// stiffness (eta' + zeta)^2 and per-block partial sums of eta' (the next volume)
// and of psi_c e_c (the compliance u^T K u h^d of the solve that produced u), each
// summed in a fixed order so that results do not depend on scheduling.  FP64.
#include "sbm_common.cuh"

namespace sbm {

namespace {

constexpr int kThr = 256;

template <int D>
__global__ void __launch_bounds__(kThr) k_topopt_step(const TopoptArgs A, const Coef<double> c,
                                                      const double *__restrict__ eta, const double *__restrict__ u,
                                                      const double *__restrict__ psi_solve,
                                                      const double *__restrict__ eta_sum, double *__restrict__ eta_out,
                                                      double *__restrict__ psi_next, double *__restrict__ part)
{
    __shared__ double red[2][kThr];
    const int mx = A.nx - 1, my = A.ny - 1, mz = D == 3 ? A.nz - 1 : 1;
    const int NC = mx * my * mz;               // node and cell indices < 2^31 (checked by the launcher)
    const int t = blockIdx.x * kThr + threadIdx.x;
    double s_eta = 0.0, s_J = 0.0;
    if (t < NC) {
        const int mxy = mx * my;
        const int ci = t % mx;
        const int cj = (t % mxy) / mx;
        const int ck = t / mxy;
        const double n = eta[t];
        // Neumann Laplacian: a missing neighbour contributes nothing
        double lap = 0.0;
        lap += (ci + 1 < mx ? eta[t + 1] - n : 0.0) + (ci > 0 ? eta[t - 1] - n : 0.0);
        lap += (cj + 1 < my ? eta[t + mx] - n : 0.0) + (cj > 0 ? eta[t - mx] - n : 0.0);
        if (D == 3) {
            lap += (ck + 1 < mz ? eta[t + mxy] - n : 0.0) + (ck > 0 ? eta[t - mxy] - n : 0.0);
        }
        lap *= A.ih2;
        // unit-psi strain energy of the cell
        const int N = A.nx * A.ny * (D == 3 ? A.nz : 1);
        double e = 0.0;
        if (D == 3) {
            double U[3][8], U0[3][8];
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                const int o = (ci + (a & 1)) + A.nx * ((cj + ((a >> 1) & 1)) + A.ny * (ck + ((a >> 2) & 1)));
#pragma unroll
                for (int p = 0; p < 3; ++p) U0[p][a] = U[p][a] = u[p * N + o];
            }
            cell_forces3<double>(U, 1.0, c);
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int p = 0; p < 3; ++p) e += U0[p][a] * U[p][a];
        } else {
            double U[2][4], U0[2][4];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int o = (ci + (a & 1)) + A.nx * (cj + ((a >> 1) & 1));
#pragma unroll
                for (int p = 0; p < 2; ++p) U0[p][a] = U[p][a] = u[p * N + o];
            }
            cell_forces2<double>(U, 1.0, c);
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int p = 0; p < 2; ++p) e += U0[p][a] * U[p][a];
        }
        const double V = A.hd * eta_sum[0];
        const double dW = 2.0 * A.alpha * n * (1.0 - n) * (1.0 - 2.0 * n) - A.beta * lap - (n + A.zeta) * e;
        const double out = n - A.dtL * (dW + A.lam * (V - A.V0));
        eta_out[t] = out;
        if (psi_next) psi_next[t] = (out + A.zeta) * (out + A.zeta);
        s_eta = out;
        s_J = psi_solve ? psi_solve[(long long)ci + A.psx * cj + A.psy * ck] * e : 0.0;
    }
    red[0][threadIdx.x] = s_eta;
    red[1][threadIdx.x] = s_J;
    __syncthreads();
    for (int w = kThr / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            red[0][threadIdx.x] += red[0][threadIdx.x + w];
            red[1][threadIdx.x] += red[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[blockIdx.x] = red[0][0];
        part[gridDim.x + blockIdx.x] = red[1][0];
    }
}

// Per-block sums of x[0..n) in a fixed order, and (eta + zeta)^2 into psi when
// psi is not null.
__global__ void __launch_bounds__(kThr) k_cell_sum(long long n, const double *__restrict__ x, double zeta,
                                                   double *__restrict__ psi, double *__restrict__ part)
{
    __shared__ double red[kThr];
    const long long t = (long long)blockIdx.x * kThr + threadIdx.x;
    double v = 0.0;
    if (t < n) {
        v = x[t];
        if (psi) psi[t] = (v + zeta) * (v + zeta);
    }
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = kThr / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

}  // namespace

int topopt_blocks(long long ncells) { return (int)((ncells + kThr - 1) / kThr); }

cudaError_t launch_topopt_step(int dim, const TopoptArgs &A, const Coef<double> &c, const double *eta,
                               const double *u, const double *psi_solve, const double *eta_sum, double *eta_out,
                               double *psi_next, double *part, cudaStream_t s)
{
    const long long NC = (long long)(A.nx - 1) * (A.ny - 1) * (dim == 3 ? A.nz - 1 : 1);
    const long long NN = (long long)A.nx * A.ny * (dim == 3 ? A.nz : 1);
    if (NN * dim >= (1ll << 31)) return cudaErrorInvalidValue;               // 32-bit indexing
    const dim3 grid((unsigned)topopt_blocks(NC));
    if (dim == 3)
        k_topopt_step<3><<<grid, kThr, 0, s>>>(A, c, eta, u, psi_solve, eta_sum, eta_out, psi_next, part);
    else
        k_topopt_step<2><<<grid, kThr, 0, s>>>(A, c, eta, u, psi_solve, eta_sum, eta_out, psi_next, part);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_cell_sum(long long n, const double *x, double zeta, double *psi, double *part, cudaStream_t s)
{
    k_cell_sum<<<topopt_blocks(n), kThr, 0, s>>>(n, x, zeta, psi, part);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace sbm
