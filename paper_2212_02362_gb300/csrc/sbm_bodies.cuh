// sbm_bodies.cuh — per-element device bodies of the stencil and transfer kernels:
// the sweep finalisation (damped Jacobi / residual / apply at one node), one cell
// of the cell-parallel FP32 3D sweep of small levels, full-weighting restriction
// and linear prolongation at one coarse node, and one row of the coarsest-level
// dense matvec.
#pragma once

#include "sbm_common.cuh"

namespace sbm {
namespace body {

template <typename T, typename TO, int MODE>
__device__ __forceinline__ void finalize(const SweepArgs<T, TO> &a, int gx, int gy, int gz, const T *Ku,
                                         T psisum, const T *uval, double &ssq)
{
    const Geom &g = a.g;
    const long long o = gidx(g, gx, gy, gz);
    if (MODE == kJacobi) {
        const T ip = T(1) / psisum;
        for (int p = 0; p < g.dim; ++p) {
            T v = uval[p];
            if (!is_dir(g, p, gx, gy, gz)) v += (a.f[p * g.cs + o] - Ku[p]) * ip * a.wk[p];
            a.out[p * g.cs + o] = TO(v);
        }
    } else if (MODE == kResidual) {
        for (int p = 0; p < g.dim; ++p) {
            T r = is_dir(g, p, gx, gy, gz) ? T(0) : a.f[p * g.cs + o] - Ku[p];
            a.out[p * g.cs + o] = TO(r);
            ssq += double(r) * double(r);
        }
    } else {
        for (int p = 0; p < g.dim; ++p) a.out[p * g.cs + o] = TO(Ku[p]);
    }
}

// finalize with the node's right-hand side already loaded (fv[p] = f[p] at the node).
template <typename T, typename TO, int MODE>
__device__ __forceinline__ void finalize_f(const SweepArgs<T, TO> &a, int gx, int gy, int gz, const T *Ku,
                                           T psisum, const T *uval, const T *fv, double &ssq)
{
    const Geom &g = a.g;
    const long long o = gidx(g, gx, gy, gz);
    if (MODE == kJacobi) {
        const T ip = T(1) / psisum;
        for (int p = 0; p < g.dim; ++p) {
            T v = uval[p];
            if (!is_dir(g, p, gx, gy, gz)) v += (fv[p] - Ku[p]) * ip * a.wk[p];
            a.out[p * g.cs + o] = TO(v);
        }
    } else if (MODE == kResidual) {
        for (int p = 0; p < g.dim; ++p) {
            T r = is_dir(g, p, gx, gy, gz) ? T(0) : fv[p] - Ku[p];
            a.out[p * g.cs + o] = TO(r);
            ssq += double(r) * double(r);
        }
    } else {
        for (int p = 0; p < g.dim; ++p) a.out[p * g.cs + o] = TO(Ku[p]);
    }
}

// Small 3D levels (FP32), one cell of a node's eight: thread c of the node's group
// of eight evaluates the cell of which node (i, j, k) is corner c (bit m = the
// node's offset along axis m within the cell) and returns the force on that
// corner and the cell's psi; cells outside the grid give zeros.
__device__ __forceinline__ void node_cell(const SweepArgs<float, float> &a, int i, int j, int k, int c,
                                          float (&F)[3], float &ps)
{
    const Geom &g = a.g;
    const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
    const int ci = i - cx, cj = j - cy, ck = k - cz;
    F[0] = F[1] = F[2] = 0.f;
    ps = 0.f;
    if (ci < 0 || cj < 0 || ck < 0 || ci >= g.nx - 1 || cj >= g.ny - 1 || ck >= g.nz - 1) return;
    ps = a.psi[gidx(g, ci, cj, ck)];
    float U[3][8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const long long o = gidx(g, ci + (b & 1), cj + ((b >> 1) & 1), ck + (b >> 2));
#pragma unroll
        for (int p = 0; p < 3; ++p) U[p][b] = a.u[p * g.cs + o];
    }
    cell_forces3<float>(U, ps, a.c);
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        float v = U[p][0];
#pragma unroll
        for (int b = 1; b < 8; ++b) v = (c == b) ? U[p][b] : v;
        F[p] = v;
    }
}

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// Fine values x = 2I-1, 2I, 2I+1 of one row, with weights 1/2, 1, 1/2 (missing
// neighbours beyond the row weigh 0).  2I is even and rows start on 8-element
// boundaries, so (2I, 2I+1) is one aligned vector load when 2I+1 is in the row.
template <typename T>
__device__ __forceinline__ T fw_row(const T *__restrict__ row, int I, int nx)
{
    using V = typename Vec2<T>::type;
    const int i = 2 * I;
    const T lo = (i > 0) ? row[i - 1] : T(0);
    T c, hi;
    if (i + 1 < nx) {
        const V v = *reinterpret_cast<const V *>(row + i);
        c = v.x;
        hi = v.y;
    } else {
        c = row[i];
        hi = T(0);
    }
    return c + T(0.5) * (lo + hi);
}

// r_c = P^T r_f / 2^d on free coarse dofs (Sec. 2.2 level transfers); coarse
// node (I,J,K) sits on fine node (2I,2J,2K), the linear weights are 1, 1/2.
// The 3^d fine rows are read with independent loads (clamped index, zero weight
// outside the grid) so they are all in flight together.
template <typename T, int D>
__device__ __forceinline__ void restrict_node(const Geom &gf, const Geom &gc, const T *__restrict__ rf,
                                              T *__restrict__ fc, int I, int J, int K)
{
    constexpr bool d3 = D == 3;
    const T scale = d3 ? T(0.125) : T(0.25);
    const long long oc = gidx(gc, I, J, K);
    constexpr int nz_rows = d3 ? 3 : 1;
#pragma unroll
    for (int p = 0; p < D; ++p) {
        T s = T(0);
        if (!is_dir(gc, p, I, J, K)) {
            const T *base = rf + p * gf.cs;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (a >= nz_rows) break;
                const int k = d3 ? 2 * K + a - 1 : 0;
                const bool kin = k >= 0 && k < gf.nz;
                const T wk = !d3 ? T(1) : (kin ? (a == 1 ? T(1) : T(0.5)) : T(0));
                const int kc = kin ? k : 2 * K;
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const int j = 2 * J + b - 1;
                    const bool jin = j >= 0 && j < gf.ny;
                    const T w = wk * (jin ? (b == 1 ? T(1) : T(0.5)) : T(0));
                    const int jc = jin ? j : 2 * J;
                    s += w * fw_row<T>(base + gidx(gf, 0, jc, kc), I, gf.nx);
                }
            }
            s *= scale;
        }
        fc[p * gc.cs + oc] = s;
    }
}

// u_f += P e_c on free fine dofs.  One thread per coarse node (I,J,K) writes the
// fine nodes (2I+a, 2J+b, 2K+c), a, b, c in {0, 1}, that exist: the coincident
// node copies e_c, the others average the 2, 4 or 8 coarse neighbours.  The x
// pair (2I, 2I+1) is read and written as one aligned vector.
template <typename T, int D>
__device__ __forceinline__ void prolong_node(const Geom &gf, const Geom &gc, const T *__restrict__ ec,
                                             T *__restrict__ uf, int I, int J, int K)
{
    using V = typename Vec2<T>::type;
    constexpr bool d3 = D == 3;
    const bool hx = I + 1 < gc.nx, hy = J + 1 < gc.ny, hz = d3 && K + 1 < gc.nz;
    const int I1 = hx ? I + 1 : I, J1 = hy ? J + 1 : J, K1 = hz ? K + 1 : K;
    const int i0 = 2 * I, j0 = 2 * J, k0 = d3 ? 2 * K : 0;
#pragma unroll
    for (int p = 0; p < D; ++p) {
        const T *e = ec + p * gc.cs;
        // coarse values of the cell above (I,J,K): [z][y][x]
        T c[2][2][2];
        c[0][0][0] = e[gidx(gc, I, J, K)];
        c[0][0][1] = e[gidx(gc, I1, J, K)];
        c[0][1][0] = e[gidx(gc, I, J1, K)];
        c[0][1][1] = e[gidx(gc, I1, J1, K)];
        c[1][0][0] = e[gidx(gc, I, J, K1)];
        c[1][0][1] = e[gidx(gc, I1, J, K1)];
        c[1][1][0] = e[gidx(gc, I, J1, K1)];
        c[1][1][1] = e[gidx(gc, I1, J1, K1)];
        T *u = uf + p * gf.cs;
#pragma unroll
        for (int zc = 0; zc < 2; ++zc) {
            if (zc == 1 && !hz) break;
#pragma unroll
            for (int yc = 0; yc < 2; ++yc) {
                if (yc == 1 && !hy) break;
                // values at x = 2I (even) and 2I+1 (odd) on this fine row
                T ev, od;
                if (zc == 0 && yc == 0) {
                    ev = c[0][0][0];
                    od = T(0.5) * (c[0][0][0] + c[0][0][1]);
                } else if (zc == 0) {
                    ev = T(0.5) * (c[0][0][0] + c[0][1][0]);
                    od = T(0.25) * ((c[0][0][0] + c[0][0][1]) + (c[0][1][0] + c[0][1][1]));
                } else if (yc == 0) {
                    ev = T(0.5) * (c[0][0][0] + c[1][0][0]);
                    od = T(0.25) * ((c[0][0][0] + c[0][0][1]) + (c[1][0][0] + c[1][0][1]));
                } else {
                    ev = T(0.25) * ((c[0][0][0] + c[0][1][0]) + (c[1][0][0] + c[1][1][0]));
                    od = T(0.125) * (((c[0][0][0] + c[0][0][1]) + (c[0][1][0] + c[0][1][1])) +
                                     ((c[1][0][0] + c[1][0][1]) + (c[1][1][0] + c[1][1][1])));
                }
                const int j = j0 + yc, k = k0 + zc;
                T *row = u + gidx(gf, 0, j, k);
                const T me = is_dir(gf, p, i0, j, k) ? T(0) : T(1);
                if (hx) {
                    const T mo = is_dir(gf, p, i0 + 1, j, k) ? T(0) : T(1);
                    V v = *reinterpret_cast<V *>(row + i0);
                    v.x += me * ev;
                    v.y += mo * od;
                    *reinterpret_cast<V *>(row + i0) = v;
                } else {
                    row[i0] += me * ev;
                }
            }
        }
    }
}

// u[gather[row]] (+)= sum_c Ainv[row][c] b[gather[c]] by one warp (lane = 0..31).
template <typename T>
__device__ __forceinline__ void bottom_row(int n, const T *__restrict__ Ainv, const int *__restrict__ gather,
                                           const T *__restrict__ b, T *__restrict__ u, int accumulate, int row,
                                           int lane)
{
    T s = T(0);
    for (int c = lane; c < n; c += 32) s += Ainv[(long long)row * n + c] * b[gather[c]];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) {
        if (accumulate) u[gather[row]] += s;
        else u[gather[row]] = s;
    }
}

}  // namespace body
}  // namespace sbm
