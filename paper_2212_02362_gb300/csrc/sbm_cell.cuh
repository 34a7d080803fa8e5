// sbm_cell.cuh — the per-cell arithmetic of the cell-flux SBM elasticity operator.
//
// One cell c with nodal displacements u[p][a] (component p, corner a, bit m of a
// = offset along axis m) contributes the nodal forces
//     F = psi_c h^-d int_c B^T C B u      (Sec. 2.1 eq. SBMLinearElasticity, with
//                                           psi in cells and u at nodes, Sec. 2.3)
// integrated exactly (the 2-point Gauss rule is exact for Q1 gradients).
//
// Sum factorisation.  Along each axis the two nodal values (v0, v1) are replaced
// by A = v0 + v1 and D = v1 - v0, i.e. the linear interpolant is A/2 + D (xi - 1/2).
// The functions 1 and (xi - 1/2) are orthogonal on [0,1] with norms 1 and 1/12, so
// in this basis the element energy splits into independent terms, one per basis
// function t of the gradient (t = which axes carry the (xi - 1/2) factor):
//     E = sum_t W(t) eps_t : C : eps_t,   W(t) = 12^-ones(t) 4^-(zeros(t)-1)
// where the gradient coefficient of d_i u_p on t is the transformed value
// U_p[t + e_i].  The force is the transpose of that map.  Per cell this costs
// ~180 adds/multiplies in 3D instead of the 576 of a dense 24 x 24 element matrix.
//
// W: 3D 1/16 (no D factor), 1/48 (one), 1/144 (two); 2D 1/4, 1/12.  Moduli are
// axis-aligned cubic (C11, C12, C44); isotropic is C11 = lambda + 2 mu, C12 =
// lambda, C44 = mu.  All constants carry the h^-2 of the FD scaling.
#pragma once

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace sbm {

// a * b + c; float and double contract to one FMA (nvcc --fmad default).
__host__ __device__ __forceinline__ float madd(float a, float b, float c) { return a * b + c; }
__host__ __device__ __forceinline__ double madd(double a, double b, double c) { return a * b + c; }

#ifdef __CUDACC__
// Two FP32 lanes in one 64-bit register pair, computed with the packed FP32x2
// instructions of sm_100+ (one FADD2 / FMUL2 / FFMA2 per pair).  The 3D FP32
// stencil evaluates two z layers of cells at once in this type.
struct F2 {
    float2 v;
    __device__ __forceinline__ F2() {}
    __device__ __forceinline__ explicit F2(float x) : v(make_float2(x, x)) {}
    __device__ __forceinline__ F2(float lo, float hi) : v(make_float2(lo, hi)) {}
};
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { F2 r; r.v = __fadd2_rn(a.v, b.v); return r; }
// a - b as one FFMA2 (b * -1 + a); there is no packed-subtract intrinsic.
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { F2 r; r.v = __ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v); return r; }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { F2 r; r.v = __fmul2_rn(a.v, b.v); return r; }
__device__ __forceinline__ F2 madd(F2 a, F2 b, F2 c) { F2 r; r.v = __ffma2_rn(a.v, b.v, c.v); return r; }
#endif

template <typename T>
struct Coef {
    T a11, a12, a44, ad;   // class 0: W0 (C11, C12, C44, C11 - C12) / h^2
    T b1, b12, b44;        // class 1: W1 (C11 + C44, C12, C44) / h^2
    T c2;                  // class 2 (3D): W2 (C11 + 2 C44) / h^2
    T kdiag[3];            // diagonal of the unit-psi cell matrix, per component
};

// Transform of one cell's nodal values to the (A, D) basis along every axis.
template <typename T>
__host__ __device__ __forceinline__ void bfly8(T (&v)[8])
{
#pragma unroll
    for (int q = 0; q < 8; q += 2) { T a = v[q] + v[q + 1], d = v[q + 1] - v[q]; v[q] = a; v[q + 1] = d; }
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int q = 4 * r; q < 4 * r + 2; ++q) { T a = v[q] + v[q + 2], d = v[q + 2] - v[q]; v[q] = a; v[q + 2] = d; }
#pragma unroll
    for (int q = 0; q < 4; ++q) { T a = v[q] + v[q + 4], d = v[q + 4] - v[q]; v[q] = a; v[q + 4] = d; }
}

// Transpose of bfly8 (lo = a - d, hi = a + d per pair), axes in reverse order.
template <typename T>
__host__ __device__ __forceinline__ void bfly8T(T (&v)[8])
{
#pragma unroll
    for (int q = 0; q < 4; ++q) { T a = v[q], d = v[q + 4]; v[q] = a - d; v[q + 4] = a + d; }
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int q = 4 * r; q < 4 * r + 2; ++q) { T a = v[q], d = v[q + 2]; v[q] = a - d; v[q + 2] = a + d; }
#pragma unroll
    for (int q = 0; q < 8; q += 2) { T a = v[q], d = v[q + 1]; v[q] = a - d; v[q + 1] = a + d; }
}

template <typename T>
__host__ __device__ __forceinline__ void bfly4(T (&v)[4])
{
    { T a = v[0] + v[1], d = v[1] - v[0]; v[0] = a; v[1] = d; }
    { T a = v[2] + v[3], d = v[3] - v[2]; v[2] = a; v[3] = d; }
    { T a = v[0] + v[2], d = v[2] - v[0]; v[0] = a; v[2] = d; }
    { T a = v[1] + v[3], d = v[3] - v[1]; v[1] = a; v[3] = d; }
}

template <typename T>
__host__ __device__ __forceinline__ void bfly4T(T (&v)[4])
{
    { T a = v[0], d = v[2]; v[0] = a - d; v[2] = a + d; }
    { T a = v[1], d = v[3]; v[1] = a - d; v[3] = a + d; }
    { T a = v[0], d = v[1]; v[0] = a - d; v[1] = a + d; }
    { T a = v[2], d = v[3]; v[2] = a - d; v[3] = a + d; }
}

// In place: nodal displacements u[p][corner] of one 3D cell -> nodal forces.
template <typename T>
__host__ __device__ __forceinline__ void cell_forces3(T (&U)[3][8], T psi, const Coef<T> &c)
{
    bfly8(U[0]);
    bfly8(U[1]);
    bfly8(U[2]);
    const T ad = psi * c.ad, a12 = psi * c.a12, a44 = psi * c.a44;
    const T b1 = psi * c.b1, b12 = psi * c.b12, b44 = psi * c.b44, c2 = psi * c.c2;
    // class 0: the mean gradient (all nine entries)
    const T ltr = a12 * (U[0][1] + U[1][2] + U[2][4]);
    const T sxx = madd(ad, U[0][1], ltr), syy = madd(ad, U[1][2], ltr), szz = madd(ad, U[2][4], ltr);
    const T sxy = a44 * (U[1][1] + U[0][2]);
    const T sxz = a44 * (U[2][1] + U[0][4]);
    const T syz = a44 * (U[2][2] + U[1][4]);
    // class 1: gradients linear along one axis
    const T S = U[2][3] + U[1][5] + U[0][6];
    const T d03 = madd(b1, U[0][3], b12 * U[2][6]);
    const T d26 = madd(b1, U[2][6], b12 * U[0][3]);
    const T d13 = madd(b1, U[1][3], b12 * U[2][5]);
    const T d25 = madd(b1, U[2][5], b12 * U[1][3]);
    const T d05 = madd(b1, U[0][5], b12 * U[1][6]);
    const T d16 = madd(b1, U[1][6], b12 * U[0][5]);
    const T d23 = b44 * (S + U[2][3]);
    const T d15 = b44 * (S + U[1][5]);
    const T d06 = b44 * (S + U[0][6]);
    // class 2: gradients bilinear in two axes
    const T d07 = c2 * U[0][7], d17 = c2 * U[1][7], d27 = c2 * U[2][7];
    U[0][0] = T(0); U[0][1] = sxx; U[0][2] = sxy; U[0][3] = d03; U[0][4] = sxz; U[0][5] = d05; U[0][6] = d06; U[0][7] = d07;
    U[1][0] = T(0); U[1][1] = sxy; U[1][2] = syy; U[1][3] = d13; U[1][4] = syz; U[1][5] = d15; U[1][6] = d16; U[1][7] = d17;
    U[2][0] = T(0); U[2][1] = sxz; U[2][2] = syz; U[2][3] = d23; U[2][4] = szz; U[2][5] = d25; U[2][6] = d26; U[2][7] = d27;
    bfly8T(U[0]);
    bfly8T(U[1]);
    bfly8T(U[2]);
}

// In place: nodal displacements u[p][corner] of one 2D (plane strain) cell -> forces.
template <typename T>
__host__ __device__ __forceinline__ void cell_forces2(T (&U)[2][4], T psi, const Coef<T> &c)
{
    bfly4(U[0]);
    bfly4(U[1]);
    const T a11 = psi * c.a11, a12 = psi * c.a12, a44 = psi * c.a44, b1 = psi * c.b1;
    const T sxx = a11 * U[0][1] + a12 * U[1][2];
    const T syy = a12 * U[0][1] + a11 * U[1][2];
    const T sxy = a44 * (U[1][1] + U[0][2]);
    const T d03 = b1 * U[0][3], d13 = b1 * U[1][3];
    U[0][0] = T(0); U[0][1] = sxx; U[0][2] = sxy; U[0][3] = d03;
    U[1][0] = T(0); U[1][1] = sxy; U[1][2] = syy; U[1][3] = d13;
    bfly4T(U[0]);
    bfly4T(U[1]);
}

// Constants for spacing h (host side, FP64, then rounded to T).
template <typename T>
inline Coef<T> make_coef(int dim, double h, double c11, double c12, double c44)
{
    const double ih2 = 1.0 / (h * h);
    double W0, W1, W2;
    if (dim == 3) { W0 = 1.0 / 16.0; W1 = 1.0 / 48.0; W2 = 1.0 / 144.0; }
    else { W0 = 1.0 / 4.0; W1 = 1.0 / 12.0; W2 = 0.0; }
    Coef<double> d;
    d.a11 = W0 * c11 * ih2;
    d.a12 = W0 * c12 * ih2;
    d.a44 = W0 * c44 * ih2;
    d.ad = W0 * (c11 - c12) * ih2;
    d.b1 = W1 * (c11 + c44) * ih2;
    d.b12 = W1 * c12 * ih2;
    d.b44 = W1 * c44 * ih2;
    d.c2 = W2 * (c11 + 2.0 * c44) * ih2;
    // diagonal entry of the unit-psi cell matrix for corner 0, from the routine itself
    for (int p = 0; p < 3; ++p) d.kdiag[p] = 0.0;
    for (int p = 0; p < dim; ++p) {
        if (dim == 3) {
            double U[3][8] = {};
            U[p][0] = 1.0;
            cell_forces3<double>(U, 1.0, d);
            d.kdiag[p] = U[p][0];
        } else {
            double U[2][4] = {};
            U[p][0] = 1.0;
            cell_forces2<double>(U, 1.0, d);
            d.kdiag[p] = U[p][0];
        }
    }
    Coef<T> t;
    t.a11 = T(d.a11); t.a12 = T(d.a12); t.a44 = T(d.a44); t.ad = T(d.ad);
    t.b1 = T(d.b1); t.b12 = T(d.b12); t.b44 = T(d.b44); t.c2 = T(d.c2);
    for (int p = 0; p < 3; ++p) t.kdiag[p] = T(d.kdiag[p]);
    return t;
}

}  // namespace sbm

namespace sbm {

// ---- plane-shared form of cell_forces3 (used by the FP64 z-streaming kernel) ----
// A node plane's in-plane transform is shared by the two cell layers it bounds,
// and the forces a layer sends to its top plane are carried in the transformed
// basis, so per layer only one in-plane forward and one in-plane transposed
// butterfly are evaluated.

// In-plane (x then y) transform of the 4 nodal values of one cell face.
template <typename T>
__host__ __device__ __forceinline__ void bfly4xy(T (&v)[4])
{
    const T a0 = v[0] + v[1], d0 = v[1] - v[0], a1 = v[2] + v[3], d1 = v[3] - v[2];
    v[0] = a0 + a1;
    v[2] = a1 - a0;
    v[1] = d0 + d1;
    v[3] = d1 - d0;
}

// Transpose of bfly4xy (y then x).
template <typename T>
__host__ __device__ __forceinline__ void bfly4xyT(T (&v)[4])
{
    const T w0 = v[0] - v[2], w2 = v[0] + v[2], w1 = v[1] - v[3], w3 = v[1] + v[3];
    v[0] = w0 - w1;
    v[1] = w0 + w1;
    v[2] = w2 - w3;
    v[3] = w2 + w3;
}

// The seven moduli constants of a 3D cell scaled by its psi, in the order
// (ad, a12, a44, b1, b12, b44, c2) of Coef.
template <typename T>
__host__ __device__ __forceinline__ void scaled_coefs(T psi, const Coef<T> &c, T (&k)[7])
{
    k[0] = psi * c.ad;
    k[1] = psi * c.a12;
    k[2] = psi * c.a44;
    k[3] = psi * c.b1;
    k[4] = psi * c.b12;
    k[5] = psi * c.b44;
    k[6] = psi * c.c2;
}

// One cell given the in-plane transforms of its bottom (Tb) and top (Tt) faces
// and its psi-scaled constants k (scaled_coefs): returns the transformed face
// forces Fb (to the bottom plane) and Ft (to the top).
template <typename T>
__host__ __device__ __forceinline__ void cell_faces3k(const T (&Tb)[3][4], const T (&Tt)[3][4], const T (&k)[7],
                                                      T (&Fb)[3][4], T (&Ft)[3][4])
{
    T U[3][8];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            U[p][s] = Tb[p][s] + Tt[p][s];
            U[p][s + 4] = Tt[p][s] - Tb[p][s];
        }
    const T ad = k[0], a12 = k[1], a44 = k[2], b1 = k[3], b12 = k[4], b44 = k[5], c2 = k[6];
    const T ltr = a12 * (U[0][1] + U[1][2] + U[2][4]);
    const T sxx = madd(ad, U[0][1], ltr), syy = madd(ad, U[1][2], ltr), szz = madd(ad, U[2][4], ltr);
    const T sxy = a44 * (U[1][1] + U[0][2]);
    const T sxz = a44 * (U[2][1] + U[0][4]);
    const T syz = a44 * (U[2][2] + U[1][4]);
    const T S = U[2][3] + U[1][5] + U[0][6];
    const T d03 = madd(b1, U[0][3], b12 * U[2][6]);
    const T d26 = madd(b1, U[2][6], b12 * U[0][3]);
    const T d13 = madd(b1, U[1][3], b12 * U[2][5]);
    const T d25 = madd(b1, U[2][5], b12 * U[1][3]);
    const T d05 = madd(b1, U[0][5], b12 * U[1][6]);
    const T d16 = madd(b1, U[1][6], b12 * U[0][5]);
    const T d23 = b44 * (S + U[2][3]);
    const T d15 = b44 * (S + U[1][5]);
    const T d06 = b44 * (S + U[0][6]);
    const T d07 = c2 * U[0][7], d17 = c2 * U[1][7], d27 = c2 * U[2][7];
    // dU[p][0] = 0; transposed z stage: bottom = dU[s] - dU[s+4], top = dU[s] + dU[s+4]
    const T dU[3][8] = {{T(0), sxx, sxy, d03, sxz, d05, d06, d07},
                        {T(0), sxy, syy, d13, syz, d15, d16, d17},
                        {T(0), sxz, syz, d23, szz, d25, d26, d27}};
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        Fb[p][0] = T(0) - dU[p][4];
        Ft[p][0] = dU[p][4];
#pragma unroll
        for (int s = 1; s < 4; ++s) {
            Fb[p][s] = dU[p][s] - dU[p][s + 4];
            Ft[p][s] = dU[p][s] + dU[p][s + 4];
        }
    }
}

template <typename T>
__host__ __device__ __forceinline__ void cell_faces3(const T (&Tb)[3][4], const T (&Tt)[3][4], T psi,
                                                     const Coef<T> &c, T (&Fb)[3][4], T (&Ft)[3][4])
{
    T k[7];
    scaled_coefs(psi, c, k);
    cell_faces3k(Tb, Tt, k, Fb, Ft);
}

}  // namespace sbm
