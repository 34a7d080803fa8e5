// k_stencil.cu — operator apply, residual (+ partial norms) and damped Jacobi
// sweep of the cell-flux SBM elasticity operator, and the 2^d-colour
// Gauss-Seidel sweep.
//
// 3D kernel organisation (one block = TX x TY cells in x/y, a chunk of z):
//   the block has (TX+1) x (TY+1) threads; thread (tx,ty) owns the cell whose
//   lower corner is node (x0+tx-1, y0+ty-1) and, when inside the tile, the node
//   (x0+tx, y0+ty).  The block streams along z one cell layer at a time: the next
//   node plane of u is staged in shared memory, every thread computes its cell's
//   24 corner forces (sbm_cell.cuh), writes them to shared memory, and every node
//   thread sums the 4 in-plane cells' bottom-corner forces plus the top-corner
//   forces carried in registers from the previous layer.  Each cell is evaluated
//   once per layer; the only redundant work is the one-cell halo ring of the tile
//   and one extra layer per z chunk.
// 2D kernel: the same with a single layer.
#include <algorithm>

#include "sbm_common.cuh"
#include "sbm_bodies.cuh"

namespace sbm {

namespace {

constexpr int TX3 = 32, TY3 = 8;     // 3D tile (cells)
constexpr int TX2 = 32, TY2 = 8;     // 2D tile (cells)

// Deterministic block reduction of ssq into part[block]: every thread stores its
// value, warp 0 folds the padded array in a fixed order and reduces by shuffles.
// (Blocks are not a multiple of 32 threads, so only warp 0, which is full, shuffles.)
template <int NT>
__device__ __forceinline__ void block_partial(double ssq, double *part, double *red)
{
    constexpr int NW = (NT + 31) / 32;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    red[tid] = ssq;
    if (tid < NW * 32 - NT) red[NT + tid] = 0.0;
    __syncthreads();
    if (tid < 32) {
        double s = 0.0;
        for (int w = 0; w < NW; ++w) s += red[w * 32 + tid];
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (tid == 0) part[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = s;
    }
}

template <typename T, typename TO, int MODE>
__global__ void __launch_bounds__((TX3 + 1) * (TY3 + 1)) k_sweep3(const SweepArgs<T, TO> a)
{
    pdl_begin();
    if (a.gate && *a.gate) return;
    constexpr int BX = TX3 + 1, BY = TY3 + 1, NT = BX * BY;
    constexpr int PX = TX3 + 2, PY = TY3 + 2, PP = PX * PY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *up = reinterpret_cast<T *>(smem_raw);           // [2][3][PY][PX]
    T *fb = up + 2 * 3 * PP;                            // [3][4][PY][PX]
    T *ft = fb + 3 * 4 * PP;                            // [3][4][PY][PX]
    T *ps = ft + 3 * 4 * PP;                            // [PY][PX]
    __shared__ double red[((NT + 31) / 32) * 32];

    const Geom &g = a.g;
    static_assert(BX == 33, "row-aligned warps need 32-cell rows");
    const int tid = threadIdx.x + BX * threadIdx.y;
    int tx, ty;
    row_warp_xy<BY>(tid, tx, ty);
    const int x0 = blockIdx.x * TX3, y0 = blockIdx.y * TY3;
    const int kz0 = blockIdx.z * a.kchunk;
    const int kz1 = min(kz0 + a.kchunk, g.nz - 1);

    // the column/row beyond the block's last cell stays zero
    for (int s = tid; s < PP; s += NT) {
        const int lx = s % PX, ly = s / PX;
        if (lx == BX || ly == BY) {
            for (int q = 0; q < 12; ++q) { fb[q * PP + s] = T(0); ft[q * PP + s] = T(0); }
            ps[s] = T(0);
        }
    }
    auto load_plane = [&](int k, int buf) {
        T *dst = up + buf * 3 * PP;
        for (int s = tid; s < PP; s += NT) {
            const int lx = s % PX, ly = s / PX;
            const int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
            const bool ok = gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny && k >= 0 && k < g.nz;
            const long long o = gidx(g, gx, gy, k);
#pragma unroll
            for (int p = 0; p < 3; ++p) dst[p * PP + s] = ok ? a.u[p * g.cs + o] : T(0);
        }
    };

    const int gx = x0 + tx, gy = y0 + ty;
    const bool own = gx < g.nx && gy < g.ny && (tx < TX3 || gx == g.nx - 1) && (ty < TY3 || gy == g.ny - 1);
    const int cx = gx - 1, cy = gy - 1;
    const bool cell_ok = cx >= 0 && cx < g.nx - 1 && cy >= 0 && cy < g.ny - 1;
    T carry[3] = {T(0), T(0), T(0)};
    T carry_ps = T(0);
    double ssq = 0.0;

    int lz = max(kz0 - 1, 0);
    load_plane(lz, lz & 1);
    for (; lz < kz1; ++lz) {
        load_plane(lz + 1, (lz + 1) & 1);
        __syncthreads();
        const T psi = cell_ok ? a.psi[gidx(g, cx, cy, lz)] : T(0);
        T U[3][8];
        {
            const T *p0 = up + (lz & 1) * 3 * PP, *p1 = up + ((lz + 1) & 1) * 3 * PP;
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                U[p][0] = p0[p * PP + ty * PX + tx];
                U[p][1] = p0[p * PP + ty * PX + tx + 1];
                U[p][2] = p0[p * PP + (ty + 1) * PX + tx];
                U[p][3] = p0[p * PP + (ty + 1) * PX + tx + 1];
                U[p][4] = p1[p * PP + ty * PX + tx];
                U[p][5] = p1[p * PP + ty * PX + tx + 1];
                U[p][6] = p1[p * PP + (ty + 1) * PX + tx];
                U[p][7] = p1[p * PP + (ty + 1) * PX + tx + 1];
            }
        }
        cell_forces3<T>(U, psi, a.c);
        const int me = ty * PX + tx;
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                fb[(p * 4 + q) * PP + me] = U[p][q];
                ft[(p * 4 + q) * PP + me] = U[p][q + 4];
            }
        ps[me] = psi;
        __syncthreads();
        if (own) {
            // node = corner 3 of cell (tx,ty), 2 of (tx+1,ty), 1 of (tx,ty+1), 0 of (tx+1,ty+1)
            T sb[3], st[3];
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                sb[p] = fb[(p * 4 + 3) * PP + me] + fb[(p * 4 + 2) * PP + me + 1] +
                        fb[(p * 4 + 1) * PP + me + PX] + fb[(p * 4 + 0) * PP + me + PX + 1];
                st[p] = ft[(p * 4 + 3) * PP + me] + ft[(p * 4 + 2) * PP + me + 1] +
                        ft[(p * 4 + 1) * PP + me + PX] + ft[(p * 4 + 0) * PP + me + PX + 1];
            }
            const T pss = ps[me] + ps[me + 1] + ps[me + PX] + ps[me + PX + 1];
            if (lz >= kz0) {
                T Ku[3], uv[3];
                const T *pl = up + (lz & 1) * 3 * PP;
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                    Ku[p] = carry[p] + sb[p];
                    uv[p] = pl[p * PP + me + PX + 1];
                }
                body::finalize<T, TO, MODE>(a, gx, gy, lz, Ku, carry_ps + pss, uv, ssq);
            }
#pragma unroll
            for (int p = 0; p < 3; ++p) carry[p] = st[p];
            carry_ps = pss;
        }
        __syncthreads();
    }
    if (kz1 == g.nz - 1 && own) {
        T uv[3];
        const T *pl = up + (kz1 & 1) * 3 * PP;
#pragma unroll
        for (int p = 0; p < 3; ++p) uv[p] = pl[p * PP + (ty + 1) * PX + tx + 1];
        body::finalize<T, TO, MODE>(a, gx, gy, kz1, carry, carry_ps, uv, ssq);
    }
    if (MODE == kResidual && a.part) block_partial<NT>(ssq, a.part, red);
}

// FP64 3D sweep.  FP64 runs at ~1/72 of the FP32 rate on this GPU, so the kernel is
// bound by FP64 instruction issue and is organised to keep the FP64 pipe fed:
// a node plane's in-plane transform is computed once and shared by the two cell
// layers it bounds, the forces a layer sends to its top plane are carried in the
// transformed basis (one transposed in-plane butterfly per plane), and the 32 x 12
// tile keeps the recomputed halo ring small.  No global load is waited on inside a
// step: node planes arrive through a three-slot shared-memory ring filled by
// cp.async two planes ahead, and the cell's psi and the node's right-hand side are
// loaded into registers one step (psi) or one compute phase (f) before their use.
// The last node plane of the grid is finalised by one extra step over an empty
// (psi = 0) layer.
constexpr int TXD = 32, TYD = 12;

// 8-byte global -> shared copy; ok = false fills zeros (src must still be valid).
__device__ __forceinline__ void cp_async8(void *sdst, const void *gsrc, bool ok)
{
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(sdst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gsrc), "r"(ok ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <typename TO, int MODE>
__global__ void __launch_bounds__((TXD + 1) * (TYD + 1)) k_sweep3_dp(const SweepArgs<double, TO> a)
{
    pdl_begin();
    if (a.gate && *a.gate) return;
    constexpr int BX = TXD + 1, BY = TYD + 1, NT = BX * BY;
    constexpr int PX = TXD + 2, PY = TYD + 2, PP = PX * PY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *up = reinterpret_cast<double *>(smem_raw);   // [3][3][PP] ring of node planes
    double *fc = up + 3 * 3 * PP;                         // [3][4][PP] corner forces of one plane
    double *ps = fc + 12 * PP;                            // [PP] psi of the cells below + above
    __shared__ double red[((NT + 31) / 32) * 32];

    const Geom &g = a.g;
    static_assert(BX == 33, "row-aligned warps need 32-cell rows");
    const int tid = threadIdx.x + BX * threadIdx.y;
    int tx, ty;
    row_warp_xy<BY>(tid, tx, ty);
    for (int s = tid; s < PP; s += NT) {
        const int lx = s % PX, ly = s / PX;
        if (lx == BX || ly == BY) {
            for (int q = 0; q < 12; ++q) fc[q * PP + s] = 0.0;
            ps[s] = 0.0;
        }
    }
    // Persistent: the units are (tile, node plane) pairs, tile-major; block b owns a
    // contiguous range of them and streams it as one z segment per tile it touches.
    const int ntx = (g.nx - 1 + TXD - 1) / TXD, nty = (g.ny - 1 + TYD - 1) / TYD;
    const long long U = (long long)ntx * nty * g.nz;
    const long long ub = U * blockIdx.x / gridDim.x, ue = U * (blockIdx.x + 1) / gridDim.x;
    double ssq = 0.0;
    for (long long su = ub; su < ue;) {
        const int tile = (int)(su / g.nz), kz0 = (int)(su % g.nz);
        const int kend = (int)min((long long)g.nz, kz0 + (ue - su)) - 1;   // last node plane finalised
        su += kend + 1 - kz0;
        const int x0 = (tile % ntx) * TXD, y0 = (tile / ntx) * TYD;
        const int kfirst = kz0 > 0 ? kz0 - 1 : 0;
        // node plane k into ring slot k % 3 (zeros outside the grid)
        auto load_plane = [&](int k) {
            double *dst = up + (k % 3) * 3 * PP;
            for (int s = tid; s < PP; s += NT) {
                const int lx = s % PX, ly = s / PX;
                const int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
                const bool ok = gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny && k >= 0 && k < g.nz;
                const long long o = ok ? gidx(g, gx, gy, k) : 0;
#pragma unroll
                for (int p = 0; p < 3; ++p) cp_async8(dst + p * PP + s, a.u + (ok ? p * g.cs + o : 0), ok);
            }
            cp_async_commit();
        };
        const int gx = x0 + tx, gy = y0 + ty;
        const bool own = gx < g.nx && gy < g.ny && (tx < TXD || gx == g.nx - 1) && (ty < TYD || gy == g.ny - 1);
        const int cx = gx - 1, cy = gy - 1;
        const bool cell_ok = cx >= 0 && cx < g.nx - 1 && cy >= 0 && cy < g.ny - 1;
        const int me = ty * PX + tx;
        auto corners = [&](int k, double (&T)[3][4]) {
            const double *pl = up + (k % 3) * 3 * PP;
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                T[p][0] = pl[p * PP + me];
                T[p][1] = pl[p * PP + me + 1];
                T[p][2] = pl[p * PP + me + PX];
                T[p][3] = pl[p * PP + me + PX + 1];
                bfly4xy(T[p]);
            }
        };
        auto cell_psi = [&](int lz) { return (cell_ok && lz <= g.nz - 2) ? a.psi[gidx(g, cx, cy, lz)] : 0.0; };

        double Tb[3][4], Cf[3][4];
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int s = 0; s < 4; ++s) Cf[p][s] = 0.0;
        double psi_prev = 0.0;
        double psi = cell_psi(kfirst);
        load_plane(kfirst);
        load_plane(kfirst + 1);
        cp_async_wait_all();
        __syncthreads();
        corners(kfirst, Tb);
        for (int lz = kfirst; lz <= kend; ++lz) {
            load_plane(lz + 2);                               // slot of plane lz - 1, free since the last barrier
            const double psi_next = cell_psi(lz + 1);
            const bool fin = own && lz >= kz0;
            double fv[3];
            const long long on = gidx(g, gx, gy, lz);
#pragma unroll
            for (int p = 0; p < 3; ++p) fv[p] = (MODE != kApply && fin) ? a.f[p * g.cs + on] : 0.0;
            double Tt[3][4], Fb[3][4], Ft[3][4];
            corners(lz + 1, Tt);
            cell_faces3<double>(Tb, Tt, psi, a.c, Fb, Ft);
#pragma unroll
            for (int p = 0; p < 3; ++p) {
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    Fb[p][s] += Cf[p][s];   // plane lz: top face of layer lz-1 + bottom face of layer lz
                    Cf[p][s] = Ft[p][s];
                    Tb[p][s] = Tt[p][s];
                }
                bfly4xyT(Fb[p]);
#pragma unroll
                for (int q = 0; q < 4; ++q) fc[(p * 4 + q) * PP + me] = Fb[p][q];
            }
            ps[me] = psi_prev + psi;
            psi_prev = psi;
            psi = psi_next;
            __syncthreads();
            if (fin) {
                double Ku[3], uv[3];
                const double *pl = up + (lz % 3) * 3 * PP;
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                    Ku[p] = (fc[(p * 4 + 3) * PP + me] + fc[(p * 4 + 2) * PP + me + 1]) +
                            (fc[(p * 4 + 1) * PP + me + PX] + fc[(p * 4 + 0) * PP + me + PX + 1]);
                    uv[p] = pl[p * PP + me + PX + 1];
                }
                const double pss = (ps[me] + ps[me + 1]) + (ps[me + PX] + ps[me + PX + 1]);
                body::finalize_f<double, TO, MODE>(a, gx, gy, lz, Ku, pss, uv, fv, ssq);
            }
            cp_async_wait_all();                              // plane lz + 2 in this thread's copies
            __syncthreads();
        }
    }
    if (MODE == kResidual && a.part) block_partial<NT>(ssq, a.part, red);
}

constexpr size_t smem_dp() { return sizeof(double) * (3 * 3 + 12 + 1) * (TXD + 2) * (TYD + 2); }

template <typename T, typename TO, int MODE>
__global__ void __launch_bounds__((TX2 + 1) * (TY2 + 1)) k_sweep2(const SweepArgs<T, TO> a)
{
    pdl_begin();
    if (a.gate && *a.gate) return;
    constexpr int BX = TX2 + 1, BY = TY2 + 1, NT = BX * BY;
    constexpr int PX = TX2 + 2, PY = TY2 + 2, PP = PX * PY;
    __shared__ T up[2 * PP];
    __shared__ T fc[2 * 4 * PP];
    __shared__ T ps[PP];
    __shared__ double red[((NT + 31) / 32) * 32];
    const Geom &g = a.g;
    static_assert(BX == 33, "row-aligned warps need 32-cell rows");
    const int tid = threadIdx.x + BX * threadIdx.y;
    int tx, ty;
    row_warp_xy<BY>(tid, tx, ty);
    const int x0 = blockIdx.x * TX2, y0 = blockIdx.y * TY2;
    for (int s = tid; s < PP; s += NT) {
        const int lx = s % PX, ly = s / PX;
        const int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
        const bool ok = gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny;
        const long long o = gidx(g, gx, gy, 0);
        up[s] = ok ? a.u[o] : T(0);
        up[PP + s] = ok ? a.u[g.cs + o] : T(0);
        if (lx == BX || ly == BY) {
            for (int q = 0; q < 8; ++q) fc[q * PP + s] = T(0);
            ps[s] = T(0);
        }
    }
    __syncthreads();
    const int gx = x0 + tx, gy = y0 + ty;
    const int cx = gx - 1, cy = gy - 1;
    const bool cell_ok = cx >= 0 && cx < g.nx - 1 && cy >= 0 && cy < g.ny - 1;
    const T psi = cell_ok ? a.psi[gidx(g, cx, cy, 0)] : T(0);
    const int me = ty * PX + tx;
    T U[2][4];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        U[p][0] = up[p * PP + me];
        U[p][1] = up[p * PP + me + 1];
        U[p][2] = up[p * PP + me + PX];
        U[p][3] = up[p * PP + me + PX + 1];
    }
    cell_forces2<T>(U, psi, a.c);
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) fc[(p * 4 + q) * PP + me] = U[p][q];
    ps[me] = psi;
    __syncthreads();
    double ssq = 0.0;
    const bool own = gx < g.nx && gy < g.ny && (tx < TX2 || gx == g.nx - 1) && (ty < TY2 || gy == g.ny - 1);
    if (own) {
        T Ku[2], uv[2];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            Ku[p] = fc[(p * 4 + 3) * PP + me] + fc[(p * 4 + 2) * PP + me + 1] + fc[(p * 4 + 1) * PP + me + PX] +
                    fc[(p * 4 + 0) * PP + me + PX + 1];
            uv[p] = up[p * PP + me + PX + 1];
        }
        const T pss = ps[me] + ps[me + 1] + ps[me + PX] + ps[me + PX + 1];
        body::finalize<T, TO, MODE>(a, gx, gy, 0, Ku, pss, uv, ssq);
    }
    if (MODE == kResidual && a.part) block_partial<NT>(ssq, a.part, red);
}

template <typename T>
constexpr size_t smem3()
{
    return sizeof(T) * (2 * 3 + 12 + 12 + 1) * (TX3 + 2) * (TY3 + 2);
}

// ---------------------------------------------------------------- Gauss-Seidel
// One colour pass: every node of colour (cx, cy, cz) = (i&1, j&1, k&1) is relaxed.
// Nodes of one colour do not couple through the 3^d stencil; within a node the
// components are relaxed in order x, y, z with the latest values (the coupling
// to the node's own earlier components is applied through the self block).
// Ke is the unit-psi cell matrix for this level, row = corner*d + component.
template <typename T, int D>
__global__ void k_gs(const Geom g, const T *__restrict__ psi, const T *__restrict__ Ke,
                     const T *__restrict__ f, T *__restrict__ u, int colour, const int *gate)
{
    pdl_begin();
    if (gate && *gate) return;
    constexpr int NC = 1 << D, ND = NC * D;
    const int cxb = colour & 1, cyb = (colour >> 1) & 1, czb = (colour >> 2) & 1;
    const int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x) + cxb;
    const int j = 2 * (blockIdx.y * blockDim.y + threadIdx.y) + cyb;
    const int k = (D == 3) ? 2 * (blockIdx.z * blockDim.z + threadIdx.z) + czb : 0;
    if (i >= g.nx || j >= g.ny || k >= g.nz) return;
    T Ku[D], S[D][D], dg[D];
#pragma unroll
    for (int p = 0; p < D; ++p) {
        Ku[p] = T(0);
        dg[p] = T(0);
#pragma unroll
        for (int q = 0; q < D; ++q) S[p][q] = T(0);
    }
#pragma unroll
    for (int a = 0; a < NC; ++a) {        // node is corner a of cell (i,j,k) - offset(a)
        const int ci = i - (a & 1), cj = j - ((a >> 1) & 1), ck = (D == 3) ? k - ((a >> 2) & 1) : 0;
        if (ci < 0 || cj < 0 || ck < 0 || ci >= g.nx - 1 || cj >= g.ny - 1 || (D == 3 && ck >= g.nz - 1))
            continue;
        const T pc = psi[gidx(g, ci, cj, ck)];
#pragma unroll
        for (int b = 0; b < NC; ++b) {
            const long long o = gidx(g, ci + (b & 1), cj + ((b >> 1) & 1), (D == 3) ? ck + ((b >> 2) & 1) : 0);
#pragma unroll
            for (int q = 0; q < D; ++q) {
                const T uv = u[q * g.cs + o];
#pragma unroll
                for (int p = 0; p < D; ++p) Ku[p] += pc * Ke[(a * D + p) * ND + b * D + q] * uv;
            }
        }
#pragma unroll
        for (int p = 0; p < D; ++p)
#pragma unroll
            for (int q = 0; q < D; ++q) S[p][q] += pc * Ke[(a * D + p) * ND + a * D + q];
    }
    const long long o = gidx(g, i, j, k);
#pragma unroll
    for (int p = 0; p < D; ++p) {
        if (is_dir(g, p, i, j, k)) continue;
        const T du = (f[p * g.cs + o] - Ku[p]) / S[p][p];
        u[p * g.cs + o] += du;
#pragma unroll
        for (int q = 0; q < D; ++q) Ku[q] += S[q][p] * du;
    }
    (void)dg;
}

// 2D colour Gauss-Seidel, one launch per sweep.  A block owns a 32 x 32 tile of
// nodes and stages u, f and psi on the tile plus a four-node halo; the four colour
// phases then run in shared memory, phase q relaxing its colour on the tile grown by
// 3 - q nodes, so every value a phase reads (its 3 x 3 neighbourhood) was produced by
// the phases before it exactly as in four separate colour passes.  Halo nodes are
// relaxed redundantly by each block that stages them and only the tile is written,
// to a second buffer (the sweep reads the old values of other tiles' nodes).  Per
// relaxed node the row of K is formed cell by cell, the unit-psi cell matrix rows
// applied first and psi_c once per cell (16 + 2 multiply-adds per cell).
constexpr int GST = 32, GSH = 4, GSN = GST + 2 * GSH, GSC = GSN - 1, GSF = GSN - 2;
constexpr int kGsThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kGsThreads) k_gs2_tile(const Geom g, const T *__restrict__ psi,
                                                         const T *__restrict__ Ke, const T *__restrict__ f,
                                                         const T *__restrict__ uin, T *__restrict__ uout,
                                                         int descending, const int *gate)
{
    pdl_begin();
    if (gate && *gate) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *su = reinterpret_cast<T *>(smem_raw);   // [2][GSN][GSN] staged nodes
    T *sf = su + 2 * GSN * GSN;                 // [2][GSF][GSF] right-hand side of staged nodes 1 .. GSN-2
    T *sp = sf + 2 * GSF * GSF;                 // [GSC][GSC] psi of the staged cells (0 outside the grid)
    T *sk = sp + GSC * GSC;                     // [8][8] unit-psi cell matrix, row = corner*2 + component
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * GST - GSH, y0 = blockIdx.y * GST - GSH;   // global node of staged (0, 0)
    for (int s = tid; s < 64; s += kGsThreads) sk[s] = Ke[s];
    for (int s = tid; s < GSN * GSN; s += kGsThreads) {
        const int i = x0 + s % GSN, j = y0 + s / GSN;
        const bool ok = i >= 0 && i < g.nx && j >= 0 && j < g.ny;
        const long long o = ok ? gidx(g, i, j, 0) : 0;
        su[s] = ok ? uin[o] : T(0);
        su[GSN * GSN + s] = ok ? uin[g.cs + o] : T(0);
    }
    for (int s = tid; s < GSF * GSF; s += kGsThreads) {
        const int i = x0 + 1 + s % GSF, j = y0 + 1 + s / GSF;
        const bool ok = i >= 0 && i < g.nx && j >= 0 && j < g.ny;
        const long long o = ok ? gidx(g, i, j, 0) : 0;
        sf[s] = ok ? f[o] : T(0);
        sf[GSF * GSF + s] = ok ? f[g.cs + o] : T(0);
    }
    for (int s = tid; s < GSC * GSC; s += kGsThreads) {
        const int i = x0 + s % GSC, j = y0 + s / GSC;
        const bool ok = i >= 0 && i < g.nx - 1 && j >= 0 && j < g.ny - 1;
        sp[s] = ok ? psi[gidx(g, i, j, 0)] : T(0);
    }
    __syncthreads();
    for (int q = 0; q < 4; ++q) {
        const int c = descending ? 3 - q : q;
        const int h = 3 - q;                              // halo still relaxed in this phase
        const int lo = GSH - h, nr = (GST + 2 * h) / 2;   // first staged index, colour nodes per row
        const int lx0 = lo + ((c & 1) - lo & 1), ly0 = lo + ((c >> 1) - lo & 1);
        for (int n = tid; n < nr * nr; n += kGsThreads) {
            const int lx = lx0 + 2 * (n % nr), ly = ly0 + 2 * (n / nr);
            const int i = x0 + lx, j = y0 + ly;
            if (i < 0 || j < 0 || i >= g.nx || j >= g.ny) continue;
            T Ku[2] = {T(0), T(0)}, S[2][2] = {{T(0), T(0)}, {T(0), T(0)}};
#pragma unroll
            for (int a = 0; a < 4; ++a) {                 // the node is corner a of staged cell (cx, cy)
                const int cx = lx - (a & 1), cy = ly - (a >> 1);
                const T pc = sp[cy * GSC + cx];
                T t[2] = {T(0), T(0)};
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int o = (cy + (b >> 1)) * GSN + cx + (b & 1);
                    const T u0 = su[o], u1 = su[GSN * GSN + o];
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        t[p] = madd(sk[(a * 2 + p) * 8 + b * 2], u0, t[p]);
                        t[p] = madd(sk[(a * 2 + p) * 8 + b * 2 + 1], u1, t[p]);
                    }
                }
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    Ku[p] = madd(pc, t[p], Ku[p]);
#pragma unroll
                    for (int r = 0; r < 2; ++r) S[p][r] = madd(pc, sk[(a * 2 + p) * 8 + a * 2 + r], S[p][r]);
                }
            }
            const int me = ly * GSN + lx, mf = (ly - 1) * GSF + lx - 1;
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                if (is_dir(g, p, i, j, 0)) continue;
                const T du = (sf[p * GSF * GSF + mf] - Ku[p]) / S[p][p];
                su[p * GSN * GSN + me] += du;
#pragma unroll
                for (int r = 0; r < 2; ++r) Ku[r] = madd(S[r][p], du, Ku[r]);
            }
        }
        __syncthreads();
    }
    for (int s = tid; s < GST * GST; s += kGsThreads) {
        const int lx = GSH + s % GST, ly = GSH + s / GST;
        const int i = x0 + lx, j = y0 + ly;
        if (i >= g.nx || j >= g.ny) continue;
        const long long o = gidx(g, i, j, 0);
        uout[o] = su[ly * GSN + lx];
        uout[g.cs + o] = su[GSN * GSN + ly * GSN + lx];
    }
}

template <typename T>
constexpr size_t smem_gs2()
{
    return sizeof(T) * (2 * GSN * GSN + 2 * GSF * GSF + GSC * GSC + 64);
}

}  // namespace

// Persistent FP64 sweep: one block per SM of the 152 (one fits per SM), at most one
// per (tile, node plane) unit.
static void sweep_grid_dp(const Geom &g, int *grid, int *kchunk)
{
    const long long units = (long long)((g.nx - 1 + TXD - 1) / TXD) * ((g.ny - 1 + TYD - 1) / TYD) * g.nz;
    grid[0] = (int)std::min<long long>(152, units);
    grid[1] = grid[2] = 1;
    *kchunk = 0;
}

void sweep_grid(const Geom &g, int *grid, int *kchunk)
{
    if (g.dim == 3) {
        grid[0] = (g.nx - 1 + TX3 - 1) / TX3;
        grid[1] = (g.ny - 1 + TY3 - 1) / TY3;
        const int nzc = g.nz - 1;
        const int nc = choose_chunks((long long)grid[0] * grid[1], nzc, 2 * 152, false);
        const int ch = (nzc + nc - 1) / nc;
        grid[2] = (nzc + ch - 1) / ch;
        *kchunk = ch;
    } else {
        grid[0] = (g.nx - 1 + TX2 - 1) / TX2;
        grid[1] = (g.ny - 1 + TY2 - 1) / TY2;
        grid[2] = 1;
        *kchunk = 1;
    }
}

long long sweep_blocks(const Geom &g, bool fp64)
{
    int grid[3], ch;
    if (fp64 && g.dim == 3) sweep_grid_dp(g, grid, &ch);
    else sweep_grid(g, grid, &ch);
    return (long long)grid[0] * grid[1] * grid[2];
}

// Small 3D levels (FP32): eight consecutive threads per node, thread c evaluating
// the cell of which the node is corner c; the node's force and psi sum are summed
// over the eight lanes by shuffles and the first lane finalises.  There is no
// shared memory, no barrier and no z streaming, and each thread's dependent
// chain is one cell: on coarse levels, whose cost is latency, a launch takes
// little more than one cell evaluation.
constexpr int kNodeThreads = 256;

template <int MODE>
__global__ void __launch_bounds__(kNodeThreads) k_sweep3_node(const SweepArgs<float, float> a)
{
    pdl_begin();
    if (a.gate && *a.gate) return;
    const Geom &g = a.g;
    const long long n = (long long)g.nx * g.ny * g.nz;
    const long long node = (long long)blockIdx.x * (kNodeThreads / 8) + (threadIdx.x >> 3);
    const int c = threadIdx.x & 7;
    const bool valid = node < n;
    int i = 0, j = 0, k = 0;
    if (valid) {
        i = (int)(node % g.nx);
        const long long t = node / g.nx;
        j = (int)(t % g.ny);
        k = (int)(t / g.ny);
    }
    float F[3] = {0.f, 0.f, 0.f}, ps = 0.f;
    if (valid) body::node_cell(a, i, j, k, c, F, ps);
    // every lane takes part in the sums; the xor partners stay in the group of eight
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) {
#pragma unroll
        for (int p = 0; p < 3; ++p) F[p] += __shfl_xor_sync(0xffffffffu, F[p], off);
        ps += __shfl_xor_sync(0xffffffffu, ps, off);
    }
    if (valid && c == 0) {
        const long long o = gidx(g, i, j, k);
        const float uv[3] = {a.u[o], a.u[g.cs + o], a.u[2 * g.cs + o]};
        double ssq = 0.0;
        body::finalize<float, float, MODE>(a, i, j, k, F, ps, uv, ssq);
    }
}

cudaError_t launch_sweep_node(int mode, const SweepArgs<float, float> &a, cudaStream_t s)
{
    const long long n = (long long)a.g.nx * a.g.ny * a.g.nz;
    const dim3 b(kNodeThreads), gr((unsigned)((n + kNodeThreads / 8 - 1) / (kNodeThreads / 8)));
    cudaError_t e;
    switch (mode) {
    case kApply: e = launch_pdl(k_sweep3_node<kApply>, gr, b, 0, s, a); break;
    case kResidual: e = launch_pdl(k_sweep3_node<kResidual>, gr, b, 0, s, a); break;
    case kJacobi: e = launch_pdl(k_sweep3_node<kJacobi>, gr, b, 0, s, a); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    ++g_launches;
    return cudaGetLastError();
}

template <typename T, typename TO, int MODE>
static cudaError_t launch_mode(const SweepArgs<T, TO> &a0, cudaStream_t s)
{
    SweepArgs<T, TO> a = a0;
    int grid[3];
    if (a.g.dim == 3 && sizeof(T) == 8) {
        sweep_grid_dp(a.g, grid, &a.kchunk);
        const size_t sm = smem_dp();
        static std::atomic<unsigned long long> attr_dp{0};
        cudaError_t ea = smem_attr_once(reinterpret_cast<const void *>(k_sweep3_dp<TO, MODE>), sm, attr_dp);
        if (ea != cudaSuccess) return ea;
        cudaError_t e = launch_pdl(k_sweep3_dp<TO, MODE>, dim3(grid[0], grid[1], grid[2]), dim3(TXD + 1, TYD + 1), sm, s,
                                   reinterpret_cast<const SweepArgs<double, TO> &>(a));
        if (e != cudaSuccess) return e;
        ++g_launches;
        return cudaGetLastError();
    }
    sweep_grid(a.g, grid, &a.kchunk);
    if (a.g.dim == 3) {
        const size_t sm = smem3<T>();
        static std::atomic<unsigned long long> attr_done{0};
        cudaError_t ea = smem_attr_once(reinterpret_cast<const void *>(k_sweep3<T, TO, MODE>), sm, attr_done);
        if (ea != cudaSuccess) return ea;
        cudaError_t e = launch_pdl(k_sweep3<T, TO, MODE>, dim3(grid[0], grid[1], grid[2]), dim3(TX3 + 1, TY3 + 1), sm, s, a);
        if (e != cudaSuccess) return e;
    } else {
        cudaError_t e = launch_pdl(k_sweep2<T, TO, MODE>, dim3(grid[0], grid[1], 1), dim3(TX2 + 1, TY2 + 1), 0, s, a);
        if (e != cudaSuccess) return e;
    }
    ++g_launches;
    return cudaGetLastError();
}

template <typename T, typename TO>
cudaError_t launch_sweep(int mode, const SweepArgs<T, TO> &a, cudaStream_t s)
{
    switch (mode) {
    case kApply: return launch_mode<T, TO, kApply>(a, s);
    case kResidual: return launch_mode<T, TO, kResidual>(a, s);
    case kJacobi: return launch_mode<T, TO, kJacobi>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_sweep<double, double>(int, const SweepArgs<double, double> &, cudaStream_t);
template cudaError_t launch_sweep<float, float>(int, const SweepArgs<float, float> &, cudaStream_t);
template cudaError_t launch_sweep<double, float>(int, const SweepArgs<double, float> &, cudaStream_t);

template <typename T>
cudaError_t launch_gs(const Geom &g, const T *psi, const T *Ke, const T *f, T *u, int colour, cudaStream_t s,
                      const int *gate)
{
    if (g.dim == 3) {
        dim3 b(32, 4, 2);
        dim3 gr(((g.nx + 1) / 2 + b.x - 1) / b.x, ((g.ny + 1) / 2 + b.y - 1) / b.y, ((g.nz + 1) / 2 + b.z - 1) / b.z);
        cudaError_t e = launch_pdl(k_gs<T, 3>, gr, b, 0, s, g, psi, Ke, f, u, colour, gate);
        if (e != cudaSuccess) return e;
    } else {
        dim3 b(32, 8, 1);
        dim3 gr(((g.nx + 1) / 2 + b.x - 1) / b.x, ((g.ny + 1) / 2 + b.y - 1) / b.y, 1);
        cudaError_t e = launch_pdl(k_gs<T, 2>, gr, b, 0, s, g, psi, Ke, f, u, colour, gate);
        if (e != cudaSuccess) return e;
    }
    ++g_launches;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gs2_sweep(const Geom &g, const T *psi, const T *Ke, const T *f, const T *uin, T *uout,
                             int descending, cudaStream_t s, const int *gate)
{
    if (g.dim != 2 || uin == uout) return cudaErrorInvalidValue;
    const size_t sm = smem_gs2<T>();
    static std::atomic<unsigned long long> attr_done{0};
    cudaError_t ea = smem_attr_once(reinterpret_cast<const void *>(k_gs2_tile<T>), sm, attr_done);
    if (ea != cudaSuccess) return ea;
    dim3 gr((g.nx + GST - 1) / GST, (g.ny + GST - 1) / GST, 1);
    cudaError_t e = launch_pdl(k_gs2_tile<T>, gr, dim3(kGsThreads), sm, s, g, psi, Ke, f, uin, uout, descending, gate);
    if (e != cudaSuccess) return e;
    ++g_launches;
    return cudaGetLastError();
}

template cudaError_t launch_gs2_sweep<double>(const Geom &, const double *, const double *, const double *,
                                              const double *, double *, int, cudaStream_t, const int *);
template cudaError_t launch_gs2_sweep<float>(const Geom &, const float *, const float *, const float *,
                                             const float *, float *, int, cudaStream_t, const int *);

template cudaError_t launch_gs<double>(const Geom &, const double *, const double *, const double *, double *, int, cudaStream_t,
                                       const int *);
template cudaError_t launch_gs<float>(const Geom &, const float *, const float *, const float *, float *, int, cudaStream_t,
                                      const int *);

}  // namespace sbm
