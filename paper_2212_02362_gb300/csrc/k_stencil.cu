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

// FP64 3D sweep.  FP64 runs at 1/64 of the FP32 rate on this GPU, so the kernel is
// bound by FP64 instruction issue and is organised to minimise FP64 operations:
// a node plane's in-plane transform is computed once and shared by the two cell
// layers it bounds, the forces a layer sends to its top plane are carried in the
// transformed basis (one transposed in-plane butterfly per plane), and the 32 x 12
// tile keeps the recomputed halo ring small.  The last node plane of the grid is
// finalised by one extra step over an empty (psi = 0) layer.
constexpr int TXD = 32, TYD = 12;

template <typename TO, int MODE>
__global__ void __launch_bounds__((TXD + 1) * (TYD + 1)) k_sweep3_dp(const SweepArgs<double, TO> a)
{
    pdl_begin();
    if (a.gate && *a.gate) return;
    constexpr int BX = TXD + 1, BY = TYD + 1, NT = BX * BY;
    constexpr int PX = TXD + 2, PY = TYD + 2, PP = PX * PY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *up = reinterpret_cast<double *>(smem_raw);   // [2][3][PP] node planes
    double *fc = up + 2 * 3 * PP;                         // [3][4][PP] corner forces of one plane
    double *ps = fc + 12 * PP;                            // [PP] psi of the cells below + above
    __shared__ double red[((NT + 31) / 32) * 32];

    const Geom &g = a.g;
    static_assert(BX == 33, "row-aligned warps need 32-cell rows");
    const int tid = threadIdx.x + BX * threadIdx.y;
    int tx, ty;
    row_warp_xy<BY>(tid, tx, ty);
    const int x0 = blockIdx.x * TXD, y0 = blockIdx.y * TYD;
    const int kz0 = blockIdx.z * a.kchunk;
    const int kz1 = min(kz0 + a.kchunk, g.nz - 1);
    const int kend = (kz1 == g.nz - 1) ? g.nz - 1 : kz1 - 1;
    const int kfirst = kz0 > 0 ? kz0 - 1 : 0;

    for (int s = tid; s < PP; s += NT) {
        const int lx = s % PX, ly = s / PX;
        if (lx == BX || ly == BY) {
            for (int q = 0; q < 12; ++q) fc[q * PP + s] = 0.0;
            ps[s] = 0.0;
        }
    }
    auto load_plane = [&](int k, int buf) {
        double *dst = up + buf * 3 * PP;
        for (int s = tid; s < PP; s += NT) {
            const int lx = s % PX, ly = s / PX;
            const int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
            const bool ok = gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny && k >= 0 && k < g.nz;
            const long long o = gidx(g, gx, gy, k);
#pragma unroll
            for (int p = 0; p < 3; ++p) dst[p * PP + s] = ok ? a.u[p * g.cs + o] : 0.0;
        }
    };
    const int gx = x0 + tx, gy = y0 + ty;
    const bool own = gx < g.nx && gy < g.ny && (tx < TXD || gx == g.nx - 1) && (ty < TYD || gy == g.ny - 1);
    const int cx = gx - 1, cy = gy - 1;
    const bool cell_ok = cx >= 0 && cx < g.nx - 1 && cy >= 0 && cy < g.ny - 1;
    const int me = ty * PX + tx;
    auto corners = [&](int buf, double (&T)[3][4]) {
        const double *pl = up + buf * 3 * PP;
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            T[p][0] = pl[p * PP + me];
            T[p][1] = pl[p * PP + me + 1];
            T[p][2] = pl[p * PP + me + PX];
            T[p][3] = pl[p * PP + me + PX + 1];
            bfly4xy(T[p]);
        }
    };

    double Tb[3][4], Cf[3][4];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int s = 0; s < 4; ++s) Cf[p][s] = 0.0;
    double psi_prev = 0.0, ssq = 0.0;
    load_plane(kfirst, kfirst & 1);
    __syncthreads();
    corners(kfirst & 1, Tb);
    for (int lz = kfirst; lz <= kend; ++lz) {
        load_plane(lz + 1, (lz + 1) & 1);
        __syncthreads();
        const double psi = (cell_ok && lz <= g.nz - 2) ? a.psi[gidx(g, cx, cy, lz)] : 0.0;
        double Tt[3][4], Fb[3][4], Ft[3][4];
        corners((lz + 1) & 1, Tt);
        cell_faces3<double>(Tb, Tt, psi, a.c, Fb, Ft);
#pragma unroll
        for (int p = 0; p < 3; ++p) {
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                Fb[p][s] += Cf[p][s];       // plane lz: top face of layer lz-1 + bottom face of layer lz
                Cf[p][s] = Ft[p][s];
                Tb[p][s] = Tt[p][s];
            }
            bfly4xyT(Fb[p]);
#pragma unroll
            for (int q = 0; q < 4; ++q) fc[(p * 4 + q) * PP + me] = Fb[p][q];
        }
        ps[me] = psi_prev + psi;
        psi_prev = psi;
        __syncthreads();
        if (own && lz >= kz0) {
            double Ku[3], uv[3];
            const double *pl = up + (lz & 1) * 3 * PP;
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                Ku[p] = (fc[(p * 4 + 3) * PP + me] + fc[(p * 4 + 2) * PP + me + 1]) +
                        (fc[(p * 4 + 1) * PP + me + PX] + fc[(p * 4 + 0) * PP + me + PX + 1]);
                uv[p] = pl[p * PP + me + PX + 1];
            }
            const double pss = (ps[me] + ps[me + 1]) + (ps[me + PX] + ps[me + PX + 1]);
            body::finalize<double, TO, MODE>(a, gx, gy, lz, Ku, pss, uv, ssq);
        }
        __syncthreads();
    }
    if (MODE == kResidual && a.part) block_partial<NT>(ssq, a.part, red);
}

constexpr size_t smem_dp() { return sizeof(double) * (2 * 3 + 12 + 1) * (TXD + 2) * (TYD + 2); }

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

}  // namespace

static void sweep_grid_dp(const Geom &g, int *grid, int *kchunk)
{
    grid[0] = (g.nx - 1 + TXD - 1) / TXD;
    grid[1] = (g.ny - 1 + TYD - 1) / TYD;
    const int nzc = g.nz - 1;
    const int nc = choose_chunks((long long)grid[0] * grid[1], nzc, 152, false);   // one block per SM
    const int ch = (nzc + nc - 1) / nc;
    grid[2] = (nzc + ch - 1) / ch;
    *kchunk = ch;
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

template cudaError_t launch_gs<double>(const Geom &, const double *, const double *, const double *, double *, int, cudaStream_t,
                                       const int *);
template cudaError_t launch_gs<float>(const Geom &, const float *, const float *, const float *, float *, int, cudaStream_t,
                                      const int *);

}  // namespace sbm
