// k_stencil_tma.cu — FP32 3D apply / residual / damped-Jacobi sweep of the
// cell-flux SBM elasticity operator: a persistent kernel with TMA plane staging
// and packed FP32x2 arithmetic (sm_100+ FFMA2 / FADD2 / FMUL2).
//
// Work split.  The grid's cells are cut into tiles of 32 x 12 cells in x/y; a
// tile's node planes (one per z index) are the units of work.  One CTA runs per
// SM and owns a contiguous range of units in (tile, plane) order, so every CTA
// finalises the same number of node planes to within one and streams them as a
// few long z segments (a range crosses at most a couple of tile boundaries).
// The TMA ring runs across segment boundaries without draining.
//
// A CTA has 33 x 13 threads, one per cell column of the tile plus the one-cell
// halo column and row (warps aligned with the 32-cell rows, the 33rd column in a
// warp of its own).  Each step handles two cell layers (k, k+1) in the two lanes
// of the packed type.  The in-plane (x, y) transform of a node plane is computed
// once and shared by the two layers it bounds (the previous plane's transform is
// carried in registers), and the forces a layer sends to its top plane are
// carried in the transformed basis, so a step costs two in-plane transforms and
// two transposed ones for two cell layers.
//
// Ring.  Node plane p of u, the f values of the tile's own nodes on plane p and
// cell layer p of psi are fetched by the Tensor Memory Accelerator into a 10-slot
// shared-memory ring (zero fill outside the grid), completion on one mbarrier per
// slot.  A step reads the raw u of planes k+1 and k+2 and the f and psi of planes
// k and k+1 before its single block barrier, after which the slots of planes k
// and k+1 are free and thread 0 refills them with the planes 10 sequence places
// ahead.  The in-plane corner forces are exchanged through a double-buffered
// shared tile (one barrier per step suffices: a buffer is written again only two
// barriers after it was read).  The compute loop issues no global loads.
//
// Every mbarrier wait is bounded: on timeout the block records an error code,
// waits (bounded) for the copies it has in flight and returns.  The grid swept may
// sit inside a larger storage at an offset (a refinement patch's view inside its
// padded box); the tensor maps then describe the storage and each tile aligns its
// boxes itself.
#include <cuda.h>

#include "sbm_common.cuh"

namespace sbm {

namespace {

constexpr int TXP = 32, TYP = 12;                // cells per tile in x, y
constexpr int BXP = TXP + 1, BYP = TYP + 1;      // threads per CTA in x, y
constexpr int NTP = BXP * BYP;                   // 429: 14 warps, so 128 registers a thread
constexpr int PXF = TXP + 2, PYF = TYP + 2, PPF = PXF * PYF;   // exchange grid (last row/column zero)
// Boxes (x width a multiple of 4 floats; each starts at a 16-byte aligned x):
constexpr int UW = 40, UH = TYP + 2;             // u: nodes x0-1 .. x0+32, y0-1 .. y0+TYP
constexpr int FW = 36, FH = TYP + 1;             // f: nodes x0 .. x0+32, y0 .. y0+TYP
constexpr int CW = 40, CH = TYP + 2;             // psi: cells x0-1 .. x0+32, y0-1 .. y0+TYP
constexpr int U_FLOATS = 3 * UH * UW, F_FLOATS = 3 * FH * FW, C_FLOATS = CH * CW;
constexpr int up32(int n) { return (n + 31) / 32 * 32; }   // 128-byte aligned TMA destinations
constexpr int F_OFF = up32(U_FLOATS), C_OFF = F_OFF + up32(F_FLOATS), SLOT_FLOATS = up32(C_OFF + C_FLOATS);
constexpr int TX_BYTES = (U_FLOATS + F_FLOATS + C_FLOATS) * 4;   // bytes one plane's three copies deliver
constexpr int RING = 10;
constexpr int NXQ = 9;                           // exchanged corner forces per cell: corners 0..2 x 3 comps
constexpr long long kSpinLimit = 1LL << 24;      // mbarrier polls before giving up
constexpr size_t kSmemBytes = 128 + (size_t)RING * SLOT_FLOATS * 4 + (size_t)2 * NXQ * PPF * 8 + RING * 8;
static_assert(kSmemBytes <= 227 * 1024, "one CTA per SM must fit");
static_assert((size_t)RING * SLOT_FLOATS * 4 >= 32 * 32 * 8, "the ring doubles as the reduction buffer");

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (long long i = 0; i < kSpinLimit; ++i)
        if (mbar_try(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y, int z, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int x, int y, int z, int c,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(c), "r"(bar)
        : "memory");
}

// 1 / x by the hardware's approximate reciprocal (PTX rcp.approx, within one ulp):
// the Jacobi scaling 1 / sum(psi) of a smoother needs no correctly rounded quotient.
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void prefetch_map(const CUtensorMap *map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Dirichlet bits (bit p = component p) of node (gx, gy, *) from the x and y faces;
// the z faces are added per plane.
__device__ __forceinline__ unsigned dir_xy(const Geom &g, int gx, int gy)
{
    unsigned b = 0;
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const unsigned m = g.dm[p];
        if (((m & 1u) && gx == 0) || ((m & 2u) && gx == g.nx - 1) || ((m & 4u) && gy == 0) ||
            ((m & 8u) && gy == g.ny - 1))
            b |= 1u << p;
    }
    return b;
}

__device__ __forceinline__ unsigned dir_z(const Geom &g, int gz)
{
    unsigned b = 0;
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const unsigned m = g.dm[p];
        if (((m & 16u) && gz == 0) || ((m & 32u) && gz == g.nz - 1)) b |= 1u << p;
    }
    return b;
}

// Segments of a CTA's unit range: units are (tile, node plane) in tile-major order
// with nz planes per tile.  Node planes [p0, p1] of tile t need cell layers
// p0-1 .. p1 (those inside the grid); they are swept as npairs steps of two
// layers from kfirst, reading planes kfirst .. kfirst + 2 npairs (planes beyond
// the grid read zeros).
struct Seg {
    int t, p0, p1, kfirst, npairs;
};

__device__ __forceinline__ Seg make_seg(int u, int ue, int nz)
{
    Seg s;
    s.t = u / nz;
    const int base = s.t * nz;
    s.p0 = u - base;
    s.p1 = min(ue - base, nz) - 1;
    s.kfirst = s.p0 > 0 ? s.p0 - 1 : 0;
    // a step from layer k finalises node planes k and k+1, so the last step must
    // start at p1 - 1 or later; layers beyond the grid (k >= nz - 1) read psi = 0
    s.npairs = (s.p1 - s.kfirst) / 2 + 1;
    return s;
}

// Cursor of the plane producer (thread 0).
struct Prod {
    int u;            // first unit of the next segment
    int seq;          // sequence number of the next plane to issue
    int t, next, last;   // current segment: tile, next plane to issue, last plane
};

// Tile origin (cells / nodes) and the 4-aligned box starts of a tile.
struct TileBox {
    int x0, y0;       // first owned node (and the cell to its upper right) of the tile
    int xs, xoff;     // u and psi boxes start at node / cell xs = x0 - 1 + org.x - xoff
    int xsf, xofff;   // f box starts at node xsf = x0 + org.x - xofff
};

__device__ __forceinline__ TileBox tile_box(int t, int ntx, int3 org)
{
    TileBox b;
    b.x0 = (t % ntx) * TXP;
    b.y0 = (t / ntx) * TYP;
    const int xv = b.x0 - 1 + org.x;
    b.xoff = ((xv % 4) + 4) % 4;
    b.xs = xv - b.xoff;
    const int xf = b.x0 + org.x;
    b.xofff = xf % 4;
    b.xsf = xf - b.xofff;
    return b;
}

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
        if (tid == 0) part[blockIdx.x] = s;
    }
}

template <int MODE>
__device__ __forceinline__ void finalize_node(const SweepArgs<float, float> &a, float *outc, unsigned dm, int gz,
                                              const float (&Ku)[3], float ip, const float (&uv)[3],
                                              const float (&fv)[3], double &ssq)
{
    const Geom &g = a.g;
    float *o = outc + (long long)g.sy * gz;
    if (MODE == kJacobi) {
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            float v = uv[p];
            if (!((dm >> p) & 1u)) v = madd((fv[p] - Ku[p]) * ip, a.wk[p], v);
            o[p * g.cs] = v;
        }
    } else if (MODE == kResidual) {
        float s = 0.f;
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            const float r = ((dm >> p) & 1u) ? 0.0f : fv[p] - Ku[p];
            o[p * g.cs] = r;
            s = fmaf(r, r, s);
        }
        if (a.part) ssq += double(s);
    } else {
#pragma unroll
        for (int p = 0; p < 3; ++p) o[p * g.cs] = Ku[p];
    }
}

template <int MODE>
__global__ void __launch_bounds__(NTP, 1) k_sweep3_f2(const __grid_constant__ CUtensorMap tmap,
                                                       const __grid_constant__ CUtensorMap tmap_f,
                                                       const __grid_constant__ CUtensorMap tmap_psi,
                                                       const SweepArgs<float, float> a, const int3 org, int *err)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    float *ring = reinterpret_cast<float *>(base);
    float2 *fx = reinterpret_cast<float2 *>(base + (size_t)RING * SLOT_FLOATS * 4);   // [2][NXQ][PPF]
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(fx + 2 * NXQ * PPF);

    const Geom &g = a.g;
    const int tid = threadIdx.x + BXP * threadIdx.y;
    int tx, ty;
    row_warp_xy<BYP>(tid, tx, ty);

    // set-up that reads nothing a predecessor kernel writes
    if (tid == 0) {
        for (int s = 0; s < RING; ++s) mbar_init(smem_addr(&bar[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        prefetch_map(&tmap);
        prefetch_map(&tmap_f);
        prefetch_map(&tmap_psi);
    }
    // the exchange grid's last row and column (no cell beyond the tile) stay zero
    for (int s = tid; s < PPF; s += NTP) {
        const int lx = s % PXF, ly = s / PXF;
        if (lx == BXP || ly == BYP)
            for (int q = 0; q < 2 * NXQ; ++q) fx[q * PPF + s] = make_float2(0.f, 0.f);
    }
    pdl_begin();
    if (a.gate && *a.gate) return;
    __syncthreads();

    const int ntx = (g.nx - 2) / TXP + 1, nty = (g.ny - 2) / TYP + 1;
    const long long U = (long long)ntx * nty * g.nz;   // < 2^31 (checked by the launcher)
    const int ub = (int)(U * blockIdx.x / gridDim.x), ue = (int)(U * (blockIdx.x + 1) / gridDim.x);

    // ---- producer (thread 0): issues the planes of the CTA's segments in order.
    // Its cursor lives in shared memory, so the other threads hold no registers for it.
    __shared__ Prod prod;
    auto issue_upto = [&](int limit) {   // issue every plane with sequence number < limit
        Prod P = prod;
        while (P.seq < limit) {
            if (P.next > P.last) {
                if (P.u >= ue) break;
                const Seg s = make_seg(P.u, ue, g.nz);
                P.u = s.t * g.nz + s.p1 + 1;
                P.t = s.t;
                P.next = s.kfirst;
                P.last = s.kfirst + 2 * s.npairs;
            }
            const TileBox b = tile_box(P.t, ntx, org);
            const int slot = (int)(P.seq % RING);
            const uint32_t mb = smem_addr(&bar[slot]);
            float *dst = ring + slot * SLOT_FLOATS;
            mbar_expect_tx(mb, TX_BYTES);
            tma_load_4d(smem_addr(dst), &tmap, b.xs, b.y0 - 1 + org.y, P.next + org.z, 0, mb);
            tma_load_4d(smem_addr(dst + F_OFF), &tmap_f, b.xsf, b.y0 + org.y, P.next + org.z, 0, mb);
            tma_load_3d(smem_addr(dst + C_OFF), &tmap_psi, b.xs, b.y0 - 1 + org.y, P.next + org.z, mb);
            ++P.next;
            ++P.seq;
        }
        prod = P;
    };
    if (tid == 0) {
        prod.u = ub;
        prod.seq = 0;
        prod.t = 0;
        prod.next = 0;
        prod.last = -1;
        issue_upto(RING);
    }

    const int me = ty * PXF + tx;
    double ssq = 0.0;
    bool failed = false;
    // the consumer's position in the plane sequence: slot and phase parity of the
    // plane a step starts from, and its sequence number
    int cseq = 0, cslot = 0;
    uint32_t cpar = 0;
    int buf = 0;
    auto nxt = [](int &slot, uint32_t &par) {
        if (++slot == RING) {
            slot = 0;
            par ^= 1u;
        }
    };
    auto full_wait = [&](int slot, uint32_t par) { return mbar_wait(smem_addr(&bar[slot]), par); };

    for (int u = ub; u < ue && !failed;) {
        const Seg s = make_seg(u, ue, g.nz);
        u = s.t * g.nz + s.p1 + 1;
        const TileBox b = tile_box(s.t, ntx, org);
        const int gx = b.x0 + tx, gy = b.y0 + ty;
        const bool own = gx < g.nx && gy < g.ny && (tx < TXP || gx == g.nx - 1) && (ty < TYP || gy == g.ny - 1);
        float *const outc = a.out + (own ? gx + (long long)g.sx * gy : 0);
        const unsigned dxy = own ? dir_xy(g, gx, gy) : 0u;
        const int ou = ty * UW + tx + b.xoff;     // corner 0 of this thread's cell in the u box
        const int oc = ty * CW + tx + b.xoff;     // this thread's cell in the psi box
        const int of = ty * FW + tx + b.xofff;    // the owned node in the f box

        // prime: the in-plane transform of plane kfirst
        float Tc[3][4];
        {
            int ok = full_wait(cslot, cpar);
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            const float *P = ring + cslot * SLOT_FLOATS;
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                const float *Q = P + p * UH * UW + ou;
                Tc[p][0] = Q[0];
                Tc[p][1] = Q[1];
                Tc[p][2] = Q[UW];
                Tc[p][3] = Q[UW + 1];
                bfly4xy(Tc[p]);
            }
        }
        float Fc[3][4];
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) Fc[p][q] = 0.f;
        float sprev = 0.f;                       // in-plane psi sum of the layer below (Jacobi)

#pragma unroll 2
        for (int it = 0; it < s.npairs; ++it) {
            const int k = s.kfirst + 2 * it;
            // planes k, k+1, k+2 in slots s0, s1, s2
            int s1 = cslot, s2;
            uint32_t r1 = cpar, r2;
            nxt(s1, r1);
            s2 = s1;
            r2 = r1;
            nxt(s2, r2);
            const int ok = full_wait(s1, r1) && full_wait(s2, r2);
            const float *P0 = ring + cslot * SLOT_FLOATS, *P1 = ring + s1 * SLOT_FLOATS, *P2 = ring + s2 * SLOT_FLOATS;
            const bool fin0 = own && k >= s.p0 && k <= s.p1;
            const bool fin1 = own && k + 1 >= s.p0 && k + 1 <= s.p1;

            // raw u of planes k+1, k+2 at the cell's four in-plane corners, then the
            // in-plane transform of both planes in one packed pass
            F2 Tt[3][4];
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                const int o = p * UH * UW + ou;
                Tt[p][0] = F2(P1[o], P2[o]);
                Tt[p][1] = F2(P1[o + 1], P2[o + 1]);
                Tt[p][2] = F2(P1[o + UW], P2[o + UW]);
                Tt[p][3] = F2(P1[o + UW + 1], P2[o + UW + 1]);
                bfly4xy(Tt[p]);
            }
            F2 Tb[3][4];
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    Tb[p][q] = F2(Tc[p][q], Tt[p][q].v.x);
                    Tc[p][q] = Tt[p][q].v.y;
                }
            // psi of the cell in layers k, k+1 times the moduli constants (scalar
            // products with the constant-bank parameters)
            F2 kc[7];
            {
                const float q0v = P0[C_OFF + oc], q1v = P1[C_OFF + oc];
                const float cc[7] = {a.c.ad, a.c.a12, a.c.a44, a.c.b1, a.c.b12, a.c.b44, a.c.c2};
#pragma unroll
                for (int i = 0; i < 7; ++i) kc[i] = F2(q0v * cc[i], q1v * cc[i]);
            }
            F2 Fb[3][4], Ft[3][4];
            cell_faces3k<F2>(Tb, Tt, kc, Fb, Ft);
            // node planes k (top of layer k-1 + bottom of layer k) and k+1 (top of k +
            // bottom of k+1), transformed back to the four in-plane corners
            F2 N[3][4];
#pragma unroll
            for (int p = 0; p < 3; ++p) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    N[p][q] = F2(Fc[p][q] + Fb[p][q].v.x, Ft[p][q].v.x + Fb[p][q].v.y);
                    Fc[p][q] = Ft[p][q].v.y;
                }
                bfly4xyT(N[p]);
            }
            float2 *X = fx + buf * NXQ * PPF;
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int c = 0; c < 3; ++c) X[(p * 3 + c) * PPF + me] = N[p][c].v;

            // what the finalisation needs from planes k and k+1, read before the
            // barrier (their slots are refilled right after it): u and f at the owned
            // node and, for Jacobi, the psi of the eight cells around it
            float uv0[3] = {0.f, 0.f, 0.f}, uv1[3] = {0.f, 0.f, 0.f};
            float fv0[3] = {0.f, 0.f, 0.f}, fv1[3] = {0.f, 0.f, 0.f};
            float sp0 = 0.f, sp1 = 0.f;
            if (own) {
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                    if (MODE == kJacobi) {
                        uv0[p] = P0[p * UH * UW + ou + UW + 1];
                        uv1[p] = P1[p * UH * UW + ou + UW + 1];
                    }
                    if (MODE != kApply) {
                        fv0[p] = P0[F_OFF + p * FH * FW + of];
                        fv1[p] = P1[F_OFF + p * FH * FW + of];
                    }
                }
                if (MODE == kJacobi) {
                    const float *C0 = P0 + C_OFF + oc, *C1 = P1 + C_OFF + oc;
                    sp0 = (C0[0] + C0[1]) + (C0[CW] + C0[CW + 1]);
                    sp1 = (C1[0] + C1[1]) + (C1[CW] + C1[CW + 1]);
                }
            }

            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            cseq += 2;
            cslot = s2;
            cpar = r2;
            if (tid == 0) {
                // planes k and k+1 are no longer read (after the segment's last step
                // plane k+2 is not either)
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue_upto(cseq + (it + 1 == s.npairs ? 1 : 0) + RING);
            }
            if (own) {
                // node = corner 3 of this cell, 2 of (tx+1,ty), 1 of (tx,ty+1), 0 of (tx+1,ty+1)
                F2 Ku2[3];
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                    F2 a1, a2, a3;
                    a1.v = X[(p * 3 + 2) * PPF + me + 1];
                    a2.v = X[(p * 3 + 1) * PPF + me + PXF];
                    a3.v = X[(p * 3 + 0) * PPF + me + PXF + 1];
                    Ku2[p] = (N[p][3] + a1) + (a2 + a3);
                }
                if (fin0) {
                    const float Ku[3] = {Ku2[0].v.x, Ku2[1].v.x, Ku2[2].v.x};
                    const float ip = MODE == kJacobi ? rcp_approx(sprev + sp0) : 0.f;
                    finalize_node<MODE>(a, outc, dxy | dir_z(g, k), k, Ku, ip, uv0, fv0, ssq);
                }
                if (fin1) {
                    const float Ku[3] = {Ku2[0].v.y, Ku2[1].v.y, Ku2[2].v.y};
                    const float ip = MODE == kJacobi ? rcp_approx(sp0 + sp1) : 0.f;
                    finalize_node<MODE>(a, outc, dxy | dir_z(g, k + 1), k + 1, Ku, ip, uv1, fv1, ssq);
                }
            }
            sprev = sp1;
            buf ^= 1;
        }
        if (!failed) {                           // past the segment's last plane
            ++cseq;
            nxt(cslot, cpar);
        }
    }
    if (failed) {
        if (tid == 0) {
            atomicExch(err, 1);
            // wait (bounded) for the copies still in flight: the last RING issued
            // (earlier ones have completed or were consumed)
            for (int q = max(cseq, prod.seq - RING); q < prod.seq; ++q)
                mbar_wait(smem_addr(&bar[q % RING]), (uint32_t)((q / RING) & 1));
        }
        __syncthreads();
        return;
    }
    if (MODE == kResidual && a.part) {
        __syncthreads();                          // every copy has been consumed: reuse the ring
        block_partial<NTP>(ssq, a.part, reinterpret_cast<double *>(ring));
    }
}

int sm_count()
{
    static int count[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (count[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
        count[dev] = n;
    }
    return count[dev];
}

// CTAs of one launch: one per SM, fewer when a CTA would get less than two node
// planes (small levels).
int ctas_f2(const Geom &g)
{
    const long long ntx = (g.nx - 2) / TXP + 1, nty = (g.ny - 2) / TYP + 1;
    const long long units = ntx * nty * g.nz;
    return (int)std::max(1LL, std::min((long long)sm_count(), units / 2));
}

}  // namespace

void tma_box_shapes(int u[2], int f[2], int c[2])
{
    u[0] = UW; u[1] = UH;
    f[0] = FW; f[1] = FH;
    c[0] = CW; c[1] = CH;
}

template <int MODE>
static cudaError_t launch_f2_mode(const SweepArgs<float, float> &a, const CUtensorMap *tmap, int *err, cudaStream_t s,
                                  int3 org)
{
    static std::atomic<unsigned long long> attr_done{0};
    cudaError_t ea = smem_attr_once(reinterpret_cast<const void *>(k_sweep3_f2<MODE>), kSmemBytes, attr_done);
    if (ea != cudaSuccess) return ea;
    cudaError_t e = launch_pdl(k_sweep3_f2<MODE>, dim3(ctas_f2(a.g)), dim3(BXP, BYP), kSmemBytes, s, tmap[0], tmap[1],
                               tmap[2], a, org, err);
    if (e != cudaSuccess) return e;
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_sweep_f2(int mode, const SweepArgs<float, float> &a, const void *tmap, int *err, cudaStream_t s,
                            int3 org)
{
    const CUtensorMap *m = static_cast<const CUtensorMap *>(tmap);
    if (org.x < 0 || org.y < 0 || org.z < 0 || a.g.dim != 3 || a.g.nx < 2 || a.g.ny < 2 || a.g.nz < 2)
        return cudaErrorInvalidValue;
    // the work split counts (tile, plane) units in 32-bit integers
    if ((long long)((a.g.nx - 2) / TXP + 1) * ((a.g.ny - 2) / TYP + 1) * a.g.nz >= (1LL << 31))
        return cudaErrorInvalidValue;
    switch (mode) {
    case kApply: return launch_f2_mode<kApply>(a, m, err, s, org);
    case kResidual: return launch_f2_mode<kResidual>(a, m, err, s, org);
    case kJacobi: return launch_f2_mode<kJacobi>(a, m, err, s, org);
    default: return cudaErrorInvalidValue;
    }
}

long long sweep_blocks_f2(const Geom &g) { return ctas_f2(g); }

}  // namespace sbm
