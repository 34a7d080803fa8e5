// k_stencil_tma.cu — FP32 3D apply / residual / damped-Jacobi sweep of the
// cell-flux SBM elasticity operator with TMA plane staging and packed FP32x2
// arithmetic (sm_100+ FFMA2 / FADD2 / FMUL2).
//
// Block = 32 x 8 cells in x/y (33 x 9 threads, one cell column each, the first
// row/column being the one-cell halo; warps aligned with the 32-cell rows),
// streaming a chunk of z.  Each step handles
// two cell layers (k, k+1) at once: every thread evaluates its two cells in the
// two lanes of the packed type, so one packed instruction does the work of two.
// Node planes of u and f and cell layers of psi are fetched by the Tensor Memory
// Accelerator into a 6-deep shared-memory ring (40 x 10 x 3 boxes of u and f and a
// 40 x 10 box of psi per slot, out-of-range elements zero filled), two pairs ahead
// of use, completion signalled by one mbarrier per slot; the compute loop issues
// no global loads.  Corner
// forces of both node planes a cell touches in this step are exchanged as one
// float2 per corner and component; the top-plane forces of layer k+1 stay in
// registers and join the next step.  Every mbarrier wait is bounded: on timeout
// the block records an error code, waits (bounded) for its copies in flight and
// returns.  The grid swept may sit inside a larger storage at an offset (a
// refinement patch's view inside its padded box); the tensor maps then describe
// the storage and each block aligns its boxes itself.
#include <cuda.h>

#include "sbm_common.cuh"

namespace sbm {

namespace {

constexpr int TXP = 32, TYP = 8;                 // cells per block in x, y
constexpr int BXP = TXP + 1, BYP = TYP + 1;      // threads per block in x, y
constexpr int NTP = BXP * BYP;
constexpr int PXF = TXP + 2, PYF = TYP + 2, PPF = PXF * PYF;   // exchange tiles
constexpr int WX = 40;                           // TMA box width: 34 nodes x0-1 .. x0+32 plus alignment
constexpr int PLANE_FLOATS = 3 * PYF * WX;       // one staged plane: 3 comps x 10 rows x 40
constexpr int PSI_FLOATS = PYF * WX;             // one staged cell layer of psi
// A ring slot holds node plane p of u, node plane p of f and cell layer p of psi.
// Every TMA destination starts on a 128-byte boundary.
constexpr int PLANE_STRIDE = (PLANE_FLOATS * 4 + 127) / 128 * 128 / 4;   // floats
constexpr int F_OFF = PLANE_STRIDE, PSI_OFF = 2 * PLANE_STRIDE;
constexpr int SLOT_FLOATS = ((PSI_OFF + PSI_FLOATS) * 4 + 127) / 128 * 128 / 4;
constexpr int TX_BYTES = (2 * PLANE_FLOATS + PSI_FLOATS) * 4;           // bytes the three copies deliver
static_assert((F_OFF * 4) % 128 == 0 && (PSI_OFF * 4) % 128 == 0 && (SLOT_FLOATS * 4) % 128 == 0,
              "TMA destinations must be 128-byte aligned");
constexpr int RING = 6;
constexpr long long kSpinLimit = 1LL << 24;      // mbarrier polls before giving up

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

template <int NT>
__device__ __forceinline__ void block_partial_f(double ssq, double *part, double *red)
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

// out: this thread's node column (gx, gy) of component 0; dxy: its x/y Dirichlet
// bits.  The residual's sum of squares is formed only when a norm is wanted.
template <int MODE>
__device__ __forceinline__ void finalize_f(const SweepArgs<float, float> &a, float *outc, unsigned dxy, int gz,
                                           const float *Ku, float pss, const float *uv, const float *fv, double &ssq)
{
    const Geom &g = a.g;
    float *o = outc + (long long)g.sy * gz;
    const unsigned dm = dxy | dir_z(g, gz);
    if (MODE == kJacobi) {
        const float ip = __frcp_rn(pss);
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
__global__ void __launch_bounds__(NTP) k_sweep3_f2(const __grid_constant__ CUtensorMap tmap,
                                                    const __grid_constant__ CUtensorMap tmap_f,
                                                    const __grid_constant__ CUtensorMap tmap_psi,
                                                    const SweepArgs<float, float> a, const int3 org, int *err)
{
    pdl_begin();
    if (a.gate && *a.gate) return;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    float *ring = reinterpret_cast<float *>(base);
    float2 *fx = reinterpret_cast<float2 *>(base + RING * SLOT_FLOATS * 4);   // [3][4][PPF]
    float2 *ps = fx + 12 * PPF;                                               // [PPF]
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(ps + PPF);
    __shared__ double red[((NTP + 31) / 32) * 32];

    const Geom &g = a.g;
    const int tid = threadIdx.x + BXP * threadIdx.y;
    int tx, ty;
    row_warp_xy<BYP>(tid, tx, ty);
    const int x0 = blockIdx.x * TXP, y0 = blockIdx.y * TYP;
    // The tensor maps describe the storage the sweep's grid sits in at offset org
    // (0 for a whole level, the view origin for a refinement patch).  The boxes
    // start at the multiple of 4 at or below node x0-1 (a TMA box's x coordinate
    // must be 16-byte aligned), xoff in 0..3 being node x0-1's box-local x; the
    // 40-wide box covers the 34 nodes x0-1 .. x0+32 for any xoff.
    const int xv = x0 - 1 + org.x;
    const int xs = xv - (((xv % 4) + 4) % 4);
    const int xoff = xv - xs;
    const int ybox = y0 - 1 + org.y;
    const int kz0 = blockIdx.z * a.kchunk;
    const int kz1 = min(kz0 + a.kchunk, g.nz - 1);
    const int kend = (kz1 == g.nz - 1) ? g.nz - 1 : kz1 - 1;   // last plane finalised here
    const int kfirst = kz0 > 0 ? kz0 - 1 : 0;
    const int npairs = (kend - kfirst) / 2 + 1;
    const int pmax = kfirst + 2 * (npairs - 1) + 2;            // last plane the block reads

    if (tid == 0) {
        for (int s = 0; s < RING; ++s) mbar_init(smem_addr(&bar[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int s = tid; s < PPF; s += NTP) {
        const int lx = s % PXF, ly = s / PXF;
        if (lx == BXP || ly == BYP) {
            for (int q = 0; q < 12; ++q) fx[q * PPF + s] = make_float2(0.f, 0.f);
            ps[s] = make_float2(0.f, 0.f);
        }
    }
    __syncthreads();

    auto slot_of = [&](int p) { return (p - kfirst) % RING; };
    auto parity_of = [&](int p) { return (uint32_t)(((p - kfirst) / RING) & 1); };
    auto issue = [&](int p) {
        if (p > pmax) return;
        const int s = slot_of(p);
        const uint32_t b = smem_addr(&bar[s]);
        mbar_expect_tx(b, TX_BYTES);
        float *slot = ring + s * SLOT_FLOATS;
        tma_load_4d(smem_addr(slot), &tmap, xs, ybox, p + org.z, 0, b);
        tma_load_4d(smem_addr(slot + F_OFF), &tmap_f, xs, ybox, p + org.z, 0, b);
        tma_load_3d(smem_addr(slot + PSI_OFF), &tmap_psi, xs, ybox, p + org.z, b);
    };
    if (tid == 0)
        for (int j = 0; j < RING; ++j) issue(kfirst + j);
    int issued_last = kfirst + RING - 1;

    Coef<F2> c2;
    c2.ad = F2(a.c.ad); c2.a12 = F2(a.c.a12); c2.a44 = F2(a.c.a44); c2.a11 = F2(a.c.a11);
    c2.b1 = F2(a.c.b1); c2.b12 = F2(a.c.b12); c2.b44 = F2(a.c.b44); c2.c2 = F2(a.c.c2);

    const int gx = x0 + tx, gy = y0 + ty;
    const bool own = gx < g.nx && gy < g.ny && (tx < TXP || gx == g.nx - 1) && (ty < TYP || gy == g.ny - 1);
    float *const outc = a.out + (own ? gx + (long long)g.sx * gy : 0);
    const unsigned dxy = own ? dir_xy(g, gx, gy) : 0u;
    const int me = ty * PXF + tx;
    float carry[3][4];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) carry[p][q] = 0.f;
    float psi_prev = 0.f;
    double ssq = 0.0;
    bool failed = false;

    // lanes of this thread's warp (the last warp of the block is partial)
    const int lane = tid & 31, wlanes = min(32, NTP - (tid & ~31));
    const unsigned wmask = wlanes == 32 ? 0xffffffffu : ((1u << wlanes) - 1u);
    for (int it = 0; it < npairs; ++it) {
        const int k = kfirst + 2 * it;
        // one lane per warp polls the barriers of planes k..k+2 (bounded); the warp
        // proceeds when its lane 0 has seen them complete
        int ok = 1;
        if (lane == 0)
            ok = mbar_wait(smem_addr(&bar[slot_of(k)]), parity_of(k)) &&
                 mbar_wait(smem_addr(&bar[slot_of(k + 1)]), parity_of(k + 1)) &&
                 mbar_wait(smem_addr(&bar[slot_of(k + 2)]), parity_of(k + 2));
        ok = __shfl_sync(wmask, ok, 0);
        // every lane then observes the completed phases itself (acquiring the copied
        // data); a timed-out wait is reported at the exchange barrier below and
        // this warp's values are then never used
        if (ok)
            ok = mbar_try(smem_addr(&bar[slot_of(k)]), parity_of(k)) &&
                 mbar_try(smem_addr(&bar[slot_of(k + 1)]), parity_of(k + 1)) &&
                 mbar_try(smem_addr(&bar[slot_of(k + 2)]), parity_of(k + 2));
        const float *P0 = ring + slot_of(k) * SLOT_FLOATS;
        const float *P1 = ring + slot_of(k + 1) * SLOT_FLOATS;
        const float *P2 = ring + slot_of(k + 2) * SLOT_FLOATS;
        // cell (x0+tx-1, y0+ty-1) of layers k, k+1; the tensor map zero-fills cells
        // outside the grid, so no bounds test is needed
        const float p0 = P0[PSI_OFF + ty * WX + tx + xoff];
        const float p1 = P1[PSI_OFF + ty * WX + tx + xoff];
        F2 U[3][8];
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int off = p * PYF * WX + (ty + (q >> 1)) * WX + tx + (q & 1) + xoff;
                const float v0 = P0[off], v1 = P1[off], v2 = P2[off];
                U[p][q] = F2(v0, v1);        // lower corners of cells k, k+1
                U[p][q + 4] = F2(v1, v2);    // upper corners
            }
        cell_forces3<F2>(U, F2(p0, p1), c2);
        // this thread's cell contributions to node plane k (carry + layer k bottom) and
        // node plane k+1 (layer k top + layer k+1 bottom); layer k+1 top is carried
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                fx[(p * 4 + q) * PPF + me] = make_float2(carry[p][q] + U[p][q].v.x, U[p][q + 4].v.x + U[p][q].v.y);
                carry[p][q] = U[p][q + 4].v.y;
            }
        ps[me] = make_float2(psi_prev + p0, p0 + p1);
        psi_prev = p1;
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        if (own) {
            // node = corner 3 of cell (tx,ty), 2 of (tx+1,ty), 1 of (tx,ty+1), 0 of (tx+1,ty+1)
            F2 Ku2[3];
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                F2 s0, s1, s2, s3;
                s0.v = fx[(p * 4 + 3) * PPF + me];
                s1.v = fx[(p * 4 + 2) * PPF + me + 1];
                s2.v = fx[(p * 4 + 1) * PPF + me + PXF];
                s3.v = fx[(p * 4 + 0) * PPF + me + PXF + 1];
                Ku2[p] = (s0 + s1) + (s2 + s3);
            }
            F2 q0, q1, q2, q3;
            q0.v = ps[me];
            q1.v = ps[me + 1];
            q2.v = ps[me + PXF];
            q3.v = ps[me + PXF + 1];
            const F2 pss = (q0 + q1) + (q2 + q3);
            const int onode = (ty + 1) * WX + tx + 1 + xoff;
            if (k >= kz0 && k <= kend) {
                const float Ku[3] = {Ku2[0].v.x, Ku2[1].v.x, Ku2[2].v.x};
                const float uv[3] = {P0[onode], P0[PYF * WX + onode], P0[2 * PYF * WX + onode]};
                const float fv[3] = {P0[F_OFF + onode], P0[F_OFF + PYF * WX + onode], P0[F_OFF + 2 * PYF * WX + onode]};
                finalize_f<MODE>(a, outc, dxy, k, Ku, pss.v.x, uv, fv, ssq);
            }
            if (k + 1 >= kz0 && k + 1 <= kend) {
                const float Ku[3] = {Ku2[0].v.y, Ku2[1].v.y, Ku2[2].v.y};
                const float uv[3] = {P1[onode], P1[PYF * WX + onode], P1[2 * PYF * WX + onode]};
                const float fv[3] = {P1[F_OFF + onode], P1[F_OFF + PYF * WX + onode], P1[F_OFF + 2 * PYF * WX + onode]};
                finalize_f<MODE>(a, outc, dxy, k + 1, Ku, pss.v.y, uv, fv, ssq);
            }
        }
        __syncthreads();
        if (tid == 0) {
            // planes k and k+1 are no longer read: refill their slots
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(k + RING);
            issue(k + 1 + RING);
            issued_last = k + 1 + RING;
        }
    }
    if (failed) {
        if (tid == 0) {
            atomicExch(err, 1);
            // wait (bounded) for every copy this block issued that has not been consumed
            const int last = min(issued_last, pmax);
            for (int p = max(kfirst, last - RING + 1); p <= last; ++p) mbar_wait(smem_addr(&bar[slot_of(p)]), parity_of(p));
        }
        __syncthreads();
        return;
    }
    if (MODE == kResidual && a.part) block_partial_f<NTP>(ssq, a.part, red);
}

constexpr size_t smem_f2()
{
    return 128 + (size_t)RING * SLOT_FLOATS * 4 + (size_t)13 * PPF * 8 + RING * 8;
}

}  // namespace

void sweep_grid_f2(const Geom &g, int *grid, int *kchunk)
{
    grid[0] = (g.nx - 1 + TXP - 1) / TXP;
    grid[1] = (g.ny - 1 + TYP - 1) / TYP;
    const int nzc = g.nz - 1;
    const int nc = choose_chunks((long long)grid[0] * grid[1], nzc, 2 * 152, true);   // two blocks per SM
    const int ch = (nzc + nc - 1) / nc;
    grid[2] = (nzc + ch - 1) / ch;
    *kchunk = ch;
}

template <int MODE>
static cudaError_t launch_f2_mode(const SweepArgs<float, float> &a0, const CUtensorMap *tmap, int *err, cudaStream_t s,
                                  int3 org)
{
    SweepArgs<float, float> a = a0;
    int grid[3];
    sweep_grid_f2(a.g, grid, &a.kchunk);
    static std::atomic<unsigned long long> attr_done{0};
    const size_t sm = smem_f2();
    cudaError_t ea = smem_attr_once(reinterpret_cast<const void *>(k_sweep3_f2<MODE>), sm, attr_done);
    if (ea != cudaSuccess) return ea;
    cudaError_t e = launch_pdl(k_sweep3_f2<MODE>, dim3(grid[0], grid[1], grid[2]), dim3(BXP, BYP), sm, s, tmap[0], tmap[1],
                               tmap[2], a, org, err);
    if (e != cudaSuccess) return e;
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_sweep_f2(int mode, const SweepArgs<float, float> &a, const void *tmap, int *err, cudaStream_t s,
                            int3 org)
{
    const CUtensorMap *m = static_cast<const CUtensorMap *>(tmap);
    if (org.x < 0 || org.y < 0 || org.z < 0) return cudaErrorInvalidValue;
    switch (mode) {
    case kApply: return launch_f2_mode<kApply>(a, m, err, s, org);
    case kResidual: return launch_f2_mode<kResidual>(a, m, err, s, org);
    case kJacobi: return launch_f2_mode<kJacobi>(a, m, err, s, org);
    default: return cudaErrorInvalidValue;
    }
}

long long sweep_blocks_f2(const Geom &g)
{
    int grid[3], ch;
    sweep_grid_f2(g, grid, &ch);
    return (long long)grid[0] * grid[1] * grid[2];
}

}  // namespace sbm
