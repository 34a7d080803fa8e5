// sbm_api.cu — the C ABI (include/sbm.h): grid and level hierarchy, set-up of
// psi / moduli / boundary conditions, the multigrid driver (FP64 V-cycles, or
// FP32 V-cycles inside an FP64 defect correction), CUDA-graph replay of one
// outer iteration, the adjoint solve and the single-step entry points.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <chrono>
#include <atomic>
#include <type_traits>
#include <string>
#include <vector>

#include "../../include/sbm.h"
#include "sbm_common.cuh"

using namespace sbm;

bool sbm::is_dev_ptr(const void *p, int dev)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

namespace {

thread_local std::string g_lib_error;
// Cap on the device bytes one grid may allocate (0: none), for tests of the
// out-of-memory path without real memory pressure.
std::atomic<unsigned long long> g_alloc_cap{0};

struct Level {
    Geom g{};
    double h = 0;
    double *psi64 = nullptr;
    float *psi32 = nullptr;
    double *du[2] = {nullptr, nullptr}, *df = nullptr, *dr = nullptr;
    float *su[2] = {nullptr, nullptr}, *sf = nullptr, *sr = nullptr;
    Coef<double> c64{};
    Coef<float> c32{};
    double *Ke64 = nullptr;   // unit-psi cell matrix (GS smoother)
    float *Ke32 = nullptr;
    CUtensorMap tm32[2][3];   // TMA descriptors {su[i], sf, psi32} for input su[i] (3D levels)
    bool has_tm = false;
};

// One refinement patch (block-structured AMR level a >= 1): node box [lo, hi] in
// level-a indices, stored with one padding node per side.
struct Patch {
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    int level = 0;            // refinement level (1 = children of the base)
    int parent = 0;           // parent patch index (0 = the base level, else 1 .. npatch)
    Geom s{};                 // padded storage (no Dirichlet faces)
    Geom v{};                 // view of the box: interface faces fixed, domain faces as the domain
    long long voff = 0;       // element offset of the view origin in the storage
    double h = 0;
    AmrInfo info{};
    double *psi64 = nullptr;
    float *psi32 = nullptr;
    double *u64 = nullptr, *f64 = nullptr, *r64 = nullptr;
    double *de[2] = {nullptr, nullptr}, *drhs = nullptr, *dres = nullptr;
    float *se[2] = {nullptr, nullptr}, *srhs = nullptr, *sres = nullptr;
    float *psiv32 = nullptr;  // psi32 on the view's cells, 0 on the padding (TMA sweep input)
    double *psi_set = nullptr;  // psi as set (floored), before coarse means of children replace cells
    CUtensorMap tm32[2][3];   // 3D: TMA maps of (se[i], srhs, psiv32) over the storage
    bool has_tm = false;
    Coef<double> c64{};
    Coef<float> c32{};
    double *Ke64 = nullptr;
    float *Ke32 = nullptr;
};

constexpr int kBranches = 8;   // side streams for concurrent patches

struct GraphSlot {
    bool valid = false;
    cudaGraphExec_t exec = nullptr;
    int mixed = 0, smoother = 0, nu1 = 0, nu2 = 0, inner = 0, max_cycles = 0;
    double omega = 0, inner_rtol = 0, tol = 0;
    const double *hist = nullptr;
    const double *rhs = nullptr;
    unsigned version = 0;
    long long body_launches = 0;
};

}  // namespace

struct sbm_grid_s {
    sbm_grid_desc desc{};
    cudaStream_t st = nullptr;
    bool own_stream = false;
    int dev = 0;
    int nl = 0;
    Level L[kMaxLevels];
    double mod[3] = {0, 0, 0};
    bool has_moduli = false, has_psi = false;
    int bct[6][3] = {};
    double bcv[6][3] = {};
    double *fsrc = nullptr, *fadj = nullptr;     // finest-level right-hand sides (level layout)
    double *psi_raw = nullptr, *rho = nullptr;    // packed finest cells
    int density = 0;
    double psi_min = 0, q = 3;
    double *part = nullptr;
    long long npart = 0;
    int *derr = nullptr;        // device error flag of the TMA kernels
    int *dgate = nullptr;       // adaptive inner cycles: [0] gate flag, [1] FP32 V-cycles run
    const int *cur_gate = nullptr;   // gate applied to the launches being enqueued (or null)
    double gate_rtol = 0, gate_tol = 0;
    double *scal = nullptr;     // device scalars, see k_norm_final
    double *hscal = nullptr;    // pinned host copy
    int *dbad = nullptr;
    int nb = 0;                 // bottom dofs
    double *A64 = nullptr, *gjtmp = nullptr;
    unsigned *gjbar = nullptr;  // grid-barrier words of the bottom-level inversion
    long long gj_spins = 0;     // polls per grid barrier before it gives up (0: the default)
    double *dhist = nullptr;    // batched FP64 V-cycles: relres per cycle (device)
    int dhist_cap = 0;
    size_t allocated = 0;       // device bytes allocated for the grid (checked against the cap)
    float *A32 = nullptr;
    int *gather = nullptr;
    bool bottom_ready = false;
    unsigned version = 1;
    GraphSlot slots[2];
    GraphSlot amr_slot;         // one outer iteration of the composite solve
    cudaStream_t side[kBranches] = {};   // branches for the patches of one level
    cudaEvent_t fork_ev = nullptr, join_ev[kBranches] = {};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::string err;
    int npatch = 0;
    Patch P[kMaxPatch];
    AmrInfo base_info{};
    bool amr_psi_dirty = false;
    double *amr_part = nullptr;   // partial sums of the composite norm
    long long amr_npart = 0;
    double *amr_u0 = nullptr, *amr_r0 = nullptr;   // composite solution / residual on the base level
    double *adj[9][kMaxPatch + 1] = {};                // adjoint iteration vectors [vector][patch]
    double *top = nullptr;      // topology optimisation: psi, eta scratch, partial sums, scalars
    double *src_sig = nullptr;  // source terms: cell stresses of the eigenstrain
    size_t src_bytes = 0;
};

namespace {

// cudaMalloc of grid storage, refused (as cudaErrorMemoryAllocation) when the
// grid's total would exceed the cap set by sbm_set_alloc_limit.
cudaError_t gmalloc(sbm_grid G, void **p, size_t bytes)
{
    const unsigned long long cap = g_alloc_cap.load();
    if (cap && G->allocated + bytes > cap) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) G->allocated += bytes;
    return e;
}

sbm_status fail(sbm_grid G, sbm_status st, const std::string &msg)
{
    if (G) G->err = msg;
    else g_lib_error = msg;
    return st;
}

#define CK(...)                                                                               \
    do {                                                                                      \
        cudaError_t e_ = (__VA_ARGS__);                                                       \
        if (e_ != cudaSuccess)                                                                \
            return fail(G, e_ == cudaErrorMemoryAllocation ? SBM_ERR_OOM : SBM_ERR_CUDA,      \
                        std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_));           \
    } while (0)

#define CKE(...)                                  \
    do {                                          \
        cudaError_t e_ = (__VA_ARGS__);           \
        if (e_ != cudaSuccess) return e_;         \
    } while (0)

long long nnodes(const Geom &g) { return (long long)g.nx * g.ny * g.nz; }
long long ncells_h(const Geom &g) { return (long long)(g.nx - 1) * (g.ny - 1) * (g.dim == 3 ? g.nz - 1 : 1); }

template <typename T> struct P;
template <> struct P<double> {
    static double *u(Level &L, int i) { return L.du[i]; }
    static double *f(Level &L) { return L.df; }
    static double *r(Level &L) { return L.dr; }
    static const double *psi(Level &L) { return L.psi64; }
    static const Coef<double> &c(Level &L) { return L.c64; }
    static const double *Ke(Level &L) { return L.Ke64; }
    static const double *A(sbm_grid G) { return G->A64; }
};
template <> struct P<float> {
    static float *u(Level &L, int i) { return L.su[i]; }
    static float *f(Level &L) { return L.sf; }
    static float *r(Level &L) { return L.sr; }
    static const float *psi(Level &L) { return L.psi32; }
    static const Coef<float> &c(Level &L) { return L.c32; }
    static const float *Ke(Level &L) { return L.Ke32; }
    static const float *A(sbm_grid G) { return G->A32; }
};

struct Opts {
    sbm_opts o;
};

template <typename T>
cudaError_t sweep(sbm_grid G, int l, int mode, const T *u, const T *f, T *out, double *part, double omega)
{
    Level &L = G->L[l];
    SweepArgs<T, T> a;
    a.g = L.g;
    a.u = u;
    a.f = f;
    a.psi = P<T>::psi(L);
    a.out = out;
    a.part = part;
    a.c = P<T>::c(L);
    for (int p = 0; p < 3; ++p) a.wk[p] = (L.c64.kdiag[p] != 0.0) ? T(omega / L.c64.kdiag[p]) : T(0);
    a.kchunk = 0;
    a.gate = G->cur_gate;
    return launch_sweep<T, T>(mode, a, G->st);
}

// FP32 3D sweeps: levels of at most kNodeKernelMaxNodes nodes (no norm wanted) use
// the cell-parallel per-node kernel; larger ones whose input is one of the level's
// TMA-described buffers the TMA + packed-FP32x2 block kernel; everything else the
// generic kernel.
template <>
cudaError_t sweep<float>(sbm_grid G, int l, int mode, const float *u, const float *f, float *out, double *part,
                         double omega)
{
    Level &L = G->L[l];
    SweepArgs<float, float> a;
    a.g = L.g;
    a.u = u;
    a.f = f;
    a.psi = L.psi32;
    a.out = out;
    a.part = part;
    a.c = L.c32;
    for (int p = 0; p < 3; ++p) a.wk[p] = (L.c64.kdiag[p] != 0.0) ? float(omega / L.c64.kdiag[p]) : 0.f;
    a.kchunk = 0;
    a.gate = G->cur_gate;
    if (L.g.dim == 3 && part == nullptr && (long long)L.g.nx * L.g.ny * L.g.nz <= kNodeKernelMaxNodes)
        return launch_sweep_node(mode, a, G->st);
    if (L.has_tm && (u == L.su[0] || u == L.su[1]) && (mode == kApply || f == L.sf))
        return launch_sweep_f2(mode, a, L.tm32[u == L.su[0] ? 0 : 1], G->derr, G->st);
    return launch_sweep<float, float>(mode, a, G->st);
}

long long sweep_nblocks(sbm_grid G, int l, bool fp32, const void *u, const void *f)
{
    Level &L = G->L[l];
    if (fp32 && L.has_tm && (u == L.su[0] || u == L.su[1]) && f == L.sf) return sweep_blocks_f2(L.g);
    return sweep_blocks(L.g, !fp32);
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// 3D map of an FP32 cell array (cells at the node index of their lower corner),
// box w x h x 1 cells, zero fill outside the grid's cells.
bool encode_cell_map(CUtensorMap *m, float *buf, const Geom &g, int w, int h)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)(g.nx - 1), (cuuint64_t)(g.ny - 1), (cuuint64_t)(g.nz - 1)};
    cuuint64_t strides[2] = {(cuuint64_t)g.sx * 4, (cuuint64_t)g.sy * 4};
    cuuint32_t box[3] = {(cuuint32_t)w, (cuuint32_t)h, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, buf, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 4D (x, y, z, component) map of one FP32 level buffer; box w x h x 1 x 3 nodes,
// zero fill outside the grid.
bool encode_plane_map(CUtensorMap *m, float *buf, const Geom &g, int w, int h)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, 3};
    cuuint64_t strides[3] = {(cuuint64_t)g.sx * 4, (cuuint64_t)g.sy * 4, (cuuint64_t)g.cs * 4};
    cuuint32_t box[4] = {(cuuint32_t)w, (cuuint32_t)h, 1, 3};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, buf, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The three maps of the TMA sweep for input buffer u, right-hand side f and cells psi.
bool encode_sweep_maps(CUtensorMap (&m)[3], float *u, float *f, float *psi, const Geom &g)
{
    int bu[2], bf[2], bc[2];
    tma_box_shapes(bu, bf, bc);
    return encode_plane_map(&m[0], u, g, bu[0], bu[1]) && encode_plane_map(&m[1], f, g, bf[0], bf[1]) &&
           encode_cell_map(&m[2], psi, g, bc[0], bc[1]);
}

template <typename T>
cudaError_t smooth(sbm_grid G, int l, int &cur, const sbm_opts &o, int nsweeps, bool descending, const T *f)
{
    Level &L = G->L[l];
    const int ncol = 1 << L.g.dim;
    for (int s = 0; s < nsweeps; ++s) {
        if (o.smoother == SBM_MCGS && L.g.dim == 2) {
            CKE(launch_gs2_sweep<T>(L.g, P<T>::psi(L), P<T>::Ke(L), f, P<T>::u(L, cur), P<T>::u(L, 1 - cur),
                                    descending ? 1 : 0, G->st, G->cur_gate));
            cur ^= 1;
        } else if (o.smoother == SBM_MCGS) {
            for (int c = 0; c < ncol; ++c)
                CKE(launch_gs<T>(L.g, P<T>::psi(L), P<T>::Ke(L), f, P<T>::u(L, cur), descending ? ncol - 1 - c : c, G->st,
                                 G->cur_gate));
        } else {
            CKE(sweep<T>(G, l, kJacobi, P<T>::u(L, cur), f, P<T>::u(L, 1 - cur), nullptr, o.omega));
            cur ^= 1;
        }
    }
    return cudaSuccess;
}

size_t level_bytes(const Level &L, size_t elem) { return (size_t)L.g.dim * L.g.cs * elem; }

// V(nu1, nu2) on level l: u = P<T>::u(L, cur), right-hand side f.  Coarse levels
// start from a zero correction; the coarsest is solved with the dense inverse.
template <typename T>
cudaError_t vcycle(sbm_grid G, int l, int &cur, const sbm_opts &o, const T *f)
{
    Level &L = G->L[l];
    if (l == 0) {
        if (G->nl == 1) {
            CKE(sweep<T>(G, 0, kResidual, P<T>::u(L, cur), f, P<T>::r(L), nullptr, 0.0));
            CKE(launch_bottom_apply<T>(G->nb, P<T>::A(G), G->gather, P<T>::r(L), P<T>::u(L, cur), 1, G->st,
                                       G->cur_gate));
        } else {
            CKE(launch_bottom_apply<T>(G->nb, P<T>::A(G), G->gather, f, P<T>::u(L, cur), 0, G->st, G->cur_gate));
        }
        return cudaSuccess;
    }
    Level &C = G->L[l - 1];
    CKE(smooth<T>(G, l, cur, o, o.nu1, false, f));
    if (G->cur_gate && l == G->nl - 1 && std::is_same<T, float>::value) {
        // adaptive inner cycles: the norm of this residual decides whether the
        // FP32 V-cycles of the outer iteration go on
        CKE(sweep<T>(G, l, kResidual, P<T>::u(L, cur), f, P<T>::r(L), G->part, 0.0));
        CKE(launch_inner_gate(G->part, (int)sweep_nblocks(G, l, true, P<T>::u(L, cur), f), G->scal, G->gate_rtol,
                              G->gate_tol, G->dgate, G->dgate + 1, G->st));
    } else {
        CKE(sweep<T>(G, l, kResidual, P<T>::u(L, cur), f, P<T>::r(L), nullptr, 0.0));
    }
    // the restriction also zeroes the coarse correction (the coarsest level's is
    // overwritten by the dense solve), keeping the cycle a chain of kernels
    CKE(launch_restrict<T>(L.g, C.g, P<T>::r(L), P<T>::f(C), G->st, G->cur_gate, l - 1 > 0 ? P<T>::u(C, 0) : nullptr));
    int cc = 0;
    CKE(vcycle<T>(G, l - 1, cc, o, P<T>::f(C)));
    CKE(launch_prolong_add<T>(L.g, C.g, P<T>::u(C, cc), P<T>::u(L, cur), G->st, G->cur_gate));
    CKE(smooth<T>(G, l, cur, o, o.nu2, true, f));
    return cudaSuccess;
}

// FP64 residual of the finest level with block partial sums -> scal[which..].
// In mixed mode the residual is written rounded to FP32 as the inner right-hand side.
cudaError_t residual64(sbm_grid G, const double *rhs, int mixed, int which)
{
    Level &L = G->L[G->nl - 1];
    cudaError_t e;
    if (mixed) {
        SweepArgs<double, float> a;
        a.g = L.g;
        a.u = L.du[0];
        a.f = rhs;
        a.psi = L.psi64;
        a.out = L.sf;
        a.part = G->part;
        a.c = L.c64;
        a.wk[0] = a.wk[1] = a.wk[2] = 0.0;
        a.kchunk = 0;
        e = launch_sweep<double, float>(kResidual, a, G->st);
    } else {
        e = sweep<double>(G, G->nl - 1, kResidual, L.du[0], rhs, L.dr, G->part, 0.0);
    }
    if (e != cudaSuccess) return e;
    return launch_norm_final(G->part, (int)sweep_blocks(L.g, true), G->scal, which, G->st, G->cur_gate);
}

// One outer iteration: V-cycle(s) and the FP64 residual + norm of the result.
cudaError_t enqueue_body(sbm_grid G, const sbm_opts &o, const double *rhs)
{
    const int fine = G->nl - 1;
    Level &L = G->L[fine];
    if (G->desc.precision == SBM_MIXED) {
        CKE(cudaMemsetAsync(L.su[0], 0, level_bytes(L, sizeof(float)), G->st));
        int cur = 0;
        if (o.inner_rtol > 0.0) {
            CKE(cudaMemsetAsync(G->dgate, 0, sizeof(int), G->st));
            G->cur_gate = G->dgate;
            G->gate_rtol = o.inner_rtol;
            G->gate_tol = 0.5 * o.tol;      // margin: the FP32 residual may underestimate the FP64 one
        }
        cudaError_t e = cudaSuccess;
        for (int it = 0; it < o.inner_cycles && e == cudaSuccess; ++it) e = vcycle<float>(G, fine, cur, o, L.sf);
        G->cur_gate = nullptr;
        CKE(e);
        CKE(launch_add<float>((long long)L.g.dim * L.g.cs, L.su[cur], L.du[0], G->st));
        return residual64(G, rhs, 1, 2);
    }
    int cur = 0;
    CKE(vcycle<double>(G, fine, cur, o, rhs));
    if (cur != 0) CKE(cudaMemcpyAsync(L.du[0], L.du[1], level_bytes(L, sizeof(double)), cudaMemcpyDeviceToDevice, G->st));
    return residual64(G, rhs, 0, 2);
}

// FP64 mode with inner_cycles = batch > 1: `batch` V-cycles, each followed by its
// FP64 residual, norm and the device gate that records relres, counts the cycle
// and stops the rest of the batch (every later kernel sees the flag dgate[0] and
// returns) once the tolerance is met or the iteration diverges.
cudaError_t enqueue_fp64_batch(sbm_grid G, const sbm_opts &o, const double *rhs, int batch)
{
    const int fine = G->nl - 1;
    Level &L = G->L[fine];
    G->cur_gate = G->dgate;
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < batch && e == cudaSuccess; ++b) {
        int cur = 0;
        e = vcycle<double>(G, fine, cur, o, rhs);
        if (e == cudaSuccess && cur != 0)
            e = launch_copy_gated((long long)L.g.dim * L.g.cs, L.du[1], L.du[0], G->dgate, G->st);
        if (e == cudaSuccess) e = residual64(G, rhs, 0, 2);
        if (e == cudaSuccess) e = launch_outer_gate(G->scal, o.tol, o.max_cycles, G->dhist, G->dgate, G->st);
    }
    G->cur_gate = nullptr;
    return e;
}

sbm_status setup_bottom(sbm_grid G)
{
    if (G->bottom_ready) return SBM_OK;
    Level &B = G->L[0];
    const long long n = G->nb;
    CK(cudaMemsetAsync(G->A64, 0, sizeof(double) * n * n, G->st));
    CK(launch_bottom_assemble(B.g, B.psi64, B.c64, G->A64, G->st));
    CK(launch_bottom_dirichlet(B.g, G->A64, G->st));
    CK(launch_gauss_jordan(B.g, (int)n, G->A64, G->gjtmp, G->gjbar, G->gj_spins, G->st));
    {
        unsigned hbar[4] = {0, 0, 0, 0};
        CK(cudaMemcpyAsync(hbar, G->gjbar, sizeof(hbar), cudaMemcpyDeviceToHost, G->st));
        CK(cudaStreamSynchronize(G->st));
        if (hbar[2]) return fail(G, SBM_ERR_CUDA, "a grid barrier of the bottom-level inversion timed out");
    }
    CK(launch_round(n * n, G->A64, G->A32, G->st));
    G->bottom_ready = true;
    return SBM_OK;
}

void make_level_coefs(sbm_grid G)
{
    for (int l = 0; l < G->nl; ++l) {
        Level &L = G->L[l];
        L.c64 = make_coef<double>(L.g.dim, L.h, G->mod[0], G->mod[1], G->mod[2]);
        L.c32 = make_coef<float>(L.g.dim, L.h, G->mod[0], G->mod[1], G->mod[2]);
    }
}

sbm_status upload_Ke(sbm_grid G)
{
    for (int l = 0; l < G->nl; ++l) {
        Level &L = G->L[l];
        const int d = L.g.dim, nc = 1 << d, nd = nc * d;
        std::vector<double> Ke(nd * nd);
        std::vector<float> Kf(nd * nd);
        for (int b = 0; b < nc; ++b)
            for (int q = 0; q < d; ++q) {
                if (d == 3) {
                    double U[3][8] = {};
                    U[q][b] = 1.0;
                    cell_forces3<double>(U, 1.0, L.c64);
                    for (int a = 0; a < 8; ++a)
                        for (int p = 0; p < 3; ++p) Ke[(a * 3 + p) * nd + b * 3 + q] = U[p][a];
                } else {
                    double U[2][4] = {};
                    U[q][b] = 1.0;
                    cell_forces2<double>(U, 1.0, L.c64);
                    for (int a = 0; a < 4; ++a)
                        for (int p = 0; p < 2; ++p) Ke[(a * 2 + p) * nd + b * 2 + q] = U[p][a];
                }
            }
        for (int e = 0; e < nd * nd; ++e) Kf[e] = float(Ke[e]);
        CK(cudaMemcpy(L.Ke64, Ke.data(), sizeof(double) * nd * nd, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(L.Ke32, Kf.data(), sizeof(float) * nd * nd, cudaMemcpyHostToDevice));
    }
    return SBM_OK;
}

sbm_status check_ready(sbm_grid G)
{
    if (!G) return fail(nullptr, SBM_ERR_ARG, "null grid");
    if (!G->has_moduli) return fail(G, SBM_ERR_STATE, "moduli not set (sbm_set_moduli)");
    if (!G->has_psi) return fail(G, SBM_ERR_STATE, "psi not set (sbm_set_psi / sbm_set_density)");
    return SBM_OK;
}

sbm_status validate_opts(sbm_grid G, const sbm_opts &o)
{
    if (!(o.tol >= 0.0) || o.max_cycles < 1 || o.nu1 < 0 || o.nu2 < 0 || o.nu1 + o.nu2 < 1 ||
        (o.smoother != SBM_JACOBI && o.smoother != SBM_MCGS) || !(o.omega > 0.0 && o.omega < 2.0) ||
        o.inner_cycles < 1 || !(o.inner_rtol >= 0.0 && std::isfinite(o.inner_rtol)))
        return fail(G, SBM_ERR_ARG, "invalid sbm_opts");
    return SBM_OK;
}

void set_dirichlet_bits(sbm_grid G)
{
    for (int l = 0; l < G->nl; ++l)
        for (int p = 0; p < 3; ++p) {
            unsigned m = 0;
            for (int f = 0; f < 6; ++f)
                if (G->bct[f][p] != SBM_FREE) m |= 1u << f;
            G->L[l].g.dm[p] = (p < G->desc.dim) ? m : 0u;
        }
}

// Run outer iterations until relres <= tol.  u lives in the finest du[0].
sbm_status run_solve(sbm_grid G, const sbm_opts &o, const double *rhs, sbm_info *info, int slot)
{
    sbm_status st = setup_bottom(G);
    if (st != SBM_OK) return st;
    const int mixed = G->desc.precision == SBM_MIXED;
    const long long launches0 = g_launches;
    long long replayed = 0;
    CK(cudaEventRecord(G->ev0, G->st));
    CK(residual64(G, rhs, mixed, 0));
    CK(cudaMemcpyAsync(G->hscal, G->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, G->st));
    CK(cudaStreamSynchronize(G->st));
    const double r0 = G->hscal[1];
    if (info) {
        info->r0 = r0;
        info->levels = G->nl;
        if (info->history && info->history_capacity > 0) info->history[0] = 1.0;
    }
    GraphSlot &gs = G->slots[slot];
    const int batch = mixed ? 1 : o.inner_cycles;
    if (batch > 1 && G->dhist_cap < o.max_cycles + 1) {
        if (G->dhist) cudaFree(G->dhist);
        G->dhist = nullptr;
        G->dhist_cap = 0;
        CK(gmalloc(G, (void **)&G->dhist, sizeof(double) * (o.max_cycles + 1)));
        G->dhist_cap = o.max_cycles + 1;
    }
    auto body = [&]() { return batch > 1 ? enqueue_fp64_batch(G, o, rhs, batch) : enqueue_body(G, o, rhs); };
    if (o.use_graph) {
        const bool match = gs.valid && gs.mixed == mixed && gs.smoother == o.smoother && gs.nu1 == o.nu1 &&
                           gs.nu2 == o.nu2 && gs.inner == o.inner_cycles && gs.omega == o.omega && gs.rhs == rhs &&
                           gs.inner_rtol == o.inner_rtol && gs.version == G->version &&
                           (batch == 1 || (gs.tol == o.tol && gs.max_cycles == o.max_cycles && gs.hist == G->dhist));
        if (!match) {
            if (gs.valid) cudaGraphExecDestroy(gs.exec);
            gs.valid = false;
            cudaGraph_t graph;
            CK(cudaStreamBeginCapture(G->st, cudaStreamCaptureModeThreadLocal));
            const long long c0 = g_launches;
            cudaError_t e = body();
            const long long nbody = g_launches - c0;
            g_launches = c0;
            cudaError_t e2 = cudaStreamEndCapture(G->st, &graph);
            if (e != cudaSuccess || e2 != cudaSuccess) {
                if (e2 == cudaSuccess) cudaGraphDestroy(graph);
                return fail(G, SBM_ERR_CUDA, std::string("graph capture: ") +
                                                 cudaGetErrorString(e != cudaSuccess ? e : e2));
            }
            e = cudaGraphInstantiate(&gs.exec, graph, 0ULL);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return fail(G, SBM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
            gs.valid = true;
            gs.mixed = mixed;
            gs.smoother = o.smoother;
            gs.nu1 = o.nu1;
            gs.nu2 = o.nu2;
            gs.inner = o.inner_cycles;
            gs.omega = o.omega;
            gs.inner_rtol = o.inner_rtol;
            gs.rhs = rhs;
            gs.version = G->version;
            gs.tol = o.tol;
            gs.max_cycles = o.max_cycles;
            gs.hist = G->dhist;
            gs.body_launches = nbody;
        }
    }
    int cyc = 0;
    double rel = 1.0;
    sbm_status status = SBM_ERR_NOCONV;
    if (r0 == 0.0) {
        status = SBM_OK;
        rel = 0.0;
    }
    const bool gated = mixed && o.inner_rtol > 0.0;
    if (gated) CK(cudaMemsetAsync(G->dgate + 1, 0, sizeof(int), G->st));
    if (batch > 1 && status == SBM_ERR_NOCONV) {
        // batched FP64 V-cycles: one host read of {done, count} per batch
        CK(cudaMemsetAsync(G->dgate, 0, 2 * sizeof(int), G->st));
        int state[2] = {0, 0};
        while (!state[0]) {
            if (o.use_graph) {
                CK(cudaGraphLaunch(gs.exec, G->st));
                replayed += gs.body_launches;
            } else {
                CK(body());
            }
            CK(cudaMemcpyAsync(state, G->dgate, sizeof(state), cudaMemcpyDeviceToHost, G->st));
            CK(cudaStreamSynchronize(G->st));
        }
        cyc = state[1];
        std::vector<double> hist(cyc + 1, 1.0);
        if (cyc > 0) CK(cudaMemcpy(hist.data() + 1, G->dhist + 1, sizeof(double) * cyc, cudaMemcpyDeviceToHost));
        if (info && info->history)
            for (int c = 1; c <= cyc && c < info->history_capacity; ++c) info->history[c] = hist[c];
        rel = cyc > 0 ? hist[cyc] : 1.0;
        if (!std::isfinite(rel) || rel > 1e10) status = SBM_ERR_DIVERGED;
        else if (rel <= o.tol) status = SBM_OK;
    }
    while (status == SBM_ERR_NOCONV && cyc < o.max_cycles && batch == 1) {
        if (o.use_graph) {
            CK(cudaGraphLaunch(gs.exec, G->st));
            replayed += gs.body_launches;
        } else {
            CK(body());
        }
        CK(cudaMemcpyAsync(G->hscal + 4, G->scal + 4, sizeof(double), cudaMemcpyDeviceToHost, G->st));
        CK(cudaStreamSynchronize(G->st));
        ++cyc;
        rel = G->hscal[4];
        if (info && info->history && cyc < info->history_capacity) info->history[cyc] = rel;
        if (!std::isfinite(rel) || rel > 1e10) status = SBM_ERR_DIVERGED;
        else if (rel <= o.tol) status = SBM_OK;
    }
    CK(cudaEventRecord(G->ev1, G->st));
    CK(cudaEventSynchronize(G->ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, G->ev0, G->ev1);
    {
        int herr = 0;
        CK(cudaMemcpy(&herr, G->derr, sizeof(int), cudaMemcpyDeviceToHost));
        if (herr) {
            cudaMemset(G->derr, 0, sizeof(int));
            return fail(G, SBM_ERR_CUDA, "a TMA pipeline wait timed out in the FP32 sweep kernel");
        }
    }
    int vrun = cyc * (mixed ? o.inner_cycles : 1);
    if (gated) CK(cudaMemcpy(&vrun, G->dgate + 1, sizeof(int), cudaMemcpyDeviceToHost));
    if (info) {
        info->status = status;
        info->cycles = cyc;
        info->vcycles = vrun;
        info->relres = rel;
        info->solve_ms = ms;
        info->launches = g_launches - launches0 + replayed;
    }
    if (status == SBM_ERR_NOCONV) G->err = "max_cycles reached before the tolerance";
    if (status == SBM_ERR_DIVERGED) G->err = "relative residual not finite or above 1e10";
    return status;
}

sbm_status check_level(sbm_grid G, int level)
{
    if (!G) return fail(nullptr, SBM_ERR_ARG, "null grid");
    if (level < 0 || level >= G->nl) return fail(G, SBM_ERR_ARG, "level out of range");
    return SBM_OK;
}


// ===================================================== block-structured refinement

int level_N(sbm_grid G, int a, int ax)
{
    if (ax >= G->desc.dim) return 1;
    return (G->desc.n[ax] - 1) * (1 << a) + 1;
}

void amr_refresh_infos(sbm_grid G)
{
    const int d = G->desc.dim;
    unsigned dm[3] = {0, 0, 0};
    for (int p = 0; p < 3; ++p)
        for (int f = 0; f < 6; ++f)
            if (p < d && G->bct[f][p] != SBM_FREE) dm[p] |= 1u << f;
    AmrInfo &B = G->base_info;
    B = AmrInfo{};
    B.dim = d;
    for (int ax = 0; ax < 3; ++ax) {
        B.N[ax] = level_N(G, 0, ax);
        B.dm[ax] = dm[ax];
    }
    B.is_base = 1;
    for (int a = 1; a <= G->npatch; ++a) {
        Patch &Pt = G->P[a - 1];
        AmrInfo &L = Pt.info;
        L = AmrInfo{};
        L.dim = d;
        for (int ax = 0; ax < 3; ++ax) {
            L.N[ax] = level_N(G, Pt.level, ax);
            L.lo[ax] = Pt.lo[ax];
            L.hi[ax] = Pt.hi[ax];
            L.org[ax] = ax < d ? Pt.lo[ax] - 1 : 0;
            L.dm[ax] = dm[ax];
        }
        // view faces: interface faces fixed for every component, domain faces as the domain
        unsigned vdm[3] = {0, 0, 0};
        for (int ax = 0; ax < d; ++ax)
            for (int side = 0; side < 2; ++side) {
                const int f = 2 * ax + side;
                const bool on_domain = side == 0 ? Pt.lo[ax] == 0 : Pt.hi[ax] == L.N[ax] - 1;
                for (int p = 0; p < d; ++p)
                    if (!on_domain || ((dm[p] >> f) & 1u)) vdm[p] |= 1u << f;
            }
        for (int p = 0; p < 3; ++p) Pt.v.dm[p] = vdm[p];
    }
    for (int c = 1; c <= G->npatch; ++c) {
        const Patch &C = G->P[c - 1];
        AmrInfo &L = C.parent == 0 ? G->base_info : G->P[C.parent - 1].info;
        for (int ax = 0; ax < 3; ++ax) {
            L.clo[L.nchild][ax] = C.lo[ax];
            L.chi[L.nchild][ax] = C.hi[ax];
        }
        ++L.nchild;
    }
}

// Patch a's geometry and role info (a = 0: the base level), its parent, its FP64
// solution array and, inside a correction cycle, its correction and right-hand side.
const Geom &amr_geom(sbm_grid G, int a) { return a == 0 ? G->L[G->nl - 1].g : G->P[a - 1].s; }
const AmrInfo &amr_info(sbm_grid G, int a) { return a == 0 ? G->base_info : G->P[a - 1].info; }
int amr_parent(sbm_grid G, int a) { return G->P[a - 1].parent; }
double *amr_u64(sbm_grid G, int a) { return a == 0 ? G->amr_u0 : G->P[a - 1].u64; }

// The patches of each refinement level (index = level), in patch order.
std::vector<std::vector<int>> amr_by_level(sbm_grid G)
{
    std::vector<std::vector<int>> out(1);
    for (int a = 1; a <= G->npatch; ++a) {
        const int L = G->P[a - 1].level;
        if ((int)out.size() <= L) out.resize(L + 1);
        out[L].push_back(a);
    }
    return out;
}

// work(a) for every patch a of `list`, the patches spread over the grid's side
// streams (each branch ordered after everything enqueued on the grid stream so
// far; the grid stream then waits for all branches).  Patches of one level touch
// disjoint data (their own storage; a child's restriction writes only the parent
// nodes it covers), so their kernels may run concurrently; under stream capture
// the branches become parallel paths of the graph.
template <typename F>
cudaError_t amr_branches(sbm_grid G, const std::vector<int> &list, F &&work)
{
    if (list.size() <= 1 || !G->side[0]) {
        for (int a : list) CKE(work(a));
        return cudaSuccess;
    }
    cudaStream_t main = G->st;
    const int nb = std::min((int)list.size(), kBranches);
    CKE(cudaEventRecord(G->fork_ev, main));
    for (int b = 0; b < nb; ++b) CKE(cudaStreamWaitEvent(G->side[b], G->fork_ev, 0));
    cudaError_t err = cudaSuccess;
    for (size_t i = 0; i < list.size() && err == cudaSuccess; ++i) {
        G->st = G->side[i % nb];
        err = work(list[i]);
    }
    G->st = main;
    for (int b = 0; b < nb; ++b) {
        cudaError_t e = cudaEventRecord(G->join_ev[b], G->side[b]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(main, G->join_ev[b], 0);
        if (err == cudaSuccess) err = e;
    }
    return err;
}

template <typename T> struct PP;
template <> struct PP<double> {
    static double *e(Patch &P, int i) { return P.de[i]; }
    static double *rhs(Patch &P) { return P.drhs; }
    static double *res(Patch &P) { return P.dres; }
    static const double *psi(Patch &P) { return P.psi64; }
    static const Coef<double> &c(Patch &P) { return P.c64; }
    static const double *Ke(Patch &P) { return P.Ke64; }
};
template <> struct PP<float> {
    static float *e(Patch &P, int i) { return P.se[i]; }
    static float *rhs(Patch &P) { return P.srhs; }
    static float *res(Patch &P) { return P.sres; }
    static const float *psi(Patch &P) { return P.psi32; }
    static const Coef<float> &c(Patch &P) { return P.c32; }
    static const float *Ke(Patch &P) { return P.Ke32; }
};

template <typename T>
T *amr_rhs(sbm_grid G, int a)
{
    Level &B = G->L[G->nl - 1];
    if (a > 0) return PP<T>::rhs(G->P[a - 1]);
    return std::is_same<T, double>::value ? (T *)B.df : (T *)B.sf;
}

template <typename T>
T *amr_e(sbm_grid G, int a, const int *cur, int cb)
{
    return a == 0 ? P<T>::u(G->L[G->nl - 1], cb) : PP<T>::e(G->P[a - 1], cur[a]);
}

template <typename T>
cudaError_t sweep_view(sbm_grid G, Patch &Pt, int mode, const T *u, const T *f, T *out, double omega)
{
    if constexpr (std::is_same<T, float>::value) {
        // 3D FP32 views of the patch's own buffers: the TMA sweep over the storage's
        // tensor maps, the view starting at storage node (1, 1, 1)
        if (Pt.has_tm && (u == Pt.se[0] || u == Pt.se[1]) && (mode == kApply || f == Pt.srhs)) {
            SweepArgs<float, float> a;
            a.g = Pt.v;
            a.u = u + Pt.voff;
            a.f = f ? f + Pt.voff : nullptr;
            a.psi = Pt.psiv32 + Pt.voff;
            a.out = out + Pt.voff;
            a.part = nullptr;
            a.c = Pt.c32;
            for (int p = 0; p < 3; ++p) a.wk[p] = (Pt.c64.kdiag[p] != 0.0) ? float(omega / Pt.c64.kdiag[p]) : 0.f;
            a.kchunk = 0;
            return launch_sweep_f2(mode, a, Pt.tm32[u == Pt.se[0] ? 0 : 1], G->derr, G->st, make_int3(1, 1, 1));
        }
    }
    SweepArgs<T, T> a;
    a.g = Pt.v;
    a.u = u + Pt.voff;
    a.f = f ? f + Pt.voff : nullptr;
    a.psi = PP<T>::psi(Pt) + Pt.voff;
    a.out = out + Pt.voff;
    a.part = nullptr;
    a.c = PP<T>::c(Pt);
    for (int p = 0; p < 3; ++p) a.wk[p] = (Pt.c64.kdiag[p] != 0.0) ? T(omega / Pt.c64.kdiag[p]) : T(0);
    a.kchunk = 0;
    return launch_sweep<T, T>(mode, a, G->st);
}

template <typename T>
cudaError_t patch_smooth(sbm_grid G, Patch &Pt, int &cur, const sbm_opts &o, int n, bool desc)
{
    const int ncol = 1 << Pt.v.dim;
    for (int s = 0; s < n; ++s) {
        if (o.smoother == SBM_MCGS && Pt.v.dim == 2) {
            CKE(launch_gs2_sweep<T>(Pt.v, PP<T>::psi(Pt) + Pt.voff, PP<T>::Ke(Pt), PP<T>::rhs(Pt) + Pt.voff,
                                    PP<T>::e(Pt, cur) + Pt.voff, PP<T>::e(Pt, 1 - cur) + Pt.voff, desc ? 1 : 0, G->st));
            cur ^= 1;
        } else if (o.smoother == SBM_MCGS) {
            for (int c = 0; c < ncol; ++c)
                CKE(launch_gs<T>(Pt.v, PP<T>::psi(Pt) + Pt.voff, PP<T>::Ke(Pt), PP<T>::rhs(Pt) + Pt.voff,
                                 PP<T>::e(Pt, cur) + Pt.voff, desc ? ncol - 1 - c : c, G->st));
        } else {
            CKE(sweep_view<T>(G, Pt, kJacobi, PP<T>::e(Pt, cur), PP<T>::rhs(Pt), PP<T>::e(Pt, 1 - cur), o.omega));
            cur ^= 1;
        }
    }
    return cudaSuccess;
}

size_t patch_bytes(const Patch &Pt, size_t elem) { return (size_t)Pt.s.dim * Pt.s.cs * elem; }

// Injection into covered parents (finest first), then ghost fill (coarsest first).
cudaError_t amr_fill(sbm_grid G)
{
    // patches are numbered parents first, so descending order is finest first
    for (int a = G->npatch; a >= 1; --a) {
        Patch &Pt = G->P[a - 1];
        const int pa = Pt.parent;
        CKE(launch_amr_inject(Pt.s, Pt.info, amr_geom(G, pa), amr_info(G, pa), Pt.u64, amr_u64(G, pa), G->st));
    }
    for (int a = 1; a <= G->npatch; ++a) {
        Patch &Pt = G->P[a - 1];
        const int pa = Pt.parent;
        CKE(launch_amr_ghost<double>(Pt.s, Pt.info, amr_geom(G, pa), amr_info(G, pa), Pt.u64, amr_u64(G, pa), 0, G->st));
    }
    return cudaSuccess;
}

// Composite FP64 residual of every level, its norm into scal[which..] and the
// residual rounded to T as the right-hand side of the correction cycle.
template <typename T>
cudaError_t amr_residual(sbm_grid G, int which)
{
    Level &B = G->L[G->nl - 1];
    CKE(amr_fill(G));
    CKE(sweep<double>(G, G->nl - 1, kResidual, G->amr_u0, G->fsrc, G->amr_r0, nullptr, 0.0));
    CKE(launch_amr_mask(B.g, G->base_info, G->amr_r0, G->st));
    T *base_rhs = std::is_same<T, double>::value ? (T *)B.df : (T *)B.sf;
    long long off = 0;
    CKE(launch_amr_sumsq_round<T>(B.g, G->base_info, G->amr_r0, base_rhs, G->amr_part, G->st));
    off += amr_blocks(B.g);
    std::vector<long long> offs(G->npatch + 1, 0);
    std::vector<int> all;
    for (int a = 1; a <= G->npatch; ++a) {
        offs[a] = off;
        off += amr_blocks(G->P[a - 1].s);
        all.push_back(a);
    }
    CKE(amr_branches(G, all, [&](int a) -> cudaError_t {
        Patch &Pt = G->P[a - 1];
        CKE(sweep_view<double>(G, Pt, kResidual, Pt.u64, Pt.f64, Pt.r64, 0.0));
        CKE(launch_amr_mask(Pt.s, Pt.info, Pt.r64, G->st));
        return launch_amr_sumsq_round<T>(Pt.s, Pt.info, Pt.r64, PP<T>::rhs(Pt), G->amr_part + offs[a], G->st);
    }));
    return launch_norm_final(G->amr_part, (int)off, G->scal, which, G->st);
}

// One correction cycle: patches top-down (smooth, residual, restrict to covered
// parent nodes), the base multigrid V-cycle, patches bottom-up (prolongate the
// parent correction, fill ghosts, smooth), then u += e on owned dofs.
// cur_out / cb_out (optional): which of the two correction buffers of each patch /
// of the base level holds the final correction.
template <typename T>
cudaError_t amr_cycle(sbm_grid G, const sbm_opts &o, double *const *target = nullptr, int *cur_out = nullptr,
                      int *cb_out = nullptr)
{
    const int A = G->npatch;
    Level &B = G->L[G->nl - 1];
    int cur[kMaxPatch + 1] = {0};
    const std::vector<std::vector<int>> lev = amr_by_level(G);
    // finest level first (every child before its parent); the patches of a level concurrently
    for (int L = (int)lev.size() - 1; L >= 1; --L)
        CKE(amr_branches(G, lev[L], [&](int a) -> cudaError_t {
            Patch &Pt = G->P[a - 1];
            CKE(cudaMemsetAsync(PP<T>::e(Pt, 0), 0, patch_bytes(Pt, sizeof(T)), G->st));
            CKE(cudaMemsetAsync(PP<T>::e(Pt, 1), 0, patch_bytes(Pt, sizeof(T)), G->st));
            cur[a] = 0;
            CKE(patch_smooth<T>(G, Pt, cur[a], o, o.nu1, false));
            CKE(sweep_view<T>(G, Pt, kResidual, PP<T>::e(Pt, cur[a]), PP<T>::rhs(Pt), PP<T>::res(Pt), 0.0));
            const int pa = Pt.parent;
            return launch_amr_restrict<T>(Pt.s, Pt.info, amr_geom(G, pa), amr_info(G, pa), PP<T>::res(Pt),
                                          amr_rhs<T>(G, pa), G->st);
        }));
    T *base_rhs = std::is_same<T, double>::value ? (T *)B.df : (T *)B.sf;
    CKE(cudaMemsetAsync(P<T>::u(B, 0), 0, level_bytes(B, sizeof(T)), G->st));
    int cb = 0;
    CKE(vcycle<T>(G, G->nl - 1, cb, o, base_rhs));
    // coarsest level first (every parent's final correction before its children)
    for (int L = 1; L < (int)lev.size(); ++L)
        CKE(amr_branches(G, lev[L], [&](int a) -> cudaError_t {
            Patch &Pt = G->P[a - 1];
            const int pa = Pt.parent;
            CKE(launch_amr_ghost<T>(Pt.s, Pt.info, amr_geom(G, pa), amr_info(G, pa), PP<T>::e(Pt, cur[a]),
                                    amr_e<T>(G, pa, cur, cb), 1, G->st));
            return patch_smooth<T>(G, Pt, cur[a], o, o.nu2, true);
        }));
    // u += e on owned free dofs (target: the composite solution, or other level arrays)
    CKE(launch_amr_update<T>(B.g, G->base_info, P<T>::u(B, cb), target ? target[0] : G->amr_u0, G->st));
    std::vector<int> all;
    for (int a = 1; a <= A; ++a) all.push_back(a);
    CKE(amr_branches(G, all, [&](int a) -> cudaError_t {
        Patch &Pt = G->P[a - 1];
        return launch_amr_update<T>(Pt.s, Pt.info, PP<T>::e(Pt, cur[a]), target ? target[a] : Pt.u64, G->st);
    }));
    if (cur_out)
        for (int a = 0; a <= A; ++a) cur_out[a] = cur[a];
    if (cb_out) *cb_out = cb;
    return cudaSuccess;
}

// Mixed-precision inner iterations: once an FP32 correction cycle has added its
// correction e to u, the cycle's FP32 right-hand side becomes the residual of the
// correction equation, r <- r - A e, on the owned free rows of every level, so the
// next FP32 cycle needs no FP64 residual.  A e is the composite operator applied
// to e filled like a solution: e injected into the covered parent nodes (finest
// first; the cycle left each patch's ghosts interpolated from its parent's final
// correction, and the ghosts depend on uncovered parent nodes only), then K of
// every level on its nodes.
cudaError_t amr_inner_residual(sbm_grid G, const int *cur, int cb)
{
    const int A = G->npatch;
    Level &B = G->L[G->nl - 1];
    for (int a = A; a >= 1; --a) {
        Patch &Pt = G->P[a - 1];
        const int pa = Pt.parent;
        CKE(launch_amr_inject<float>(Pt.s, Pt.info, amr_geom(G, pa), amr_info(G, pa), Pt.se[cur[a]],
                                     amr_e<float>(G, pa, cur, cb), G->st));
    }
    CKE(sweep<float>(G, G->nl - 1, kResidual, B.su[cb], B.sf, B.sr, nullptr, 0.0));
    CKE(launch_amr_mask_to<float>(B.g, G->base_info, B.sr, B.sf, G->st));
    for (int a = 1; a <= A; ++a) {
        Patch &Pt = G->P[a - 1];
        CKE(sweep_view<float>(G, Pt, kResidual, Pt.se[cur[a]], Pt.srhs, Pt.sres, 0.0));
        CKE(launch_amr_mask_to<float>(Pt.s, Pt.info, Pt.sres, Pt.srhs, G->st));
    }
    return cudaSuccess;
}

// ------------------------------------------------ adjoint of the composite problem
//
// Composite vectors: one FP64 array per level in the level layout, nonzero only on
// the owned free dofs.  A^T is applied as the transpose of "fill, apply K_a, keep
// owned rows": K_a on every level, then the ghost values go back to the parent
// (transposed interpolation, finest first) and the covered values to the finer
// level (transposed injection, coarsest first), then the owned free rows are kept.

size_t amr_vec_len(sbm_grid G, int a) { const Geom &g = amr_geom(G, a); return (size_t)g.dim * g.cs; }

cudaError_t cv_zero(sbm_grid G, double *const *x)
{
    for (int a = 0; a <= G->npatch; ++a) CKE(cudaMemsetAsync(x[a], 0, sizeof(double) * amr_vec_len(G, a), G->st));
    return cudaSuccess;
}

cudaError_t cv_lincomb(sbm_grid G, double al, double *const *x, double be, double *const *y, double ga,
                       double *const *z, double *const *out)
{
    for (int a = 0; a <= G->npatch; ++a)
        CKE(launch_lincomb((long long)amr_vec_len(G, a), al, x[a], be, y[a], ga, z ? z[a] : nullptr, out[a], G->st));
    return cudaSuccess;
}

// <x, y> over the owned free dofs into scal[slot] (device)
cudaError_t cv_dot(sbm_grid G, double *const *x, double *const *y, int slot)
{
    long long off = 0;
    for (int a = 0; a <= G->npatch; ++a) {
        CKE(launch_amr_dot(amr_geom(G, a), amr_info(G, a), x[a], y[a], G->amr_part + off, G->st));
        off += amr_blocks(amr_geom(G, a));
    }
    return launch_sum_parts(G->amr_part, (int)off, G->scal + slot, G->st);
}

cudaError_t amr_apply_T(sbm_grid G, double *const *x, double *const *out)
{
    const int A = G->npatch;
    CKE(cv_zero(G, out));
    CKE(sweep<double>(G, G->nl - 1, kApply, x[0], nullptr, out[0], nullptr, 0.0));
    for (int a = 1; a <= A; ++a) CKE(sweep_view<double>(G, G->P[a - 1], kApply, x[a], nullptr, out[a], 0.0));
    for (int a = A; a >= 1; --a) {
        const int pa = amr_parent(G, a);
        CKE(launch_amr_ghostT(amr_geom(G, a), amr_info(G, a), amr_geom(G, pa), amr_info(G, pa), out[a], out[pa], 0,
                              G->st));
    }
    for (int c = 1; c <= A; ++c) {
        const int pa = amr_parent(G, c);
        CKE(launch_amr_injectT(amr_geom(G, c), amr_info(G, c), amr_geom(G, pa), amr_info(G, pa), out[pa], out[c],
                               G->st));
    }
    for (int a = 0; a <= A; ++a) CKE(launch_amr_mask(amr_geom(G, a), amr_info(G, a), out[a], G->st));
    return cudaSuccess;
}

// out = A^T x with the stencil products in FP32 (x rounded into the FP32 buffers of
// each level, the FP32 apply, the products widened into the FP64 vectors), the
// ghost, injection and ownership transposes in FP64: the operator of the inner
// transposed iterations on mixed-precision grids.
cudaError_t amr_apply_T32(sbm_grid G, double *const *x, double *const *out)
{
    const int A = G->npatch;
    Level &B = G->L[G->nl - 1];
    CKE(cv_zero(G, out));
    const long long n0 = (long long)amr_vec_len(G, 0);
    CKE(launch_round(n0, x[0], B.su[0], G->st));
    CKE(sweep<float>(G, G->nl - 1, kApply, B.su[0], nullptr, B.sr, nullptr, 0.0));
    CKE(launch_add<float>(n0, B.sr, out[0], G->st));
    for (int a = 1; a <= A; ++a) {
        Patch &Pt = G->P[a - 1];
        CKE(launch_round((long long)amr_vec_len(G, a), x[a], Pt.se[0], G->st));
        CKE(sweep_view<float>(G, Pt, kApply, Pt.se[0], nullptr, Pt.sres, 0.0));
        CKE(launch_axpy_view<float>(Pt.v, Pt.voff, 1.0, Pt.sres, out[a], G->st));
    }
    for (int a = A; a >= 1; --a) {
        const int pa = amr_parent(G, a);
        CKE(launch_amr_ghostT(amr_geom(G, a), amr_info(G, a), amr_geom(G, pa), amr_info(G, pa), out[a], out[pa], 0,
                              G->st));
    }
    for (int c = 1; c <= A; ++c) {
        const int pa = amr_parent(G, c);
        CKE(launch_amr_injectT(amr_geom(G, c), amr_info(G, c), amr_geom(G, pa), amr_info(G, pa), out[pa], out[c],
                               G->st));
    }
    for (int a = 0; a <= A; ++a) CKE(launch_amr_mask(amr_geom(G, a), amr_info(G, a), out[a], G->st));
    return cudaSuccess;
}

// eb -= K_a x on patch a's view, the product taken in FP32 on mixed-precision grids:
// x is rounded into the patch's FP32 correction buffer (or used as is on FP64
// grids), the stencil writes every view node of the residual buffer, and those are
// subtracted.  Inside the transposed correction cycle this is enough: the cycle only
// preconditions the adjoint iteration, whose fixed point A^T lambda = g is set by
// the FP64 A^T alone.
cudaError_t view_apply_sub(sbm_grid G, Patch &Pt, const double *x, double *eb, size_t n)
{
    if (G->desc.precision != SBM_MIXED) {
        CKE(sweep_view<double>(G, Pt, kApply, x, nullptr, Pt.dres, 0.0));
        return launch_axpy_view<double>(Pt.v, Pt.voff, -1.0, Pt.dres, eb, G->st);
    }
    CKE(launch_round((long long)n, x, Pt.se[0], G->st));
    CKE(sweep_view<float>(G, Pt, kApply, Pt.se[0], nullptr, Pt.sres, 0.0));
    return launch_axpy_view<float>(Pt.v, Pt.voff, -1.0, Pt.sres, eb, G->st);
}

// One transposed (damped-Jacobi) sweep on patch a's solved dofs: eb <- eb - K_a W eb
// and rb += W eb, with W the Jacobi scaling (the transpose of e <- e + W (r - K e)).
// W (vector 5 of adj, set by amr_adjoint_scaling) is 0 off the solved free dofs; the
// scaled vector goes straight into the stencil's input buffer.
cudaError_t patch_jacobiT(sbm_grid G, int a, double *eb, double *rb)
{
    Patch &Pt = G->P[a - 1];
    const long long n = (long long)amr_vec_len(G, a);
    const double *W = G->adj[5][a];
    if (G->desc.precision != SBM_MIXED) {
        CKE(launch_amr_jacT_scale<double>(n, W, eb, rb, Pt.de[0], G->st));
        CKE(sweep_view<double>(G, Pt, kApply, Pt.de[0], nullptr, Pt.dres, 0.0));
        return launch_axpy_view<double>(Pt.v, Pt.voff, -1.0, Pt.dres, eb, G->st);
    }
    CKE(launch_amr_jacT_scale<float>(n, W, eb, rb, Pt.se[0], G->st));
    CKE(sweep_view<float>(G, Pt, kApply, Pt.se[0], nullptr, Pt.sres, 0.0));
    return launch_axpy_view<float>(Pt.v, Pt.voff, -1.0, Pt.sres, eb, G->st);
}

// W of every patch for relaxation weight omega (vector 5 of adj).
cudaError_t amr_adjoint_scaling(sbm_grid G, double omega)
{
    for (int a = 1; a <= G->npatch; ++a) {
        Patch &Pt = G->P[a - 1];
        CKE(launch_amr_scaleW(Pt.s, Pt.info, Pt.psi64, omega, Pt.c64.kdiag, nullptr, G->adj[5][a], G->st));
    }
    return cudaSuccess;
}

// z = B^T y: the transpose of one correction cycle (Jacobi smoother; its stencil
// products and base V-cycle in FP32 on mixed-precision grids, see view_apply_sub), taken
// step by step in reverse: the update's mask; per patch, finest first, the
// post-smoothing sweeps transposed and the correction prolongation transposed
// (into the parent's adjoint); the base V-cycle (symmetric); per patch, coarsest
// first, the restriction onto covered parents transposed, the residual
// transposed and the pre-smoothing sweeps transposed; z = the right-hand sides'
// adjoints on the owned free dofs.  y is overwritten (it becomes the corrections'
// adjoints).  Scratch: vector 7 of adj (5 holds W).
cudaError_t amr_precondT(sbm_grid G, const sbm_opts &o, double *const *y, double *const *z)
{
    const int A = G->npatch;
    Level &B = G->L[G->nl - 1];
    double *const *EB = y;             // adjoints of the corrections e_a (y is consumed)
    double *const *T1 = G->adj[7];
    // z holds the right-hand sides' adjoints while they accumulate
    CKE(cv_zero(G, z));
    for (int a = A; a >= 1; --a) {
        for (int s_ = 0; s_ < o.nu2; ++s_) CKE(patch_jacobiT(G, a, EB[a], z[a]));
        const int pa = amr_parent(G, a);
        CKE(launch_amr_ghostT(amr_geom(G, a), amr_info(G, a), amr_geom(G, pa), amr_info(G, pa), EB[a], EB[pa], 1,
                              G->st));
        CKE(launch_amr_mask_solved(amr_geom(G, a), amr_info(G, a), EB[a], G->st));
    }
    // base: rhs adjoint = V_0 (adjoint of its output); the FP32 V-cycle on mixed grids
    const size_t n0 = amr_vec_len(G, 0);
    int cb = 0;
    if (G->desc.precision == SBM_MIXED) {
        CKE(launch_round((long long)n0, EB[0], B.sf, G->st));
        CKE(cudaMemsetAsync(P<float>::u(B, 0), 0, level_bytes(B, sizeof(float)), G->st));
        CKE(vcycle<float>(G, G->nl - 1, cb, o, B.sf));
        CKE(launch_add<float>((long long)n0, P<float>::u(B, cb), z[0], G->st));
    } else {
        CKE(cudaMemcpyAsync(B.df, EB[0], sizeof(double) * n0, cudaMemcpyDeviceToDevice, G->st));
        CKE(cudaMemsetAsync(P<double>::u(B, 0), 0, level_bytes(B, sizeof(double)), G->st));
        CKE(vcycle<double>(G, G->nl - 1, cb, o, B.df));
        CKE(launch_lincomb((long long)n0, 1.0, z[0], 1.0, P<double>::u(B, cb), 0.0, nullptr, z[0], G->st));
    }
    for (int a = 1; a <= A; ++a) {
        // restriction onto the covered parent nodes, transposed: residual adjoint
        const int pa = amr_parent(G, a);
        CKE(launch_amr_restrictT(amr_geom(G, a), amr_info(G, a), amr_geom(G, pa), amr_info(G, pa), z[pa], T1[a],
                                 G->st));
        CKE(launch_amr_mask_solved(amr_geom(G, a), amr_info(G, a), T1[a], G->st));
        // residual r = rhs - K e (solved dofs): rhs_adj += res_adj, e_adj -= K res_adj
        const size_t n = amr_vec_len(G, a);
        CKE(launch_lincomb((long long)n, 1.0, z[a], 1.0, T1[a], 0.0, nullptr, z[a], G->st));
        CKE(view_apply_sub(G, G->P[a - 1], T1[a], EB[a], n));
        for (int s_ = 0; s_ < o.nu1; ++s_) CKE(patch_jacobiT(G, a, EB[a], z[a]));
    }
    for (int a = 0; a <= A; ++a) CKE(launch_amr_mask(amr_geom(G, a), amr_info(G, a), z[a], G->st));
    return cudaSuccess;
}

sbm_status amr_alloc_adjoint(sbm_grid G)
{
    for (auto &vec : G->adj)
        for (int a = 0; a <= G->npatch; ++a)
            if (!vec[a]) {
                CK(gmalloc(G, (void **)&vec[a], sizeof(double) * amr_vec_len(G, a)));
                CK(cudaMemset(vec[a], 0, sizeof(double) * amr_vec_len(G, a)));
            }
    return SBM_OK;
}

sbm_status amr_prepare(sbm_grid G)
{
    amr_refresh_infos(G);
    if (!G->side[0] && G->npatch > 1) {
        for (int b = 0; b < kBranches; ++b) {
            CK(cudaStreamCreateWithFlags(&G->side[b], cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&G->join_ev[b], cudaEventDisableTiming));
        }
        CK(cudaEventCreateWithFlags(&G->fork_ev, cudaEventDisableTiming));
    }
    for (int a = 1; a <= G->npatch; ++a) {
        Patch &Pt = G->P[a - 1];
        Pt.c64 = make_coef<double>(Pt.s.dim, Pt.h, G->mod[0], G->mod[1], G->mod[2]);
        Pt.c32 = make_coef<float>(Pt.s.dim, Pt.h, G->mod[0], G->mod[1], G->mod[2]);
        const int d = Pt.s.dim, nc = 1 << d, nd = nc * d;
        std::vector<double> Ke(nd * nd);
        std::vector<float> Kf(nd * nd);
        for (int b = 0; b < nc; ++b)
            for (int q = 0; q < d; ++q) {
                if (d == 3) {
                    double U[3][8] = {};
                    U[q][b] = 1.0;
                    cell_forces3<double>(U, 1.0, Pt.c64);
                    for (int c = 0; c < 8; ++c)
                        for (int p = 0; p < 3; ++p) Ke[(c * 3 + p) * nd + b * 3 + q] = U[p][c];
                } else {
                    double U[2][4] = {};
                    U[q][b] = 1.0;
                    cell_forces2<double>(U, 1.0, Pt.c64);
                    for (int c = 0; c < 4; ++c)
                        for (int p = 0; p < 2; ++p) Ke[(c * 2 + p) * nd + b * 2 + q] = U[p][c];
                }
            }
        for (int e = 0; e < nd * nd; ++e) Kf[e] = float(Ke[e]);
        CK(cudaMemcpyAsync(Pt.Ke64, Ke.data(), sizeof(double) * nd * nd, cudaMemcpyHostToDevice, G->st));
        CK(cudaMemcpyAsync(Pt.Ke32, Kf.data(), sizeof(float) * nd * nd, cudaMemcpyHostToDevice, G->st));
        CK(cudaStreamSynchronize(G->st));
    }
    if (G->amr_psi_dirty) {
        Level &B = G->L[G->nl - 1];
        for (int a = G->npatch; a >= 1; --a) {
            Patch &Pt = G->P[a - 1];
            const int pa = Pt.parent;
            double *psip = pa == 0 ? B.psi64 : G->P[pa - 1].psi64;
            CK(launch_amr_coarsen_psi(Pt.s, Pt.info, amr_geom(G, pa), amr_info(G, pa), Pt.psi64, psip, G->st));
        }
        for (int a = 1; a <= G->npatch; ++a) {
            CK(launch_round(G->P[a - 1].s.cs, G->P[a - 1].psi64, G->P[a - 1].psi32, G->st));
            CK(launch_amr_view_cells(G->P[a - 1].s, G->P[a - 1].psi32, G->P[a - 1].psiv32, G->st));
        }
        for (int l = G->nl - 1; l > 0; --l)
            CK(launch_coarsen_psi(G->L[l].g, G->L[l - 1].g, G->L[l].psi64, G->L[l - 1].psi64, G->st));
        for (int l = 0; l < G->nl; ++l) CK(launch_round_cells(G->L[l].g, G->L[l].psi64, G->L[l].psi32, G->st));
        G->bottom_ready = false;
        G->amr_psi_dirty = false;
    }
    return SBM_OK;
}

template <typename T>
sbm_status amr_run(sbm_grid G, const sbm_opts &o, sbm_info *info)
{
    sbm_status st = setup_bottom(G);
    if (st != SBM_OK) return st;
    const long long launches0 = g_launches;
    CK(cudaEventRecord(G->ev0, G->st));
    CK(amr_residual<T>(G, 0));
    CK(cudaMemcpyAsync(G->hscal, G->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, G->st));
    CK(cudaStreamSynchronize(G->st));
    const double r0 = G->hscal[1];
    if (info) {
        info->r0 = r0;
        info->levels = G->nl + G->npatch;
        if (info->history && info->history_capacity > 0) info->history[0] = 1.0;
    }
    int cyc = 0;
    double rel = 1.0;
    sbm_status status = SBM_ERR_NOCONV;
    if (r0 == 0.0) {
        status = SBM_OK;
        rel = 0.0;
    }
    // SBM_MIXED: inner_cycles FP32 correction cycles per FP64 residual
    const int inner = std::is_same<T, float>::value ? o.inner_cycles : 1;
    // one outer iteration: the correction cycles and the FP64 composite residual
    // with its norm in scal[4]; captured once as a CUDA graph and replayed
    auto body = [&]() -> cudaError_t {
        for (int it = 0; it < inner; ++it) {
            int cur[kMaxPatch + 1], cb = 0;
            CKE(amr_cycle<T>(G, o, nullptr, cur, &cb));
            if constexpr (std::is_same<T, float>::value)
                if (it + 1 < inner) CKE(amr_inner_residual(G, cur, cb));
        }
        return amr_residual<T>(G, 2);
    };
    GraphSlot &gs = G->amr_slot;
    const int mixed = std::is_same<T, float>::value ? 1 : 0;
    if (o.use_graph) {
        const bool match = gs.valid && gs.mixed == mixed && gs.smoother == o.smoother && gs.nu1 == o.nu1 &&
                           gs.nu2 == o.nu2 && gs.inner == inner && gs.omega == o.omega && gs.version == G->version;
        if (!match) {
            if (gs.valid) cudaGraphExecDestroy(gs.exec);
            gs.valid = false;
            cudaGraph_t graph;
            CK(cudaStreamBeginCapture(G->st, cudaStreamCaptureModeThreadLocal));
            const long long c0 = g_launches;
            cudaError_t e = body();
            const long long nbody = g_launches - c0;
            g_launches = c0;
            cudaError_t e2 = cudaStreamEndCapture(G->st, &graph);
            if (e != cudaSuccess || e2 != cudaSuccess) {
                if (e2 == cudaSuccess) cudaGraphDestroy(graph);
                return fail(G, SBM_ERR_CUDA, std::string("graph capture: ") +
                                                 cudaGetErrorString(e != cudaSuccess ? e : e2));
            }
            e = cudaGraphInstantiate(&gs.exec, graph, 0ULL);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return fail(G, SBM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
            gs.valid = true;
            gs.mixed = mixed;
            gs.smoother = o.smoother;
            gs.nu1 = o.nu1;
            gs.nu2 = o.nu2;
            gs.inner = inner;
            gs.omega = o.omega;
            gs.version = G->version;
            gs.body_launches = nbody;
        }
    }
    int ncycles = 0;
    while (status == SBM_ERR_NOCONV && cyc < o.max_cycles) {
        if (o.use_graph) {
            CK(cudaGraphLaunch(gs.exec, G->st));
            g_launches += gs.body_launches;
        } else {
            CK(body());
        }
        ncycles += inner;
        CK(cudaMemcpyAsync(G->hscal + 4, G->scal + 4, sizeof(double), cudaMemcpyDeviceToHost, G->st));
        CK(cudaStreamSynchronize(G->st));
        ++cyc;
        rel = G->hscal[4];
        if (info && info->history && cyc < info->history_capacity) info->history[cyc] = rel;
        if (!std::isfinite(rel) || rel > 1e10) status = SBM_ERR_DIVERGED;
        else if (rel <= o.tol) status = SBM_OK;
    }
    CK(amr_fill(G));
    CK(cudaEventRecord(G->ev1, G->st));
    CK(cudaEventSynchronize(G->ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, G->ev0, G->ev1);
    {
        int herr = 0;
        CK(cudaMemcpy(&herr, G->derr, sizeof(int), cudaMemcpyDeviceToHost));
        if (herr) {
            cudaMemset(G->derr, 0, sizeof(int));
            return fail(G, SBM_ERR_CUDA, "a TMA pipeline wait timed out in the FP32 sweep kernel");
        }
    }
    if (info) {
        info->status = status;
        info->cycles = cyc;
        info->vcycles = ncycles;
        info->relres = rel;
        info->solve_ms = ms;
        info->launches = g_launches - launches0;
    }
    if (status == SBM_ERR_NOCONV) G->err = "max_cycles reached before the tolerance";
    if (status == SBM_ERR_DIVERGED) G->err = "relative residual not finite or above 1e10";
    return status;
}

sbm_status amr_pack_u(sbm_grid G, double *const *u)
{
    Level &F = G->L[G->nl - 1];
    if (!is_dev_ptr(u[0], G->dev)) return fail(G, SBM_ERR_ARG, "u[0] is not a device pointer");
    CK(launch_pack<double, double>(F.g, F.g.dim, u[0], G->amr_u0, G->st));
    for (int f = 0; f < 2 * F.g.dim; ++f)
        for (int p = 0; p < F.g.dim; ++p)
            if (G->bct[f][p] == SBM_DIRICHLET) CK(launch_set_face(F.g, f, p, G->bcv[f][p], G->amr_u0, G->st));
    for (int a = 1; a <= G->npatch; ++a) {
        if (!is_dev_ptr(u[a], G->dev)) return fail(G, SBM_ERR_ARG, "u[a] is not a device pointer");
        Patch &Pt = G->P[a - 1];
        CK(launch_pack<double, double>(Pt.s, Pt.s.dim, u[a], Pt.u64, G->st));
    }
    return SBM_OK;
}

sbm_status amr_unpack(sbm_grid G, double *base, double *const *pat, bool residual)
{
    Level &F = G->L[G->nl - 1];
    CK(launch_unpack<double, double>(F.g, F.g.dim, residual ? G->amr_r0 : G->amr_u0, base, G->st));
    for (int a = 1; a <= G->npatch; ++a) {
        Patch &Pt = G->P[a - 1];
        CK(launch_unpack<double, double>(Pt.s, Pt.s.dim, residual ? Pt.r64 : Pt.u64, pat[a], G->st));
    }
    return SBM_OK;
}

void free_patch(Patch &Pt)
{
    void *ptrs[] = {Pt.psi64, Pt.psi32, Pt.u64, Pt.f64, Pt.r64, Pt.de[0], Pt.de[1], Pt.drhs, Pt.dres,
                    Pt.se[0], Pt.se[1], Pt.srhs, Pt.sres, Pt.psiv32, Pt.Ke64, Pt.Ke32, Pt.psi_set};
    for (void *p : ptrs)
        if (p) cudaFree(p);
}

}  // namespace

void sbm::set_library_error(const char *msg) { g_lib_error = msg; }

// ========================================================================= ABI

extern "C" {

void sbm_default_opts(sbm_opts *o)
{
    if (!o) return;
    o->tol = 1e-10;
    o->max_cycles = 500;
    o->nu1 = 2;
    o->nu2 = 2;
    o->omega = 2.0 / 3.0;
    o->smoother = SBM_JACOBI;
    o->inner_cycles = 1;
    o->use_graph = 1;
    o->inner_rtol = 0.0;
}

const char *sbm_status_string(int s)
{
    switch (s) {
    case SBM_OK: return "SBM_OK";
    case SBM_ERR_ARG: return "SBM_ERR_ARG";
    case SBM_ERR_STATE: return "SBM_ERR_STATE";
    case SBM_ERR_CUDA: return "SBM_ERR_CUDA";
    case SBM_ERR_OOM: return "SBM_ERR_OOM";
    case SBM_ERR_NOCONV: return "SBM_ERR_NOCONV";
    case SBM_ERR_DIVERGED: return "SBM_ERR_DIVERGED";
    default: return "unknown status";
    }
}

const char *sbm_last_error(sbm_grid G) { return G ? G->err.c_str() : g_lib_error.c_str(); }

sbm_status sbm_grid_destroy(sbm_grid G)
{
    if (!G) return SBM_OK;
    cudaSetDevice(G->dev);
    if (G->st) cudaStreamSynchronize(G->st);
    for (auto &s : G->slots)
        if (s.valid) cudaGraphExecDestroy(s.exec);
    if (G->amr_slot.valid) cudaGraphExecDestroy(G->amr_slot.exec);
    for (int b = 0; b < kBranches; ++b) {
        if (G->side[b]) cudaStreamDestroy(G->side[b]);
        if (G->join_ev[b]) cudaEventDestroy(G->join_ev[b]);
    }
    if (G->fork_ev) cudaEventDestroy(G->fork_ev);
    for (int l = 0; l < G->nl; ++l) {
        Level &L = G->L[l];
        void *ptrs[] = {L.psi64, L.psi32, L.du[0], L.du[1], L.df, L.dr, L.su[0], L.su[1], L.sf, L.sr, L.Ke64, L.Ke32};
        for (void *p : ptrs)
            if (p) cudaFree(p);
    }
    for (int a = 0; a < G->npatch; ++a) free_patch(G->P[a]);
    for (auto &vec : G->adj)
        for (double *q : vec)
            if (q) cudaFree(q);
    void *ptrs[] = {G->fsrc, G->fadj, G->psi_raw, G->rho, G->part, G->scal, G->dbad, G->A64, G->A32, G->gjtmp, G->gjbar, G->gather,
                    G->derr, G->dgate, G->amr_part, G->amr_u0, G->amr_r0, G->dhist, G->top, G->src_sig};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (G->hscal) cudaFreeHost(G->hscal);
    if (G->ev0) cudaEventDestroy(G->ev0);
    if (G->ev1) cudaEventDestroy(G->ev1);
    if (G->own_stream && G->st) cudaStreamDestroy(G->st);
    delete G;
    return SBM_OK;
}

// Everything of sbm_grid_create after the descriptor checks: the stream, the level
// hierarchy and its storage.  On failure the caller destroys the partial grid.
static sbm_status grid_create_impl(const sbm_grid_desc *d, sbm_grid G)
{
    CK(cudaSetDevice(G->dev));
    if (d->stream) {
        G->st = (cudaStream_t)d->stream;
    } else {
        CK(cudaStreamCreate(&G->st));   // blocking: ordered after legacy-stream work
        G->own_stream = true;
    }
    // hierarchy: halve while every (n-1) is even and stays >= 4 after halving
    int n[3] = {d->n[0], d->n[1], d->n[2]};
    double h = d->h;
    std::vector<std::pair<std::vector<int>, double>> shapes;
    shapes.push_back({{n[0], n[1], n[2]}, h});
    while ((int)shapes.size() < kMaxLevels) {
        bool ok = true;
        for (int a = 0; a < d->dim; ++a) {
            const int m = n[a] - 1;
            if (m % 2 != 0 || m / 2 < 4) ok = false;
        }
        if (!ok) break;
        for (int a = 0; a < d->dim; ++a) n[a] = (n[a] - 1) / 2 + 1;
        h *= 2.0;
        shapes.push_back({{n[0], n[1], n[2]}, h});
    }
    G->nl = (int)shapes.size();
    {
        // the coarsest level is solved densely: refuse before allocating anything
        const auto &c = shapes.back().first;
        const long long nb = (long long)c[0] * c[1] * c[2] * d->dim;
        if (nb * nb > (1LL << 28)) return fail(G, SBM_ERR_ARG, "coarsest level too large for the dense bottom solve");
    }
    for (int l = 0; l < G->nl; ++l) {
        const auto &sh = shapes[G->nl - 1 - l];   // level 0 = coarsest
        Level &L = G->L[l];
        L.h = sh.second;
        Geom &g = L.g;
        g.dim = d->dim;
        g.nx = sh.first[0];
        g.ny = sh.first[1];
        g.nz = sh.first[2];
        g.sx = (g.nx + 7) / 8 * 8;
        g.sy = (long long)g.sx * g.ny;
        g.cs = (g.sy * g.nz + 63) / 64 * 64;
        const size_t nd = (size_t)g.dim * g.cs;
        CK(gmalloc(G, (void **)&L.psi64, sizeof(double) * g.cs));
        CK(gmalloc(G, (void **)&L.psi32, sizeof(float) * g.cs));
        CK(cudaMemset(L.psi64, 0, sizeof(double) * g.cs));
        CK(cudaMemset(L.psi32, 0, sizeof(float) * g.cs));
        double **dptrs[] = {&L.du[0], &L.du[1], &L.df, &L.dr};
        for (double **p : dptrs) {
            CK(gmalloc(G, (void **)p, sizeof(double) * nd));
            CK(cudaMemset(*p, 0, sizeof(double) * nd));
        }
        float **sptrs[] = {&L.su[0], &L.su[1], &L.sf, &L.sr};
        for (float **p : sptrs) {
            CK(gmalloc(G, (void **)p, sizeof(float) * nd));
            CK(cudaMemset(*p, 0, sizeof(float) * nd));
        }
        if (g.dim == 3) {
            L.has_tm = true;
            for (int i = 0; i < 2; ++i)
                L.has_tm = L.has_tm && encode_sweep_maps(L.tm32[i], L.su[i], L.sf, L.psi32, g);
        }
        const int nk = (1 << g.dim) * g.dim;
        CK(gmalloc(G, (void **)&L.Ke64, sizeof(double) * nk * nk));
        CK(gmalloc(G, (void **)&L.Ke32, sizeof(float) * nk * nk));
    }
    Level &F = G->L[G->nl - 1];
    const size_t nfd = (size_t)F.g.dim * F.g.cs;
    CK(gmalloc(G, (void **)&G->fsrc, sizeof(double) * nfd));
    CK(cudaMemset(G->fsrc, 0, sizeof(double) * nfd));
    CK(gmalloc(G, (void **)&G->fadj, sizeof(double) * nfd));
    CK(cudaMemset(G->fadj, 0, sizeof(double) * nfd));
    const long long nc = ncells_h(F.g);
    CK(gmalloc(G, (void **)&G->psi_raw, sizeof(double) * nc));
    CK(gmalloc(G, (void **)&G->rho, sizeof(double) * nc));
    G->npart = 1;
    for (int l = 0; l < G->nl; ++l)
        G->npart = std::max({G->npart, sweep_blocks(G->L[l].g, false), sweep_blocks(G->L[l].g, true),
                             sweep_blocks_f2(G->L[l].g)});
    CK(gmalloc(G, (void **)&G->part, sizeof(double) * G->npart));
    CK(gmalloc(G, (void **)&G->derr, sizeof(int)));
    CK(gmalloc(G, (void **)&G->dgate, 2 * sizeof(int)));
    CK(cudaMemset(G->dgate, 0, 2 * sizeof(int)));
    CK(cudaMemset(G->derr, 0, sizeof(int)));
    CK(gmalloc(G, (void **)&G->scal, sizeof(double) * 16));
    CK(cudaMemset(G->scal, 0, sizeof(double) * 16));
    CK(cudaMallocHost(&G->hscal, sizeof(double) * 16));
    CK(gmalloc(G, (void **)&G->dbad, sizeof(int)));
    // bottom
    Level &B = G->L[0];
    G->nb = (int)(nnodes(B.g) * B.g.dim);
    CK(gmalloc(G, (void **)&G->A64, sizeof(double) * G->nb * G->nb));
    CK(gmalloc(G, (void **)&G->A32, sizeof(float) * G->nb * G->nb));
    CK(gmalloc(G, (void **)&G->gjtmp, sizeof(double) * 4 * 16 * G->nb));   // 2 buffers x (16 rows + 16 columns)
    CK(gmalloc(G, (void **)&G->gjbar, sizeof(unsigned) * 4));
    CK(gmalloc(G, (void **)&G->gather, sizeof(int) * G->nb));
    {
        std::vector<int> gi(G->nb);
        const long long N = nnodes(B.g);
        for (int p = 0; p < B.g.dim; ++p)
            for (int k = 0; k < B.g.nz; ++k)
                for (int j = 0; j < B.g.ny; ++j)
                    for (int i = 0; i < B.g.nx; ++i)
                        gi[p * N + i + (long long)B.g.nx * (j + (long long)B.g.ny * k)] = (int)(p * B.g.cs + gidx(B.g, i, j, k));
        CK(cudaMemcpy(G->gather, gi.data(), sizeof(int) * G->nb, cudaMemcpyHostToDevice));
    }
    CK(cudaEventCreate(&G->ev0));
    CK(cudaEventCreate(&G->ev1));
    for (int f = 0; f < 6; ++f)
        for (int p = 0; p < 3; ++p) G->bct[f][p] = SBM_FREE;
    set_dirichlet_bits(G);
    return SBM_OK;
}

sbm_status sbm_grid_create(const sbm_grid_desc *d, sbm_grid *out)
{
    sbm_grid G = nullptr;
    if (!d || !out) return fail(nullptr, SBM_ERR_ARG, "null descriptor or output");
    *out = nullptr;
    if (d->dim != 2 && d->dim != 3) return fail(nullptr, SBM_ERR_ARG, "dim must be 2 or 3");
    if (d->n[0] < 2 || d->n[1] < 2 || (d->dim == 3 && d->n[2] < 2) || (d->dim == 2 && d->n[2] != 1))
        return fail(nullptr, SBM_ERR_ARG, "node counts must be >= 2 (n[2] == 1 in 2D)");
    if (!(d->h > 0.0) || !std::isfinite(d->h)) return fail(nullptr, SBM_ERR_ARG, "h must be positive");
    if (d->precision != SBM_FP64 && d->precision != SBM_MIXED) return fail(nullptr, SBM_ERR_ARG, "bad precision");
    const double nodes = (double)d->n[0] * d->n[1] * d->n[2];
    if (nodes > 2.0e9) return fail(nullptr, SBM_ERR_ARG, "grid too large");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || d->device < 0 || d->device >= ndev) {
        cudaGetLastError();
        return fail(nullptr, SBM_ERR_CUDA, "no CUDA device with the requested ordinal");
    }
    G = new sbm_grid_s();
    G->desc = *d;
    G->dev = d->device;
    const sbm_status st = grid_create_impl(d, G);
    if (st != SBM_OK) {
        // nothing of a failed creation is kept: free what was allocated and report
        // the failure through the library's message (there is no handle)
        const std::string msg = G->err;
        sbm_grid_destroy(G);
        return fail(nullptr, st, msg);
    }
    *out = G;
    return SBM_OK;
}

void sbm_set_alloc_limit(size_t bytes) { g_alloc_cap.store((unsigned long long)bytes); }

sbm_status sbm_set_wait_limit(sbm_grid G, long long spins)
{
    if (!G) return fail(G, SBM_ERR_ARG, "null grid");
    if (spins < 0) return fail(G, SBM_ERR_ARG, "spins must be >= 0");
    G->gj_spins = spins;
    G->bottom_ready = false;        // the next solve inverts the bottom matrix again
    return SBM_OK;
}

sbm_status sbm_grid_levels(sbm_grid G, int *nl)
{
    if (!G || !nl) return fail(G, SBM_ERR_ARG, "null argument");
    *nl = G->nl;
    return SBM_OK;
}

sbm_status sbm_grid_level_shape(sbm_grid G, int level, int n[3], double *h)
{
    sbm_status s = check_level(G, level);
    if (s != SBM_OK) return s;
    if (n) {
        n[0] = G->L[level].g.nx;
        n[1] = G->L[level].g.ny;
        n[2] = G->L[level].g.nz;
    }
    if (h) *h = G->L[level].h;
    return SBM_OK;
}

static sbm_status finish_psi(sbm_grid G)
{
    for (int l = G->nl - 1; l > 0; --l)
        CK(launch_coarsen_psi(G->L[l].g, G->L[l - 1].g, G->L[l].psi64, G->L[l - 1].psi64, G->st));
    for (int l = 0; l < G->nl; ++l) CK(launch_round_cells(G->L[l].g, G->L[l].psi64, G->L[l].psi32, G->st));
    int bad = 0;
    CK(cudaMemcpyAsync(&bad, G->dbad, sizeof(int), cudaMemcpyDeviceToHost, G->st));
    CK(cudaStreamSynchronize(G->st));
    if (bad) {
        G->has_psi = false;
        return fail(G, SBM_ERR_ARG, "psi/rho contains non-finite or negative values");
    }
    G->has_psi = true;
    G->bottom_ready = false;
    return SBM_OK;
}

// psi of the finest level from a device array: raw copy, floor, coarsening.
static sbm_status set_psi_dev(sbm_grid G, const double *psi, double psi_min)
{
    Level &F = G->L[G->nl - 1];
    CK(cudaMemsetAsync(G->dbad, 0, sizeof(int), G->st));
    CK(cudaMemcpyAsync(G->psi_raw, psi, sizeof(double) * ncells_h(F.g), cudaMemcpyDeviceToDevice, G->st));
    CK(launch_set_psi(F.g, psi, psi_min, F.psi64, G->dbad, G->st));
    G->density = 0;
    G->psi_min = psi_min;
    if (G->npatch > 0) G->amr_psi_dirty = true;   // covered cells are re-averaged at the next solve
    return finish_psi(G);
}

sbm_status sbm_set_psi(sbm_grid G, int level, const double *psi, double psi_min)
{
    if (!G) return fail(nullptr, SBM_ERR_ARG, "null grid");
    if (level != G->nl - 1) return fail(G, SBM_ERR_ARG, "psi must be given on the finest level");
    if (!is_dev_ptr(psi, G->dev)) return fail(G, SBM_ERR_ARG, "psi is not a device pointer of the grid's device");
    if (!(psi_min > 0.0) || !std::isfinite(psi_min)) return fail(G, SBM_ERR_ARG, "psi_min must be positive");
    CK(cudaSetDevice(G->dev));
    return set_psi_dev(G, psi, psi_min);
}

sbm_status sbm_set_density(sbm_grid G, int level, const double *rho, double psi_min, double q)
{
    if (!G) return fail(nullptr, SBM_ERR_ARG, "null grid");
    if (level != G->nl - 1) return fail(G, SBM_ERR_ARG, "rho must be given on the finest level");
    if (!is_dev_ptr(rho, G->dev)) return fail(G, SBM_ERR_ARG, "rho is not a device pointer of the grid's device");
    if (!(psi_min > 0.0 && psi_min < 1.0) || !(q >= 1.0)) return fail(G, SBM_ERR_ARG, "need 0 < psi_min < 1, q >= 1");
    CK(cudaSetDevice(G->dev));
    Level &F = G->L[G->nl - 1];
    CK(cudaMemsetAsync(G->dbad, 0, sizeof(int), G->st));
    CK(cudaMemcpyAsync(G->rho, rho, sizeof(double) * ncells_h(F.g), cudaMemcpyDeviceToDevice, G->st));
    CK(launch_set_density(F.g, rho, psi_min, q, F.psi64, G->dbad, G->st));
    G->density = 1;
    G->psi_min = psi_min;
    G->q = q;
    return finish_psi(G);
}

sbm_status sbm_set_moduli(sbm_grid G, int kind, const double p[3])
{
    if (!G || !p) return fail(G, SBM_ERR_ARG, "null argument");
    double c11, c12, c44;
    if (kind == SBM_CUBIC) {
        c11 = p[0];
        c12 = p[1];
        c44 = p[2];
    } else if (kind == SBM_ISO_LAME) {
        c11 = p[0] + 2.0 * p[1];
        c12 = p[0];
        c44 = p[1];
    } else if (kind == SBM_ISO_ENU) {
        const double E = p[0], nu = p[1];
        if (!(nu > -1.0 && nu < 0.5)) return fail(G, SBM_ERR_ARG, "Poisson ratio must be in (-1, 0.5)");
        const double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), mu = E / (2.0 * (1.0 + nu));
        c11 = lam + 2.0 * mu;
        c12 = lam;
        c44 = mu;
    } else {
        return fail(G, SBM_ERR_ARG, "unknown moduli kind");
    }
    if (!moduli_definite(G->desc.dim, c11, c12, c44)) return fail(G, SBM_ERR_ARG, "moduli are not positive definite");
    CK(cudaSetDevice(G->dev));
    G->mod[0] = c11;
    G->mod[1] = c12;
    G->mod[2] = c44;
    make_level_coefs(G);
    sbm_status s = upload_Ke(G);
    if (s != SBM_OK) return s;
    G->has_moduli = true;
    G->bottom_ready = false;
    ++G->version;
    return SBM_OK;
}

sbm_status sbm_set_bc(sbm_grid G, int face, int comp, int type, double value)
{
    if (!G) return fail(nullptr, SBM_ERR_ARG, "null grid");
    if (face < 0 || face >= 2 * G->desc.dim) return fail(G, SBM_ERR_ARG, "face out of range");
    if (comp < 0 || comp >= G->desc.dim) return fail(G, SBM_ERR_ARG, "component out of range");
    if (type != SBM_FREE && type != SBM_DIRICHLET && type != SBM_DIRICHLET_FROM_U)
        return fail(G, SBM_ERR_ARG, "unknown face condition");
    if (!std::isfinite(value)) return fail(G, SBM_ERR_ARG, "non-finite boundary value");
    G->bct[face][comp] = type;
    G->bcv[face][comp] = value;
    set_dirichlet_bits(G);
    G->bottom_ready = false;
    ++G->version;
    return SBM_OK;
}

sbm_status sbm_set_source(sbm_grid G, int level, const double *f)
{
    if (!G) return fail(nullptr, SBM_ERR_ARG, "null grid");
    if (level != G->nl - 1) return fail(G, SBM_ERR_ARG, "the source must be given on the finest level");
    if (!is_dev_ptr(f, G->dev)) return fail(G, SBM_ERR_ARG, "f is not a device pointer of the grid's device");
    CK(cudaSetDevice(G->dev));
    Level &F = G->L[G->nl - 1];
    CK(launch_pack<double, double>(F.g, F.g.dim, f, G->fsrc, G->st));
    CK(cudaStreamSynchronize(G->st));
    return SBM_OK;
}

sbm_status sbm_solve(sbm_grid G, double *u, const sbm_opts *opts, sbm_info *info)
{
    sbm_status s = check_ready(G);
    if (s != SBM_OK) return s;
    if (!is_dev_ptr(u, G->dev)) return fail(G, SBM_ERR_ARG, "u is not a device pointer of the grid's device");
    sbm_opts o;
    sbm_default_opts(&o);
    if (opts) o = *opts;
    if ((s = validate_opts(G, o)) != SBM_OK) return s;
    CK(cudaSetDevice(G->dev));
    Level &F = G->L[G->nl - 1];
    CK(launch_pack<double, double>(F.g, F.g.dim, u, F.du[0], G->st));
    for (int f = 0; f < 2 * F.g.dim; ++f)
        for (int p = 0; p < F.g.dim; ++p)
            if (G->bct[f][p] == SBM_DIRICHLET) CK(launch_set_face(F.g, f, p, G->bcv[f][p], F.du[0], G->st));
    s = run_solve(G, o, G->fsrc, info, 0);
    if (s != SBM_OK && s != SBM_ERR_NOCONV && s != SBM_ERR_DIVERGED) return s;
    CK(launch_unpack<double, double>(F.g, F.g.dim, F.du[0], u, G->st));
    CK(cudaStreamSynchronize(G->st));
    return s;
}

sbm_status sbm_adjoint(sbm_grid G, const double *u, const double *dJdu, double *lambda, double *dJdpsi,
                       double *dJdrho, const sbm_opts *opts, sbm_info *info)
{
    sbm_status s = check_ready(G);
    if (s != SBM_OK) return s;
    if (!is_dev_ptr(u, G->dev) || !is_dev_ptr(dJdu, G->dev) || !is_dev_ptr(lambda, G->dev) ||
        !is_dev_ptr(dJdpsi, G->dev) || (dJdrho && !is_dev_ptr(dJdrho, G->dev)))
        return fail(G, SBM_ERR_ARG, "u, dJdu, lambda, dJdpsi (and dJdrho) must be device pointers of the grid's device");
    sbm_opts o;
    sbm_default_opts(&o);
    if (opts) o = *opts;
    if ((s = validate_opts(G, o)) != SBM_OK) return s;
    CK(cudaSetDevice(G->dev));
    Level &F = G->L[G->nl - 1];
    CK(launch_pack<double, double>(F.g, F.g.dim, dJdu, G->fadj, G->st));
    CK(cudaMemsetAsync(F.du[0], 0, level_bytes(F, sizeof(double)), G->st));   // lambda_0 = 0, homogeneous Dirichlet
    s = run_solve(G, o, G->fadj, info, 1);
    if (s != SBM_OK && s != SBM_ERR_NOCONV && s != SBM_ERR_DIVERGED) return s;
    CK(launch_unpack<double, double>(F.g, F.g.dim, F.du[0], lambda, G->st));
    CK(launch_dJdpsi(F.g, F.c64, u, lambda, dJdpsi, dJdrho, G->rho, G->psi_raw, G->psi_min, G->q, G->density, G->st));
    CK(cudaStreamSynchronize(G->st));
    return s;
}

// ------------------------------------------------------------------ steps

sbm_status sbm_apply(sbm_grid G, int level, int fp32, const double *u, double *Ku)
{
    sbm_status s = check_level(G, level);
    if (s != SBM_OK) return s;
    if (!G->has_moduli || !G->has_psi) return check_ready(G);
    if (!is_dev_ptr(u, G->dev) || !is_dev_ptr(Ku, G->dev)) return fail(G, SBM_ERR_ARG, "u and Ku must be device pointers");
    CK(cudaSetDevice(G->dev));
    Level &L = G->L[level];
    if (fp32) {
        CK(launch_pack<double, float>(L.g, L.g.dim, u, L.su[1], G->st));
        CK(sweep<float>(G, level, kApply, L.su[1], nullptr, L.sr, nullptr, 0.0));
        CK(launch_unpack<float, double>(L.g, L.g.dim, L.sr, Ku, G->st));
    } else {
        CK(launch_pack<double, double>(L.g, L.g.dim, u, L.du[1], G->st));
        CK(sweep<double>(G, level, kApply, L.du[1], nullptr, L.dr, nullptr, 0.0));
        CK(launch_unpack<double, double>(L.g, L.g.dim, L.dr, Ku, G->st));
    }
    CK(cudaStreamSynchronize(G->st));
    return SBM_OK;
}

sbm_status sbm_residual(sbm_grid G, int level, int fp32, const double *f, const double *u, double *r, double *norm)
{
    sbm_status s = check_level(G, level);
    if (s != SBM_OK) return s;
    if (!G->has_moduli || !G->has_psi) return check_ready(G);
    if (!is_dev_ptr(u, G->dev) || !is_dev_ptr(f, G->dev) || !is_dev_ptr(r, G->dev))
        return fail(G, SBM_ERR_ARG, "f, u and r must be device pointers");
    CK(cudaSetDevice(G->dev));
    Level &L = G->L[level];
    const int nb = (int)sweep_nblocks(G, level, fp32 != 0, fp32 ? (const void *)L.su[1] : (const void *)L.du[1],
                                      fp32 ? (const void *)L.sf : (const void *)L.df);
    if (fp32) {
        CK(launch_pack<double, float>(L.g, L.g.dim, u, L.su[1], G->st));
        CK(launch_pack<double, float>(L.g, L.g.dim, f, L.sf, G->st));
        CK(sweep<float>(G, level, kResidual, L.su[1], L.sf, L.sr, G->part, 0.0));
        CK(launch_unpack<float, double>(L.g, L.g.dim, L.sr, r, G->st));
    } else {
        CK(launch_pack<double, double>(L.g, L.g.dim, u, L.du[1], G->st));
        CK(launch_pack<double, double>(L.g, L.g.dim, f, L.df, G->st));
        CK(sweep<double>(G, level, kResidual, L.du[1], L.df, L.dr, G->part, 0.0));
        CK(launch_unpack<double, double>(L.g, L.g.dim, L.dr, r, G->st));
    }
    CK(launch_norm_final(G->part, nb, G->scal, 5, G->st));
    CK(cudaMemcpyAsync(G->hscal + 5, G->scal + 5, 2 * sizeof(double), cudaMemcpyDeviceToHost, G->st));
    CK(cudaStreamSynchronize(G->st));
    if (norm) *norm = G->hscal[6];
    return SBM_OK;
}

sbm_status sbm_smooth(sbm_grid G, int level, int fp32, int smoother, double omega, int descending, const double *f,
                      double *u)
{
    sbm_status s = check_level(G, level);
    if (s != SBM_OK) return s;
    if (!G->has_moduli || !G->has_psi) return check_ready(G);
    if (!is_dev_ptr(u, G->dev) || !is_dev_ptr(f, G->dev)) return fail(G, SBM_ERR_ARG, "f and u must be device pointers");
    if (smoother != SBM_JACOBI && smoother != SBM_MCGS) return fail(G, SBM_ERR_ARG, "unknown smoother");
    CK(cudaSetDevice(G->dev));
    sbm_opts o;
    sbm_default_opts(&o);
    o.smoother = smoother;
    o.omega = omega;
    Level &L = G->L[level];
    int cur = 0;
    if (fp32) {
        CK(launch_pack<double, float>(L.g, L.g.dim, u, L.su[0], G->st));
        CK(launch_pack<double, float>(L.g, L.g.dim, f, L.sf, G->st));
        CK(smooth<float>(G, level, cur, o, 1, descending != 0, L.sf));
        CK(launch_unpack<float, double>(L.g, L.g.dim, L.su[cur], u, G->st));
    } else {
        CK(launch_pack<double, double>(L.g, L.g.dim, u, L.du[0], G->st));
        CK(launch_pack<double, double>(L.g, L.g.dim, f, L.df, G->st));
        CK(smooth<double>(G, level, cur, o, 1, descending != 0, L.df));
        CK(launch_unpack<double, double>(L.g, L.g.dim, L.du[cur], u, G->st));
    }
    CK(cudaStreamSynchronize(G->st));
    return SBM_OK;
}

sbm_status sbm_restrict(sbm_grid G, int level, int fp32, const double *rf, double *rc)
{
    sbm_status s = check_level(G, level);
    if (s != SBM_OK) return s;
    if (level < 1) return fail(G, SBM_ERR_ARG, "restriction needs a fine level >= 1");
    if (!is_dev_ptr(rf, G->dev) || !is_dev_ptr(rc, G->dev)) return fail(G, SBM_ERR_ARG, "device pointers required");
    CK(cudaSetDevice(G->dev));
    Level &L = G->L[level], &C = G->L[level - 1];
    if (fp32) {
        CK(launch_pack<double, float>(L.g, L.g.dim, rf, L.sr, G->st));
        CK(launch_restrict<float>(L.g, C.g, L.sr, C.sf, G->st));
        CK(launch_unpack<float, double>(C.g, C.g.dim, C.sf, rc, G->st));
    } else {
        CK(launch_pack<double, double>(L.g, L.g.dim, rf, L.dr, G->st));
        CK(launch_restrict<double>(L.g, C.g, L.dr, C.df, G->st));
        CK(launch_unpack<double, double>(C.g, C.g.dim, C.df, rc, G->st));
    }
    CK(cudaStreamSynchronize(G->st));
    return SBM_OK;
}

sbm_status sbm_prolong_add(sbm_grid G, int level, int fp32, const double *ec, double *uf)
{
    sbm_status s = check_level(G, level);
    if (s != SBM_OK) return s;
    if (level < 1) return fail(G, SBM_ERR_ARG, "prolongation needs a fine level >= 1");
    if (!is_dev_ptr(ec, G->dev) || !is_dev_ptr(uf, G->dev)) return fail(G, SBM_ERR_ARG, "device pointers required");
    CK(cudaSetDevice(G->dev));
    Level &L = G->L[level], &C = G->L[level - 1];
    if (fp32) {
        CK(launch_pack<double, float>(C.g, C.g.dim, ec, C.su[1], G->st));
        CK(launch_pack<double, float>(L.g, L.g.dim, uf, L.su[1], G->st));
        CK(launch_prolong_add<float>(L.g, C.g, C.su[1], L.su[1], G->st));
        CK(launch_unpack<float, double>(L.g, L.g.dim, L.su[1], uf, G->st));
    } else {
        CK(launch_pack<double, double>(C.g, C.g.dim, ec, C.du[1], G->st));
        CK(launch_pack<double, double>(L.g, L.g.dim, uf, L.du[1], G->st));
        CK(launch_prolong_add<double>(L.g, C.g, C.du[1], L.du[1], G->st));
        CK(launch_unpack<double, double>(L.g, L.g.dim, L.du[1], uf, G->st));
    }
    CK(cudaStreamSynchronize(G->st));
    return SBM_OK;
}

sbm_status sbm_get_psi(sbm_grid G, int level, double *psi)
{
    sbm_status s = check_level(G, level);
    if (s != SBM_OK) return s;
    if (!G->has_psi) return fail(G, SBM_ERR_STATE, "psi not set");
    if (!is_dev_ptr(psi, G->dev)) return fail(G, SBM_ERR_ARG, "psi must be a device pointer");
    CK(cudaSetDevice(G->dev));
    CK(launch_get_cells(G->L[level].g, G->L[level].psi64, psi, G->st));
    CK(cudaStreamSynchronize(G->st));
    return SBM_OK;
}

sbm_status sbm_bottom_correct(sbm_grid G, int fp32, const double *f, double *u)
{
    sbm_status s = check_ready(G);
    if (s != SBM_OK) return s;
    if (!is_dev_ptr(u, G->dev) || !is_dev_ptr(f, G->dev)) return fail(G, SBM_ERR_ARG, "f and u must be device pointers");
    CK(cudaSetDevice(G->dev));
    if ((s = setup_bottom(G)) != SBM_OK) return s;
    Level &B = G->L[0];
    if (fp32) {
        CK(launch_pack<double, float>(B.g, B.g.dim, u, B.su[1], G->st));
        CK(launch_pack<double, float>(B.g, B.g.dim, f, B.sf, G->st));
        CK(sweep<float>(G, 0, kResidual, B.su[1], B.sf, B.sr, nullptr, 0.0));
        CK(launch_bottom_apply<float>(G->nb, G->A32, G->gather, B.sr, B.su[1], 1, G->st));
        CK(launch_unpack<float, double>(B.g, B.g.dim, B.su[1], u, G->st));
    } else {
        CK(launch_pack<double, double>(B.g, B.g.dim, u, B.du[1], G->st));
        CK(launch_pack<double, double>(B.g, B.g.dim, f, B.df, G->st));
        CK(sweep<double>(G, 0, kResidual, B.du[1], B.df, B.dr, nullptr, 0.0));
        CK(launch_bottom_apply<double>(G->nb, G->A64, G->gather, B.dr, B.du[1], 1, G->st));
        CK(launch_unpack<double, double>(B.g, B.g.dim, B.du[1], u, G->st));
    }
    CK(cudaStreamSynchronize(G->st));
    return SBM_OK;
}

sbm_status sbm_dJdpsi(sbm_grid G, const double *u, const double *lam, double *g)
{
    sbm_status s = check_ready(G);
    if (s != SBM_OK) return s;
    if (!is_dev_ptr(u, G->dev) || !is_dev_ptr(lam, G->dev) || !is_dev_ptr(g, G->dev))
        return fail(G, SBM_ERR_ARG, "u, lambda and dJdpsi must be device pointers");
    CK(cudaSetDevice(G->dev));
    Level &F = G->L[G->nl - 1];
    CK(launch_dJdpsi(F.g, F.c64, u, lam, g, nullptr, nullptr, nullptr, 0.0, 3.0, 0, G->st));
    CK(cudaStreamSynchronize(G->st));
    return SBM_OK;
}

sbm_status sbm_apply_product(sbm_grid G, int variant, const double *psi, const double *u, double *Ku)
{
    if (!G) return fail(G, SBM_ERR_ARG, "null grid");
    if (variant != SBM_OP_PRODUCT_NODE && variant != SBM_OP_PRODUCT_CELL) return fail(G, SBM_ERR_ARG, "unknown variant");
    if (!G->has_moduli) return fail(G, SBM_ERR_STATE, "moduli not set (sbm_set_moduli)");
    if (!is_dev_ptr(psi, G->dev) || !is_dev_ptr(u, G->dev) || !is_dev_ptr(Ku, G->dev))
        return fail(G, SBM_ERR_ARG, "psi, u and Ku must be device pointers");
    CK(cudaSetDevice(G->dev));
    const Level &L = G->L[G->nl - 1];
    const int n[3] = {L.g.nx, L.g.ny, L.g.nz};
    CK(launch_product(0, L.g.dim, n, L.h, G->mod, L.g.dm, variant, 0.0, psi, u, nullptr, Ku, G->st));
    CK(cudaStreamSynchronize(G->st));
    return SBM_OK;
}

sbm_status sbm_source_terms(sbm_grid G, int level, const double *psi, const double *eps0, const double *b,
                            const double *t, double *f)
{
    if (!G) return fail(G, SBM_ERR_ARG, "null grid");
    if (!G->has_moduli) return fail(G, SBM_ERR_STATE, "moduli not set (sbm_set_moduli)");
    if (level < 0 || level >= G->nl) return fail(G, SBM_ERR_ARG, "level out of range");
    if (!is_dev_ptr(psi, G->dev) || !is_dev_ptr(f, G->dev))
        return fail(G, SBM_ERR_ARG, "psi and f must be device pointers");
    if ((eps0 && !is_dev_ptr(eps0, G->dev)) || (b && !is_dev_ptr(b, G->dev)) || (t && !is_dev_ptr(t, G->dev)))
        return fail(G, SBM_ERR_ARG, "eps0, b and t must be device pointers or NULL");
    CK(cudaSetDevice(G->dev));
    const Level &L = G->L[level];
    const int n[3] = {L.g.nx, L.g.ny, L.g.nz};
    double *sig = nullptr;
    if (eps0) {
        const size_t bytes = sizeof(double) * (L.g.dim == 3 ? 6 : 3) * (size_t)ncells_h(L.g);
        if (G->src_bytes < bytes) {
            if (G->src_sig) cudaFree(G->src_sig);
            G->src_sig = nullptr;
            G->src_bytes = 0;
            CK(gmalloc(G, (void **)&G->src_sig, bytes));
            G->src_bytes = bytes;
        }
        sig = G->src_sig;
    }
    CK(launch_source_terms(L.g.dim, n, L.h, G->mod, psi, eps0, b, t, f, sig, G->st));
    CK(cudaStreamSynchronize(G->st));
    return SBM_OK;
}

// ------------------------------------------------- topology optimisation (Sec. 3.3)

static sbm_status topopt_check(sbm_grid G, const sbm_topopt_params *p)
{
    if (!G) return fail(nullptr, SBM_ERR_ARG, "null grid");
    if (!p) return fail(G, SBM_ERR_ARG, "null parameters");
    const double v[] = {p->alpha, p->beta, p->zeta, p->lambda, p->lambda_rate, p->V0, p->mobility, p->dt, p->psi_min};
    for (double x : v)
        if (!std::isfinite(x)) return fail(G, SBM_ERR_ARG, "non-finite topology-optimisation parameter");
    if (p->alpha < 0 || p->beta < 0 || p->lambda < 0 || p->lambda_rate < 0 || !(p->mobility > 0) || !(p->dt > 0) ||
        !(p->psi_min > 0) || p->zeta < 0)
        return fail(G, SBM_ERR_ARG, "need alpha, beta, zeta, lambda, lambda_rate >= 0 and mobility, dt, psi_min > 0");
    if (!G->has_moduli) return fail(G, SBM_ERR_STATE, "moduli not set (sbm_set_moduli)");
    if (G->npatch > 0) return fail(G, SBM_ERR_STATE, "topology optimisation runs on single-level grids");
    if (!G->top) {
        const long long NC = ncells_h(G->L[G->nl - 1].g);
        const long long B = topopt_blocks(NC);
        CK(gmalloc(G, (void **)&G->top, sizeof(double) * (2 * NC + 2 * B + 8)));
    }
    return SBM_OK;
}

static TopoptArgs topopt_args(sbm_grid G, const sbm_topopt_params *p, int step)
{
    const Level &F = G->L[G->nl - 1];
    TopoptArgs A;
    A.nx = F.g.nx;
    A.ny = F.g.ny;
    A.nz = F.g.nz;
    A.alpha = p->alpha;
    A.beta = p->beta;
    A.zeta = p->zeta;
    A.lam = p->lambda + p->lambda_rate * step * p->dt;
    A.V0 = p->V0;
    A.dtL = p->dt * p->mobility;
    A.hd = std::pow(F.h, F.g.dim);
    A.ih2 = 1.0 / (F.h * F.h);
    A.psx = F.g.sx;
    A.psy = F.g.sy;
    return A;
}

sbm_status sbm_topopt_step(sbm_grid G, const sbm_topopt_params *p, int step, const double *eta, const double *u,
                           double *eta_out, double *volume, double *compliance)
{
    sbm_status st = topopt_check(G, p);
    if (st != SBM_OK) return st;
    if (step < 0) return fail(G, SBM_ERR_ARG, "step must be >= 0");
    if (!is_dev_ptr(eta, G->dev) || !is_dev_ptr(u, G->dev) || !is_dev_ptr(eta_out, G->dev))
        return fail(G, SBM_ERR_ARG, "eta, u and eta_out must be device pointers of the grid's device");
    if (eta == eta_out) return fail(G, SBM_ERR_ARG, "eta_out must not alias eta");
    CK(cudaSetDevice(G->dev));
    const Level &F = G->L[G->nl - 1];
    const long long NC = ncells_h(F.g);
    const int B = topopt_blocks(NC);
    double *part = G->top + 2 * NC, *scal = part + 2 * B;
    const TopoptArgs A = topopt_args(G, p, step);
    CK(launch_cell_sum(NC, eta, 0.0, nullptr, part, G->st));
    CK(launch_sum_parts(part, B, scal, G->st));
    CK(launch_topopt_step(F.g.dim, A, F.c64, eta, u, G->has_psi ? F.psi64 : nullptr, scal, eta_out, nullptr, part,
                          G->st));
    CK(launch_sum_parts(part, B, scal + 1, G->st));
    CK(launch_sum_parts(part + B, B, scal + 2, G->st));
    double h[3];
    CK(cudaMemcpyAsync(h, scal, sizeof(h), cudaMemcpyDeviceToHost, G->st));
    CK(cudaStreamSynchronize(G->st));
    if (volume) *volume = A.hd * h[1];
    if (compliance) *compliance = A.hd * h[2];
    return SBM_OK;
}

sbm_status sbm_topopt_run(sbm_grid G, const sbm_topopt_params *p, int steps, double *eta, double *u,
                          const sbm_opts *opts, sbm_topopt_info *info)
{
    sbm_status st = topopt_check(G, p);
    if (st != SBM_OK) return st;
    if (steps < 0) return fail(G, SBM_ERR_ARG, "steps must be >= 0");
    if (!is_dev_ptr(eta, G->dev) || !is_dev_ptr(u, G->dev))
        return fail(G, SBM_ERR_ARG, "eta and u must be device pointers of the grid's device");
    sbm_opts o;
    sbm_default_opts(&o);
    if (opts) o = *opts;
    if ((st = validate_opts(G, o)) != SBM_OK) return st;
    CK(cudaSetDevice(G->dev));
    if (info) info->steps = 0;
    Level &F = G->L[G->nl - 1];
    const long long NC = ncells_h(F.g);
    const int B = topopt_blocks(NC);
    double *psi = G->top, *scratch = G->top + NC, *part = G->top + 2 * NC, *scal = part + 2 * B;
    double *cur = eta, *nxt = scratch;
    const auto t0 = std::chrono::steady_clock::now();
    // psi of the first solve and the volume of the initial eta
    CK(launch_cell_sum(NC, eta, p->zeta, psi, part, G->st));
    CK(launch_sum_parts(part, B, scal, G->st));
    for (int s = 0; s < steps; ++s) {
        if ((st = set_psi_dev(G, psi, p->psi_min)) != SBM_OK) return st;
        CK(launch_pack<double, double>(F.g, F.g.dim, u, F.du[0], G->st));
        for (int f = 0; f < 2 * F.g.dim; ++f)
            for (int q = 0; q < F.g.dim; ++q)
                if (G->bct[f][q] == SBM_DIRICHLET) CK(launch_set_face(F.g, f, q, G->bcv[f][q], F.du[0], G->st));
        sbm_info si{};
        st = run_solve(G, o, G->fsrc, &si, 0);
        if (st != SBM_OK && st != SBM_ERR_NOCONV && st != SBM_ERR_DIVERGED) return st;
        CK(launch_unpack<double, double>(F.g, F.g.dim, F.du[0], u, G->st));
        if (st != SBM_OK) {
            if (cur != eta) CK(cudaMemcpyAsync(eta, cur, sizeof(double) * NC, cudaMemcpyDeviceToDevice, G->st));
            CK(cudaStreamSynchronize(G->st));
            return st;
        }
        const TopoptArgs A = topopt_args(G, p, s);
        CK(launch_topopt_step(F.g.dim, A, F.c64, cur, u, F.psi64, scal, nxt, psi, part, G->st));
        CK(launch_sum_parts(part, B, scal, G->st));
        CK(launch_sum_parts(part + B, B, scal + 1, G->st));
        double h[2];
        CK(cudaMemcpyAsync(h, scal, sizeof(h), cudaMemcpyDeviceToHost, G->st));
        CK(cudaStreamSynchronize(G->st));
        if (info) {
            if (s < info->capacity) {
                if (info->compliance) info->compliance[s] = A.hd * h[1];
                if (info->volume) info->volume[s] = A.hd * h[0];
                if (info->cycles) info->cycles[s] = si.cycles;
            }
            info->steps = s + 1;
        }
        std::swap(cur, nxt);
    }
    if (cur != eta) CK(cudaMemcpyAsync(eta, cur, sizeof(double) * NC, cudaMemcpyDeviceToDevice, G->st));
    CK(cudaStreamSynchronize(G->st));
    if (info) info->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return SBM_OK;
}

sbm_status sbm_jacobi_product(sbm_grid G, int variant, const double *psi, const double *f, double *u, double omega,
                              int sweeps)
{
    if (!G) return fail(G, SBM_ERR_ARG, "null grid");
    if (variant != SBM_OP_PRODUCT_NODE && variant != SBM_OP_PRODUCT_CELL) return fail(G, SBM_ERR_ARG, "unknown variant");
    if (sweeps < 0 || !(omega > 0.0 && omega < 2.0)) return fail(G, SBM_ERR_ARG, "sweeps >= 0 and 0 < omega < 2");
    if (!G->has_moduli) return fail(G, SBM_ERR_STATE, "moduli not set (sbm_set_moduli)");
    if (!is_dev_ptr(psi, G->dev) || !is_dev_ptr(u, G->dev) || !is_dev_ptr(f, G->dev))
        return fail(G, SBM_ERR_ARG, "psi, f and u must be device pointers");
    CK(cudaSetDevice(G->dev));
    set_dirichlet_bits(G);
    Level &L = G->L[G->nl - 1];
    const int n[3] = {L.g.nx, L.g.ny, L.g.nz};
    const size_t bytes = sizeof(double) * L.g.dim * (size_t)nnodes(L.g);
    // ping-pong through the finest level's two work buffers (each holds dim * cs >= dim * N)
    double *buf[2] = {L.du[0], L.du[1]};
    CK(cudaMemcpyAsync(buf[0], u, bytes, cudaMemcpyDeviceToDevice, G->st));
    int cur = 0;
    for (int s = 0; s < sweeps; ++s) {
        CK(launch_product(1, L.g.dim, n, L.h, G->mod, L.g.dm, variant, omega, psi, buf[cur], f, buf[1 - cur], G->st));
        cur ^= 1;
    }
    CK(cudaMemcpyAsync(u, buf[cur], bytes, cudaMemcpyDeviceToDevice, G->st));
    CK(cudaStreamSynchronize(G->st));
    return SBM_OK;
}

sbm_status sbm_time_kernel(sbm_grid G, int which, int reps, int flush_l2, double *ms, double *bytes, double *flops)
{
    sbm_status s = check_ready(G);
    if (s != SBM_OK) return s;
    if (which < SBM_K_RESIDUAL64 || which > SBM_K_GS || reps < 1) return fail(G, SBM_ERR_ARG, "bad kernel id or reps");
    if (which == SBM_K_GS && G->desc.dim != 2) return fail(G, SBM_ERR_ARG, "SBM_K_GS times the 2D colour sweep");
    CK(cudaSetDevice(G->dev));
    const int fine = G->nl - 1;
    Level &L = G->L[fine];
    const int mixed = G->desc.precision == SBM_MIXED;
    const int d = L.g.dim;
    const double nn = (double)nnodes(L.g), nc = (double)ncells_h(L.g);
    const double cellf = d == 3 ? 195.0 : 38.0, nodef = d == 3 ? 41.0 : 26.0;
    // scratch inputs of the source-term and topology-step kernels (packed arrays)
    const int nv = d == 3 ? 6 : 3;
    const long long NC = ncells_h(L.g), NN = nnodes(L.g);
    const int TB = topopt_blocks(NC);
    double *scr = nullptr;
    struct FreeOnExit {
        double *&p;
        ~FreeOnExit()
        {
            if (p) cudaFree(p);
        }
    } free_scr{scr};
    int nsm = 0;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, G->dev));
    const int fma_blocks = 8 * nsm, fma_threads = 256, fma_iters = which == SBM_K_FMA64 ? 1 << 11 : 1 << 14;
    if (which == SBM_K_FMA64 || which == SBM_K_FMA32) {
        CK(cudaMalloc(&scr, 64));
    } else if (which >= SBM_K_SOURCE) {
        const size_t n = (size_t)NC * (2 * nv + 4) + (size_t)NN * d * 3 + 2 * TB + 8;
        CK(cudaMalloc(&scr, sizeof(double) * n));
        CK(cudaMemsetAsync(scr, 0, sizeof(double) * n, G->st));
    }
    double *s_eps = scr, *s_eta = scr + NC * nv, *s_eta2 = s_eta + NC, *s_psi = s_eta2 + NC, *s_psi2 = s_psi + NC,
           *s_b = s_psi2 + NC, *s_t = s_b + NN * d, *s_f = s_t + NN * d, *s_part = s_f + NN * d,
           *s_scal = s_part + 2 * TB, *s_sig = s_scal + 8;
    sbm_topopt_params tp{200.0, 0.01, 0.01, 400.0, 0.0, 0.25, 1.0, 1e-4, 1e-6};
    const TopoptArgs TA = topopt_args(G, &tp, 0);
    const int nsz[3] = {L.g.nx, L.g.ny, L.g.nz};
    auto launch = [&]() -> cudaError_t {
        if (which == SBM_K_RESIDUAL64) return residual64(G, G->fsrc, mixed, 5);
        if (which == SBM_K_SOURCE)
            return launch_source_terms(d, nsz, L.h, G->mod, G->psi_raw, s_eps, s_b, s_t, s_f, s_sig, G->st);
        if (which == SBM_K_TOPOPT)
            return launch_topopt_step(d, TA, L.c64, s_eta, s_b, L.psi64, s_scal, s_eta2, s_psi2, s_part, G->st);
        if (which == SBM_K_FMA64 || which == SBM_K_FMA32)
            return launch_fma_rate(which == SBM_K_FMA64, fma_blocks, fma_threads, fma_iters, scr, G->st);
        int cur = 0;
        sbm_opts o;
        sbm_default_opts(&o);
        o.nu1 = 1;
        if (which == SBM_K_GS) o.smoother = SBM_MCGS;
        if (which == SBM_K_JACOBI || which == SBM_K_GS) {
            if (mixed) return smooth<float>(G, fine, cur, o, 1, false, L.sf);
            return smooth<double>(G, fine, cur, o, 1, false, L.df);
        }
        if (mixed) return sweep<float>(G, fine, kResidual, L.su[0], L.sf, L.sr, nullptr, 0.0);
        return sweep<double>(G, fine, kResidual, L.du[0], L.df, L.dr, nullptr, 0.0);
    };
    {
        cudaError_t e = launch();
        if (e != cudaSuccess) return fail(G, SBM_ERR_CUDA, std::string("sbm_time_kernel: ") + cudaGetErrorString(e));
    }
    float t = 0.f;
    if (flush_l2) {
        // flush: write 256 MB, then read a second 256 MB buffer, so that the launch
        // finds neither its inputs nor dirty lines (whose write-back would be charged
        // to it) in the 126 MB L2
        const size_t fb = 256ull << 20;
        void *flush = nullptr;
        CK(cudaMalloc(&flush, 2 * fb + 64));
        CK(cudaMemsetAsync(flush, 0, 2 * fb + 64, G->st));
        void *clean = static_cast<char *>(flush) + fb;
        float *sink = reinterpret_cast<float *>(static_cast<char *>(flush) + 2 * fb);
        for (int r = 0; r < reps; ++r) {
            cudaError_t e = cudaMemsetAsync(flush, r & 0xff, fb, G->st);
            if (e == cudaSuccess) e = launch_l2_read(clean, fb, sink, G->st);
            if (e == cudaSuccess) e = cudaEventRecord(G->ev0, G->st);
            if (e == cudaSuccess) e = launch();
            if (e == cudaSuccess) e = cudaEventRecord(G->ev1, G->st);
            if (e == cudaSuccess) e = cudaEventSynchronize(G->ev1);
            float tr = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&tr, G->ev0, G->ev1);
            if (e != cudaSuccess) {
                cudaFree(flush);
                return fail(G, SBM_ERR_CUDA, std::string("sbm_time_kernel: ") + cudaGetErrorString(e));
            }
            t += tr;
        }
        CK(cudaFree(flush));
    } else {
        CK(cudaEventRecord(G->ev0, G->st));
        for (int r = 0; r < reps; ++r) CK(launch());
        CK(cudaEventRecord(G->ev1, G->st));
        CK(cudaEventSynchronize(G->ev1));
        CK(cudaEventElapsedTime(&t, G->ev0, G->ev1));
    }
    if (ms) *ms = t / reps;
    if (which == SBM_K_SOURCE) {
        if (bytes) *bytes = 8.0 * (NC * (1.0 + nv) + NN * 3.0 * d);
        if (flops) *flops = (double)NC * (d == 3 ? 60.0 : 24.0) + (double)NN * (d == 3 ? 60.0 : 40.0);
        return SBM_OK;
    }
    if (which == SBM_K_TOPOPT) {
        if (bytes) *bytes = 8.0 * (NC * 4.0 + NN * d);
        if (flops) *flops = (double)NC * (cellf + 50.0);
        return SBM_OK;
    }
    if (which == SBM_K_FMA64 || which == SBM_K_FMA32) {
        if (bytes) *bytes = 0.0;
        if (flops) *flops = 16.0 * fma_iters * (double)fma_blocks * fma_threads;
        return SBM_OK;
    }
    // per node: read u and f (d values each), psi (one cell per node), write d outputs
    double per_node;
    if (which == SBM_K_RESIDUAL64) per_node = mixed ? (8.0 * d + 8.0 * d + 8.0 + 4.0 * d) : (8.0 * (3 * d + 1));
    else per_node = (mixed ? 4.0 : 8.0) * (3 * d + 1);
    if (bytes) *bytes = per_node * nn;
    if (which == SBM_K_GS) {
        // per relaxed node: 4 cells x (16 + 2 + 4) multiply-adds, then the 2-component update
        if (flops) *flops = 190.0 * nn;
        return SBM_OK;
    }
    if (flops) *flops = cellf * nc + (which == SBM_K_JACOBI ? nodef : nodef - 11.0) * nn;
    return SBM_OK;
}

// ------------------------------------------------------------------- BSAMR

// Storage of patch level a (box already checked and recorded in Pt) and the
// composite-solve buffers it needs; on failure the caller frees the patch.
static sbm_status patch_alloc(sbm_grid G, int a, Patch &Pt)
{
    const int d = G->desc.dim;
    const Geom &g = Pt.s;
    const size_t nd = (size_t)d * g.cs;
    CK(gmalloc(G, (void **)&Pt.psi64, sizeof(double) * g.cs));
    CK(cudaMemset(Pt.psi64, 0, sizeof(double) * g.cs));
    CK(gmalloc(G, (void **)&Pt.psi32, sizeof(float) * g.cs));
    CK(cudaMemset(Pt.psi32, 0, sizeof(float) * g.cs));
    double **dp[] = {&Pt.u64, &Pt.f64, &Pt.r64, &Pt.de[0], &Pt.de[1], &Pt.drhs, &Pt.dres};
    for (double **q : dp) {
        CK(gmalloc(G, (void **)q, sizeof(double) * nd));
        CK(cudaMemset(*q, 0, sizeof(double) * nd));
    }
    float **fp[] = {&Pt.se[0], &Pt.se[1], &Pt.srhs, &Pt.sres};
    for (float **q : fp) {
        CK(gmalloc(G, (void **)q, sizeof(float) * nd));
        CK(cudaMemset(*q, 0, sizeof(float) * nd));
    }
    CK(gmalloc(G, (void **)&Pt.psiv32, sizeof(float) * g.cs));
    CK(cudaMemset(Pt.psiv32, 0, sizeof(float) * g.cs));
    CK(gmalloc(G, (void **)&Pt.psi_set, sizeof(double) * g.cs));
    CK(cudaMemset(Pt.psi_set, 0, sizeof(double) * g.cs));
    if (d == 3) {
        Pt.has_tm = true;
        for (int i = 0; i < 2; ++i)
            Pt.has_tm = Pt.has_tm && encode_sweep_maps(Pt.tm32[i], Pt.se[i], Pt.srhs, Pt.psiv32, g);
    }
    const int nk = (1 << d) * d;
    CK(gmalloc(G, (void **)&Pt.Ke64, sizeof(double) * nk * nk));
    CK(gmalloc(G, (void **)&Pt.Ke32, sizeof(float) * nk * nk));
    Level &F = G->L[G->nl - 1];
    if (!G->amr_u0) {
        const size_t nb = (size_t)F.g.dim * F.g.cs;
        CK(gmalloc(G, (void **)&G->amr_u0, sizeof(double) * nb));
        CK(cudaMemset(G->amr_u0, 0, sizeof(double) * nb));
        CK(gmalloc(G, (void **)&G->amr_r0, sizeof(double) * nb));
        CK(cudaMemset(G->amr_r0, 0, sizeof(double) * nb));
    }
    long long need = amr_blocks(F.g);
    for (int b = 1; b <= a; ++b) need += amr_blocks(G->P[b - 1].s);
    if (need > G->amr_npart) {
        if (G->amr_part) cudaFree(G->amr_part);
        G->amr_part = nullptr;
        G->amr_npart = 0;
        CK(gmalloc(G, (void **)&G->amr_part, sizeof(double) * need));
        G->amr_npart = need;
    }
    return SBM_OK;
}

// Checks of a new box at `level` (>= 1): even corners inside the level, at least two
// nodes thick, nested one parent cell inside exactly one patch of level-1 (the base
// for level 1) unless on the domain boundary, and apart from every patch of the same
// level (at least two parent cells between the boxes on some axis).  Returns the
// parent's patch index, or -1 with the grid's error set.
static int amr_check_box(sbm_grid G, int level, const sbm_box *box)
{
    const int d = G->desc.dim;
    for (int ax = 0; ax < 3; ++ax) {
        const int lo = box->lo[ax], hi = box->hi[ax], N = level_N(G, level, ax);
        if (ax >= d) {
            if (lo != 0 || hi != 0) return fail(G, SBM_ERR_ARG, "2D boxes have lo[2] = hi[2] = 0"), -1;
            continue;
        }
        if ((lo & 1) || (hi & 1) || lo < 0 || hi > N - 1 || hi - lo < 2)
            return fail(G, SBM_ERR_ARG, "box corners must be even, inside the level and at least 2 apart"), -1;
    }
    int parent = level == 1 ? 0 : -1;
    if (level > 1) {
        int found = 0;
        for (int q = 1; q <= G->npatch; ++q) {
            const Patch &Pp = G->P[q - 1];
            if (Pp.level != level - 1) continue;
            bool inside = true;
            for (int ax = 0; ax < d; ++ax) {
                const int lo = box->lo[ax], hi = box->hi[ax], N = level_N(G, level, ax), Np = level_N(G, level - 1, ax);
                const bool lo_ok = (lo == 0 && Pp.lo[ax] == 0) || lo >= 2 * Pp.lo[ax] + 2;
                const bool hi_ok = (hi == N - 1 && Pp.hi[ax] == Np - 1) || hi <= 2 * Pp.hi[ax] - 2;
                inside = inside && lo_ok && hi_ok;
            }
            if (inside) {
                parent = q;
                ++found;
            }
        }
        if (found != 1) return fail(G, SBM_ERR_ARG, "box must lie inside one patch of the next coarser level by one parent cell"), -1;
    }
    for (int q = 1; q <= G->npatch; ++q) {
        const Patch &Ps = G->P[q - 1];
        if (Ps.level != level) continue;
        bool apart = false;
        for (int ax = 0; ax < d; ++ax)
            apart = apart || box->lo[ax] >= Ps.hi[ax] + 4 || Ps.lo[ax] >= box->hi[ax] + 4;
        if (!apart) return fail(G, SBM_ERR_ARG, "boxes of one level must be at least two parent cells apart"), -1;
    }
    const AmrInfo &Lp = parent == 0 ? G->base_info : G->P[parent - 1].info;
    if (Lp.nchild >= kMaxChild) return fail(G, SBM_ERR_ARG, "at most 8 child patches per patch"), -1;
    return parent;
}

sbm_status sbm_amr_add_box(sbm_grid G, int level, const sbm_box *box, int *index)
{
    if (!G || !box) return fail(G, SBM_ERR_ARG, "null argument");
    if (G->npatch >= kMaxPatch) return fail(G, SBM_ERR_ARG, "at most 64 patches");
    int deepest = 0;
    for (int q = 1; q <= G->npatch; ++q) deepest = std::max(deepest, G->P[q - 1].level);
    if (level < 1 || level > deepest + 1) return fail(G, SBM_ERR_ARG, "level must be 1 .. (deepest level + 1)");
    CK(cudaSetDevice(G->dev));
    amr_refresh_infos(G);
    const int parent = amr_check_box(G, level, box);
    if (parent < 0) return SBM_ERR_ARG;
    const int a = G->npatch + 1, d = G->desc.dim;
    Patch &Pt = G->P[a - 1];
    Pt = Patch();
    for (int ax = 0; ax < 3; ++ax) {
        Pt.lo[ax] = box->lo[ax];
        Pt.hi[ax] = box->hi[ax];
    }
    Pt.level = level;
    Pt.parent = parent;
    Pt.h = G->desc.h / (double)(1 << level);
    Geom &g = Pt.s;
    g.dim = d;
    g.nx = Pt.hi[0] - Pt.lo[0] + 3;
    g.ny = Pt.hi[1] - Pt.lo[1] + 3;
    g.nz = d == 3 ? Pt.hi[2] - Pt.lo[2] + 3 : 1;
    g.sx = (g.nx + 7) / 8 * 8;
    g.sy = (long long)g.sx * g.ny;
    g.cs = (g.sy * g.nz + 63) / 64 * 64;
    g.dm[0] = g.dm[1] = g.dm[2] = 0;
    Pt.v = g;
    Pt.v.nx = g.nx - 2;
    Pt.v.ny = g.ny - 2;
    Pt.v.nz = d == 3 ? g.nz - 2 : 1;
    Pt.voff = 1 + g.sx + (d == 3 ? g.sy : 0);
    const sbm_status st = patch_alloc(G, a, Pt);
    if (st != SBM_OK) {
        // the patch is not added: free its storage and leave the grid as it was
        free_patch(Pt);
        Pt = Patch();
        return st;
    }
    G->npatch = a;
    amr_refresh_infos(G);
    G->amr_psi_dirty = true;
    ++G->version;               // captured cycles hold the old patch set
    if (index) *index = a;
    return SBM_OK;
}

// ------------------------------------------------------- regridding (host clustering)

namespace {

struct IBox {
    int lo[3], hi[3];
};

bool boxes_apart(const IBox &a, const IBox &b, int d)
{
    for (int ax = 0; ax < d; ++ax)
        if (a.lo[ax] >= b.hi[ax] + 4 || b.lo[ax] >= a.hi[ax] + 4) return true;
    return false;
}

IBox box_union(const IBox &a, const IBox &b, int d)
{
    IBox u{};
    for (int ax = 0; ax < d; ++ax) {
        u.lo[ax] = std::min(a.lo[ax], b.lo[ax]);
        u.hi[ax] = std::max(a.hi[ax], b.hi[ax]);
    }
    return u;
}

long long box_volume(const IBox &b, int d)
{
    long long v = 1;
    for (int ax = 0; ax < d; ++ax) v *= b.hi[ax] - b.lo[ax];
    return v;
}

// Boxes of one parent from its tags (storage cells n[0] x n[1] x n[2], x fastest,
// global cell = storage cell + org): dilation by `grow` cells (Chebyshev distance,
// separable), restriction to the allowed cells [cmin, cmax], connected components
// (face, edge or corner neighbours) numbered in the order of their first cell,
// bounding boxes in child nodes clipped to [amin, amax] (thinner than 2 dropped),
// merging of boxes closer than two parent cells and, beyond max_children, of the
// pair whose union adds the least volume; sorted by (lo, hi), x first.
std::vector<IBox> cluster_tags(std::vector<unsigned char> &tag, const int n[3], int d, const int org[3], int grow,
                               const int cmin[3], const int cmax[3], const int amin[3], const int amax[3],
                               int max_children)
{
    auto at = [&](int i, int j, int k) -> long long { return i + (long long)n[0] * (j + (long long)n[1] * k); };
    for (int ax = 0; ax < d && grow > 0; ++ax) {
        std::vector<unsigned char> out(tag.size(), 0);
        for (int k = 0; k < n[2]; ++k)
            for (int j = 0; j < n[1]; ++j)
                for (int i = 0; i < n[0]; ++i) {
                    const int l[3] = {i, j, k};
                    unsigned char v = 0;
                    for (int off = -grow; off <= grow && !v; ++off) {
                        int q[3] = {i, j, k};
                        q[ax] = l[ax] + off;
                        if (q[ax] < 0 || q[ax] >= n[ax]) continue;
                        v = tag[at(q[0], q[1], q[2])];
                    }
                    out[at(i, j, k)] = v;
                }
        tag.swap(out);
    }
    for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
            for (int i = 0; i < n[0]; ++i) {
                const int C[3] = {i + org[0], j + org[1], k + org[2]};
                for (int ax = 0; ax < d; ++ax)
                    if (C[ax] < cmin[ax] || C[ax] > cmax[ax]) tag[at(i, j, k)] = 0;
            }
    std::vector<IBox> boxes;
    std::vector<int> seen(tag.size(), 0);
    std::vector<long long> stack;
    for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
            for (int i = 0; i < n[0]; ++i) {
                if (!tag[at(i, j, k)] || seen[at(i, j, k)]) continue;
                int lo[3] = {i, j, k}, hi[3] = {i, j, k};
                stack.assign(1, at(i, j, k));
                seen[at(i, j, k)] = 1;
                while (!stack.empty()) {
                    const long long c = stack.back();
                    stack.pop_back();
                    const int ci = (int)(c % n[0]), cj = (int)((c / n[0]) % n[1]), ck = (int)(c / ((long long)n[0] * n[1]));
                    const int cc[3] = {ci, cj, ck};
                    for (int ax = 0; ax < 3; ++ax) {
                        lo[ax] = std::min(lo[ax], cc[ax]);
                        hi[ax] = std::max(hi[ax], cc[ax]);
                    }
                    for (int dz = (d == 3 ? -1 : 0); dz <= (d == 3 ? 1 : 0); ++dz)
                        for (int dy = -1; dy <= 1; ++dy)
                            for (int dx = -1; dx <= 1; ++dx) {
                                const int q[3] = {ci + dx, cj + dy, ck + dz};
                                if (q[0] < 0 || q[1] < 0 || q[2] < 0 || q[0] >= n[0] || q[1] >= n[1] || q[2] >= n[2])
                                    continue;
                                const long long e = at(q[0], q[1], q[2]);
                                if (tag[e] && !seen[e]) {
                                    seen[e] = 1;
                                    stack.push_back(e);
                                }
                            }
                }
                IBox b{};
                bool thick = true;
                for (int ax = 0; ax < d; ++ax) {
                    b.lo[ax] = std::max(2 * (lo[ax] + org[ax]), amin[ax]);
                    b.hi[ax] = std::min(2 * (hi[ax] + 1 + org[ax]), amax[ax]);
                    thick = thick && b.hi[ax] - b.lo[ax] >= 2;
                }
                if (thick) boxes.push_back(b);
            }
    for (bool changed = true; changed;) {
        changed = false;
        for (size_t a = 0; a < boxes.size() && !changed; ++a)
            for (size_t b = a + 1; b < boxes.size(); ++b)
                if (!boxes_apart(boxes[a], boxes[b], d)) {
                    boxes[a] = box_union(boxes[a], boxes[b], d);
                    boxes.erase(boxes.begin() + b);
                    changed = true;
                    break;
                }
        if (!changed && (int)boxes.size() > max_children) {
            long long best = 0;
            size_t bi = 0, bj = 1;
            bool have = false;
            for (size_t a = 0; a < boxes.size(); ++a)
                for (size_t b = a + 1; b < boxes.size(); ++b) {
                    const long long cost = box_volume(box_union(boxes[a], boxes[b], d), d) - box_volume(boxes[a], d) -
                                           box_volume(boxes[b], d);
                    if (!have || cost < best) {
                        best = cost;
                        bi = a;
                        bj = b;
                        have = true;
                    }
                }
            boxes[bi] = box_union(boxes[bi], boxes[bj], d);
            boxes.erase(boxes.begin() + bj);
            changed = true;
        }
    }
    std::sort(boxes.begin(), boxes.end(), [](const IBox &x, const IBox &y) {
        for (int ax = 0; ax < 3; ++ax)
            if (x.lo[ax] != y.lo[ax]) return x.lo[ax] < y.lo[ax];
        for (int ax = 0; ax < 3; ++ax)
            if (x.hi[ax] != y.hi[ax]) return x.hi[ax] < y.hi[ax];
        return false;
    });
    return boxes;
}

}  // namespace

sbm_status sbm_amr_regrid(sbm_grid G, int level, double threshold, int grow, int *nadded)
{
    if (!G) return fail(nullptr, SBM_ERR_ARG, "null grid");
    if (nadded) *nadded = 0;
    if (!G->has_psi) return fail(G, SBM_ERR_STATE, "psi not set (sbm_set_psi)");
    int deepest = 0;
    for (int q = 1; q <= G->npatch; ++q) deepest = std::max(deepest, G->P[q - 1].level);
    if (level != deepest + 1) return fail(G, SBM_ERR_ARG, "regridding builds the level below the deepest one");
    if (!(threshold >= 0.0) || !std::isfinite(threshold) || grow < 0 || grow > 64)
        return fail(G, SBM_ERR_ARG, "need threshold >= 0 and 0 <= grow <= 64");
    CK(cudaSetDevice(G->dev));
    amr_refresh_infos(G);
    const int d = G->desc.dim;
    std::vector<std::pair<int, IBox>> found;
    for (int p = 0; p <= G->npatch; ++p) {
        if ((p == 0 ? 0 : G->P[p - 1].level) != level - 1) continue;
        const Geom &s = amr_geom(G, p);
        const AmrInfo &L = amr_info(G, p);
        const double *psi = p == 0 ? G->L[G->nl - 1].psi64 : G->P[p - 1].psi64;
        int amin[3] = {0, 0, 0}, amax[3] = {0, 0, 0}, cmin[3] = {0, 0, 0}, cmax[3] = {0, 0, 0};
        for (int ax = 0; ax < d; ++ax) {
            const int Np = level_N(G, level - 1, ax), N = 2 * (Np - 1) + 1;
            if (p == 0) {
                amin[ax] = 0;
                amax[ax] = N - 1;
            } else {
                const Patch &Pp = G->P[p - 1];
                amin[ax] = Pp.lo[ax] == 0 ? 0 : 2 * Pp.lo[ax] + 2;
                amax[ax] = Pp.hi[ax] == Np - 1 ? N - 1 : 2 * Pp.hi[ax] - 2;
            }
            cmin[ax] = amin[ax] / 2;
            cmax[ax] = amax[ax] / 2 - 1;
        }
        const int n[3] = {s.nx - 1, s.ny - 1, d == 3 ? s.nz - 1 : 1};
        const size_t nt = (size_t)n[0] * n[1] * n[2];
        unsigned char *dtag = nullptr;
        CK(cudaMalloc(&dtag, nt));
        std::vector<unsigned char> tag(nt);
        cudaError_t e = launch_amr_tag(s, L, psi, threshold, cmin, cmax, dtag, G->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tag.data(), dtag, nt, cudaMemcpyDeviceToHost, G->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(G->st);
        cudaFree(dtag);
        if (e != cudaSuccess) return fail(G, SBM_ERR_CUDA, std::string("regrid tags: ") + cudaGetErrorString(e));
        const int org[3] = {L.org[0], L.org[1], L.org[2]};
        for (const IBox &b : cluster_tags(tag, n, d, org, grow, cmin, cmax, amin, amax, kMaxChild))
            found.push_back({p, b});
    }
    int added = 0;
    for (const auto &pb : found) {
        sbm_box box{};
        for (int ax = 0; ax < 3; ++ax) {
            box.lo[ax] = pb.second.lo[ax];
            box.hi[ax] = pb.second.hi[ax];
        }
        int idx = 0;
        sbm_status st = sbm_amr_add_box(G, level, &box, &idx);
        if (st != SBM_OK) return st;
        if (G->P[idx - 1].parent != pb.first) return fail(G, SBM_ERR_STATE, "regridded box found another parent");
        ++added;
        if (nadded) *nadded = added;
    }
    return SBM_OK;
}

sbm_status sbm_amr_remove_levels(sbm_grid G, int level)
{
    if (!G) return fail(nullptr, SBM_ERR_ARG, "null grid");
    if (level < 1) return fail(G, SBM_ERR_ARG, "level must be >= 1");
    CK(cudaSetDevice(G->dev));
    CK(cudaStreamSynchronize(G->st));
    int remap[kMaxPatch + 1];
    remap[0] = 0;
    int w = 0;
    for (int a = 1; a <= G->npatch; ++a) {
        if (G->P[a - 1].level >= level) {
            free_patch(G->P[a - 1]);
            G->P[a - 1] = Patch();
            remap[a] = -1;
        } else {
            remap[a] = ++w;
            if (w != a) {
                G->P[w - 1] = G->P[a - 1];
                G->P[a - 1] = Patch();
            }
        }
    }
    for (int a = 1; a <= w; ++a) G->P[a - 1].parent = remap[G->P[a - 1].parent];   // parents are kept
    G->npatch = w;
    // the adjoint vectors of the patches are sized per patch: reallocated on demand
    for (auto &vec : G->adj)
        for (int a = 1; a <= kMaxPatch; ++a)
            if (vec[a]) {
                cudaFree(vec[a]);
                vec[a] = nullptr;
            }
    // psi as set: the base level's from its raw input, each kept patch's from its copy
    // (the cells a removed child had replaced by coarse means get their own values back)
    if (G->has_psi) {
        Level &F = G->L[G->nl - 1];
        CK(cudaMemsetAsync(G->dbad, 0, sizeof(int), G->st));
        if (G->density) CK(launch_set_density(F.g, G->rho, G->psi_min, G->q, F.psi64, G->dbad, G->st));
        else CK(launch_set_psi(F.g, G->psi_raw, G->psi_min, F.psi64, G->dbad, G->st));
        sbm_status st = finish_psi(G);
        if (st != SBM_OK) return st;
    }
    for (int a = 1; a <= w; ++a) {
        Patch &Pt = G->P[a - 1];
        CK(cudaMemcpyAsync(Pt.psi64, Pt.psi_set, sizeof(double) * Pt.s.cs, cudaMemcpyDeviceToDevice, G->st));
    }
    CK(cudaStreamSynchronize(G->st));
    G->amr_psi_dirty = true;
    ++G->version;
    amr_refresh_infos(G);
    return SBM_OK;
}

sbm_status sbm_amr_get_box(sbm_grid G, int a, sbm_box *box, int *level, int *parent)
{
    if (!G) return fail(nullptr, SBM_ERR_ARG, "null grid");
    if (a < 1 || a > G->npatch) return fail(G, SBM_ERR_ARG, "patch index out of range");
    const Patch &Pt = G->P[a - 1];
    if (box)
        for (int ax = 0; ax < 3; ++ax) {
            box->lo[ax] = Pt.lo[ax];
            box->hi[ax] = Pt.hi[ax];
        }
    if (level) *level = Pt.level;
    if (parent) *parent = Pt.parent;
    return SBM_OK;
}

sbm_status sbm_amr_add_level(sbm_grid G, const sbm_box *box)
{
    if (!G) return fail(nullptr, SBM_ERR_ARG, "null grid");
    int deepest = 0;
    for (int q = 1; q <= G->npatch; ++q) deepest = std::max(deepest, G->P[q - 1].level);
    return sbm_amr_add_box(G, deepest + 1, box, nullptr);
}

sbm_status sbm_amr_set_psi(sbm_grid G, int a, const double *psi, double psi_min)
{
    if (!G) return fail(nullptr, SBM_ERR_ARG, "null grid");
    if (a < 1 || a > G->npatch) return fail(G, SBM_ERR_ARG, "patch index out of range");
    if (!is_dev_ptr(psi, G->dev)) return fail(G, SBM_ERR_ARG, "psi is not a device pointer of the grid's device");
    if (!(psi_min > 0.0)) return fail(G, SBM_ERR_ARG, "psi_min must be positive");
    CK(cudaSetDevice(G->dev));
    Patch &Pt = G->P[a - 1];
    CK(cudaMemsetAsync(G->dbad, 0, sizeof(int), G->st));
    CK(launch_amr_set_cells(Pt.s, psi, psi_min, Pt.psi64, G->dbad, G->st));
    CK(cudaMemcpyAsync(Pt.psi_set, Pt.psi64, sizeof(double) * Pt.s.cs, cudaMemcpyDeviceToDevice, G->st));
    int bad = 0;
    CK(cudaMemcpyAsync(&bad, G->dbad, sizeof(int), cudaMemcpyDeviceToHost, G->st));
    CK(cudaStreamSynchronize(G->st));
    if (bad) return fail(G, SBM_ERR_ARG, "psi contains non-finite values");
    G->amr_psi_dirty = true;
    return SBM_OK;
}

sbm_status sbm_amr_set_source(sbm_grid G, int a, const double *f)
{
    if (!G) return fail(nullptr, SBM_ERR_ARG, "null grid");
    if (a < 1 || a > G->npatch) return fail(G, SBM_ERR_ARG, "patch index out of range");
    if (!is_dev_ptr(f, G->dev)) return fail(G, SBM_ERR_ARG, "f is not a device pointer of the grid's device");
    CK(cudaSetDevice(G->dev));
    Patch &Pt = G->P[a - 1];
    CK(launch_pack<double, double>(Pt.s, Pt.s.dim, f, Pt.f64, G->st));
    CK(cudaStreamSynchronize(G->st));
    return SBM_OK;
}

sbm_status sbm_amr_solve(sbm_grid G, double *const *u, const sbm_opts *opts, sbm_info *info)
{
    sbm_status s = check_ready(G);
    if (s != SBM_OK) return s;
    if (!u) return fail(G, SBM_ERR_ARG, "null u");
    sbm_opts o;
    sbm_default_opts(&o);
    if (opts) o = *opts;
    if ((s = validate_opts(G, o)) != SBM_OK) return s;
    CK(cudaSetDevice(G->dev));
    if (G->npatch == 0) return sbm_solve(G, u[0], opts, info);
    if ((s = amr_prepare(G)) != SBM_OK) return s;
    if ((s = amr_pack_u(G, u)) != SBM_OK) return s;
    s = G->desc.precision == SBM_MIXED ? amr_run<float>(G, o, info) : amr_run<double>(G, o, info);
    if (s != SBM_OK && s != SBM_ERR_NOCONV && s != SBM_ERR_DIVERGED) return s;
    sbm_status s2 = amr_unpack(G, u[0], u, false);
    if (s2 != SBM_OK) return s2;
    CK(cudaStreamSynchronize(G->st));
    return s;
}

sbm_status sbm_amr_adjoint(sbm_grid G, double *const *u, double *const *dJdu, double *const *lambda,
                           double *const *dJdpsi, const sbm_opts *opts, sbm_info *info)
{
    sbm_status s = check_ready(G);
    if (s != SBM_OK) return s;
    if (!u || !dJdu || !lambda) return fail(G, SBM_ERR_ARG, "null argument");
    if (G->npatch == 0) return fail(G, SBM_ERR_STATE, "no patch levels: use sbm_adjoint");
    sbm_opts o;
    sbm_default_opts(&o);
    if (opts) o = *opts;
    if ((s = validate_opts(G, o)) != SBM_OK) return s;
    CK(cudaSetDevice(G->dev));
    for (int a = 0; a <= G->npatch; ++a) {
        if (!is_dev_ptr(dJdu[a], G->dev) || !is_dev_ptr(lambda[a], G->dev) || (dJdpsi && !is_dev_ptr(dJdpsi[a], G->dev)))
            return fail(G, SBM_ERR_ARG, "dJdu[a], lambda[a] and dJdpsi[a] must be device pointers");
    }
    if ((s = amr_prepare(G)) != SBM_OK) return s;
    if ((s = setup_bottom(G)) != SBM_OK) return s;
    if ((s = amr_alloc_adjoint(G)) != SBM_OK) return s;
    CK(amr_adjoint_scaling(G, o.omega));
    const int A = G->npatch;
    double *const *X = G->adj[0], *const *Gv = G->adj[1], *const *R = G->adj[2], *const *Zv = G->adj[3];
    const long long launches0 = g_launches;
    CK(cudaEventRecord(G->ev0, G->st));
    // right-hand side g = dJ/du on the owned free dofs
    for (int a = 0; a <= A; ++a) {
        CK(launch_pack<double, double>(amr_geom(G, a), amr_geom(G, a).dim, dJdu[a], Gv[a], G->st));
        CK(launch_amr_mask(amr_geom(G, a), amr_info(G, a), Gv[a], G->st));
    }
    CK(cv_zero(G, X));
    double hs[2];
    auto norm_of = [&](double *const *v, double *out) -> cudaError_t {
        cudaError_t e = cv_dot(G, v, v, 8);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hs, G->scal + 8, sizeof(double), cudaMemcpyDeviceToHost, G->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(G->st);
        *out = std::sqrt(hs[0]);
        return e;
    };
    double bnorm = 0.0;
    CK(norm_of(Gv, &bnorm));
    if (info) {
        info->r0 = bnorm;
        info->levels = G->nl + G->npatch;
        if (info->history && info->history_capacity > 0) info->history[0] = 1.0;
    }
    // lambda <- lambda + B^T (g - A^T lambda): the transposed correction iteration,
    // which converges at the rate of the forward one
    // On mixed-precision grids with inner_cycles k > 1, each outer iteration runs k
    // transposed cycles on the correction equation A^T d = r, their residual updates
    // with FP32 stencil products (amr_apply_T32), before lambda += d and the FP64
    // residual, as the forward solve runs k FP32 cycles per FP64 residual.
    double rel = bnorm > 0.0 ? 1.0 : 0.0;
    int it = 0, inner = 0;
    const int kin = (G->desc.precision == SBM_MIXED && o.inner_cycles > 1) ? o.inner_cycles : 1;
    sbm_status status = bnorm > 0.0 ? SBM_ERR_NOCONV : SBM_OK;
    CK(cv_lincomb(G, 1.0, Gv, 0.0, Gv, 0.0, nullptr, R));
    while (status == SBM_ERR_NOCONV && inner < o.max_cycles) {
        if (kin == 1) {
            CK(amr_precondT(G, o, R, Zv));
            CK(cv_lincomb(G, 1.0, X, 1.0, Zv, 0.0, nullptr, X));
            ++inner;
        } else {
            double *const *D = G->adj[4], *const *RI = G->adj[6], *const *Zi = G->adj[8];
            CK(cv_zero(G, D));
            CK(cv_lincomb(G, 1.0, R, 0.0, R, 0.0, nullptr, RI));
            for (int m = 0; m < kin && inner < o.max_cycles; ++m) {
                CK(amr_precondT(G, o, RI, Zi));
                CK(cv_lincomb(G, 1.0, D, 1.0, Zi, 0.0, nullptr, D));
                ++inner;
                if (m + 1 < kin && inner < o.max_cycles) {
                    CK(amr_apply_T32(G, D, Zv));
                    CK(cv_lincomb(G, 1.0, R, -1.0, Zv, 0.0, nullptr, RI));
                }
            }
            CK(cv_lincomb(G, 1.0, X, 1.0, D, 0.0, nullptr, X));
        }
        CK(amr_apply_T(G, X, Zv));
        CK(cv_lincomb(G, 1.0, Gv, -1.0, Zv, 0.0, nullptr, R));
        double rn = 0.0;
        CK(norm_of(R, &rn));
        ++it;
        rel = rn / bnorm;
        if (info && info->history && it < info->history_capacity) info->history[it] = rel;
        if (!std::isfinite(rel) || rel > 1e10) status = SBM_ERR_DIVERGED;
        else if (rel <= o.tol) status = SBM_OK;
    }
    double *const *T = G->adj[4];
    for (int a = 0; a <= A; ++a)
        CK(launch_unpack<double, double>(amr_geom(G, a), amr_geom(G, a).dim, X[a], lambda[a], G->st));
    if (dJdpsi) {
        // filled solution, per-level cell gradients, coarse-to-fine chain, floor mask
        if ((s = amr_pack_u(G, u)) != SBM_OK) return s;
        CK(amr_fill(G));
        for (int a = 0; a <= A; ++a) {
            const Coef<double> &c = a == 0 ? G->L[G->nl - 1].c64 : G->P[a - 1].c64;
            CK(launch_amr_dJdpsi(amr_geom(G, a), amr_info(G, a), c, a == 0 ? G->amr_u0 : G->P[a - 1].u64, X[a], T[a],
                                 G->st));
        }
        for (int c = 1; c <= A; ++c) {    // coarse to fine: a parent before its children
            const int pa = amr_parent(G, c);
            CK(launch_amr_grad_chain(amr_geom(G, c), amr_info(G, c), amr_geom(G, pa), amr_info(G, pa), T[pa], T[c],
                                     G->st));
        }
        for (int a = 0; a <= A; ++a)
            CK(launch_amr_get_cells(amr_geom(G, a), T[a], a == 0 ? G->L[G->nl - 1].psi64 : G->P[a - 1].psi64,
                                    G->psi_min, dJdpsi[a], G->st));
    }
    CK(cudaEventRecord(G->ev1, G->st));
    CK(cudaEventSynchronize(G->ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, G->ev0, G->ev1);
    if (info) {
        info->status = status;
        info->cycles = it;
        info->vcycles = inner;
        info->relres = rel;
        info->solve_ms = ms;
        info->launches = g_launches - launches0;
    }
    if (status == SBM_ERR_NOCONV) G->err = "max_cycles reached before the tolerance";
    if (status == SBM_ERR_DIVERGED) G->err = "relative residual not finite or above 1e10";
    return status;
}

sbm_status sbm_amr_residual(sbm_grid G, double *const *u, double *const *r, double *norm)
{
    sbm_status s = check_ready(G);
    if (s != SBM_OK) return s;
    if (!u || !r) return fail(G, SBM_ERR_ARG, "null argument");
    if (G->npatch == 0) return fail(G, SBM_ERR_STATE, "no patch levels: use sbm_residual");
    CK(cudaSetDevice(G->dev));
    if ((s = amr_prepare(G)) != SBM_OK) return s;
    if ((s = amr_pack_u(G, u)) != SBM_OK) return s;
    for (int a = 0; a <= G->npatch; ++a)
        if (!is_dev_ptr(r[a], G->dev)) return fail(G, SBM_ERR_ARG, "r[a] is not a device pointer");
    CK(amr_residual<double>(G, 5));
    if ((s = amr_unpack(G, r[0], r, true)) != SBM_OK) return s;
    CK(cudaMemcpyAsync(G->hscal + 5, G->scal + 5, 2 * sizeof(double), cudaMemcpyDeviceToHost, G->st));
    CK(cudaStreamSynchronize(G->st));
    if (norm) *norm = G->hscal[6];
    return SBM_OK;
}

}  // extern "C"
