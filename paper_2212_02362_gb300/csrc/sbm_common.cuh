// sbm_common.cuh — level geometry, kernel argument structs and launcher
// declarations shared by the translation units of libsbm.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "sbm_cell.cuh"

namespace sbm {

constexpr int kMaxLevels = 16;

// Internal layout of one level: node (i,j,k), component p at
//   p*cs + i + sx*(j + ny*k)
// with the x pitch sx a multiple of 8 elements (rows start 32-byte aligned for
// FP32, 64-byte for FP64).  Cells use the same indexing (cell (i,j,k) has lower
// corner node (i,j,k)); the last row/column/plane of the cell array is unused.
struct Geom {
    int dim;
    int nx, ny, nz;
    int sx;
    long long sy;          // plane stride (sx * ny for a full level)
    long long cs;          // component stride (>= sy * nz, multiple of 64)
    unsigned dm[3];        // Dirichlet face bits per component (faces 0..5)
};

// sy is the plane stride; it equals sx * ny for a full level, and is larger for a
// view of a sub-box of a padded patch (extents nx, ny, nz, strides of the storage).
__host__ __device__ __forceinline__ long long gidx(const Geom &g, int i, int j, int k)
{
    return (long long)i + (long long)g.sx * j + g.sy * k;
}

__host__ __device__ __forceinline__ bool is_dir(const Geom &g, int p, int i, int j, int k)
{
    const unsigned m = g.dm[p];
    return ((m & 1u) && i == 0) || ((m & 2u) && i == g.nx - 1) || ((m & 4u) && j == 0) ||
           ((m & 8u) && j == g.ny - 1) || ((m & 16u) && k == 0) || ((m & 32u) && k == g.nz - 1);
}

// Thread layout of the tiled 3D/2D sweeps: a block of 33 x BY threads, one cell
// column (cell row in 2D) each, the first row and column being the one-cell halo.
// Warps cover whole 32-cell rows and the last, partial warp the 33rd column, so the
// shared-memory accesses of a warp along a row are contiguous and free of bank
// conflicts (a warp spanning the end of one row and the start of the next would hit
// the same banks twice).
template <int BY>
__device__ __forceinline__ void row_warp_xy(int tid, int &tx, int &ty)
{
    if (tid < 32 * BY) {
        tx = tid & 31;
        ty = tid >> 5;
    } else {
        tx = 32;
        ty = tid - 32 * BY;
    }
}

// Programmatic dependent launch: the kernels of the V-cycle path are launched
// with the programmatic-serialisation attribute, so a launch is processed while
// its predecessor drains; each of them first waits for its predecessor to
// complete (griddepcontrol.wait: memory visible) and then lets its own successor
// be scheduled.  Launched without the attribute, both are no-ops.
__device__ __forceinline__ void pdl_begin()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

enum SweepMode { kApply = 0, kResidual = 1, kJacobi = 2 };

template <typename T, typename TO>
struct SweepArgs {
    Geom g;
    const T *u;            // input displacement (level layout)
    const T *f;            // right-hand side (residual / Jacobi)
    const T *psi;          // cells
    TO *out;               // Ku, r, or the smoothed u (must not alias u for Jacobi)
    double *part;          // per-block partial sums of r^2 (residual), may be null
    Coef<T> c;
    T wk[3];               // Jacobi: omega / kdiag[p]
    int kchunk;            // node planes per block along z (3D)
    const int *gate = nullptr;   // device flag: when set, the launch does nothing
};

// Number of z chunks for a z-streaming stencil launch: minimises
// waves x (layers per block), where a wave is `slots` resident blocks (the
// kernel's blocks per SM x 152 SMs), a block streams ceil(nzc/nc) layers plus one
// halo layer, and `pair` counts layers two at a time (the packed FP32 kernel).
inline int choose_chunks(long long xy, int nzc, int slots, bool pair)
{
    int best = 1;
    long long best_cost = -1;
    for (int nc = 1; nc <= nzc; ++nc) {
        const int ch = (nzc + nc - 1) / nc;
        const int nblk_z = (nzc + ch - 1) / ch;
        if (nblk_z != nc) continue;                       // same chunking as a smaller nc
        const long long waves = (xy * nc + slots - 1) / slots;
        const long long layers = ch + (nc > 1 ? 1 : 0);
        const long long cost = waves * (pair ? (layers + 1) / 2 : layers);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = nc;
        }
    }
    return best;
}

// ---- launchers (defined in k_stencil.cu / k_misc.cu) ----------------------

// Number of kernels the launchers have enqueued from the calling host thread
// (graph capture included).  Entry points report the difference over a call, so
// the counter is per thread: handles used from different threads do not mix.
extern thread_local long long g_launches;

// Raise a kernel's dynamic shared-memory limit on the current device.  The
// attribute belongs to the device context, so it is set once per device (bit
// `dev` of `done`); setting it twice from racing threads is harmless.
inline cudaError_t smem_attr_once(const void *kernel, size_t bytes, std::atomic<unsigned long long> &done)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
    return e;
}

// True when p is device (or managed) memory of device dev (sbm_api.cu).
bool is_dev_ptr(const void *p, int dev);

// Axis-aligned cubic moduli (C11, C12, C44) give a positive-definite stiffness:
// finite, C44 > 0, C11 > |C12|, and in 3D C11 + 2 C12 > 0 (the bulk mode).
inline bool moduli_definite(int dim, double c11, double c12, double c44)
{
    const bool fin = c11 - c11 == 0.0 && c12 - c12 == 0.0 && c44 - c44 == 0.0;   // finite (no NaN / Inf)
    if (!fin || !(c44 > 0.0) || !(c11 > (c12 < 0 ? -c12 : c12))) return false;
    return dim != 3 || c11 + 2.0 * c12 > 0.0;
}

// Message returned by sbm_last_error(NULL) (defined in sbm_api.cu).
void set_library_error(const char *msg);

// Tile shape of the stencil kernels (cells per block along x and y).
void sweep_grid(const Geom &g, int *grid, int *kchunk);   // grid[3] of the generic kernel
// Blocks (= partial sums written) of launch_sweep in FP64 (fp64) or FP32.
long long sweep_blocks(const Geom &g, bool fp64);

template <typename T, typename TO>
cudaError_t launch_sweep(int mode, const SweepArgs<T, TO> &a, cudaStream_t s);

// FP32 3D sweep with TMA plane staging and packed FP32x2 arithmetic, one
// persistent CTA per SM (k_stencil_tma.cu).  tmap: three CUtensorMaps of the
// storage that a.g's grid sits in at offset org (>= 0; zero for a whole level):
// u and f as 4D (x, y, z, component) maps, psi as a 3D cell map, with the box
// shapes tma_box_shapes gives ({x, y} extents; z 1, components 3).  psi must be 0
// on the cells of that storage outside a.g's grid (beyond the storage the tensor
// maps read zeros).  a.out is written at a.g's nodes.  err: device flag set when
// an mbarrier wait times out.
cudaError_t launch_sweep_f2(int mode, const SweepArgs<float, float> &a, const void *tmap, int *err,
                            cudaStream_t s, int3 org = make_int3(0, 0, 0));
// Partial sums (= CTAs) of one launch of launch_sweep_f2 on the current device.
long long sweep_blocks_f2(const Geom &g);
// Box extents {x, y} of the u, f and psi tensor maps of launch_sweep_f2.
void tma_box_shapes(int u[2], int f[2], int c[2]);

template <typename T>
cudaError_t launch_gs(const Geom &g, const T *psi, const T *Ke, const T *f, T *u, int colour,
                      cudaStream_t s, const int *gate = nullptr);

// One 2D colour Gauss-Seidel sweep (all four colours, ascending or descending) in one
// launch, reading uin and writing every node of the grid to uout (uout != uin).
template <typename T>
cudaError_t launch_gs2_sweep(const Geom &g, const T *psi, const T *Ke, const T *f, const T *uin, T *uout,
                             int descending, cudaStream_t s, const int *gate = nullptr);

template <typename T>
cudaError_t launch_restrict(const Geom &gf, const Geom &gc, const T *rf, T *fc, cudaStream_t s,
                            const int *gate = nullptr, T *zero_uc = nullptr);

template <typename T>
cudaError_t launch_prolong_add(const Geom &gf, const Geom &gc, const T *ec, T *uf, cudaStream_t s,
                               const int *gate = nullptr);

cudaError_t launch_coarsen_psi(const Geom &gf, const Geom &gc, const double *pf, double *pc,
                               cudaStream_t s);

// packed (user) <-> level layout copies, with conversion
template <typename TS, typename TD>
cudaError_t launch_pack(const Geom &g, int ncomp, const TS *packed, TD *lev, cudaStream_t s);
template <typename TS, typename TD>
cudaError_t launch_unpack(const Geom &g, int ncomp, const TS *lev, TD *packed, cudaStream_t s);
// cells: packed (nx-1)(ny-1)(nz-1) <-> level layout; floor with psi_min, count non-finite
cudaError_t launch_set_psi(const Geom &g, const double *packed, double psi_min, double *lev,
                           int *bad, cudaStream_t s);
cudaError_t launch_set_density(const Geom &g, const double *rho, double psi_min, double q,
                               double *lev, int *bad, cudaStream_t s);
cudaError_t launch_get_cells(const Geom &g, const double *lev, double *packed, cudaStream_t s);
cudaError_t launch_round_cells(const Geom &g, const double *src, float *dst, cudaStream_t s);
// write a face value into Dirichlet dofs of one component
cudaError_t launch_set_face(const Geom &g, int face, int comp, double value, double *u,
                            cudaStream_t s);
// u64 += e (FP32 or FP64) over n elements
template <typename TE>
cudaError_t launch_add(long long n, const TE *e, double *u, cudaStream_t s);
// deterministic final reduction of block partials: out[0] = sum, optional relres
cudaError_t launch_norm_final(const double *part, int nparts, double *scal, int which,
                              cudaStream_t s, const int *gate = nullptr);
// Batched FP64 V-cycles (see k_misc.cu): state = {done, count}, hist[count] = relres.
cudaError_t launch_outer_gate(const double *scal, double tol, int max_cycles, double *hist, int *state, cudaStream_t s);
// dst <- src unless *gate (gate may be null).
cudaError_t launch_copy_gated(long long n, const double *src, double *dst, const int *gate, cudaStream_t s);
// bottom: dense assembly, Dirichlet rows/cols, Gauss-Jordan inverse, matvec
cudaError_t launch_bottom_assemble(const Geom &g, const double *psi, const Coef<double> &c,
                                   double *A, cudaStream_t s);
cudaError_t launch_bottom_dirichlet(const Geom &g, double *A, cudaStream_t s);
// FP32 3D sweep, eight threads (one per cell) per node (small levels; no partial sums).
cudaError_t launch_sweep_node(int mode, const SweepArgs<float, float> &a, cudaStream_t s);
// Levels with at most this many nodes use the cell-parallel per-node FP32 kernel.
constexpr long long kNodeKernelMaxNodes = 20000;

// Inverse of the coarsest-level matrix in place (one cooperative launch);
// bar: 4 device words, bar[2] != 0 afterwards if a grid barrier timed out.
// spins: polls a block makes at one grid barrier before giving up (<= 0: default).
cudaError_t launch_gauss_jordan(const Geom &g, int n, double *A, double *tmp, unsigned *bar, long long spins,
                                cudaStream_t s);
cudaError_t launch_round(long long n, const double *src, float *dst, cudaStream_t s);
template <typename T>
cudaError_t launch_bottom_apply(int n, const T *Ainv, const int *gather, const T *b, T *u,
                                int accumulate, cudaStream_t s, const int *gate = nullptr);
// Adaptive inner cycles: sum the partial sums of the FP32 residual of this V-cycle
// and set *gate when its norm <= max(rtol * scal[7], tol_frac * scal[1]) (scal[7]:
// the latest FP64 residual norm, scal[1]: the initial one); counts the V-cycles
// run in *count.  Skipped itself once the gate is set.
cudaError_t launch_inner_gate(const double *part, int nparts, const double *scal, double rtol, double tol_frac,
                              int *gate, int *count, cudaStream_t s);
// dJ/dpsi_c = -lambda_c^T S_c u_c (packed u, lambda; packed cell output) and the
// optional chain rule through the SIMP map or the psi_min floor.
cudaError_t launch_dJdpsi(const Geom &g, const Coef<double> &c, const double *u, const double *lam,
                          double *g_out, double *grho_out, const double *rho, const double *psi_raw,
                          double psi_min, double q, int density, cudaStream_t s);

// ---- block-structured refinement (k_amr.cu) ---------------------------------

// Roles of the nodes of one refinement level (see k_amr.cu).
constexpr int kMaxChild = 8;                      // child patches of one patch (or of the base)
constexpr int kMaxPatch = 64;                     // refinement patches of a grid
struct AmrInfo {
    int dim;
    int N[3];              // global nodes per axis at this level
    int lo[3], hi[3];      // the patch box (level indices); unused on the base level
    int org[3];            // global index of storage node (0, 0, 0)
    int is_base;
    int nchild;            // child patches (boxes disjoint and apart)
    int clo[kMaxChild][3], chi[kMaxChild][3];   // their boxes (child-level indices)
    unsigned dm[3];        // Dirichlet faces of the domain, per component
};

cudaError_t launch_lincomb(long long n, double a, const double *x, double b, const double *y, double c,
                           const double *z, double *out, cudaStream_t s);
cudaError_t launch_sum_parts(const double *part, int n, double *out, cudaStream_t s);
// Product-rule strong form of Sec. 2.3 (k_variant.cu), FP64 packed arrays: mode 0
// out = K u; mode 1 one damped Jacobi sweep from u into out.  variant 1: psi at
// nodes, 2: psi in cells.
cudaError_t launch_product(int mode, int dim, const int n[3], double h, const double mod[3], const unsigned dm[3],
                           int variant, double omega, const double *psi, const double *u, const double *f, double *out,
                           cudaStream_t s);
// Source terms of eq. SBMLinearElasticity (k_source.cu), FP64 packed arrays: the
// load f of K u = f from a per-cell eigenstrain (Voigt, may be null), a nodal body
// force b and a nodal diffuse traction t (either may be null).  sig: scratch for the
// cell stresses (d(d+1)/2 doubles per cell), needed when eps0 is given.
cudaError_t launch_source_terms(int dim, const int n[3], double h, const double mod[3], const double *psi,
                                const double *eps0, const double *b, const double *t, double *f, double *sig,
                                cudaStream_t s);
// Phase-field topology optimisation step (k_topopt.cu): node counts, the
// coefficients of eq. topop_evolution and the grid factors.
struct TopoptArgs {
    int nx, ny, nz;
    double alpha, beta, zeta;
    double lam, V0;        // lambda(t) of this step and the target volume
    double dtL;            // dt * mobility
    double hd, ih2;        // h^d and 1 / h^2
    long long psx, psy;    // strides of psi_solve (the level layout: cell (i,j,k) at i + psx j + psy k)
};
int topopt_blocks(long long ncells);
// eta_out = one explicit step from eta (cells, packed) at the equilibrium u (nodes,
// packed); psi_next (may be null) = (eta_out + zeta)^2; part[0..B) = per-block sums of
// eta_out, part[B..2B) of psi_solve_c e_c (B = topopt_blocks(cells); psi_solve may be
// null); eta_sum: device scalar, the sum of eta over the cells.
cudaError_t launch_topopt_step(int dim, const TopoptArgs &A, const Coef<double> &c, const double *eta,
                               const double *u, const double *psi_solve, const double *eta_sum, double *eta_out,
                               double *psi_next, double *part, cudaStream_t s);
// part[0..B) = per-block sums of x[0..n); psi (may be null) = (x + zeta)^2.
cudaError_t launch_cell_sum(long long n, const double *x, double zeta, double *psi, double *part, cudaStream_t s);
// FMA throughput probe (measurement): blocks x threads threads, 8 chains of `iters`
// multiply-adds each (16 iters flops per thread), FP64 or FP32.
cudaError_t launch_fma_rate(int fp64, int blocks, int threads, int iters, void *sink, cudaStream_t s);
// Reads a buffer (measurement: leaves L2 holding clean lines of it).
cudaError_t launch_l2_read(const void *buf, size_t bytes, float *sink, cudaStream_t s);
// adjoint of the composite problem
cudaError_t launch_amr_ghostT(const Geom &sc, const AmrInfo &Lc, const Geom &sp, const AmrInfo &Lp, const double *wc,
                              double *wp, int with_solved, cudaStream_t st);
cudaError_t launch_amr_mask_solved(const Geom &s, const AmrInfo &L, double *x, cudaStream_t st);
// regridding: tags of h |grad psi| > thr on the storage cells whose global index is
// in [cmin, cmax] (packed over the storage cells)
cudaError_t launch_amr_tag(const Geom &s, const AmrInfo &L, const double *psi, double thr, const int cmin[3],
                           const int cmax[3], unsigned char *tags, cudaStream_t st);
cudaError_t launch_amr_scaleW(const Geom &s, const AmrInfo &L, const double *psi, double omega, const double kdiag[3],
                              const double *x, double *out, cudaStream_t st);
// t = W eb, rb += t (n elements; t rounded to TS): the scaling half of a transposed
// damped-Jacobi sweep, W from launch_amr_scaleW with x = null.
template <typename TS>
cudaError_t launch_amr_jacT_scale(long long n, const double *W, const double *eb, double *rb, TS *t, cudaStream_t st);
// eb += alpha y on the nodes of view v (storage strides; the view at element offset voff).
template <typename TS>
cudaError_t launch_axpy_view(const Geom &v, long long voff, double alpha, const TS *y, double *eb, cudaStream_t st);
cudaError_t launch_amr_restrictT(const Geom &sc, const AmrInfo &Lc, const Geom &sp, const AmrInfo &Lp,
                                 const double *rp, double *rc, cudaStream_t st);
cudaError_t launch_amr_injectT(const Geom &sc, const AmrInfo &Lc, const Geom &sp, const AmrInfo &Lp, const double *wp,
                               double *wc, cudaStream_t st);
cudaError_t launch_amr_dot(const Geom &s, const AmrInfo &L, const double *x, const double *y, double *part,
                           cudaStream_t st);
cudaError_t launch_amr_dJdpsi(const Geom &s, const AmrInfo &L, const Coef<double> &c, const double *u,
                              const double *lam, double *g, cudaStream_t st);
cudaError_t launch_amr_grad_chain(const Geom &sc, const AmrInfo &Lc, const Geom &sp, const AmrInfo &Lp, double *gp,
                                  double *gc, cudaStream_t st);
cudaError_t launch_amr_get_cells(const Geom &s, const double *lev, const double *psi, double psi_min, double *packed,
                                 cudaStream_t st);
long long amr_blocks(const Geom &s);
bool amr_owned_host(const AmrInfo &L, int i, int j, int k);
cudaError_t launch_amr_mask(const Geom &s, const AmrInfo &L, double *r, cudaStream_t st);
template <typename T>
cudaError_t launch_amr_inject(const Geom &sc, const AmrInfo &Lc, const Geom &sp, const AmrInfo &Lp, const T *uc, T *up,
                              cudaStream_t st);
// psi of a patch view's cells, 0 on the storage's padding cells (for the TMA sweep).
cudaError_t launch_amr_view_cells(const Geom &s, const float *src, float *dst, cudaStream_t st);
// out <- r on owned free rows, 0 elsewhere (every storage node of the level).
template <typename T>
cudaError_t launch_amr_mask_to(const Geom &s, const AmrInfo &L, const T *r, T *out, cudaStream_t st);
template <typename T>
cudaError_t launch_amr_ghost(const Geom &sc, const AmrInfo &Lc, const Geom &sp, const AmrInfo &Lp, T *uc, const T *up,
                             int mode, cudaStream_t st);
template <typename T>
cudaError_t launch_amr_restrict(const Geom &sc, const AmrInfo &Lc, const Geom &sp, const AmrInfo &Lp, const T *rc,
                                T *rhsp, cudaStream_t st);
template <typename T>
cudaError_t launch_amr_update(const Geom &s, const AmrInfo &L, const T *e, double *u, cudaStream_t st);
template <typename TO>
cudaError_t launch_amr_sumsq_round(const Geom &s, const AmrInfo &L, const double *r, TO *out, double *part,
                                   cudaStream_t st);
cudaError_t launch_amr_coarsen_psi(const Geom &sc, const AmrInfo &Lc, const Geom &sp, const AmrInfo &Lp,
                                   const double *psic, double *psip, cudaStream_t st);
// padded-box cells: packed user layout <-> node-indexed storage (floor psi_min)
cudaError_t launch_amr_set_cells(const Geom &s, const double *packed, double psi_min, double *lev, int *bad,
                                 cudaStream_t st);

}  // namespace sbm
