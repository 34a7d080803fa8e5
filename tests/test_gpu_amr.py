"""Block-structured refinement on the GPU against the oracle's composite problem.

Composite residual parity covers the injection, ghost fill (coarse-to-fine
interpolation), coarse psi under patches and the ownership masks; the composite
solve is compared with the oracle's dense composite solve on small hierarchies,
with the uniformly refined solve when a patch covers the whole domain, and, at
the 2D (129^2 base + 3 levels, colour Gauss-Seidel, FP64) and 3D (mixed
precision) test sizes, through the oracle's composite residual of the GPU result.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from _amr import dense_solve, dense_system
from _sbm import cuda, host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2212_02362_gb300 as sbm  # noqa: E402


@pytest.fixture(scope="module")
def built():
    from paper_2212_02362_gb300 import build
    build.build()
    oracle.build()
    return True


def _custom(dim, n0, boxes, precision="fp64", smoother="jacobi"):
    wk = W.voids_amr(dim, n0, len(boxes), count=2, rmin=0.1, rmax=0.2)
    wk.boxes = boxes
    wk.precision = precision
    wk.smoother = smoother
    return wk


def _gpu(wk, precision=None):
    g = sbm.Grid(wk.dim, wk.n, wk.h, precision=precision or wk.precision)
    g.set_moduli(sbm.SBM_CUBIC, wk.moduli)
    for face, comp, _ in wk.bcs:
        g.set_bc(face, comp, sbm.SBM_DIRICHLET_FROM_U)
    g.set_psi(cuda(wk.level_psi(0)), wk.psi_min)
    for a, b in enumerate(wk.boxes, start=1):
        assert g.amr_add_box(wk.level(a), b[0], b[1]) == a
    for a in range(1, len(wk.boxes) + 1):
        g.amr_set_psi(a, cuda(wk.level_psi(a)), wk.psi_min)
    return g


def _oracle(wk):
    P = oracle.Problem(wk.dim, wk.n, wk.h, *wk.moduli, dirichlet=wk.dirichlet_bits())
    A = oracle.Amr(P, [(b[0][:wk.dim], b[1][:wk.dim], wk.parent(a)) for a, b in enumerate(wk.boxes, start=1)])
    psis = [np.ascontiguousarray(np.maximum(wk.level_psi(a), wk.psi_min)) for a in range(A.nlev)]
    oracle.amr_coarsen_psi(A, psis)
    return A, psis


def _zeros_f(A):
    return [np.zeros(A.level_problem(a).ndofs) for a in range(A.nlev)]


SMALL = {
    "2d_two_patches": lambda: _custom(2, 9, [((4, 4, 0), (12, 12, 0)), ((10, 10, 0), (22, 22, 0))]),
    "2d_touching_boundary": lambda: _custom(2, 9, [((0, 4, 0), (12, 16, 0))]),
    "3d_one_patch": lambda: _custom(3, 5, [((2, 2, 2), (6, 6, 6))]),
    # several patches per level: (lo, hi, parent), siblings apart, children nested
    "2d_multibox": lambda: _custom(2, 9, [((2, 2, 0), (6, 6, 0), 0), ((10, 8, 0), (16, 16, 0), 0),
                                          ((6, 6, 0), (10, 10, 0), 1), ((22, 18, 0), (32, 32, 0), 2)]),
    "3d_two_slabs": lambda: _custom(3, 5, [((0, 0, 0), (2, 8, 8), 0), ((6, 2, 0), (8, 8, 6), 0)]),
}


@pytest.mark.parametrize("case", list(SMALL))
def test_composite_residual_parity(built, case):
    wk = SMALL[case]()
    g = _gpu(wk)
    A, psis = _oracle(wk)
    us = [np.ascontiguousarray(wk.level_u0(a) + W.uniform(70 + a, A.level_problem(a).ndofs, -1e-3, 1e-3))
          for a in range(A.nlev)]
    fs = _zeros_f(A)
    ref = oracle.amr_residual(A, psis, fs, [u.copy() for u in us])
    rs, nrm = g.amr_residual([cuda(u) for u in us])
    scale = max(np.abs(r).max() for r in ref)
    for a in range(A.nlev):
        assert np.abs(host(rs[a]) - ref[a]).max() <= 1e-12 * scale, a
    assert np.isclose(nrm, np.sqrt(sum((r ** 2).sum() for r in ref)), rtol=1e-12)


@pytest.mark.parametrize("case", list(SMALL))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_composite_solve_matches_dense_oracle(built, case, precision):
    wk = SMALL[case]()
    A, psis = _oracle(wk)
    us0 = [np.ascontiguousarray(wk.level_u0(a)) for a in range(A.nlev)]
    ref = dense_solve(A, psis, _zeros_f(A), us0)
    g = _gpu(wk, precision)
    us = [cuda(u) for u in us0]
    info = g.amr_solve(us, tol=1e-10, omega=wk.omega, smoother=wk.smoother)
    assert info.converged
    num = np.sqrt(sum(((host(us[a]) - ref[a]) ** 2).sum() for a in range(A.nlev)))
    den = np.sqrt(sum((ref[a] ** 2).sum() for a in range(A.nlev)))
    assert num <= 1e-8 * den, (num / den, info.cycles)


@pytest.mark.parametrize("case", list(SMALL))
@pytest.mark.parametrize("inner", [3, 8])
def test_composite_mixed_inner_cycles(built, case, inner):
    """Mixed precision with several FP32 correction cycles per FP64 residual (the
    FP32 right-hand side becomes r - A e in between): the dense oracle's solution,
    with fewer FP64 residuals than one cycle each and about as many cycles."""
    wk = SMALL[case]()
    A, psis = _oracle(wk)
    us0 = [np.ascontiguousarray(wk.level_u0(a)) for a in range(A.nlev)]
    ref = dense_solve(A, psis, _zeros_f(A), us0)
    g = _gpu(wk, "mixed")
    one = g.amr_solve([cuda(u) for u in us0], tol=1e-10, omega=wk.omega, smoother=wk.smoother)
    us = [cuda(u) for u in us0]
    info = g.amr_solve(us, tol=1e-10, omega=wk.omega, smoother=wk.smoother, inner_cycles=inner)
    assert info.converged
    num = np.sqrt(sum(((host(us[a]) - ref[a]) ** 2).sum() for a in range(A.nlev)))
    den = np.sqrt(sum((ref[a] ** 2).sum() for a in range(A.nlev)))
    assert num <= 1e-8 * den, (num / den, info.cycles, info.vcycles)
    assert info.vcycles == info.cycles * inner
    assert info.cycles < one.cycles, (info.cycles, one.cycles)
    assert info.vcycles <= one.vcycles + 2 * inner, (info.vcycles, one.vcycles)


def test_P10_patch_over_domain_equals_uniform_fine_gpu_solve(built):
    n0 = 17
    wk = _custom(2, n0, [((0, 0, 0), (32, 32, 0))])
    g = _gpu(wk)
    us = [cuda(wk.level_u0(a)) for a in range(2)]
    g.amr_solve(us, tol=1e-12)
    # the same fine problem as a single-level grid
    nf = 2 * (n0 - 1) + 1
    fine = W.Workload("fine", 2, (nf, nf, 1), wk.h / 2, wk.moduli, wk.bcs,
                      wk.level_psi(1).reshape(nf + 1, nf + 1)[1:-1, 1:-1].reshape(-1), wk.psi_min,
                      np.zeros(2 * nf * nf), W.initial_guess(2, (nf, nf, 1), wk.bcs))
    gf = sbm.Grid(2, fine.n, fine.h)
    gf.set_moduli(sbm.SBM_CUBIC, fine.moduli)
    for face, comp, v in fine.bcs:
        gf.set_bc(face, comp, sbm.SBM_DIRICHLET, float(v))
    gf.set_psi(cuda(fine.psi), fine.psi_min)
    uf = cuda(fine.u0)
    gf.solve(uf, tol=1e-12)
    patch = host(us[1]).reshape(2, nf + 2, nf + 2)[:, 1:-1, 1:-1].reshape(-1)
    assert np.linalg.norm(patch - host(uf)) <= 1e-9 * np.linalg.norm(host(uf))


@pytest.mark.parametrize("dim,n0,levels,precision,inner", [(2, 129, 3, "fp64", 1), (3, 33, 2, "mixed", 1),
                                                           (3, 33, 2, "mixed", 6)])
def test_full_hierarchy_converges_with_oracle_residual(built, dim, n0, levels, precision, inner):
    """The refinement recipes of the 2D (GS, FP64) and 3D (mixed) AMR workloads:
    the oracle's composite residual of the GPU solution is at the tolerance."""
    wk = W.voids_amr(dim, n0, levels) if dim == 2 else W.voids_amr(3, n0, levels, count=16, rmin=0.04, rmax=0.12)
    g = _gpu(wk, precision)
    A, psis = _oracle(wk)
    us0 = [np.ascontiguousarray(wk.level_u0(a)) for a in range(A.nlev)]
    us = [cuda(u) for u in us0]
    info = g.amr_solve(us, tol=1e-10, omega=wk.omega, smoother=wk.smoother, max_cycles=300, inner_cycles=inner)
    assert info.converged, info
    fs = _zeros_f(A)
    r0 = oracle.amr_residual(A, psis, fs, [u.copy() for u in us0])
    r = oracle.amr_residual(A, psis, fs, [host(u).copy() for u in us])
    n0_ = np.sqrt(sum((x ** 2).sum() for x in r0))
    n1_ = np.sqrt(sum((x ** 2).sum() for x in r))
    assert n1_ / n0_ <= 2e-10, (n1_ / n0_, info.cycles)


def _samples(wk, A, count, seed):
    """Random owned-or-not dofs of every level plus dofs next to each patch's
    coarse/fine interface (global level indices)."""
    rng = np.random.default_rng(seed)
    lev, nodes, comps = [], [], []
    for a in range(A.nlev):
        n = wk.storage_shape(a)
        o = wk.origin(a)
        pts = rng.integers(0, n, size=(count, 3))
        if a > 0:                        # rows on and next to the interface
            lo, hi = wk.boxes[a - 1][:2]
            face = pts.copy()
            ax = rng.integers(0, wk.dim, size=count)
            side = rng.integers(0, 2, size=count)
            off = rng.integers(-1, 3, size=count)
            for s_ in range(count):
                x = ax[s_]
                face[s_, x] = (lo[x] - o[x] + off[s_]) if side[s_] == 0 else (hi[x] - o[x] - off[s_])
            pts = np.concatenate([pts, np.clip(face, 0, np.array(n) - 1)])
        g = pts + np.array(o)
        lev += [a] * len(g)
        nodes.append(g)
        comps.append(rng.integers(0, wk.dim, size=len(g)))
    return np.array(lev), np.concatenate(nodes), np.concatenate(comps)


def _at(wk, arrs, lev, nodes, comps):
    out = np.empty(len(lev))
    for i, (a, g, p) in enumerate(zip(lev, nodes, comps)):
        n, o = wk.storage_shape(a), wk.origin(a)
        loc = (g[0] - o[0]) + n[0] * ((g[1] - o[1]) + n[1] * (g[2] - o[2]))
        out[i] = arrs[a][p * n[0] * n[1] * n[2] + loc]
    return out


def test_C5_full_size_sampled_parity(built):
    """3D refinement at full size (129^3 base + 2 levels around 16 spherical voids,
    triaxial loading, mixed precision): at sampled dofs of every level (random and
    next to the interfaces) the GPU composite residual of the initial guess equals
    the oracle's, and the oracle's composite residual of the GPU solution is at the
    tolerance relative to the initial residual."""
    wk = W.voids_amr(3, 129, 2, count=16, rmin=0.04, rmax=0.12)
    raw = [np.ascontiguousarray(wk.level_psi(a)) for a in range(3)]
    g = sbm.Grid(3, wk.n, wk.h, precision="mixed")
    g.set_moduli(sbm.SBM_CUBIC, wk.moduli)
    for face, comp, _ in wk.bcs:
        g.set_bc(face, comp, sbm.SBM_DIRICHLET_FROM_U)
    g.set_psi(cuda(raw[0]), wk.psi_min)
    for lo, hi, *_ in wk.boxes:
        g.amr_add_level(lo, hi)
    for a in (1, 2):
        g.amr_set_psi(a, cuda(raw[a]), wk.psi_min)
    P = oracle.Problem(3, wk.n, wk.h, *wk.moduli, dirichlet=wk.dirichlet_bits())
    A = oracle.Amr(P, [tuple(b[:2]) for b in wk.boxes])
    psis = [np.ascontiguousarray(np.maximum(r, wk.psi_min)) for r in raw]
    del raw
    oracle.amr_coarsen_psi(A, psis)
    fs = [np.zeros(A.level_problem(a).ndofs) for a in range(3)]
    us0 = [np.ascontiguousarray(wk.level_u0(a)) for a in range(3)]
    lev, nodes, comps = _samples(wk, A, 1500, 77)
    # residual of the initial guess
    rs, nrm0 = g.amr_residual([cuda(u) for u in us0])
    got = _at(wk, [host(r) for r in rs], lev, nodes, comps)
    del rs
    ref = oracle.amr_residual_at(A, psis, fs, us0, lev, nodes, comps)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    # solve, then the oracle's residual of the GPU solution
    us = [cuda(u) for u in us0]
    info = g.amr_solve(us, tol=1e-10, omega=wk.omega, smoother=wk.smoother, max_cycles=200)
    assert info.converged, info
    sol = [host(u) for u in us]
    r = oracle.amr_residual_at(A, psis, fs, sol, lev, nodes, comps)
    assert np.abs(r).max() <= 2e-10 * nrm0, (np.abs(r).max() / nrm0, info.cycles)


def _filled_dense_solution(A, psis, fs, us0):
    unk, M, b = dense_system(A, psis, fs, us0)
    x = np.linalg.solve(M, b)
    us = [u.copy() for u in us0]
    for (a, e), v in zip(unk, x):
        us[a][e] += v
    oracle.amr_fill(A, us)
    return unk, M, us


@pytest.mark.parametrize("case", list(SMALL))
@pytest.mark.parametrize("precision,inner", [("fp64", 1), ("mixed", 1), ("mixed", 6)])
@pytest.mark.parametrize("smoother", ["jacobi", "gs"])
def test_composite_adjoint_matches_dense_oracle(built, case, precision, inner, smoother):
    """lambda of A^T lambda = g and dJ/dpsi per level against the oracle's dense
    transpose solve and its composite gradient (floor cells masked); the
    transposed correction iteration converges like the forward one, also on grids
    whose smoother is colour Gauss-Seidel (Jacobi patch sweeps in B^T, the colour
    smoother in the base V-cycle), and with 6 inner transposed cycles per FP64
    A^T lambda whose residual updates take FP32 stencil products."""
    wk = SMALL[case]()
    A, psis = _oracle(wk)
    fs = [W.uniform(800 + a, A.level_problem(a).ndofs, -1, 1) for a in range(A.nlev)]
    us0 = [np.ascontiguousarray(wk.level_u0(a)) for a in range(A.nlev)]
    unk, M, us = _filled_dense_solution(A, psis, fs, us0)
    gs = [W.uniform(900 + a, A.level_problem(a).ndofs, -1, 1) for a in range(A.nlev)]
    gvec = np.array([gs[a][e] for a, e in unk])
    lam = np.linalg.solve(M.T, gvec)
    lams = [np.zeros_like(u) for u in us]
    for (a, e), v in zip(unk, lam):
        lams[a][e] = v
    ref = oracle.amr_dJdpsi(A, us, lams)
    g = _gpu(wk, precision)
    lg, gg, info = g.amr_adjoint([cuda(u) for u in us], [cuda(x) for x in gs], tol=1e-12, max_cycles=300,
                                 omega=wk.omega, smoother=smoother, inner_cycles=inner)
    assert info.converged, info
    assert info.vcycles <= 80, info.vcycles
    num = np.sqrt(sum(((host(lg[a]) - lams[a]) ** 2).sum() for a in range(A.nlev)))
    assert num <= 1e-9 * np.linalg.norm(lam), num / np.linalg.norm(lam)
    scale = max(np.abs(r).max() for r in ref)
    for a in range(A.nlev):
        mask = np.maximum(wk.level_psi(a), wk.psi_min) > wk.psi_min
        assert np.abs(host(gg[a]) - np.where(mask, ref[a], 0.0)).max() <= 1e-9 * scale, a


def test_C5_full_size_adjoint_directional_derivative(built):
    """3D refinement at full size: one adjoint solve for J = g.u, then the predicted
    change of J along a smooth psi perturbation of every level against central
    differences of two forward solves."""
    wk = W.voids_amr(3, 129, 2, count=16, rmin=0.04, rmax=0.12)
    raw = [np.ascontiguousarray(wk.level_psi(a)) for a in range(3)]
    g = sbm.Grid(3, wk.n, wk.h, precision="mixed")
    g.set_moduli(sbm.SBM_CUBIC, wk.moduli)
    for face, comp, _ in wk.bcs:
        g.set_bc(face, comp, sbm.SBM_DIRICHLET_FROM_U)
    g.set_psi(cuda(raw[0]), wk.psi_min)
    for lo, hi, *_ in wk.boxes:
        g.amr_add_level(lo, hi)
    for a in (1, 2):
        g.amr_set_psi(a, cuda(raw[a]), wk.psi_min)
    us0 = [cuda(wk.level_u0(a)) for a in range(3)]
    # J = g.u over the owned free dofs: the composite residual of a random field is
    # zero exactly off them
    rnd = [torch.from_numpy(W.uniform(1100 + a, u.numel(), -1, 1)).cuda() for a, u in enumerate(us0)]
    rs, _ = g.amr_residual(rnd)
    gs = [torch.from_numpy(W.uniform(1000 + a, u.numel(), -1, 1)).cuda() * (r != 0) for a, (u, r) in
          enumerate(zip(us0, rs))]
    del rnd, rs
    opts = dict(omega=wk.omega, smoother=wk.smoother, max_cycles=300)

    def J(psi_levels):
        g.set_psi(cuda(psi_levels[0]), wk.psi_min)
        for a in (1, 2):
            g.amr_set_psi(a, cuda(psi_levels[a]), wk.psi_min)
        us = [u.clone() for u in us0]
        g.amr_solve(us, tol=1e-12, **opts)
        tot = 0.0
        for a in range(3):
            tot += float((gs[a] * us[a]).sum())
        return tot, us

    J0, us = J(raw)
    lams, grads, info = g.amr_adjoint(us, gs, tol=1e-10, **opts)
    assert info.converged, info
    rng = np.random.default_rng(5)
    dpsi = []
    for a in range(3):
        X = np.arange(raw[a].size)
        d = 0.01 * raw[a] * np.sin(0.37 * X + rng.uniform(0, 6))
        d[np.maximum(raw[a], wk.psi_min) <= 1.5 * wk.psi_min] = 0.0
        dpsi.append(d)
    pred = sum(float((host(grads[a]) * dpsi[a]).sum()) for a in range(3))
    eps = 1e-3
    Jp, _ = J([r + eps * d for r, d in zip(raw, dpsi)])
    Jm, _ = J([r - eps * d for r, d in zip(raw, dpsi)])
    fd = (Jp - Jm) / (2 * eps)
    assert abs(fd - pred) <= 1e-4 * abs(pred), (fd, pred, info.cycles)

