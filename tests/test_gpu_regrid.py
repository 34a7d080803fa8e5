"""Regridding in the library (sbm_amr_regrid: tags on the device, clustering on the
host) against the oracle's restatement (oracle.regrid_boxes): the same boxes and
parents, integer for integer, for a step interface, separated and merged discs, a
field with more blobs than the child limit, two levels in 2D and two levels of a 3D
void field; then the regridded 3D hierarchy is solved and checked by the oracle's
composite residual."""
import numpy as np
import pytest

import oracle
import workloads as W
from _sbm import cuda, host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2212_02362_gb300 as sbm  # noqa: E402

PSI_MIN = 1e-6


@pytest.fixture(scope="module")
def built():
    from paper_2212_02362_gb300 import build
    build.build()
    oracle.build()
    return True


def _cells(dim, n, o, h, fn):
    """fn at the cell centres of a storage box with n nodes per axis, origin o."""
    ncz = n[2] - 1 if dim == 3 else 1
    k, j, i = np.meshgrid(np.arange(ncz), np.arange(n[1] - 1), np.arange(n[0] - 1), indexing="ij")
    X, Y = (i + o[0] + 0.5) * h, (j + o[1] + 0.5) * h
    Z = (k + o[2] + 0.5) * h if dim == 3 else np.zeros(X.shape)
    return np.ascontiguousarray(fn(X, Y, Z).reshape(-1), dtype=np.float64)


def _regrid_both(dim, n0, fn, levels, threshold=0.1, grow=2):
    n = (n0, n0, n0 if dim == 3 else 1)
    h0 = 1.0 / (n0 - 1)
    P = oracle.Problem(dim, n, h0, 1.0, 0.6, 0.5)
    g = sbm.Grid(dim, n, h0)
    g.set_moduli(sbm.SBM_CUBIC, (1.0, 0.6, 0.5))
    base = _cells(dim, n, (0, 0, 0), h0, fn)
    g.set_psi(cuda(base), PSI_MIN)
    A = oracle.Amr(P, [])
    psis = [np.maximum(base, PSI_MIN)]
    for L in range(1, levels + 1):
        ref = oracle.regrid_boxes(A, psis, L, threshold, grow)
        got = g.amr_regrid(L, threshold, grow)
        got_full = []
        for lo, hi, a in got:
            box = sbm._capi.sbm_box()
            lvl, par = sbm.C.c_int(), sbm.C.c_int()
            sbm.lib().sbm_amr_get_box(g._h, a, sbm.C.byref(box), sbm.C.byref(lvl), sbm.C.byref(par))
            assert lvl.value == L
            got_full.append((tuple(box.lo), tuple(box.hi), par.value))
        assert got_full == [(tuple(lo) + (0,) * (3 - len(lo)), tuple(hi) + (0,) * (3 - len(hi)), p)
                            for lo, hi, p in ref], (L, got_full, ref)
        A = oracle.Amr(P, list(A.boxes) + [(lo[:dim], hi[:dim], p) for lo, hi, p in ref])
        for a in range(len(psis), A.nlev):
            Pa = A.level_problem(a)
            v = _cells(dim, Pa.n, A.origin(a), Pa.h, fn)
            g.amr_set_psi(a, cuda(v), PSI_MIN)
            psis.append(np.maximum(v, PSI_MIN))
    return g, A, psis


def _disc(cx, cy, r, w):
    return lambda X, Y, Z: 0.5 * (1 + np.tanh((np.hypot(X - cx, Y - cy) - r) / w))


def test_step_interface(built):
    for grow, box in ((0, ((14, 0), (18, 32), 0)), (2, ((10, 0), (22, 32), 0))):
        g, A, _ = _regrid_both(2, 17, lambda X, Y, Z: (X > 0.5).astype(float), 1, grow=grow)
        assert A.boxes == [box]


def test_separated_and_merged_discs(built):
    h = 1.0 / 64
    f1, f2 = _disc(0.25, 0.3, 0.08, 2 * h), _disc(0.72, 0.7, 0.1, 2 * h)
    _, A, _ = _regrid_both(2, 65, lambda X, Y, Z: f1(X, Y, Z) * f2(X, Y, Z), 1)
    assert A.nlev == 3
    g1, g2 = _disc(0.4, 0.5, 0.08, 2 * h), _disc(0.62, 0.5, 0.08, 2 * h)
    _, A, _ = _regrid_both(2, 65, lambda X, Y, Z: g1(X, Y, Z) * g2(X, Y, Z), 1)
    assert A.nlev == 2


def test_child_limit(built):
    h = 1.0 / 128
    fs = [_disc(0.12 + 0.25 * i, 0.12 + 0.25 * j, 0.04, 2 * h) for i in range(4) for j in range(3)]
    _, A, _ = _regrid_both(2, 129, lambda X, Y, Z: np.prod([f(X, Y, Z) for f in fs], axis=0), 1)
    assert A.nlev == 9


def test_two_levels_2d(built):
    h0 = 1.0 / 32
    fs = [_disc(0.3, 0.3, 0.1, h0 / 2), _disc(0.72, 0.66, 0.12, h0 / 2)]
    _, A, _ = _regrid_both(2, 33, lambda X, Y, Z: np.prod([f(X, Y, Z) for f in fs], axis=0), 2)
    assert max(A.level(a) for a in range(A.nlev)) == 2


def test_two_levels_3d_and_solve(built):
    """Four spheres in a 33^3 base, two regridded levels, then a mixed-precision
    composite solve (triaxial affine loading) checked by the oracle's composite
    residual."""
    wk = W.voids_amr(3, 33, 2, count=4, rmin=0.08, rmax=0.12, clustered=True)
    g, A, psis = _regrid_both(3, 33, wk.psi_fn, 2)
    assert A.nlev >= 3
    # solve on the regridded hierarchy (the grid above is FP64; a mixed grid with the same boxes)
    gm = sbm.Grid(3, wk.n, wk.h, precision="mixed")
    gm.set_moduli(sbm.SBM_CUBIC, wk.moduli)
    for face, comp, _ in wk.bcs:
        gm.set_bc(face, comp, sbm.SBM_DIRICHLET_FROM_U)
    gm.set_psi(cuda(psis[0]), wk.psi_min)
    wk.boxes = [(tuple(lo), tuple(hi), p) for lo, hi, p in A.boxes]
    for a, b in enumerate(wk.boxes, start=1):
        assert gm.amr_add_box(wk.level(a), b[0], b[1]) == a
        gm.amr_set_psi(a, cuda(wk.level_psi(a)), wk.psi_min)
    us0 = [np.ascontiguousarray(wk.level_u0(a)) for a in range(A.nlev)]
    us = [cuda(u) for u in us0]
    info = gm.amr_solve(us, tol=1e-10, omega=wk.omega, max_cycles=300, inner_cycles=6)
    assert info.converged, info
    P = oracle.Problem(3, wk.n, wk.h, *wk.moduli, dirichlet=wk.dirichlet_bits())
    Ao = oracle.Amr(P, [(b[0], b[1], b[2]) for b in wk.boxes])
    ps = [np.ascontiguousarray(np.maximum(wk.level_psi(a), wk.psi_min)) for a in range(Ao.nlev)]
    oracle.amr_coarsen_psi(Ao, ps)
    fs = [np.zeros(Ao.level_problem(a).ndofs) for a in range(Ao.nlev)]
    r0 = oracle.amr_residual(Ao, ps, fs, [u.copy() for u in us0])
    r = oracle.amr_residual(Ao, ps, fs, [host(u).copy() for u in us])
    rel = np.sqrt(sum((x ** 2).sum() for x in r)) / np.sqrt(sum((x ** 2).sum() for x in r0))
    assert rel <= 2e-10, rel


def _grid2d(n0, fn, boxes_psi=None, bcs=True):
    n = (n0, n0, 1)
    h0 = 1.0 / (n0 - 1)
    g = sbm.Grid(2, n, h0)
    g.set_moduli(sbm.SBM_CUBIC, (1.0, 0.6, 0.5))
    if bcs:
        g.set_bc("-y", 0, sbm.SBM_DIRICHLET, 0.0)
        g.set_bc("-y", 1, sbm.SBM_DIRICHLET, 0.0)
        g.set_bc("+y", 0, sbm.SBM_DIRICHLET, 0.0)
        g.set_bc("+y", 1, sbm.SBM_DIRICHLET, 0.01)
    g.set_psi(cuda(_cells(2, n, (0, 0, 0), h0, fn)), PSI_MIN)
    return g


def _patch_psi(g, a, fn):
    lo, hi = g.patches[a - 1][0], g.patches[a - 1][1]
    lvl = g.patches[a - 1][2]
    h = g.h / 2 ** lvl
    n = (hi[0] - lo[0] + 3, hi[1] - lo[1] + 3, 1)
    return _cells(2, n, (lo[0] - 1, lo[1] - 1, 0), h, fn)


def _solve_all(g):
    us = [torch.zeros(2 * g.nnodes(), dtype=torch.float64, device="cuda")]
    for lo, hi, lvl, a in g.patches:
        us.append(torch.zeros(2 * (hi[0] - lo[0] + 3) * (hi[1] - lo[1] + 3), dtype=torch.float64, device="cuda"))
    info = g.amr_solve(us, tol=1e-12, max_cycles=400)
    assert info.converged
    return [host(u) for u in us]


def test_remove_levels_and_regrid(built):
    """Regrid two levels and solve; remove level 2: the solution equals that of a
    fresh grid holding the level-1 patches only; remove level 1 as well: it equals
    the single-grid solve; regrid again after the discs moved: the oracle's boxes of
    the new psi (the psi the removed patches had overwritten is restored)."""
    h0 = 1.0 / 64
    fs = [_disc(0.3, 0.3, 0.1, h0), _disc(0.7, 0.68, 0.12, h0)]
    fn = lambda X, Y, Z: np.prod([f(X, Y, Z) for f in fs], axis=0)
    g = _grid2d(65, fn)
    for L in (1, 2):
        for lo, hi, a in g.amr_regrid(L, 0.1, 2):
            g.amr_set_psi(a, cuda(_patch_psi(g, a, fn)), PSI_MIN)
    assert max(p[2] for p in g.patches) == 2
    _solve_all(g)
    g.amr_remove_levels(2)
    assert all(p[2] == 1 for p in g.patches) and len(g.patches) >= 2
    got = _solve_all(g)
    fresh = _grid2d(65, fn)
    for lo, hi, lvl, a in g.patches:
        assert fresh.amr_add_box(1, lo, hi) == a
        fresh.amr_set_psi(a, cuda(_patch_psi(fresh, a, fn)), PSI_MIN)
    ref = _solve_all(fresh)
    scale = max(np.abs(r).max() for r in ref)
    for x, y in zip(got, ref):
        assert np.abs(x - y).max() <= 1e-12 * scale
    g.amr_remove_levels(1)
    assert not g.patches
    u = torch.zeros(2 * g.nnodes(), dtype=torch.float64, device="cuda")
    g.solve(u, tol=1e-12, max_cycles=400)
    single = _grid2d(65, fn)
    u1 = torch.zeros_like(u)
    single.solve(u1, tol=1e-12, max_cycles=400)
    assert np.abs(host(u) - host(u1)).max() <= 1e-12 * np.abs(host(u1)).max()
    # the discs move: new base psi, regrid against the oracle
    ms = [_disc(0.45, 0.35, 0.1, h0), _disc(0.5, 0.75, 0.08, h0)]
    fm = lambda X, Y, Z: np.prod([f(X, Y, Z) for f in ms], axis=0)
    base = _cells(2, (65, 65, 1), (0, 0, 0), h0, fm)
    g.set_psi(cuda(base), PSI_MIN)
    got = g.amr_regrid(1, 0.1, 2)
    P = oracle.Problem(2, (65, 65, 1), h0, 1.0, 0.6, 0.5)
    ref = oracle.regrid_boxes(oracle.Amr(P, []), [np.maximum(base, PSI_MIN)], 1, 0.1, 2)
    assert [(tuple(lo), tuple(hi)) for lo, hi, _ in got] == [(tuple(lo), tuple(hi)) for lo, hi, _ in ref]
