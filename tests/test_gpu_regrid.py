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
