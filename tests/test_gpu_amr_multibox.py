"""Several refinement patches per level on the GPU (sbm_amr_add_box): the
composite residual of a 3D hierarchy with two patches on level 1 and a child in
one of them against the oracle's composite residual; the clustered 2D and 3D void
hierarchies (tagging and clustering on the host, up to 23 patches) solved on the
GPU and checked by the oracle's composite residual; and the box rules (siblings
apart, one parent, at most 8 children) refused on the host side of the library.
The oracle records of the clustered workloads at full size are compared in
tests/test_gpu_full_size.py."""
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
from paper_2212_02362_gb300 import _capi  # noqa: E402


@pytest.fixture(scope="module")
def built():
    from paper_2212_02362_gb300 import build
    build.build()
    oracle.build()
    return True


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


def _nested3d(precision="fp64"):
    wk = W.voids_amr(3, 9, 2, count=2, rmin=0.1, rmax=0.2)
    wk.boxes = [((2, 2, 2), (8, 8, 8), 0), ((12, 2, 2), (16, 10, 16), 0), ((6, 6, 6), (12, 12, 12), 1)]
    wk.precision = precision
    return wk


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nested_multibox_composite_residual_parity(built, precision):
    wk = _nested3d(precision)
    g = _gpu(wk)
    A, psis = _oracle(wk)
    us = [np.ascontiguousarray(wk.level_u0(a) + W.uniform(170 + a, A.level_problem(a).ndofs, -1e-3, 1e-3))
          for a in range(A.nlev)]
    fs = [np.zeros(A.level_problem(a).ndofs) for a in range(A.nlev)]
    ref = oracle.amr_residual(A, psis, fs, [u.copy() for u in us])
    rs, nrm = g.amr_residual([cuda(u) for u in us])
    scale = max(np.abs(r).max() for r in ref)
    for a in range(A.nlev):
        assert np.abs(host(rs[a]) - ref[a]).max() <= 1e-12 * scale, a
    assert np.isclose(nrm, np.sqrt(sum((r ** 2).sum() for r in ref)), rtol=1e-12)


@pytest.mark.parametrize("dim,precision,inner", [(2, "fp64", 1), (3, "mixed", 6)])
def test_clustered_hierarchy_converges_with_oracle_residual(built, dim, precision, inner):
    """The clustered void hierarchies (2D: 129^2 base + 3 levels, 23 patches; 3D:
    65^3 base + 2 levels): the oracle's composite residual of the GPU solution is at
    the tolerance."""
    wk = (W.voids_amr(2, 129, 3, clustered=True) if dim == 2 else
          W.voids_amr(3, 65, 2, count=8, rmin=0.04, rmax=0.08, clustered=True))
    assert len(wk.boxes) > wk.level(len(wk.boxes))       # more patches than levels
    g = _gpu(wk, precision)
    A, psis = _oracle(wk)
    us0 = [np.ascontiguousarray(wk.level_u0(a)) for a in range(A.nlev)]
    us = [cuda(u) for u in us0]
    info = g.amr_solve(us, tol=1e-10, omega=wk.omega, smoother=wk.smoother, max_cycles=300, inner_cycles=inner)
    assert info.converged, info
    fs = [np.zeros(A.level_problem(a).ndofs) for a in range(A.nlev)]
    r0 = oracle.amr_residual(A, psis, fs, [u.copy() for u in us0])
    r = oracle.amr_residual(A, psis, fs, [host(u).copy() for u in us])
    rel = np.sqrt(sum((x ** 2).sum() for x in r)) / np.sqrt(sum((x ** 2).sum() for x in r0))
    assert rel <= 2e-10, (rel, info.cycles)


def test_box_rules(built):
    wk = W.voids_amr(2, 17, 1, count=2, rmin=0.1, rmax=0.2)
    g = sbm.Grid(2, wk.n, wk.h)
    g.set_moduli(sbm.SBM_CUBIC, wk.moduli)
    g.set_psi(cuda(wk.level_psi(0)), wk.psi_min)
    assert g.amr_add_box(1, (4, 4), (12, 12)) == 1
    for lvl, lo, hi in [(1, (14, 4), (20, 12)),          # 2 nodes from patch 1: closer than two parent cells
                        (2, (40, 40), (50, 50)),        # level 2 outside every level-1 patch
                        (3, (8, 8), (12, 12))]:         # skips level 2
        with pytest.raises(sbm.SBMError) as e:
            g.amr_add_box(lvl, lo, hi)
        assert e.value.status == _capi.SBM_ERR_ARG
    assert g.amr_add_box(1, (16, 4), (22, 12)) == 2      # 4 nodes apart: accepted
    assert g.amr_add_box(2, (36, 12), (40, 20)) == 3     # inside patch 2 (level-2 nodes 32..44)
    # eight children of the base at most
    g2 = sbm.Grid(2, (33, 33, 1), 1.0 / 32)
    g2.set_moduli(sbm.SBM_CUBIC, wk.moduli)
    k = 0
    for j in range(3):
        for i in range(3):
            lo, hi = (4 + 20 * i, 4 + 20 * j), (16 + 20 * i, 16 + 20 * j)
            if k < 8:
                assert g2.amr_add_box(1, lo, hi) == k + 1
            else:
                with pytest.raises(sbm.SBMError):
                    g2.amr_add_box(1, lo, hi)
            k += 1
