"""The source terms of eq. SBMLinearElasticity (Sec. 2.1) on the GPU
(sbm_source_terms) against the oracle's restatement, and the solver validated as
Sec. 3.1 does, against closed-form solutions for a plate with a hole:

  - Kirsch: a traction-free hole under uniaxial tension; the stresses along the
    line y = R tangent to the hole converge to the exact ones as the interface
    width eps decreases (the paper's L2 error against eps);
  - Lame: a pressurised hole, the pressure entering only through the diffuse
    traction source t |grad psi| (Theorem 1); the displacement converges as eps
    decreases;
  - the 3D analogue, a pressurised spherical cavity, through the 3D path.

The plates are quarter (octant) models with symmetry planes through the hole's
centre and the exact displacement on the outer faces, so the discrete problem
approximates the infinite-plate solution without finite-size error.
"""
import ctypes as C

import numpy as np
import pytest

import _exact as X
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


def _grid(dim, n, h, moduli=(1.0, 0.6, 0.5), kind=None, precision="fp64"):
    g = sbm.Grid(dim, n, h, precision=precision)
    g.set_moduli(sbm.SBM_CUBIC if kind is None else kind, moduli)
    return g


def _inputs(P, seed, psi_lo=0.0):
    nv = 3 if P.dim == 2 else 6
    psi = W.uniform(seed, P.ncells, psi_lo, 1.0)
    eps0 = W.uniform(seed + 1, nv * P.ncells, -0.01, 0.01)
    b = W.uniform(seed + 2, P.ndofs, -1.0, 1.0)
    t = W.uniform(seed + 3, P.ndofs, -1.0, 1.0)
    return psi, eps0, b, t


@pytest.mark.parametrize("dim,n", [(2, (37, 29, 1)), (3, (17, 13, 11)), (3, (21, 6, 9))])
def test_source_terms_parity(built, dim, n):
    h = 1.0 / (n[0] - 1)
    moduli = (1.0, 0.6, 0.5)
    P = oracle.Problem(dim, n, h, *moduli)
    g = _grid(dim, n, h, moduli)
    psi, eps0, b, t = _inputs(P, 900 + dim)
    for kw in ({"eps0": eps0, "b": b, "t": t}, {"eps0": eps0}, {"b": b}, {"t": t}, {}):
        ref = oracle.source_terms(P, psi, **kw)
        got = host(g.source_terms(cuda(psi), **{k: cuda(v) for k, v in kw.items()}))
        scale = max(np.abs(ref).max(), 1e-300)
        assert np.abs(got - ref).max() <= 1e-13 * scale, sorted(kw)
        if not kw:
            assert not got.any()


def test_source_terms_parity_129_cubed(built):
    """The 129^3 grid of the damage workload (6.4 M dofs), its psi, a random
    eigenstrain, body force and traction: every entry against the oracle."""
    wk = W.damage3d(129)
    P = oracle.Problem(3, wk.n, wk.h, *wk.moduli)
    g = _grid(3, wk.n, wk.h, wk.moduli)
    _, eps0, b, t = _inputs(P, 930)
    ref = oracle.source_terms(P, wk.psi, eps0=eps0, b=b, t=t)
    got = host(g.source_terms(cuda(wk.psi), eps0=cuda(eps0), b=cuda(b), t=cuda(t)))
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_source_terms_on_a_coarse_level_and_stress_free_affine_field(built):
    """On level 0 of a 3-level hierarchy: a uniform eigenstrain is balanced exactly
    by the affine displacement with that strain, K u = f (through the library's own
    operator apply)."""
    n = (33, 25, 17)
    h = 1.0 / 32
    g = _grid(3, n, h)
    g.set_psi(cuda(W.uniform(940, 32 * 24 * 16, 0.1, 1.0)), 1e-3)
    lv = 0
    nl, hl = g.level_shape(lv)
    Pl = oracle.Problem(3, nl, hl, 1.0, 0.6, 0.5)
    psi_l = g.get_psi(lv)
    E = np.array([[0.011, 0.004, -0.002], [0.004, -0.007, 0.003], [-0.002, 0.003, 0.009]])
    pairs = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    eps0 = np.concatenate([np.full(Pl.ncells, E[i, j]) for i, j in pairs])
    f = host(g.source_terms(psi_l, eps0=cuda(eps0), level=lv))
    Xn = W.node_coords(3, nl, hl)
    u = np.concatenate([sum(E[p, q] * Xn[q] for q in range(3)) for p in range(3)])
    Ku = torch.empty(3 * Pl.nnodes, dtype=torch.float64, device="cuda")
    _capi.check(sbm.lib().sbm_apply(g._h, lv, 0, sbm._ptr(cuda(u)), sbm._ptr(Ku)), g._h)
    assert np.abs(f - host(Ku)).max() <= 1e-12 * np.abs(f).max()
    assert np.abs(f - oracle.source_terms(Pl, host(psi_l), eps0=eps0)).max() <= 1e-13 * np.abs(f).max()


def test_source_terms_argument_errors(built):
    g = _grid(2, (9, 9, 1), 0.125)
    psi = cuda(np.ones(64))
    f = torch.empty(2 * 81, dtype=torch.float64, device="cuda")
    host_buf = (C.c_double * 162)()
    L = sbm.lib()
    assert L.sbm_source_terms(g._h, 0, sbm._ptr(psi), None, C.addressof(host_buf), None, sbm._ptr(f)) \
        == _capi.SBM_ERR_ARG
    assert L.sbm_source_terms(g._h, 0, C.addressof(host_buf), None, None, None, sbm._ptr(f)) == _capi.SBM_ERR_ARG
    assert L.sbm_source_terms(g._h, 7, sbm._ptr(psi), None, None, None, sbm._ptr(f)) == _capi.SBM_ERR_ARG
    g2 = sbm.Grid(2, (9, 9, 1), 0.125)
    assert L.sbm_source_terms(g2._h, 0, sbm._ptr(psi), None, None, None, sbm._ptr(f)) == _capi.SBM_ERR_STATE


# ------------------------------------------------------------ plate with a hole

E_, NU_ = 1.0, 0.3
A_ = 1.0            # hole radius


def _plate(dim, n, L, eps, exact_u, psi_min=1e-4):
    """Quarter (octant) plate [0, L]^dim, hole of radius A_ at the origin:
    psi = (1 + tanh((r - A_) / eps)) / 2 in cells, symmetry planes (normal
    displacement 0) on the faces through the origin, exact displacement on the
    outer faces.  Returns the grid, the nodal coordinates and the initial guess."""
    nn = (n, n, n if dim == 3 else 1)
    h = L / (n - 1)
    g = _grid(dim, nn, h, (E_, NU_), kind=sbm.SBM_ISO_ENU, precision="mixed")
    faces = ["-x", "+x", "-y", "+y", "-z", "+z"]
    for p in range(dim):
        g.set_bc(faces[2 * p], p, sbm.SBM_DIRICHLET_FROM_U)
        for q in range(dim):
            g.set_bc(faces[2 * q + 1], p, sbm.SBM_DIRICHLET_FROM_U)
    Xc = W.cell_centres(dim, nn, h)[:dim]
    r = np.sqrt(sum(x * x for x in Xc))
    psi = 0.5 * (1 + np.tanh((r - A_) / eps))
    g.set_psi(cuda(psi), psi_min)
    Xn = W.node_coords(dim, nn, h)[:dim]
    with np.errstate(divide="ignore", invalid="ignore"):     # the hole's centre, r = 0
        ue = np.nan_to_num(np.concatenate(exact_u(*Xn)))
    N = Xn[0].size
    u0 = np.zeros(dim * N)
    on_outer = np.zeros(N, dtype=bool)
    for q in range(dim):
        on_outer |= np.isclose(Xn[q], L)
    for p in range(dim):
        u0[p * N:(p + 1) * N][on_outer] = ue[p * N:(p + 1) * N][on_outer]
    return g, psi, Xn, ue, u0, h


def _nodal_stress_on_row(u, n, h, j, i_hi):
    """Plane-strain stresses by central differences at nodes (i, j), 1 <= i <= i_hi."""
    N = n * n
    ux = u[:N].reshape(n, n)
    uy = u[N:].reshape(n, n)
    i = np.arange(1, i_hi + 1)
    exx = (ux[j, i + 1] - ux[j, i - 1]) / (2 * h)
    eyy = (uy[j + 1, i] - uy[j - 1, i]) / (2 * h)
    exy = 0.5 * ((ux[j + 1, i] - ux[j - 1, i]) + (uy[j, i + 1] - uy[j, i - 1])) / (2 * h)
    return i * h, X.plane_strain_stress(exx, eyy, exy, E_, NU_)


def _solve(g, f, u0):
    g.set_source(cuda(f))
    u = cuda(u0)
    info = g.solve(u, tol=1e-10, max_cycles=400)
    assert info.converged
    return host(u)


def test_kirsch_plate_with_hole_converges_as_eps_decreases(built):
    """Sec. 3.1: uniaxial tension S, traction-free hole; normalised L2 error of the
    stresses along y = R (0 < x <= 4R) against Kirsch's solution, for eps = 0.8,
    0.4, 0.2, 0.1 on a 1025^2 quarter plate of side 16 R (h = R / 64)."""
    n, L, S = 1025, 16.0, 0.01
    exact = lambda x, y: X.kirsch_displacement(x, y, A_, S, E_, NU_)
    errs = []
    for eps in (0.8, 0.4, 0.2, 0.1):
        g, _, _, _, u0, h = _plate(2, n, L, eps, exact)
        u = _solve(g, np.zeros(2 * n * n), u0)
        j = int(round(A_ / h))
        x, sig = _nodal_stress_on_row(u, n, h, j, int(round(4 * A_ / h)))
        ref = X.kirsch_stress(x, np.full_like(x, A_), A_, S)
        err = np.sqrt(sum(((s - r) ** 2).sum() for s, r in zip(sig, ref)) / sum((r ** 2).sum() for r in ref))
        errs.append(err)
        g.close()
    print("kirsch eps -> L2 stress error along y = R:", dict(zip((0.8, 0.4, 0.2, 0.1), np.round(errs, 4))))
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1)), errs
    assert errs[-1] < 0.06, errs


def test_pressurised_hole_through_the_traction_source(built):
    """Lame's problem: pressure p in the hole, applied only as the diffuse traction
    t = -p e_r of eq. SBMLinearElasticity (sbm_source_terms); the displacement of
    the material (r >= R + eps) converges to the exact one as eps decreases."""
    n, L, p = 513, 8.0, 0.01
    exact = lambda x, y: X.lame_hole_displacement(x, y, A_, p, E_, NU_)
    errs = []
    for eps in (0.4, 0.2, 0.1):
        g, psi, Xn, ue, u0, h = _plate(2, n, L, eps, exact)
        r = np.hypot(*Xn)
        er = np.where(r > 0, 1.0 / np.maximum(r, 1e-300), 0.0)
        t = np.concatenate([-p * Xn[0] * er, -p * Xn[1] * er])
        f = host(g.source_terms(cuda(psi), t=cuda(t)))
        u = _solve(g, f, u0)
        m = np.tile(r >= A_ + eps, 2)
        errs.append(np.linalg.norm((u - ue)[m]) / np.linalg.norm(ue[m]))
        g.close()
    print("pressurised hole eps -> displacement error:", dict(zip((0.4, 0.2, 0.1), np.round(errs, 4))))
    assert all(errs[i + 1] < 0.6 * errs[i] for i in range(len(errs) - 1)), errs
    assert errs[-1] < 0.025, errs


def test_pressurised_spherical_cavity_3d(built):
    """The 3D analogue on a 129^3 octant of side 4 R (h = R / 32), through the 3D
    mixed-precision path: eps = 0.4 and 0.2."""
    n, L, p = 129, 4.0, 0.01
    exact = lambda x, y, z: X.cavity_displacement(x, y, z, A_, p, E_, NU_)
    errs = []
    for eps in (0.4, 0.2):
        g, psi, Xn, ue, u0, h = _plate(3, n, L, eps, exact)
        r = np.sqrt(sum(x * x for x in Xn))
        er = np.where(r > 0, 1.0 / np.maximum(r, 1e-300), 0.0)
        t = np.concatenate([-p * x * er for x in Xn])
        f = host(g.source_terms(cuda(psi), t=cuda(t)))
        u = _solve(g, f, u0)
        m = np.tile(r >= A_ + eps, 3)
        errs.append(np.linalg.norm((u - ue)[m]) / np.linalg.norm(ue[m]))
        g.close()
    print("pressurised cavity eps -> displacement error:", dict(zip((0.4, 0.2), np.round(errs, 4))))
    assert errs[1] < 0.75 * errs[0] and errs[1] < 0.07, errs
