"""Full-size parity: the CUDA library on every configuration's workload against the
oracle's records (tests/golden/*_oracle.json, written by tests/golden/make_golden.py
from the oracle alone).

For each field the oracle computed (the displacement, the adjoint and the
gradients of the cantilever) the GPU result must match the oracle's at the
record's seeded sample of entries to the parity tolerance (relative displacement
error <= 1e-8, the GPU solve at relres 1e-10 against the oracle's at 1e-14 or its
FP64 floor) and in each of the record's sketches (inner products with seeded
random vectors, which see an error wherever it sits).  The operator and the
damped-Jacobi sweep of the FP32 TMA kernel are also compared element by element
with the oracle at 129^3.
"""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W
from _sbm import cuda, gpu_grid, host, oracle_problem

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2212_02362_gb300 as sbm  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def built():
    from paper_2212_02362_gb300 import build
    build.build()
    oracle.build()
    return True


def _record(name):
    path = os.path.join(GOLDEN, f"{name}_oracle.json")
    if not os.path.exists(path):
        pytest.skip(f"no oracle record {name}")
    return json.load(open(path))


def _sketch_vectors(n, count, seed=7100):
    # the seeded vectors of tests/golden/make_golden.py (uniform in [-1, 1])
    return [W.uniform(seed + j, n, -1.0, 1.0) for j in range(count)]


def _compare(rec, x, tol, what):
    """Relative 2-norm error at the record's samples <= tol, and every sketch within
    2 tol |x_oracle| of the oracle's (an error e moves a sketch by about |e|/sqrt(3))."""
    idx = np.asarray(rec["sample_index"])
    ref = np.asarray(rec["sample"])
    err = np.linalg.norm(x[idx] - ref) / max(np.linalg.norm(ref), 1e-300)
    assert err <= tol, (what, err)
    for j, (w, s) in enumerate(zip(_sketch_vectors(x.size, len(rec["sketch"])), rec["sketch"])):
        assert abs(float(w @ x) - s) <= 2 * tol * rec["norm"], (what, j, float(w @ x) - s, rec["norm"])
    return err


# ------------------------------------------------- C3: damage_3d 129^3 (cubic)

def test_C3_fp32_operator_and_jacobi_elementwise_at_129(built):
    """The FP32 TMA kernel over the whole 129^3 grid (all tiles, both ragged edges of
    the 32 x 12 tiling, every z segment of the persistent CTAs): K u and one damped
    Jacobi sweep element by element against the oracle."""
    wk = W.damage3d(129)
    P = oracle_problem(wk)
    psi = oracle.floor_psi(wk.psi, wk.psi_min)
    g = gpu_grid(wk, precision="mixed")
    u = W.uniform(5, P.ndofs, -1, 1)
    ref = oracle.apply(P, psi, u)
    got = host(g.apply(g.finest, cuda(u), fp32=True))
    assert np.abs(got - ref).max() <= 3e-5 * np.abs(ref).max()
    u = wk.u0 + W.uniform(9, P.ndofs, -1e-2, 1e-2) * ~oracle.dirichlet_mask(P)
    ref = oracle.jacobi_sweep(P, psi, wk.f, u, wk.omega)
    got = host(g.smooth(g.finest, cuda(wk.f), cuda(u), "jacobi", wk.omega, fp32=True))
    assert np.abs((got - u) - (ref - u)).max() <= 1e-4 * np.abs(ref - u).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_C3_damage_129_solution_matches_oracle_record(built, precision):
    rec = _record("damage_3d_129")
    wk = W.damage3d(129)
    g = gpu_grid(wk, precision=precision, bc_values=True)
    u = cuda(wk.u0)
    opts = {"tol": 1e-10, "omega": wk.omega}
    if precision == "mixed":
        opts.update(inner_cycles=12, inner_rtol=1e-6)     # the bench's settings
    info = g.solve(u, **opts)
    assert info.converged and info.relres <= 1e-10
    _compare(rec["u"], host(u), 1e-8, f"u {precision}")
    if precision == "fp64":
        assert abs(info.cycles - rec["cycles_to_1e-10"]) <= 1, (info.cycles, rec["cycles_to_1e-10"])


# ------------------------------------ C4: topopt_3d 257 x 129 x 129 cantilever

def test_C4_topopt_forward_adjoint_and_gradient_match_oracle_record(built):
    """Mixed-precision forward solve, adjoint solve and dJ/drho of the compliance
    with the bench's settings, against the oracle's forward solution, adjoint
    solution and gradients (both at their FP64 floor)."""
    rec = _record("topopt_3d")
    wk = W.topopt3d()
    g = gpu_grid(wk, precision="mixed", density=True)
    u = cuda(wk.u0)
    opts = {"tol": 1e-10, "omega": wk.omega, "inner_cycles": 8}
    info = g.solve(u, **opts)
    assert info.converged
    _compare(rec["u"], host(u), 1e-8, "u")
    P = oracle_problem(wk)
    dJdu = np.where(oracle.dirichlet_mask(P), 0.0, wk.h ** 3 * wk.f)
    lam, gpsi, grho, ainfo = g.adjoint(u, cuda(dJdu), want_rho=True, **opts)
    assert ainfo.converged
    _compare(rec["lambda"], host(lam), 1e-8, "lambda")
    _compare(rec["dJdpsi"], host(gpsi), 1e-7, "dJ/dpsi")
    _compare(rec["dJdrho"], host(grho), 1e-7, "dJ/drho")
    J = wk.h ** 3 * float(torch.dot(cuda(wk.f), u))
    assert abs(J - rec["compliance"]) <= 1e-8 * abs(rec["compliance"])


# ------------------------------------------ C2 / C5: block-structured refinement

def _amr_gpu(wk, precision):
    g = sbm.Grid(wk.dim, wk.n, wk.h, precision=precision)
    g.set_moduli(sbm.SBM_CUBIC, wk.moduli)
    for face, comp, _ in wk.bcs:
        g.set_bc(face, comp, sbm.SBM_DIRICHLET_FROM_U)
    g.set_psi(cuda(wk.level_psi(0)), wk.psi_min)
    for a, b in enumerate(wk.boxes, start=1):
        assert g.amr_add_box(wk.level(a), b[0], b[1]) == a
    for a in range(1, len(wk.boxes) + 1):
        g.amr_set_psi(a, cuda(wk.level_psi(a)), wk.psi_min)
    return g


def _amr_parity(rec, wk, precision, tol, **opts):
    """Composite solve to relres tol; returns the relative error over all levels'
    samples, the largest sketch deviation in units of |u_a| and the solve info."""
    assert [[list(b[0]), list(b[1])] + ([b[2]] if len(b) > 2 else []) for b in wk.boxes] == rec["boxes"]
    g = _amr_gpu(wk, precision)
    us = [cuda(wk.level_u0(a)) for a in range(len(wk.boxes) + 1)]
    info = g.amr_solve(us, tol=tol, omega=wk.omega, smoother=wk.smoother, **opts)
    assert info.converged and info.relres <= tol
    num = den = 0.0
    sk = 0.0
    for a, lr in enumerate(rec["levels"]):
        x = host(us[a])
        idx = np.asarray(lr["sample_index"])
        ref = np.asarray(lr["sample"])
        num += float(((x[idx] - ref) ** 2).sum())
        den += float((ref ** 2).sum())
        for w, s in zip(_sketch_vectors(x.size, len(lr["sketch"])), lr["sketch"]):
            sk = max(sk, abs(float(w @ x) - s) / lr["norm"])
    return (num / den) ** 0.5, sk, info


def test_C2_voids_amr_2d_full_size_matches_oracle_record(built):
    """129^2 base + 3 refinement levels (finest h = 1/1024), FP64, colour Gauss-Seidel,
    against the oracle's composite iteration at its FP64 floor (5e-13).  At psi_min =
    1e-4 the composite problem is too ill-conditioned for relres 1e-10 to bound the
    displacement error by 1e-8 (measured: ~3e-8 at 1e-10), so the GPU solves to relres
    1e-12 for the 1e-8 bound."""
    rec = _record("voids_amr_2d")
    wk = W.voids_amr(2, 129, 3)
    err, sk, info = _amr_parity(rec, wk, "fp64", 1e-12)
    assert err <= 1e-8 and sk <= 2e-8, (err, sk, info.cycles)


@pytest.mark.parametrize("base", [33, 65])
def test_C5_voids_amr_3d_matches_oracle_record(built, base):
    """The 3D refinement workload at a 33^3 and a 65^3 base + 2 levels (65^3 is the
    largest the single-thread oracle solves offline), mixed precision with 6 FP32
    correction cycles per FP64 composite residual, as the bench runs the 129^3 base.
    As for C2, relres 1e-10 does not bound the error by 1e-8 on this ill-conditioned
    composite problem (two GPU solutions at 1e-10 differ by ~1e-7), so the GPU solves
    to relres 1e-12."""
    rec = _record(f"voids_amr_3d_{base}")
    wk = W.voids_amr(3, base, 2, count=16, rmin=0.04, rmax=0.12)
    err, sk, info = _amr_parity(rec, wk, "mixed", 1e-12, inner_cycles=6, max_cycles=500)
    assert err <= 1e-8 and sk <= 2e-8, (err, sk, info.cycles)


@pytest.mark.parametrize("name,precision,opts", [
    ("voids_amr_2d_clustered", "fp64", {}),
    ("voids_amr_3d_clustered_65", "mixed", {"inner_cycles": 6}),
    ("voids_amr_3d_clustered_129", "mixed", {"inner_cycles": 6}),
])
def test_clustered_hierarchies_match_oracle_records(built, name, precision, opts):
    """Several patches per level (host tagging and clustering): the 2D voids at a
    129^2 base + 3 levels (23 patches, FP64 colour Gauss-Seidel) and the 3D voids at
    a 65^3 and a 129^3 base + 2 levels (mixed precision), against the oracle's
    composite iteration at its FP64 floor; GPU at relres 1e-12 (D9)."""
    rec = _record(name)
    if name == "voids_amr_2d_clustered":
        wk = W.voids_amr(2, 129, 3, clustered=True)
    else:
        wk = W.voids_amr(3, int(name.rsplit("_", 1)[1]), 2, count=8, rmin=0.04, rmax=0.08, clustered=True)
    err, sk, info = _amr_parity(rec, wk, precision, 1e-12, max_cycles=500, **opts)
    assert err <= 1e-8 and sk <= 2e-8, (err, sk, info.cycles)
