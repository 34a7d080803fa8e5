"""Parity of the CUDA library (through the C ABI) with the CPU oracle.

Every step of the hot path is compared element by element with the oracle on
the same seeded inputs, at sizes that span several tiles with ragged tails;
full solves are compared with the oracle's solution converged to 1e-14.
Tolerances: FP64 steps 1e-12 of the largest output entry (summation order
differs: the kernels use the sum-factorised cell form, the oracle the dense
cell matrix); FP32 steps 3e-5 (inputs and moduli rounded to FP32, ~60 terms per
entry); solutions 1e-8 relative displacement error at relres 1e-10 (both
precisions, the FP32 path inside FP64 defect correction).
"""
import numpy as np
import pytest

import oracle
import workloads as W
from _sbm import cuda, gpu_grid, host, oracle_problem, random_workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2212_02362_gb300 as sbm  # noqa: E402

CASES = {
    "plate65": lambda: W.plate_hole(65),
    "ragged2d": lambda: random_workload(2, (73, 45), 101),
    "wide2d": lambda: random_workload(2, (161, 99), 103),
    "damage33": lambda: W.damage3d(33),
    "ragged3d": lambda: random_workload(3, (73, 45, 21), 202),
    # large enough for the warp-specialised FP32 kernel: ragged x tile (97 = 3 x 31 + 4),
    # a one-row last block row (65 = 2 x 32 + 1), Dirichlet data on several faces
    "col_ragged3d": lambda: random_workload(3, (97, 65, 33), 303, bits=(1 | 2 | 16, 4 | 8, 32)),
    # nx - 1 = 4 x 31: the last node of each row falls to lane 31 of the last tile
    "col_lastlane3d": lambda: random_workload(3, (125, 49, 17), 404, bits=(2 | 32, 1 | 16, 8)),
}


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _tol(fp32):
    return 3e-5 if fp32 else 1e-12


@pytest.fixture(scope="module")
def built():
    from paper_2212_02362_gb300 import build
    build.build()
    oracle.build()
    return True


def _floored(wk):
    return oracle.floor_psi(wk.psi, wk.psi_min)


def _level_problems(wk):
    """oracle problems and psi for every level, finest last."""
    P = oracle_problem(wk)
    psi = _floored(wk)
    probs, psis = [P], [psi]
    while oracle.can_coarsen(probs[0]):
        psis.insert(0, oracle.coarsen_psi(probs[0], psis[0]))
        probs.insert(0, oracle.coarse_problem(probs[0]))
    return probs, psis


# ------------------------------------------------------------------ steps

@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("fp32", [False, True])
def test_apply_parity(built, case, fp32):
    wk = CASES[case]()
    g = gpu_grid(wk)
    P = oracle_problem(wk)
    u = W.uniform(7, P.ndofs, -1, 1)
    ref = oracle.apply(P, _floored(wk), u)
    got = host(g.apply(g.finest, cuda(u), fp32=fp32))
    assert _rel(got, ref) <= _tol(fp32)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("fp32", [False, True])
def test_residual_and_norm_parity(built, case, fp32):
    wk = CASES[case]()
    g = gpu_grid(wk)
    P = oracle_problem(wk)
    u = wk.u0 + W.uniform(8, P.ndofs, -1e-3, 1e-3) * ~oracle.dirichlet_mask(P)
    ref = oracle.residual(P, _floored(wk), wk.f, u)
    r, nrm = g.residual(g.finest, cuda(wk.f), cuda(u), fp32=fp32)
    assert _rel(host(r), ref) <= _tol(fp32)
    assert np.isclose(nrm, oracle.norm_free(P, ref), rtol=1e-12 if not fp32 else 1e-5)
    assert np.all(host(r)[oracle.dirichlet_mask(P)] == 0.0)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("fp32", [False, True])
def test_jacobi_sweep_parity(built, case, fp32):
    wk = CASES[case]()
    g = gpu_grid(wk)
    P = oracle_problem(wk)
    u = wk.u0 + W.uniform(9, P.ndofs, -1e-2, 1e-2) * ~oracle.dirichlet_mask(P)
    ref = oracle.jacobi_sweep(P, _floored(wk), wk.f, u, 0.6)
    got = host(g.smooth(g.finest, cuda(wk.f), cuda(u), "jacobi", 0.6, fp32=fp32))
    assert _rel(got - u, ref - u) <= (1e-4 if fp32 else 1e-11)


@pytest.mark.parametrize("case", ["plate65", "ragged2d", "damage33", "ragged3d"])
@pytest.mark.parametrize("descending", [False, True])
def test_colour_gs_sweep_parity(built, case, descending):
    wk = CASES[case]()
    g = gpu_grid(wk)
    P = oracle_problem(wk)
    u = wk.u0 + W.uniform(10, P.ndofs, -1e-2, 1e-2) * ~oracle.dirichlet_mask(P)
    ref = oracle.gs_sweep(P, _floored(wk), wk.f, u, descending)
    got = host(g.smooth(g.finest, cuda(wk.f), cuda(u), "gs", descending=descending))
    assert _rel(got - u, ref - u) <= 1e-11


@pytest.mark.parametrize("case", ["plate65", "ragged2d", "wide2d"])
@pytest.mark.parametrize("descending", [False, True])
@pytest.mark.parametrize("fp32", [False, True])
def test_colour_gs_sweep_every_level(built, case, descending, fp32):
    """The one-launch 2D colour sweep (32 x 32 tiles, four-node halo) on every level of
    the hierarchy: levels of several tiles with ragged edges down to levels smaller
    than one tile, against the oracle's sequential colour sweep."""
    wk = CASES[case]()
    g = gpu_grid(wk)
    probs, psis = _level_problems(wk)
    assert g.nlevels == len(probs)
    for l in range(g.nlevels):
        P = probs[l]
        f = W.uniform(30 + l, P.ndofs, -1, 1) * ~oracle.dirichlet_mask(P)
        u = W.uniform(50 + l, P.ndofs, -1e-1, 1e-1)
        ref = oracle.gs_sweep(P, psis[l], f, u, descending)
        got = host(g.smooth(l, cuda(f), cuda(u), "gs", descending=descending, fp32=fp32))
        assert _rel(got - u, ref - u) <= (1e-4 if fp32 else 1e-11), l
        # Dirichlet dofs keep their values exactly
        mask = oracle.dirichlet_mask(P)
        assert np.array_equal(got[mask], u[mask]) if not fp32 else np.allclose(got[mask], u[mask], rtol=1e-7)


@pytest.mark.parametrize("case", ["plate65", "ragged2d", "damage33", "ragged3d"])
@pytest.mark.parametrize("fp32", [False, True])
def test_transfers_and_psi_hierarchy(built, case, fp32):
    wk = CASES[case]()
    g = gpu_grid(wk)
    probs, psis = _level_problems(wk)
    assert g.nlevels == len(probs)
    for l in range(g.nlevels):
        assert np.allclose(host(g.get_psi(l)), psis[l], rtol=1e-14, atol=0)
    for l in range(1, g.nlevels):
        Pf, Pc = probs[l], probs[l - 1]
        r = W.uniform(20 + l, Pf.ndofs, -1, 1) * ~oracle.dirichlet_mask(Pf)
        assert _rel(host(g.restrict(l, cuda(r), fp32=fp32)), oracle.restrict(Pf, r)) <= (1e-6 if fp32 else 1e-14)
        e = W.uniform(40 + l, Pc.ndofs, -1, 1) * ~oracle.dirichlet_mask(Pc)
        u = W.uniform(60 + l, Pf.ndofs, -1, 1)
        assert _rel(host(g.prolong_add(l, cuda(e), cuda(u), fp32=fp32)) - u,
                    oracle.prolong_add(Pf, e, u) - u) <= (1e-6 if fp32 else 1e-14)


@pytest.mark.parametrize("case", ["plate65", "ragged2d", "damage33", "ragged3d"])
def test_bottom_solve_parity(built, case):
    wk = CASES[case]()
    g = gpu_grid(wk)
    probs, psis = _level_problems(wk)
    Pb, pb = probs[0], psis[0]
    f = W.uniform(77, Pb.ndofs, -1, 1)
    u = W.uniform(78, Pb.ndofs, -1, 1)
    ref = oracle.direct_solve(Pb, pb, f, u)
    got = host(g.bottom_correct(cuda(f), cuda(u)))
    assert _rel(got, ref) <= 1e-9
    got32 = host(g.bottom_correct(cuda(f), cuda(u), fp32=True))
    assert _rel(got32, ref) <= 1e-2


# ------------------------------------------------------------------ solves

def _oracle_solution(wk, smoother="jacobi", omega=None):
    """Oracle solution converged to 1e-14, or to its FP64 rounding floor (the rough
    SIMP fields stagnate near 1e-13), and the oracle's cycle count to 1e-10."""
    P = oracle_problem(wk)
    res = oracle.mg_solve(P, _floored(wk), wk.f, wk.u0, smoother=smoother,
                          omega=wk.omega if omega is None else omega, tol=1e-14, max_cycles=150)
    assert res.status == 0 or (res.status == 1 and res.history.min() <= 1e-12)
    r10 = oracle.mg_solve(P, _floored(wk), wk.f, wk.u0, smoother=smoother,
                          omega=wk.omega if omega is None else omega, tol=1e-10, max_cycles=500)
    return res.u, r10.cycles


@pytest.mark.parametrize("case,precision,smoother,bcvals", [
    ("plate65", "fp64", "jacobi", False),
    ("plate65", "fp64", "gs", True),
    ("plate65", "mixed", "jacobi", False),
    ("damage33", "fp64", "jacobi", True),
    ("damage33", "mixed", "jacobi", False),
    ("ragged3d", "mixed", "jacobi", False),
])
def test_solve_parity(built, case, precision, smoother, bcvals):
    wk = CASES[case]()
    if case.startswith("ragged"):
        wk.omega = 0.5
    uref, cyc_ref = _oracle_solution(wk, smoother)
    g = gpu_grid(wk, precision=precision, bc_values=bcvals)
    u = cuda(wk.u0 if not bcvals else np.where(oracle.dirichlet_mask(oracle_problem(wk)), 0.0, wk.u0))
    info = g.solve(u, tol=1e-10, smoother=smoother, omega=wk.omega)
    err = np.linalg.norm(host(u) - uref) / np.linalg.norm(uref)
    assert info.converged and info.relres <= 1e-10
    assert err <= 1e-8, (err, info.cycles)
    if precision == "fp64":
        assert abs(info.cycles - cyc_ref) <= 1, (info.cycles, cyc_ref)
    # the oracle confirms the reported residual
    P = oracle_problem(wk)
    r = oracle.residual(P, _floored(wk), wk.f, host(u))
    r0 = oracle.residual(P, _floored(wk), wk.f, wk.u0)
    assert oracle.norm_free(P, r) / oracle.norm_free(P, r0) <= 2e-10


@pytest.mark.parametrize("case", ["plate65", "damage33", "ragged3d"])
@pytest.mark.parametrize("use_graph", [True, False])
def test_adaptive_inner_cycles(built, case, use_graph):
    """Mixed precision with the device-side stop of the FP32 V-cycles: the same
    fixed point (the oracle's solution) and about as many V-cycles as with the
    fixed count, with and without graph replay."""
    wk = CASES[case]()
    if case.startswith("ragged"):
        wk.omega = 0.5
    uref, _ = _oracle_solution(wk, "jacobi")
    g = gpu_grid(wk, precision="mixed")
    u = cuda(wk.u0)
    fixed = g.solve(u, tol=1e-10, omega=wk.omega, inner_cycles=12, use_graph=use_graph)
    u = cuda(wk.u0)
    info = g.solve(u, tol=1e-10, omega=wk.omega, inner_cycles=12, inner_rtol=1e-6, use_graph=use_graph)
    err = np.linalg.norm(host(u) - uref) / np.linalg.norm(uref)
    assert info.converged and info.relres <= 1e-10
    assert err <= 1e-8, (err, info.cycles)
    # the stop is decided one V-cycle late at most per outer iteration
    assert info.vcycles <= fixed.vcycles + info.cycles, (info.vcycles, fixed.vcycles)
    assert info.vcycles < 12 * info.cycles or info.cycles <= fixed.cycles


@pytest.mark.parametrize("case,smoother", [("plate65", "jacobi"), ("plate65", "gs"), ("damage33", "jacobi")])
@pytest.mark.parametrize("use_graph", [True, False])
def test_fp64_batched_vcycles_match_one_per_host_read(built, case, smoother, use_graph):
    """FP64 mode with several V-cycles per host read (inner_cycles > 1): the device
    stops the batch at the tolerance, so the iterates, the cycle count and the relres
    history are those of one V-cycle per read, bit for bit; max_cycles falling inside
    a batch stops there."""
    wk = CASES[case]()
    g = gpu_grid(wk)
    u1 = cuda(wk.u0)
    i1 = g.solve(u1, smoother=smoother, omega=wk.omega, use_graph=use_graph)
    for batch in (4, 8):
        ub = cuda(wk.u0)
        ib = g.solve(ub, smoother=smoother, omega=wk.omega, inner_cycles=batch, use_graph=use_graph)
        assert ib.converged and ib.cycles == i1.cycles and ib.vcycles == i1.cycles
        assert torch.equal(ub, u1)
        assert ib.history == i1.history
    u = cuda(wk.u0)
    info = g.solve(u, smoother=smoother, omega=wk.omega, inner_cycles=4, max_cycles=5, raise_on_fail=False,
                   use_graph=use_graph)
    assert info.status == sbm._capi.SBM_ERR_NOCONV and info.cycles == 5 and len(info.history) == 6
    assert info.history == i1.history[:6]


def test_solve_graph_and_eager_agree_bitwise(built):
    wk = W.damage3d(17)
    g = gpu_grid(wk, precision="mixed")
    u1, u2 = cuda(wk.u0), cuda(wk.u0)
    i1 = g.solve(u1, use_graph=True)
    i2 = g.solve(u2, use_graph=False)
    assert i1.cycles == i2.cycles
    assert torch.equal(u1, u2)
    u3 = cuda(wk.u0)
    g.solve(u3, use_graph=True)
    assert torch.equal(u1, u3)


def test_topopt_mixed_solve_and_adjoint_gradient(built):
    wk = W.topopt3d(33, 17, 17)
    P = oracle_problem(wk)
    uref, _ = _oracle_solution(wk)
    g = gpu_grid(wk, precision="mixed", density=True)
    u = cuda(wk.u0)
    info = g.solve(u, omega=wk.omega)
    assert np.linalg.norm(host(u) - uref) / np.linalg.norm(uref) <= 1e-8
    hd = wk.h ** 3
    mask = oracle.dirichlet_mask(P)
    dJdu = np.where(mask, 0.0, hd * wk.f)
    lam, gpsi, grho, ainfo = g.adjoint(u, cuda(dJdu), want_rho=True, omega=wk.omega)
    assert ainfo.converged
    # oracle gradient from its own adjoint solution
    lam_ref = oracle.mg_solve(P, _floored(wk), dJdu, np.zeros(P.ndofs), omega=wk.omega, tol=1e-14,
                              max_cycles=150).u
    g_ref = oracle.dJdpsi(P, uref, lam_ref)
    _, dpsi = oracle.simp(wk.rho, wk.psi_min)
    assert _rel(host(gpsi), g_ref) <= 1e-7
    assert _rel(host(grho), g_ref * dpsi) <= 1e-7
    assert np.all(host(gpsi) <= 1e-12 * np.abs(g_ref).max())


def test_autograd_gradient_matches_central_differences(built):
    wk = W.topopt3d(17, 9, 9)
    hd = wk.h ** 3
    g = gpu_grid(wk, precision="mixed", density=True)
    opts = {"omega": wk.omega, "tol": 1e-12}
    f = cuda(wk.f)
    rho = cuda(wk.rho).requires_grad_(True)
    u = sbm.SBMSolve.apply(rho, g, cuda(wk.u0), opts)
    J = hd * torch.dot(f, u)
    J.backward()
    grad = host(rho.grad)
    P = oracle_problem(wk)

    def J_of(r):
        # stationary form: its error is quadratic in the solve error, so the oracle's
        # multigrid solve at its FP64 floor (~1e-13) is exact enough for the difference
        psi, _ = oracle.simp(r, wk.psi_min)
        uu = oracle.mg_solve(P, psi, wk.f, wk.u0, omega=wk.omega, tol=1e-14, max_cycles=60).u
        return hd * (2 * wk.f @ uu - uu @ oracle.apply(P, psi, uu))

    cells = (W.uniform(4999, 32) * P.ncells).astype(int)
    eps = 1e-6
    for c in cells:
        rp, rm = wk.rho.copy(), wk.rho.copy()
        rp[c] += eps
        rm[c] -= eps
        fd = (J_of(rp) - J_of(rm)) / (2 * eps)
        assert abs(fd - grad[c]) <= 1e-5 * np.abs(grad).max(), (c, fd, grad[c])


# ------------------------------------------------------------- edge cases

@pytest.mark.parametrize("dim,n", [(2, (2, 2)), (2, (7, 7)), (3, (2, 2, 2)), (3, (3, 4, 5))])
def test_single_level_grids_solve_exactly(built, dim, n):
    wk = random_workload(dim, n, 303)
    P = oracle_problem(wk)
    g = gpu_grid(wk)
    assert g.nlevels == 1
    u = cuda(wk.u0)
    info = g.solve(u, tol=1e-12)
    ref = oracle.direct_solve(P, _floored(wk), wk.f, wk.u0)
    assert info.cycles <= 2
    assert _rel(host(u), ref) <= 1e-10


def test_zero_problem_returns_without_cycles(built):
    wk = W.plate_hole(17)
    wk.f[:] = 0.0
    wk.u0[:] = 0.0
    wk.bcs = [(f, c, 0.0) for f, c, _ in wk.bcs]
    g = gpu_grid(wk)
    u = cuda(wk.u0)
    info = g.solve(u)
    assert info.cycles == 0 and info.r0 == 0.0 and float(u.abs().max()) == 0.0


def test_psi_floor_and_all_void(built):
    wk = W.plate_hole(33)
    wk.psi[:] = 0.0                                     # everything at the floor
    g = gpu_grid(wk)
    assert np.all(host(g.get_psi(g.finest)) == wk.psi_min)
    uref, _ = _oracle_solution(wk)
    u = cuda(wk.u0)
    g.solve(u)
    assert np.linalg.norm(host(u) - uref) <= 1e-8 * np.linalg.norm(uref)


def test_errors_are_reported_not_raised_on_device(built):
    wk = W.plate_hole(17)
    g = sbm.Grid(2, wk.n, wk.h)
    with pytest.raises(sbm.SBMError) as e:
        g.solve(cuda(wk.u0))
    assert e.value.status == sbm._capi.SBM_ERR_STATE
    g.set_moduli(sbm.SBM_CUBIC, wk.moduli)
    bad = wk.psi.copy()
    bad[3] = np.nan
    with pytest.raises(sbm.SBMError) as e:
        g.set_psi(cuda(bad), 1e-3)
    assert e.value.status == sbm._capi.SBM_ERR_ARG
    # host pointer where a device pointer is required
    import ctypes
    hostbuf = np.zeros(wk.ncells)
    st = sbm.lib().sbm_set_psi(g._h, g.finest, hostbuf.ctypes.data_as(ctypes.c_void_p), 1e-3)
    assert st == sbm._capi.SBM_ERR_ARG
    with pytest.raises(sbm.SBMError):
        g.set_bc("-z", 0)                               # no z faces in 2D
    with pytest.raises(sbm.SBMError):
        g.set_moduli(sbm.SBM_ISO_ENU, (1.0, 0.7))       # nu >= 0.5
    # non-convergence is a status with info, not an exception when asked
    g2 = gpu_grid(wk)
    info = g2.solve(cuda(wk.u0), raise_on_fail=False, max_cycles=2)
    assert info.status == sbm._capi.SBM_ERR_NOCONV and info.cycles == 2 and len(info.history) == 3
    # divergence (omega too large for Jacobi) is detected
    info = g2.solve(cuda(wk.u0), raise_on_fail=False, omega=1.95, max_cycles=500)
    assert info.status in (sbm._capi.SBM_ERR_DIVERGED, sbm._capi.SBM_ERR_NOCONV)


def test_solves_are_deterministic(built):
    wk = W.damage3d(33)
    g = gpu_grid(wk)
    a, b = cuda(wk.u0), cuda(wk.u0)
    g.solve(a)
    g.solve(b)
    assert torch.equal(a, b)


# --------------------------------------------------- full-size workloads

@pytest.mark.slow
def test_full_size_damage_129_apply_samples_and_residual(built):
    """129^3 cubic damage field (the benchmark workload): the operator matches the
    oracle at sampled nodes, and both precisions' solutions satisfy the oracle's
    residual check at relres 1e-10."""
    wk = W.damage3d(129)
    P = oracle_problem(wk)
    psi = _floored(wk)
    u = W.uniform(5, P.ndofs, -1, 1)
    ref = oracle.apply(P, psi, u)
    for prec in ("fp64", "mixed"):
        g = gpu_grid(wk, precision=prec)
        got = host(g.apply(g.finest, cuda(u)))
        idx = (W.uniform(6, 4096) * P.ndofs).astype(int)
        assert _rel(got[idx], ref[idx]) <= 1e-12
        uu = cuda(wk.u0)
        info = g.solve(uu)
        r = oracle.residual(P, psi, wk.f, host(uu))
        r0 = oracle.residual(P, psi, wk.f, wk.u0)
        assert info.converged
        assert oracle.norm_free(P, r) / oracle.norm_free(P, r0) <= 2e-10
        del g
