"""Phase-field topology optimisation (Sec. 3.3) on the GPU: the Allen-Cahn step
(sbm_topopt_step) against the oracle's restatement, element by element, from small
ragged grids to the 257 x 129 x 129 cantilever; the staggered loop (sbm_topopt_run:
psi from eta, warm-started solve, step) against the same loop driven through the
oracle; and along the GPU loop the discrete energy the step descends (double well +
gradient energy + half the compliance + volume penalty) decreases step by step while
the volume approaches its target."""
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


def _cantilever(dim, n, moduli=(1.0, 0.4, 0.3), precision="fp64", load=1.0):
    """[0, (nx-1) h] x [0, 1] (x [0, 1]): x = 0 clamped, a downward load spread over
    the nodes of the +x face near its centre (h^d sum f_y = -load)."""
    nn = tuple(n) if dim == 3 else (n[0], n[1], 1)
    h = 1.0 / (nn[1] - 1)
    P = oracle.Problem(dim, nn, h, *moduli, dirichlet=(1,) * dim + (0,) * (3 - dim))
    X = W.node_coords(dim, nn, h)
    r2 = (X[0] - (nn[0] - 1) * h) ** 2 + (X[1] - 0.5) ** 2 + ((X[2] - 0.5) ** 2 if dim == 3 else 0.0)
    g = np.exp(-r2 / (2 * (2 * h) ** 2))
    f = np.zeros(P.ndofs)
    f[P.nnodes:2 * P.nnodes] = -load * g / (h ** dim * g.sum())
    grid = sbm.Grid(dim, nn, h, precision=precision)
    grid.set_moduli(sbm.SBM_CUBIC, moduli)
    for p in range(dim):
        grid.set_bc("-x", p, sbm.SBM_DIRICHLET, 0.0)
    grid.set_source(cuda(f))
    return P, grid, f


PRM = dict(alpha=2.0, beta=0.01, zeta=0.01, lam=5.0, lam_rate=0.0, mobility=1.0, dt=2e-3)


def _otp(P, **kw):
    d = dict(PRM, **kw)
    return oracle.TopoptParams(alpha=d["alpha"], beta=d["beta"], zeta=d["zeta"], lam=d["lam"],
                               lam_rate=d["lam_rate"], V0=d["V0"], mobility=d["mobility"], dt=d["dt"])


@pytest.mark.parametrize("dim,n", [(2, (37, 21)), (3, (19, 11, 9)), (3, (33, 17, 17))])
def test_topopt_step_parity(built, dim, n):
    P, g, _ = _cantilever(dim, n)
    V0 = 0.3 * P.ncells * P.h ** dim
    T = _otp(P, V0=V0, lam_rate=40.0)
    eta = W.uniform(300 + dim, P.ncells, -0.05, 1.05)
    u = W.uniform(310 + dim, P.ndofs, -0.1, 0.1)
    psi = W.uniform(320 + dim, P.ncells, 1e-3, 1.0)
    g.set_psi(cuda(psi), 1e-6)
    for step in (0, 3):
        ref = oracle.topopt_step(P, T, eta, u, step=step)
        out, vol, comp = g.topopt_step(cuda(eta), cuda(u), V0=V0, step=step, **PRM | {"lam_rate": 40.0})
        out = host(out)
        assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref - eta).max() + 1e-15
        assert np.isclose(vol, P.h ** dim * ref.sum(), rtol=1e-12)
        e = -oracle.dJdpsi(P, u, u)
        assert np.isclose(comp, P.h ** dim * (psi * e).sum(), rtol=1e-12)


def test_topopt_step_parity_257x129x129(built):
    """The 257 x 129 x 129 cantilever of the topology-optimisation workload
    (4.19 M cells): every cell against the oracle."""
    wk = W.topopt3d()
    P = oracle.Problem(3, wk.n, wk.h, *wk.moduli)
    g = sbm.Grid(3, wk.n, wk.h, precision="mixed")
    g.set_moduli(sbm.SBM_CUBIC, wk.moduli)
    V0 = 0.25 * 2.0
    T = _otp(P, V0=V0)
    eta = np.clip(wk.rho, 0.0, 1.0)
    u = W.uniform(330, P.ndofs, -1e-3, 1e-3)
    ref = oracle.topopt_step(P, T, eta, u)
    out, vol, _ = g.topopt_step(cuda(eta), cuda(u), V0=V0, **PRM)
    out = host(out)
    assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref - eta).max()
    assert np.isclose(vol, P.h ** 3 * ref.sum(), rtol=1e-12)


@pytest.mark.parametrize("dim,n,steps,omega", [(2, (49, 25), 6, 2.0 / 3.0), (3, (25, 9, 9), 4, 0.5)])
def test_topopt_loop_matches_the_oracle_loop(built, dim, n, steps, omega):
    """Steps of the staggered loop on a 49 x 25 and a 25 x 9 x 9 cantilever, FP64
    solves to 1e-11 (relative to each warm start's initial residual), against the
    same loop through the oracle (multigrid solve to 1e-12, then the step)."""
    P, g, f = _cantilever(dim, n)
    V0 = 0.4 * P.ncells * P.h ** dim
    T = _otp(P, V0=V0)
    eta0 = np.clip(0.5 + 0.3 * np.sin(np.arange(P.ncells) * 0.37), 0, 1)
    psi_min = 1e-6
    eta = cuda(eta0)
    u = torch.zeros(P.ndofs, dtype=torch.float64, device="cuda")
    res = g.topopt_run(eta, u, steps, V0=V0, psi_min=psi_min, tol=1e-11, max_cycles=300, omega=omega, **PRM)
    assert res["steps"] == steps
    e_ref, u_ref = eta0.copy(), np.zeros(P.ndofs)
    comps = []
    for s in range(steps):
        psi = np.maximum(oracle.psi_of_eta(T, e_ref), psi_min)
        u_ref = oracle.mg_solve(P, psi, f, u_ref, omega=omega, tol=1e-12, max_cycles=400).u
        comps.append(P.h ** dim * (psi * -oracle.dJdpsi(P, u_ref, u_ref)).sum())
        e_ref = oracle.topopt_step(P, T, e_ref, u_ref, step=s)
    got = host(eta)
    assert np.abs(got - e_ref).max() <= 1e-9 * np.abs(e_ref - eta0).max()
    assert np.allclose(res["compliance"], comps, rtol=1e-9)
    assert np.allclose(res["volume"][-1], P.h ** dim * e_ref.sum(), rtol=1e-12)
    assert np.abs(host(u) - u_ref).max() <= 1e-9 * np.abs(u_ref).max()


def test_topopt_loop_descends_the_discrete_energy(built):
    """A 2 x 1 cantilever (129 x 65 nodes, mixed precision) starting below its 40 %
    fill, its load (0.02) sized so that half the compliance is of the order of the
    volume penalty: along 30 steps of the GPU loop the discrete energy decreases at
    every step, the volume approaches V0 and, as material is added, the compliance
    falls."""
    P, g, f = _cantilever(2, (129, 65), precision="mixed", load=0.02)
    V0 = 0.4 * 2.0
    prm = dict(PRM, dt=1e-3, lam=20.0)
    T = _otp(P, V0=V0, dt=1e-3, lam=20.0)
    eta = cuda(np.full(P.ncells, 0.3) + 0.02 * W.uniform(340, P.ncells, -1, 1))
    u = torch.zeros(P.ndofs, dtype=torch.float64, device="cuda")
    energies, vols, comps = [], [], []
    for s in range(30):
        e_host = host(eta)
        res = g.topopt_run(eta, u, 1, V0=V0, tol=1e-9, **prm)
        comps.append(res["compliance"][0])
        energies.append(oracle.topopt_energy(P, T, e_host).sum() + 0.5 * res["compliance"][0])
        vols.append(P.h ** 2 * e_host.sum())
    d = np.diff(energies)
    print("topopt energies", np.round(energies[::6], 6), "volumes", np.round(vols[::6], 4),
          "compliance", np.round(comps[::6], 6))
    assert np.all(d < 0), d
    assert abs(vols[-1] - V0) < 0.5 * abs(vols[0] - V0)
    assert comps[-1] < comps[0]


def test_topopt_argument_errors(built):
    P, g, _ = _cantilever(2, (9, 5))
    eta = cuda(np.full(P.ncells, 0.5))
    u = torch.zeros(P.ndofs, dtype=torch.float64, device="cuda")
    with pytest.raises(sbm.SBMError) as e:
        g.topopt_step(eta, u, dt=-1.0)
    assert e.value.status == _capi.SBM_ERR_ARG
    with pytest.raises(sbm.SBMError) as e:
        g.topopt_step(eta, u, mobility=0.0)
    assert e.value.status == _capi.SBM_ERR_ARG
    prm = _capi.sbm_topopt_params(1, 0, 0, 0, 0, 0, 1, 1e-3, 1e-6)
    assert sbm.lib().sbm_topopt_step(g._h, prm, 0, sbm._ptr(eta), sbm._ptr(u), sbm._ptr(eta), None, None) \
        == _capi.SBM_ERR_ARG                      # eta_out aliases eta
