"""Pins of the oracle's phase-field topology optimisation step (Sec. 3.3): one
explicit Euler step of eq. topop_evolution with the energy of eq. topop_objective
and the volume constraint of eq. topop_volume_constraint, psi = (eta + zeta)^2.

  - the step is a gradient step of the discrete energy (double well + gradient
    energy + half the compliance of the equilibrium solve + the volume penalty):
    central differences of that energy, with a direct solve per evaluation, give
    h^d times the bracket of the update in every cell probed (2D and 3D);
  - each term alone against its closed form: the double well's fixed points
    0, 1/2, 1 and its sign; the Laplacian of a quadratic; conservation of the
    Neumann Laplacian; one volume step with dt L lambda |Omega| = 1 lands on V0;
    lambda(t) growing linearly with the step index;
  - the elastic term alone lowers the compliance.
"""
import numpy as np
import pytest

import workloads as W


def _cantilever(oracle, dim, n):
    """Left face clamped, a random load on the right face."""
    nn = tuple(n) if dim == 3 else (n[0], n[1], 1)
    h = 1.0 / (nn[1] - 1)
    bits = (1,) * dim + (0,) * (3 - dim)
    P = oracle.Problem(dim, nn, h, 1.0, 0.4, 0.3, dirichlet=bits)
    X = W.node_coords(dim, nn, h)
    f = np.zeros(P.ndofs)
    right = np.isclose(X[0], (nn[0] - 1) * h)
    g = W.uniform(77 + dim, P.ndofs, -1.0, 1.0)
    for p in range(dim):
        f[p * P.nnodes:(p + 1) * P.nnodes][right] = g[p * P.nnodes:(p + 1) * P.nnodes][right]
    return P, f


def _total_energy(oracle, P, T, f, eta):
    u = oracle.direct_solve(P, oracle.psi_of_eta(T, eta), f, np.zeros(P.ndofs))
    return oracle.topopt_energy(P, T, eta).sum() + 0.5 * P.h ** P.dim * f @ u, u


@pytest.mark.parametrize("dim,n", [(2, (7, 5)), (3, (5, 4, 3))])
def test_step_is_a_gradient_step_of_the_discrete_energy(oracle_lib, dim, n):
    oracle = oracle_lib
    P, f = _cantilever(oracle, dim, n)
    T = oracle.TopoptParams(alpha=3.0, beta=0.05, zeta=0.01, lam=7.0, V0=0.3, mobility=0.7, dt=1e-3)
    eta = W.uniform(81 + dim, P.ncells, 0.1, 0.9)
    E0, u = _total_energy(oracle, P, T, f, eta)
    out = oracle.topopt_step(P, T, eta, u)
    bracket = (eta - out) / (T.dt * T.mobility)
    d = 1e-6
    for c in range(0, P.ncells, max(1, P.ncells // 7)):
        e = np.zeros(P.ncells)
        e[c] = d
        Ep, _ = _total_energy(oracle, P, T, f, eta + e)
        Em, _ = _total_energy(oracle, P, T, f, eta - e)
        fd = (Ep - Em) / (2 * d)
        assert np.isclose(fd, P.h ** dim * bracket[c], rtol=1e-6, atol=1e-9 * abs(E0)), (c, fd, bracket[c])


def test_double_well_alone(oracle_lib):
    oracle = oracle_lib
    P = oracle.Problem(2, (6, 5, 1), 0.25, 1.0, 0.4, 0.3)
    T = oracle.TopoptParams(alpha=5.0, beta=0.0, lam=0.0, zeta=0.01, mobility=2.0, dt=1e-2)
    eta = np.array([0.0, 0.5, 1.0, 0.3, 0.7, -0.2, 1.2, 0.1, 0.9, 0.45] * 2)
    out = oracle.topopt_step(P, T, eta, np.zeros(P.ndofs))
    expect = eta - T.dt * T.mobility * 2 * T.alpha * eta * (1 - eta) * (1 - 2 * eta)
    assert np.allclose(out, expect, rtol=1e-15, atol=1e-15)
    assert out[0] == 0.0 and out[1] == 0.5 and out[2] == 1.0
    assert out[3] < eta[3] and out[4] > eta[4]          # towards the nearer well


def test_laplacian_of_a_quadratic_and_conservation(oracle_lib):
    oracle = oracle_lib
    nn = (9, 8, 7)
    h = 0.125
    P = oracle.Problem(3, nn, h, 1.0, 0.4, 0.3)
    T = oracle.TopoptParams(alpha=0.0, beta=0.3, lam=0.0, mobility=1.5, dt=1e-3)
    Xc = W.cell_centres(3, nn, h)
    eta = Xc[0] ** 2 + 2 * Xc[1] ** 2 - 0.5 * Xc[2] ** 2
    out = oracle.topopt_step(P, T, eta, np.zeros(P.ndofs))
    lap = (out - eta) / (T.dt * T.mobility * T.beta)
    inner = np.ones(P.ncells, dtype=bool)
    for a in range(3):
        inner &= (Xc[a] > h) & (Xc[a] < (nn[a] - 2) * h)
    assert np.allclose(lap[inner], 2 + 4 - 1, rtol=1e-10)
    # Neumann: the Laplacian of any field sums to zero over the box
    r = W.uniform(85, P.ncells, 0, 1)
    out = oracle.topopt_step(P, T, r, np.zeros(P.ndofs))
    assert abs((out - r).sum()) <= 1e-14 * P.ncells
    assert np.abs(out - r).max() > 1e-5


def test_volume_step_lands_on_the_target(oracle_lib):
    oracle = oracle_lib
    P = oracle.Problem(2, (11, 6, 1), 0.2, 1.0, 0.4, 0.3)
    area = 10 * 5 * 0.2 ** 2
    T = oracle.TopoptParams(alpha=0.0, beta=0.0, lam=50.0, V0=0.6, mobility=1.0)
    T.dt = 1.0 / (T.mobility * T.lam * area)
    eta = W.uniform(86, P.ncells, 0, 1)
    out = oracle.topopt_step(P, T, eta, np.zeros(P.ndofs))
    assert np.isclose(P.h ** 2 * out.sum(), T.V0, rtol=1e-13)
    assert np.allclose(np.diff(out - eta), 0.0, atol=1e-15)     # a uniform shift
    # lambda(t) = lam + lam_rate * step * dt
    T2 = oracle.TopoptParams(alpha=0.0, beta=0.0, lam=50.0, lam_rate=1e3, V0=0.6, mobility=1.0, dt=T.dt)
    s = 4
    shift = (oracle.topopt_step(P, T2, eta, np.zeros(P.ndofs), step=s) - eta)[0]
    assert np.isclose(shift, -T.dt * (50.0 + 1e3 * s * T.dt) * (P.h ** 2 * eta.sum() - T.V0), rtol=1e-13)


def test_elastic_term_alone_lowers_the_compliance(oracle_lib):
    oracle = oracle_lib
    P, f = _cantilever(oracle, 2, (9, 5))
    T = oracle.TopoptParams(alpha=0.0, beta=0.0, lam=0.0, zeta=0.01, mobility=1.0, dt=1e-4)
    eta = W.uniform(87, P.ncells, 0.2, 0.8)
    J = lambda e: P.h ** 2 * f @ oracle.direct_solve(P, oracle.psi_of_eta(T, e), f, np.zeros(P.ndofs))
    u = oracle.direct_solve(P, oracle.psi_of_eta(T, eta), f, np.zeros(P.ndofs))
    out = oracle.topopt_step(P, T, eta, u)
    assert np.all(out >= eta)                      # stiffening everywhere: e_c >= 0
    assert J(out) < J(eta)
