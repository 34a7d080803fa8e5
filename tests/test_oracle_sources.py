"""Pins of the oracle's source terms of eq. SBMLinearElasticity (Sec. 2.1),
div(psi C (grad u - eps0)) - psi b = t |grad psi|, in the form K u = f:

  - an affine displacement whose strain is a uniform eigenstrain is stress free, so
    K u equals the eigenstrain load exactly at every node (any psi);
  - for an eigenstrain that varies from cell to cell, the load paired with an affine
    test field equals the sum over cells of psi_c sym(G) : C : eps0_c (the discrete
    weak form), and the load is self-equilibrated;
  - psi_n and grad psi_n are exact for a linear psi;
  - Theorem 1 of the paper: the diffuse traction source integrates to the boundary
    integral, h^d sum_n w_n |grad psi|_n -> perimeter (2D) / area (3D) of the hole;
  - the body-force load integrates to -(volume) b for psi = 1.
"""
import numpy as np
import pytest

import workloads as W


def _cubicC(c11, c12, c44):
    def C(i, j, k, l):
        if i == j and k == l:
            return c11 if i == k else c12
        if i != j and ((i == k and j == l) or (i == l and j == k)):
            return c44
        return 0.0
    return C


def _voigt_pairs(d):
    return [(0, 0), (1, 1), (0, 1)] if d == 2 else [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


@pytest.mark.parametrize("dim,n", [(2, (9, 7, 1)), (3, (5, 6, 4))])
def test_uniform_eigenstrain_affine_field_is_stress_free(oracle_lib, dim, n):
    oracle = oracle_lib
    P = oracle.Problem(dim, n, 0.25, 1.0, 0.6, 0.5)
    psi = W.uniform(3, P.ncells, 1e-3, 1.0)
    E = np.array([[0.011, 0.004, -0.002], [0.004, -0.007, 0.003], [-0.002, 0.003, 0.009]])[:dim, :dim]
    eps0 = np.concatenate([np.full(P.ncells, E[i, j]) for i, j in _voigt_pairs(dim)])
    X = W.node_coords(dim, P.n, P.h)[:dim]
    u = np.concatenate([sum(E[p, q] * X[q] for q in range(dim)) for p in range(dim)])
    Ku = oracle.apply(P, psi, u)
    f = oracle.source_terms(P, psi, eps0=eps0)
    assert np.allclose(f, Ku, rtol=1e-12, atol=1e-12 * np.abs(Ku).max())
    assert np.abs(f).max() > 1e-3


@pytest.mark.parametrize("dim,n", [(2, (9, 7, 1)), (3, (5, 6, 4))])
def test_cellwise_eigenstrain_load_is_the_discrete_weak_form(oracle_lib, dim, n):
    oracle = oracle_lib
    c = (1.0, 0.6, 0.5)
    C = _cubicC(*c)
    P = oracle.Problem(dim, n, 0.25, *c)
    psi = W.uniform(4, P.ncells, 1e-3, 1.0)
    nv = 3 if dim == 2 else 6
    eps0 = W.uniform(5, nv * P.ncells, -0.01, 0.01)
    f = oracle.source_terms(P, psi, eps0=eps0)
    # self-equilibrated: no net force
    for p in range(dim):
        assert abs(f[p * P.nnodes:(p + 1) * P.nnodes].sum()) <= 1e-12 * np.abs(f).max() * P.nnodes
    # paired with an affine field v = G x: sum over cells of psi_c sym(G) : C : eps0_c (h^d f . v in FD scaling)
    G = np.array([[0.3, -0.2, 0.5], [0.7, 0.1, -0.4], [-0.6, 0.2, 0.9]])[:dim, :dim]
    X = W.node_coords(dim, P.n, P.h)[:dim]
    v = np.concatenate([sum(G[p, q] * X[q] for q in range(dim)) for p in range(dim)])
    S = 0.5 * (G + G.T)
    pairs = _voigt_pairs(dim)
    E = np.zeros((dim, dim, P.ncells))
    for m, (i, j) in enumerate(pairs):
        E[i, j] = eps0[m * P.ncells:(m + 1) * P.ncells]
        E[j, i] = E[i, j]
    expect = 0.0
    for i in range(dim):
        for j in range(dim):
            for k in range(dim):
                for l in range(dim):
                    Cv = C(i, j, k, l)
                    if Cv:
                        expect += S[i, j] * Cv * (psi * E[k, l]).sum()
    assert np.isclose(P.h ** dim * (f @ v), P.h ** dim * expect, rtol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_nodal_psi_and_gradient_exact_for_linear_psi(oracle_lib, dim):
    oracle = oracle_lib
    n = (9, 8, 7 if dim == 3 else 1)
    P = oracle.Problem(dim, n, 0.125, 1.0, 0.6, 0.5)
    a = np.array([0.7, -0.4, 0.3])[:dim]
    Xc = W.cell_centres(dim, P.n, P.h)[:dim]
    psi = 1.0 + sum(a[i] * Xc[i] for i in range(dim))
    pn, gn, w = oracle.node_psi(P, psi)
    X = W.node_coords(dim, P.n, P.h)[:dim]
    inner = np.ones(P.nnodes, dtype=bool)
    for i in range(dim):
        inner &= (X[i] > 1e-12) & (X[i] < (P.n[i] - 1) * P.h - 1e-12)
    assert np.allclose(pn[inner], (1.0 + sum(a[i] * X[i] for i in range(dim)))[inner], rtol=1e-13)
    assert np.allclose(gn[inner], np.linalg.norm(a), rtol=1e-13)
    assert np.isclose(w.sum() * P.h ** dim, np.prod([(m - 1) * P.h for m in P.n[:dim]]), rtol=1e-13)


@pytest.mark.parametrize("dim,n,R,eps", [(2, 257, 0.25, 0.02), (3, 97, 0.3, 0.04)])
def test_theorem1_diffuse_traction_integrates_to_the_boundary_measure(oracle_lib, dim, n, R, eps):
    """psi = (1 + tanh((r - R)/eps)) / 2 around a hole of radius R: the integral of
    |grad psi| over the domain is, in closed form, the perimeter 2 pi R in 2D (the
    profile's first moment vanishes) and 4 pi (R^2 + pi^2 eps^2 / 12) in 3D (its
    second moment), which tends to the area 4 pi R^2 as eps -> 0 (Theorem 1); the
    discrete sum matches to within the discretisation error."""
    oracle = oracle_lib
    nn = (n, n, n if dim == 3 else 1)
    h = 1.0 / (n - 1)
    P = oracle.Problem(dim, nn, h, 1.0, 0.6, 0.5)
    Xc = W.cell_centres(dim, nn, h)[:dim]
    r = np.sqrt(sum((Xc[i] - 0.5) ** 2 for i in range(dim)))
    psi = 0.5 * (1 + np.tanh((r - R) / eps))
    _, gn, w = oracle.node_psi(P, psi)
    integral = h ** dim * (w * gn).sum()
    exact = 2 * np.pi * R if dim == 2 else 4 * np.pi * (R ** 2 + np.pi ** 2 * eps ** 2 / 12)
    assert abs(integral - exact) <= 2e-3 * exact, (integral, exact)
    # and the traction source carries that much load: unit t_x over the domain
    t = np.zeros(P.ndofs)
    t[: P.nnodes] = 1.0
    f = oracle.source_terms(P, psi, t=t)
    assert np.isclose(-h ** dim * f[: P.nnodes].sum(), integral, rtol=1e-12)


def test_body_force_integrates_to_the_volume(oracle_lib):
    oracle = oracle_lib
    P = oracle.Problem(3, (7, 6, 5), 0.2, 1.0, 0.6, 0.5)
    b = np.concatenate([np.full(P.nnodes, v) for v in (0.3, -1.2, 0.7)])
    f = oracle.source_terms(P, np.ones(P.ncells), b=b)
    vol = 6 * 5 * 4 * 0.2 ** 3
    for p, v in enumerate((0.3, -1.2, 0.7)):
        assert np.isclose(P.h ** 3 * f[p * P.nnodes:(p + 1) * P.nnodes].sum(), -v * vol, rtol=1e-13)
