"""Pins of the oracle's block-structured refinement (composite problem of the
reflux-free reading of Sec. 2.2): exact ghost interpolation of linear fields,
coarse psi = fine means, a patch that covers the whole domain reproduces the
uniformly refined solution (P10), and the composite problem reproduces affine
displacement fields exactly (patch test through the coarse/fine interface)."""
import numpy as np
import pytest

import oracle
import workloads as W
from _amr import cells_inside_domain, dense_solve, level_coords


def _amr(dim, n0, boxes, moduli=(1.0, 0.6, 0.5), bits=(0, 0, 0)):
    n = (n0, n0, n0 if dim == 3 else 1)
    P = oracle.Problem(dim, n, 1.0 / (n0 - 1), *moduli, dirichlet=bits)
    return oracle.Amr(P, boxes)


def _zeros(A):
    return [np.zeros(A.level_problem(a).ndofs) for a in range(A.nlev)]


def _psi(A, fn):
    out = []
    for a in range(A.nlev):
        from _amr import level_cell_centres
        X, Y, Z = level_cell_centres(A, a)
        v = fn(X, Y, Z)
        if a > 0:
            v = np.where(cells_inside_domain(A, a), v, 0.0)
        out.append(np.ascontiguousarray(v, dtype=np.float64))
    return out


@pytest.mark.parametrize("dim", [2, 3])
def test_ghost_fill_is_exact_for_linear_fields(oracle_lib, dim):
    boxes = [((4, 4, 4)[:dim], (12, 10, 12)[:dim]), ((10, 10, 10)[:dim], (20, 16, 22)[:dim])]
    A = _amr(dim, 9, boxes)
    us = _zeros(A)
    lin = lambda X, Y, Z, p: 0.3 + 0.7 * X - 0.2 * Y + (0.5 * Z if dim == 3 else 0) + p
    for a in range(A.nlev):
        P = A.level_problem(a)
        X, Y, Z = level_coords(A, a)
        h = P.h
        inside = np.all([(c >= 0) & (c <= N - 1) for c, N in zip((X, Y, Z), A.global_n(a))], axis=0)
        owned = np.array([A.owned(a, int(x), int(y), int(z)) for x, y, z in zip(X, Y, Z)])
        for p in range(dim):   # linear on owned nodes, garbage on ghosts
            us[a][p * P.nnodes:(p + 1) * P.nnodes] = np.where(inside & owned, lin(X * h, Y * h, Z * h, p), 7.0)
    oracle.amr_fill(A, us)
    for a in range(1, A.nlev):
        P = A.level_problem(a)
        X, Y, Z = level_coords(A, a)
        h = P.h
        inside = np.all([(c >= 0) & (c <= N - 1) for c, N in zip((X, Y, Z), A.global_n(a))], axis=0)
        for p in range(dim):
            got = us[a][p * P.nnodes:(p + 1) * P.nnodes]
            ghost = np.array([not A.owned(a, int(x), int(y), int(z)) for x, y, z in zip(X, Y, Z)]) & inside
            assert np.allclose(got[ghost], lin(X * h, Y * h, Z * h, p)[ghost], atol=1e-14)


def test_coarse_psi_under_patch_is_fine_mean(oracle_lib):
    A = _amr(2, 9, [((4, 4), (12, 12))])
    psis = _psi(A, lambda X, Y, Z: 0.2 + X + 2 * Y ** 2)
    before = psis[0].copy()
    oracle.amr_coarsen_psi(A, psis)
    c = psis[0].reshape(8, 8)
    f = psis[1].reshape(10, 10)                 # fine cells [3, 12] (one padding cell per side)
    for J in range(8):
        for I in range(8):
            if 4 <= 2 * I and 2 * I + 2 <= 12 and 4 <= 2 * J and 2 * J + 2 <= 12:
                li, lj = 2 * I - 3, 2 * J - 3
                ref = 0.25 * (f[lj, li] + f[lj, li + 1] + f[lj + 1, li] + f[lj + 1, li + 1])
                assert np.isclose(c[J, I], ref, rtol=1e-15)
            else:
                assert c[J, I] == before.reshape(8, 8)[J, I]


@pytest.mark.parametrize("dim,n0", [(2, 9), (3, 5)])
def test_P10_patch_over_whole_domain_equals_uniform_fine_solution(oracle_lib, dim, n0):
    nf = 2 * (n0 - 1) + 1
    bits = (4, 4 | 8, 4) if dim == 2 else (16, 16, 16 | 32)
    A = _amr(dim, n0, [((0,) * dim, (nf - 1,) * dim)], bits=bits)
    rng_psi = lambda X, Y, Z: 0.05 + 0.95 * (0.5 + 0.5 * np.sin(7 * X + 3 * Y + 5 * Z))
    psis = oracle.amr_coarsen_psi(A, _psi(A, rng_psi))
    us, fs = _zeros(A), _zeros(A)
    # Dirichlet data on the fine level (top face pulled), load on the fine level
    P1 = A.level_problem(1)
    X, Y, Z = level_coords(A, 1)
    top = (Y == nf - 1) if dim == 2 else (Z == nf - 1)
    us[1][(dim - 1) * P1.nnodes:dim * P1.nnodes][top] = 0.01
    fs[1][:P1.nnodes] = W.uniform(5, P1.nnodes, -1, 1)
    sol = dense_solve(A, psis, fs, us)
    # uniform fine problem on the same nodes (strip the padding)
    Pf = oracle.Problem(dim, (nf,) * dim, 1.0 / (nf - 1), 1.0, 0.6, 0.5, dirichlet=bits)
    sl = (slice(1, -1),) * dim
    def strip(v, comps):
        shape = (comps,) + tuple(P1.n[::-1][3 - dim:])
        return v.reshape(shape)[(slice(None),) + sl[::-1]].reshape(-1)
    cells = psis[1].reshape(tuple(n - 1 for n in P1.n[::-1][3 - dim:]))[sl[::-1]].reshape(-1)
    ref = oracle.direct_solve(Pf, cells, strip(fs[1], dim), strip(us[1], dim))
    assert np.abs(strip(sol[1], dim) - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("dim,n0,boxes", [
    (2, 9, [((4, 4), (12, 10))]),
    (2, 9, [((4, 2), (12, 12)), ((10, 6), (20, 18))]),
    (3, 5, [((2, 2, 2), (6, 6, 6))]),
])
def test_composite_reproduces_affine_fields(oracle_lib, dim, n0, boxes):
    """psi = 1, affine Dirichlet data on every face, no load: the composite solution
    is the affine field on every level (exactness of the fine and coarse equations
    and of the interface interpolation for linear fields)."""
    allf = (1 << (2 * dim)) - 1
    A = _amr(dim, n0, boxes, bits=(allf,) * dim)
    Amat = np.array([[0.010, 0.004, -0.002], [-0.003, 0.020, 0.005], [0.001, -0.006, 0.015]])[:dim, :dim]
    psis = oracle.amr_coarsen_psi(A, _psi(A, lambda X, Y, Z: np.ones_like(X)))
    us, fs = _zeros(A), _zeros(A)
    exact = []
    for a in range(A.nlev):
        P = A.level_problem(a)
        X, Y, Z = level_coords(A, a)
        xyz = np.stack([X * P.h, Y * P.h, Z * P.h])[:dim]
        ex = np.concatenate([Amat[p] @ xyz for p in range(dim)])
        exact.append(ex)
        N = A.global_n(a)
        on_face = np.zeros(P.nnodes, dtype=bool)
        for ax, c in enumerate((X, Y, Z)[:dim]):
            on_face |= (c == 0) | (c == N[ax] - 1)
        for p in range(dim):
            us[a][p * P.nnodes:(p + 1) * P.nnodes][on_face] = ex[p * P.nnodes:(p + 1) * P.nnodes][on_face]
    sol = dense_solve(A, psis, fs, us)
    for a in range(A.nlev):
        P = A.level_problem(a)
        X, Y, Z = level_coords(A, a)
        N = A.global_n(a)
        inside = np.all([(c >= 0) & (c <= n - 1) for c, n in zip((X, Y, Z)[:dim], N)], axis=0)
        mask = np.tile(inside, dim)
        assert np.abs(sol[a][mask] - exact[a][mask]).max() <= 1e-12
