"""Pins of the oracle's composite problem (reflux-free reading of Sec. 2.2) with
several patches per refinement level: patches given as (lo, hi, parent), siblings
apart, each nested in its parent.

  - every point of the domain is owned by exactly one patch (brute force);
  - coarse cells under each child hold the mean of that child's fine cells, the
    other coarse cells keep their values;
  - affine displacement fields are reproduced exactly on every patch;
  - the sampled composite residual equals the full one at every dof;
  - dJ/dpsi through the coarse-to-fine chain equals central differences of dense
    composite solves, on cells of every patch;
  - the correction iteration reaches the dense composite solution;
  - mirror-image boxes on a mirror-symmetric problem give a mirror-symmetric
    solution (each child's data go to and come from its own parent region).
"""
import numpy as np
import pytest

import oracle
import workloads as W
from _amr import cells_inside_domain, dense_solve, dirichlet_dof, level_cell_centres, level_coords

# 2D: base 9^2 (level-1 nodes 17, level-2 nodes 33); two level-1 boxes, one level-2
# box in each of them.  3D: base 5^3, two level-1 slabs on opposite faces.
CASE2 = (2, 9, [((2, 2), (6, 6), 0), ((10, 8), (16, 16), 0), ((6, 6), (10, 10), 1), ((22, 18), (32, 32), 2)])
CASE3 = (3, 5, [((0, 0, 0), (2, 8, 8), 0), ((6, 2, 0), (8, 8, 6), 0)])
CASES = [CASE2, CASE3]


def _amr(dim, n0, boxes, moduli=(1.0, 0.6, 0.5), bits=(0, 0, 0)):
    n = (n0, n0, n0 if dim == 3 else 1)
    P = oracle.Problem(dim, n, 1.0 / (n0 - 1), *moduli, dirichlet=bits)
    return oracle.Amr(P, boxes)


def _zeros(A):
    return [np.zeros(A.level_problem(a).ndofs) for a in range(A.nlev)]


def _psi(A, fn):
    out = []
    for a in range(A.nlev):
        X, Y, Z = level_cell_centres(A, a)
        v = fn(X, Y, Z)
        if a > 0:
            v = np.where(cells_inside_domain(A, a), v, 0.0)
        out.append(np.ascontiguousarray(v, dtype=np.float64))
    return out


def _in_region(A, a, g):
    N = A.global_n(a)
    if a == 0:
        return all(0 <= g[ax] <= N[ax] - 1 for ax in range(A.base.dim))
    lo, hi = A.boxes[a - 1][0], A.boxes[a - 1][1]
    return all((lo[ax] < g[ax] < hi[ax]) or (g[ax] == lo[ax] == 0) or (g[ax] == hi[ax] == N[ax] - 1)
               for ax in range(A.base.dim))


@pytest.mark.parametrize("dim,n0,boxes", CASES)
def test_every_point_is_owned_by_exactly_one_patch(oracle_lib, dim, n0, boxes):
    A = _amr(dim, n0, boxes)
    top = max(A.level(a) for a in range(A.nlev))
    owners, region = {}, []
    for a in range(A.nlev):
        X, Y, Z = level_coords(A, a)
        N = A.global_n(a)
        s = 2 ** (top - A.level(a))
        for x, y, z in zip(X, Y, Z):
            g = (int(x), int(y), int(z))
            if not all(0 <= g[ax] <= N[ax] - 1 for ax in range(dim)):
                continue
            key = (g[0] * s, g[1] * s, g[2] * s if dim == 3 else 0)
            if A.owned(a, *g):
                owners[key] = owners.get(key, 0) + 1
            if _in_region(A, a, g):
                region.append(key)
    assert region and all(owners.get(k, 0) == 1 for k in region)
    # and the base level has points owned by none of the patches
    assert sum(A.owned(0, *map(int, g)) for g in zip(*level_coords(A, 0))) > 0


@pytest.mark.parametrize("dim,n0,boxes", CASES)
def test_coarse_psi_under_each_child_is_its_fine_mean(oracle_lib, dim, n0, boxes):
    A = _amr(dim, n0, boxes)
    psis = _psi(A, lambda X, Y, Z: 0.2 + X + 2 * Y ** 2 + 0.5 * Z)
    before = [p.copy() for p in psis]
    oracle.amr_coarsen_psi(A, psis)
    for a in range(A.nlev):
        Xc, Yc, Zc = level_cell_centres(A, a)
        h = A.level_problem(a).h
        children = [c for c in range(1, A.nlev) if A.parent(c) == a]
        for i, xyz in enumerate(zip(Xc, Yc, Zc)):
            C = [int(np.floor(v / h)) for v in xyz[:dim]]
            under = None
            for c in children:
                lo, hi = A.boxes[c - 1][0], A.boxes[c - 1][1]
                if all(2 * C[ax] >= lo[ax] and 2 * C[ax] + 2 <= hi[ax] for ax in range(dim)):
                    under = c
            if under is None:
                assert psis[a][i] == before[a][i]
                continue
            # mean of the child's 2^d cells (after the child's own coarsening)
            Xf, Yf, Zf = level_cell_centres(A, under)
            hf = A.level_problem(under).h
            sel = np.ones(len(Xf), dtype=bool)
            for ax, v in enumerate((Xf, Yf, Zf)[:dim]):
                f = np.floor(v / hf).astype(int)
                sel &= (f >= 2 * C[ax]) & (f <= 2 * C[ax] + 1)
            assert sel.sum() == 2 ** dim
            assert np.isclose(psis[a][i], psis[under][sel].mean(), rtol=1e-14)


@pytest.mark.parametrize("dim,n0,boxes", CASES)
def test_composite_reproduces_affine_fields(oracle_lib, dim, n0, boxes):
    allf = (1 << (2 * dim)) - 1
    A = _amr(dim, n0, boxes, bits=(allf,) * dim)
    M = np.array([[0.010, 0.004, -0.002], [-0.003, 0.020, 0.005], [0.001, -0.006, 0.015]])[:dim, :dim]
    psis = oracle.amr_coarsen_psi(A, _psi(A, lambda X, Y, Z: np.ones_like(X)))
    us, fs, exact = _zeros(A), _zeros(A), []
    for a in range(A.nlev):
        P = A.level_problem(a)
        X, Y, Z = level_coords(A, a)
        xyz = np.stack([X * P.h, Y * P.h, Z * P.h])[:dim]
        ex = np.concatenate([M[p] @ xyz for p in range(dim)])
        exact.append(ex)
        N = A.global_n(a)
        on_face = np.zeros(P.nnodes, dtype=bool)
        for ax, c in enumerate((X, Y, Z)[:dim]):
            on_face |= (c == 0) | (c == N[ax] - 1)
        us[a][np.tile(on_face, dim)] = ex[np.tile(on_face, dim)]
    sol = dense_solve(A, psis, fs, us)
    for a in range(A.nlev):
        X, Y, Z = level_coords(A, a)
        N = A.global_n(a)
        inside = np.all([(c >= 0) & (c <= n - 1) for c, n in zip((X, Y, Z)[:dim], N)], axis=0)
        assert np.abs(sol[a][np.tile(inside, dim)] - exact[a][np.tile(inside, dim)]).max() <= 1e-12, a


@pytest.mark.parametrize("dim,n0,boxes", CASES)
def test_sampled_composite_residual_equals_full(oracle_lib, dim, n0, boxes):
    bits = (1 | 4, 2 | 8, 16) if dim == 3 else (1 | 4, 8, 0)
    A = _amr(dim, n0, boxes, bits=bits)
    psis = oracle.amr_coarsen_psi(A, _psi(A, lambda X, Y, Z: 0.1 + 0.9 * (0.5 + 0.5 * np.cos(5 * X - 2 * Y + 3 * Z))))
    us = [W.uniform(600 + a, A.level_problem(a).ndofs, -1, 1) for a in range(A.nlev)]
    fs = [W.uniform(700 + a, A.level_problem(a).ndofs, -1, 1) for a in range(A.nlev)]
    full = oracle.amr_residual(A, psis, fs, [u.copy() for u in us])
    for a in range(A.nlev):
        P = A.level_problem(a)
        nodes = np.stack(level_coords(A, a), axis=1)
        for p in range(dim):
            got = oracle.amr_residual_at(A, psis, fs, us, np.full(P.nnodes, a), nodes, np.full(P.nnodes, p))
            ref = full[a][p * P.nnodes:(p + 1) * P.nnodes]
            assert np.abs(got - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max()), (a, p)


def _bc_guess(A, dim):
    us0 = []
    for a in range(A.nlev):
        P = A.level_problem(a)
        X, Y, Z = level_coords(A, a)
        u = np.zeros(P.ndofs)
        for p in range(dim):
            for n in range(P.nnodes):
                if dirichlet_dof(A, a, (int(X[n]), int(Y[n]), int(Z[n])), p):
                    u[p * P.nnodes + n] = 0.01 * (p + 1) + 0.002 * X[n] * P.h
        us0.append(u)
    return us0


@pytest.mark.parametrize("dim,n0,boxes,bits", [CASE2 + ((1 | 4, 4 | 8, 0),), CASE3 + ((16, 16 | 32, 16),)])
def test_composite_iteration_reaches_the_dense_composite_solution(oracle_lib, dim, n0, boxes, bits):
    A = _amr(dim, n0, boxes, bits=bits)
    psis = oracle.amr_coarsen_psi(A, _psi(A, lambda X, Y, Z: np.maximum(
        1e-3, 0.5 + 0.5 * np.sin(7 * X + 3 * Y - 5 * Z) * np.cos(4 * X - 6 * Y + 2 * Z))))
    fs = [W.uniform(800 + a, A.level_problem(a).ndofs, -1, 1) for a in range(A.nlev)]
    us0 = _bc_guess(A, dim)
    ref = dense_solve(A, psis, fs, [u.copy() for u in us0])
    us = [u.copy() for u in us0]
    res = oracle.amr_solve(A, psis, fs, us, omega=0.5, tol=1e-13, max_cycles=300)
    assert res.status == 0, (res.status, res.history[-3:])
    scale = max(np.abs(r).max() for r in ref)
    for a in range(A.nlev):
        assert np.abs(us[a] - ref[a]).max() <= 1e-10 * scale, a


@pytest.mark.parametrize("dim,n0,boxes,bits", [CASE2 + ((4 | 8, 4, 0),), CASE3 + ((16, 16 | 32, 16),)])
def test_composite_gradient_matches_central_differences(oracle_lib, dim, n0, boxes, bits):
    """J = g.x over the composite unknowns; dJ/dpsi from the adjoint of the dense
    composite matrix and the oracle's per-patch cell formula with its coarse-to-fine
    chain, against central differences of dense solves for cells of every patch;
    coarse cells under each child get 0."""
    from _amr import dense_system
    A = _amr(dim, n0, boxes, bits=bits)
    raw = _psi(A, lambda X, Y, Z: 0.2 + 0.8 * (0.5 + 0.5 * np.sin(6 * X + 4 * Y + 3 * Z)))
    us0, fs = _zeros(A), []
    for a in range(A.nlev):
        P = A.level_problem(a)
        X, Y, Z = level_coords(A, a)
        Na = A.global_n(a)
        top = (Y == Na[1] - 1) if dim == 2 else (Z == Na[2] - 1)
        us0[a][(dim - 1) * P.nnodes:dim * P.nnodes][top] = 0.01
        fs.append(W.uniform(900 + a, P.ndofs, -1, 1))

    def solve(raw_psis):
        psis = oracle.amr_coarsen_psi(A, [p.copy() for p in raw_psis])
        unk, M, b = dense_system(A, psis, fs, us0)
        return unk, M, np.linalg.solve(M, b)

    unk, M, x = solve(raw)
    gvec = W.uniform(950, len(unk), -1, 1)
    J = lambda xx: float(gvec @ xx)
    lam = np.linalg.solve(M.T, gvec)
    lams = [np.zeros_like(u) for u in us0]
    us = [u.copy() for u in us0]
    for (a, e), v, xv in zip(unk, lam, x):
        lams[a][e] = v
        us[a][e] += xv
    oracle.amr_fill(A, us)
    grads = oracle.amr_dJdpsi(A, us, lams)
    scale = max(np.abs(gg).max() for gg in grads)
    rng = np.random.default_rng(11)
    checked = 0
    for a in range(A.nlev):
        inside = np.nonzero(cells_inside_domain(A, a))[0]
        for c in rng.choice(inside, size=min(3, len(inside)), replace=False):
            eps = 1e-6 * raw[a][c]
            plus = [p.copy() for p in raw]
            minus = [p.copy() for p in raw]
            plus[a][c] += eps
            minus[a][c] -= eps
            fd = (J(solve(plus)[2]) - J(solve(minus)[2])) / (2 * eps)
            assert abs(fd - grads[a][c]) <= 1e-6 * scale, (a, c, fd, grads[a][c])
            checked += 1
    # a coarse cell under each child of the base: its psi is overwritten, gradient 0
    P0 = A.level_problem(0)
    for c in range(1, A.nlev):
        if A.parent(c) != 0:
            continue
        lo, hi = A.boxes[c - 1][0], A.boxes[c - 1][1]
        C0 = [(lo[ax] + hi[ax]) // 4 for ax in range(dim)] + [0] * (3 - dim)
        assert all(2 * C0[ax] >= lo[ax] and 2 * C0[ax] + 2 <= hi[ax] for ax in range(dim))
        cid = C0[0] + (P0.n[0] - 1) * (C0[1] + (P0.n[1] - 1) * C0[2])
        assert grads[0][cid] == 0.0
    assert checked >= 2 * A.nlev


def test_mirror_boxes_give_a_mirror_symmetric_solution(oracle_lib):
    """psi symmetric about x = 1/2, boxes mirror images, the bottom clamped and the
    top pulled up: u_x is odd and u_y even under x -> 1 - x on every patch."""
    n0 = 9
    boxes = [((2, 4), (6, 12), 0), ((10, 4), (14, 12), 0)]     # level-1 nodes 0..16: x -> 16 - x
    A = _amr(2, n0, boxes, bits=(4 | 8, 4 | 8, 0))
    psis = oracle.amr_coarsen_psi(A, _psi(A, lambda X, Y, Z: 0.2 + 0.8 * np.exp(-((X - 0.5) ** 2) * 9) * (1 + Y)))
    fs = _zeros(A)
    us = _zeros(A)
    for a in range(A.nlev):
        P = A.level_problem(a)
        X, Y, Z = level_coords(A, a)
        top = Y == A.global_n(a)[1] - 1
        us[a][P.nnodes:][top] = 0.01
    res = oracle.amr_solve(A, psis, fs, us, omega=0.5, tol=1e-13, max_cycles=300)
    assert res.status == 0
    P1, P2 = A.level_problem(1), A.level_problem(2)
    n1 = P1.n[0]
    ux1 = us[1][:P1.nnodes].reshape(P1.n[1], n1)
    uy1 = us[1][P1.nnodes:].reshape(P1.n[1], n1)
    ux2 = us[2][:P2.nnodes].reshape(P2.n[1], n1)
    uy2 = us[2][P2.nnodes:].reshape(P2.n[1], n1)
    # patch 1 storage x = 1..7, patch 2 storage x = 9..15: local i <-> n1 - 1 - i
    assert np.allclose(ux2, -ux1[:, ::-1], atol=1e-12) and np.allclose(uy2, uy1[:, ::-1], atol=1e-12)
    assert np.abs(uy1).max() > 1e-4
