"""Pins of the oracle's block-structured refinement (composite problem of the
reflux-free reading of Sec. 2.2): exact ghost interpolation of linear fields,
coarse psi = fine means, every point owned by exactly one level, a patch (or a
nested pair of patches) that covers the whole domain reproduces the uniformly
refined solution with the coarser levels holding its injection (P10), psi of
padding cells beyond the domain is ignored, and the composite problem reproduces
affine displacement fields exactly (patch test through the coarse/fine interface)."""
import numpy as np
import pytest

import oracle
import workloads as W
from _amr import cells_inside_domain, dense_solve, dense_system, dirichlet_dof, level_coords


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


@pytest.mark.parametrize("dim,n0,boxes", [
    (2, 9, [((4, 4), (12, 12)), ((10, 10), (22, 22)), ((22, 22), (42, 42))]),
    (2, 9, [((0, 4), (12, 16)), ((0, 10), (14, 30))]),
    (3, 5, [((2, 2, 2), (6, 6, 6)), ((6, 6, 4), (10, 10, 10))]),
])
def test_every_point_is_owned_by_exactly_one_level(oracle_lib, dim, n0, boxes):
    """Brute force over all levels: a point of the domain that lies in level a's
    box region is owned by exactly one level (the finest whose region contains it)."""
    A = _amr(dim, n0, boxes)
    top = A.nlev - 1
    owners = {}
    region = []
    for a in range(A.nlev):
        X, Y, Z = level_coords(A, a)
        N = A.global_n(a)
        s = 2 ** (top - a)
        for x, y, z in zip(X, Y, Z):
            g = (int(x), int(y), int(z))
            if not all(0 <= g[ax] <= N[ax] - 1 for ax in range(dim)):
                continue
            key = (g[0] * s, g[1] * s, g[2] * s if dim == 3 else 0)
            if A.owned(a, *g):
                owners[key] = owners.get(key, 0) + 1
            if a == 0 or all((A.boxes[a - 1][0][ax] < g[ax] < A.boxes[a - 1][1][ax])
                             or (g[ax] == A.boxes[a - 1][0][ax] == 0)
                             or (g[ax] == A.boxes[a - 1][1][ax] == N[ax] - 1) for ax in range(dim)):
                region.append(key)
    assert region and all(owners.get(k, 0) == 1 for k in region)


def _uniform_fine(dim, nf, bits, psi_cells, f, u):
    Pf = oracle.Problem(dim, (nf,) * dim, 1.0 / (nf - 1), 1.0, 0.6, 0.5, dirichlet=bits)
    return oracle.direct_solve(Pf, psi_cells, f, u)


def _strip(P, v, comps):
    """drop the padding layer of a level array (nodes: comps > 0; cells: comps = 0)"""
    d = P.dim
    sl = (slice(1, -1),) * d
    if comps == 0:
        shape = tuple(n - 1 for n in P.n[::-1][3 - d:])
        return v.reshape(shape)[sl].reshape(-1)
    shape = (comps,) + tuple(P.n[::-1][3 - d:])
    return v.reshape(shape)[(slice(None),) + sl].reshape(-1)


@pytest.mark.parametrize("dim,n0,nest", [(2, 9, 1), (3, 5, 1), (2, 5, 2), (3, 3, 2)])
def test_P10_patches_over_whole_domain_equal_uniform_fine_solution(oracle_lib, dim, n0, nest):
    """One patch (nest = 1) or two nested patches (nest = 2) covering the whole
    domain: the finest level holds the uniformly refined solution and every
    coarser level its injection.  Padding cells beyond the domain carry psi = 5,
    which must not enter the composite problem."""
    nf = (n0 - 1) * 2 ** nest + 1
    boxes = [((0,) * dim, ((n0 - 1) * 2 ** a,) * dim) for a in range(1, nest + 1)]
    bits = (4, 4 | 8, 4) if dim == 2 else (16, 16, 16 | 32)
    A = _amr(dim, n0, boxes, bits=bits)
    rng_psi = lambda X, Y, Z: 0.05 + 0.95 * (0.5 + 0.5 * np.sin(7 * X + 3 * Y + 5 * Z))
    psis = []
    for a in range(A.nlev):
        from _amr import level_cell_centres
        v = rng_psi(*level_cell_centres(A, a))
        if a > 0:
            v = np.where(cells_inside_domain(A, a), v, 5.0)
        psis.append(np.ascontiguousarray(v))
    psis = oracle.amr_coarsen_psi(A, psis)
    us, fs = _zeros(A), _zeros(A)
    Pt = A.level_problem(nest)
    for a in range(A.nlev):
        P = A.level_problem(a)
        X, Y, Z = level_coords(A, a)
        Na = A.global_n(a)
        top = (Y == Na[1] - 1) if dim == 2 else (Z == Na[2] - 1)
        us[a][(dim - 1) * P.nnodes:dim * P.nnodes][top] = 0.01
    fs[nest][:Pt.nnodes] = W.uniform(5, Pt.nnodes, -1, 1)
    sol = dense_solve(A, psis, fs, us)
    ref = _uniform_fine(dim, nf, bits, _strip(Pt, psis[nest], 0), _strip(Pt, fs[nest], dim), _strip(Pt, us[nest], dim))
    scale = np.abs(ref).max()
    assert np.abs(_strip(Pt, sol[nest], dim) - ref).max() <= 1e-11 * scale
    # coarser levels hold the injection of the fine solution
    R = ref.reshape((dim,) + (nf,) * dim)
    for a in range(nest):
        P = A.level_problem(a)
        s = 2 ** (nest - a)
        sub = (slice(None),) + (slice(None, None, s),) * dim
        got = sol[a] if a == 0 else _strip(P, sol[a], dim)
        assert np.abs(got - R[sub].reshape(-1)).max() <= 1e-11 * scale, a


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


@pytest.mark.parametrize("dim,n0,boxes", [
    (2, 9, [((4, 4), (12, 12)), ((10, 10), (22, 22)), ((22, 22), (42, 42))]),
    (2, 9, [((0, 4), (12, 16)), ((0, 10), (14, 30))]),
    (3, 5, [((2, 2, 2), (6, 6, 6)), ((6, 6, 4), (10, 10, 10))]),
])
def test_sampled_composite_residual_equals_full(oracle_lib, dim, n0, boxes):
    """The sampled composite residual (ghost and covered values evaluated on the
    fly) equals the full composite residual at every dof of every level."""
    bits = (1 | 4, 2 | 8, 16) if dim == 3 else (1 | 4, 8)
    A = _amr(dim, n0, boxes, bits=bits + (0,) * (3 - len(bits)))
    psis = oracle.amr_coarsen_psi(A, _psi(A, lambda X, Y, Z: 0.1 + 0.9 * (0.5 + 0.5 * np.cos(5 * X - 2 * Y + 3 * Z))))
    us = [W.uniform(300 + a, A.level_problem(a).ndofs, -1, 1) for a in range(A.nlev)]
    fs = [W.uniform(400 + a, A.level_problem(a).ndofs, -1, 1) for a in range(A.nlev)]
    full = oracle.amr_residual(A, psis, fs, [u.copy() for u in us])
    for a in range(A.nlev):
        P = A.level_problem(a)
        X, Y, Z = level_coords(A, a)
        nodes = np.stack([X, Y, Z], axis=1)
        for p in range(dim):
            got = oracle.amr_residual_at(A, psis, fs, us, np.full(P.nnodes, a), nodes, np.full(P.nnodes, p))
            ref = full[a][p * P.nnodes:(p + 1) * P.nnodes]
            assert np.abs(got - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max()), (a, p)


@pytest.mark.parametrize("dim,n0,boxes,bits", [
    (2, 9, [((4, 4), (12, 12)), ((10, 10), (22, 22))], (4 | 8, 4, 0)),
    (2, 9, [((0, 4), (12, 16))], (1 | 4, 4 | 8, 0)),
    (3, 5, [((2, 2, 2), (6, 6, 6))], (16, 16 | 32, 16)),
])
def test_composite_gradient_matches_central_differences(oracle_lib, dim, n0, boxes, bits):
    """dJ/dpsi of J = g.x (x the composite unknowns) from the adjoint A^T lam = g and
    the per-level cell formula with the coarse-to-fine chain rule, against central
    differences of dense composite solves, for cells on every level: outside the
    patches, under them (whose psi is overwritten by the fine mean: gradient 0) and
    on the fine levels."""
    A = _amr(dim, n0, boxes, bits=bits)
    raw = _psi(A, lambda X, Y, Z: 0.2 + 0.8 * (0.5 + 0.5 * np.sin(6 * X + 4 * Y + 3 * Z)))
    us0, fs = _zeros(A), []
    for a in range(A.nlev):
        P = A.level_problem(a)
        X, Y, Z = level_coords(A, a)
        Na = A.global_n(a)
        top = (Y == Na[1] - 1) if dim == 2 else (Z == Na[2] - 1)
        us0[a][(dim - 1) * P.nnodes:dim * P.nnodes][top] = 0.01
        fs.append(W.uniform(500 + a, P.ndofs, -1, 1))

    def solve(raw_psis):
        psis = oracle.amr_coarsen_psi(A, [p.copy() for p in raw_psis])
        unk, M, b = dense_system(A, psis, fs, us0)
        x = np.linalg.solve(M, b)
        return psis, unk, M, x

    psis, unk, M, x = solve(raw)
    gvec = W.uniform(600, len(unk), -1, 1)
    base = np.array([us0[a][e] for a, e in unk])
    J = lambda xx: float(gvec @ (base + xx))
    lam = np.linalg.solve(M.T, gvec)
    lams = [np.zeros_like(u) for u in us0]
    us = [u.copy() for u in us0]
    for (a, e), v, xv in zip(unk, lam, x):
        lams[a][e] = v
        us[a][e] += xv
    oracle.amr_fill(A, us)
    grads = oracle.amr_dJdpsi(A, us, lams)
    scale = max(np.abs(gg).max() for gg in grads)
    rng = np.random.default_rng(7)
    checked = 0
    for a in range(A.nlev):
        inside = np.nonzero(cells_inside_domain(A, a))[0]
        for c in rng.choice(inside, size=min(4, len(inside)), replace=False):
            eps = 1e-6 * raw[a][c]
            plus = [p.copy() for p in raw]
            minus = [p.copy() for p in raw]
            plus[a][c] += eps
            minus[a][c] -= eps
            fd = (J(solve(plus)[3]) - J(solve(minus)[3])) / (2 * eps)
            assert abs(fd - grads[a][c]) <= 1e-6 * scale, (a, c, fd, grads[a][c])
            checked += 1
    # a coarse cell under the first patch: its psi is overwritten, its gradient is 0
    lo, hi = A.boxes[0]
    C0 = [lo[ax] // 2 for ax in range(dim)] + [0] * (3 - dim)
    P0 = A.level_problem(0)
    cid = C0[0] + (P0.n[0] - 1) * (C0[1] + (P0.n[1] - 1) * C0[2])
    assert grads[0][cid] == 0.0
    assert checked >= 2 * A.nlev



@pytest.mark.parametrize("dim", [2, 3])
def test_composite_residual_is_affine_in_the_owned_values(oracle_lib, dim):
    """The two properties a correction cycle of the composite problem rests on:
    the residual depends on the owned values only (ghosts and covered parents are
    re-derived by the fill), and it is affine in them, r(u + e) = r(u) + r_0(e) with
    r_0 the residual for a zero load (e is zero on the Dirichlet dofs here, as a
    correction is)."""
    boxes = [((2, 2, 2)[:dim], (10, 12, 10)[:dim]), ((6, 8, 6)[:dim], (16, 18, 16)[:dim])]
    A = _amr(dim, 9, boxes, bits=(1, 1 | 4, 1))
    rng = np.random.default_rng(40 + dim)
    psis = _psi(A, lambda X, Y, Z: 0.2 + 0.8 * np.abs(np.sin(7 * X + 3 * Y + 5 * Z)))
    fs = [rng.uniform(-1, 1, A.level_problem(a).ndofs) for a in range(A.nlev)]
    zeros = _zeros(A)
    us = [rng.uniform(-1, 1, A.level_problem(a).ndofs) for a in range(A.nlev)]
    e = [rng.uniform(-1, 1, A.level_problem(a).ndofs) for a in range(A.nlev)]
    nonowned = []
    for a in range(A.nlev):
        P = A.level_problem(a)
        X, Y, Z = level_coords(A, a)
        for n in range(P.nnodes):
            g = (int(X[n]), int(Y[n]), int(Z[n]))
            own = A.owned(a, *g)
            for p in range(dim):
                if own and dirichlet_dof(A, a, g, p):
                    e[a][p * P.nnodes + n] = 0.0
                if not own:
                    nonowned.append((a, p * P.nnodes + n))
    r_u = oracle.amr_residual(A, psis, fs, [u.copy() for u in us])
    r_ue = oracle.amr_residual(A, psis, fs, [u + d for u, d in zip(us, e)])
    r0_e = oracle.amr_residual(A, psis, zeros, [d.copy() for d in e])
    scale = max(np.abs(r).max() for r in r_u)
    for a in range(A.nlev):
        assert np.abs(r_ue[a] - (r_u[a] + r0_e[a])).max() <= 1e-12 * scale, a
    # values off the owned dofs do not enter
    junk = [u.copy() for u in us]
    for a, i in nonowned:
        junk[a][i] += 3.0
    r_junk = oracle.amr_residual(A, psis, fs, junk)
    for a in range(A.nlev):
        assert np.array_equal(r_junk[a], r_u[a]), a


@pytest.mark.parametrize("dim,n0,boxes,bits", [
    (2, 9, [((4, 4), (12, 10))], (4, 4 | 8, 0)),
    (2, 9, [((4, 2), (12, 12)), ((10, 6), (20, 18))], (1 | 4, 4, 0)),
    (2, 9, [((0, 4), (12, 16)), ((0, 10), (14, 30))], (1 | 4, 8, 0)),
    (3, 5, [((2, 2, 2), (6, 6, 6))], (16, 16 | 32, 16)),
    (3, 5, [((2, 2, 2), (6, 6, 6)), ((6, 6, 4), (10, 10, 10))], (16 | 32, 16, 1 | 16)),
])
def test_composite_iteration_reaches_the_dense_composite_solution(oracle_lib, dim, n0, boxes, bits):
    """The oracle's correction iteration (orc_amr_solve) converges to the solution
    of the composite problem: the same values as the dense solve of the probed
    composite system on every dof of every level, and a composite residual, checked
    by the oracle's own residual routine, at the requested tolerance.  Cases: one
    and two nested patches, a patch on the domain boundary, 2D and 3D, random psi
    down to 1e-3, Dirichlet data on several faces, a random load."""
    A = _amr(dim, n0, boxes, bits=bits)
    psis = oracle.amr_coarsen_psi(A, _psi(A, lambda X, Y, Z: np.maximum(
        1e-3, 0.5 + 0.5 * np.sin(7 * X + 3 * Y - 5 * Z) * np.cos(4 * X - 6 * Y + 2 * Z))))
    fs = [W.uniform(500 + a, A.level_problem(a).ndofs, -1, 1) for a in range(A.nlev)]
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
    ref = dense_solve(A, psis, fs, [u.copy() for u in us0])
    us = [u.copy() for u in us0]
    res = oracle.amr_solve(A, psis, fs, us, omega=0.5, tol=1e-13, max_cycles=300)
    assert res.status == 0, (res.status, res.history[-3:])
    scale = max(np.abs(r).max() for r in ref)
    for a in range(A.nlev):
        assert np.abs(us[a] - ref[a]).max() <= 1e-10 * scale, a
    r = oracle.amr_residual(A, psis, fs, [u.copy() for u in us])
    r0 = oracle.amr_residual(A, psis, fs, [u.copy() for u in us0])
    nrm = lambda rs: np.sqrt(sum(float(x @ x) for x in rs))
    assert nrm(r) <= 1e-13 * nrm(r0) * (1 + 1e-9)
