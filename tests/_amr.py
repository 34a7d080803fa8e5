"""Helpers for BSAMR tests: level storage, unknown sets and a dense composite
solve built only from the oracle's composite residual."""
import numpy as np

import oracle


def level_coords(A, a):
    """Global level-a coordinates (X, Y, Z index arrays) of level a's storage nodes."""
    P = A.level_problem(a)
    o = A.origin(a)
    k, j, i = np.meshgrid(np.arange(P.n[2]), np.arange(P.n[1]), np.arange(P.n[0]), indexing="ij")
    return (i.reshape(-1) + o[0], j.reshape(-1) + o[1], k.reshape(-1) + o[2])


def level_cell_centres(A, a):
    """Physical centres of level a's storage cells (padding cells included)."""
    P = A.level_problem(a)
    o = A.origin(a)
    ncz = P.n[2] - 1 if P.dim == 3 else 1
    k, j, i = np.meshgrid(np.arange(ncz), np.arange(P.n[1] - 1), np.arange(P.n[0] - 1), indexing="ij")
    h = P.h
    X = (i.reshape(-1) + o[0] + 0.5) * h
    Y = (j.reshape(-1) + o[1] + 0.5) * h
    Z = (k.reshape(-1) + o[2] + 0.5) * h if P.dim == 3 else np.zeros(X.shape)
    return X, Y, Z


def cells_inside_domain(A, a):
    P = A.level_problem(a)
    o = A.origin(a)
    ncz = P.n[2] - 1 if P.dim == 3 else 1
    k, j, i = np.meshgrid(np.arange(ncz), np.arange(P.n[1] - 1), np.arange(P.n[0] - 1), indexing="ij")
    N = A.global_n(a)
    ok = (i + o[0] >= 0) & (i + o[0] < N[0] - 1) & (j + o[1] >= 0) & (j + o[1] < N[1] - 1)
    if P.dim == 3:
        ok &= (k + o[2] >= 0) & (k + o[2] < N[2] - 1)
    return ok.reshape(-1)


def dirichlet_dof(A, a, g, p):
    N = A.global_n(a)
    m = A.base.dirichlet[p]
    for ax in range(A.base.dim):
        if (m >> (2 * ax)) & 1 and g[ax] == 0:
            return True
        if (m >> (2 * ax + 1)) & 1 and g[ax] == N[ax] - 1:
            return True
    return False


def unknowns(A):
    """[(level, flat dof index)] of every owned free dof."""
    out = []
    for a in range(A.nlev):
        P = A.level_problem(a)
        X, Y, Z = level_coords(A, a)
        Nn = P.nnodes
        for n in range(Nn):
            g = (int(X[n]), int(Y[n]), int(Z[n]))
            if not A.owned(a, *g):
                continue
            for p in range(P.dim):
                if not dirichlet_dof(A, a, g, p):
                    out.append((a, p * Nn + n))
    return out


def dense_system(A, psis, fs, us0):
    """The composite operator M (d residual / d unknowns, negated) and the residual
    b of us0, by probing the oracle's (affine) composite residual column by column:
    the composite problem is M x = b for the correction x of the unknowns."""
    unk = unknowns(A)
    r0 = oracle.amr_residual(A, psis, fs, [u.copy() for u in us0])

    def vec(rs):
        return np.array([rs[a][e] for a, e in unk])

    b = vec(r0)
    M = np.zeros((len(unk), len(unk)))
    for col, (a, e) in enumerate(unk):
        ue = [u.copy() for u in us0]
        ue[a][e] += 1.0
        M[:, col] = b - vec(oracle.amr_residual(A, psis, fs, ue))
    return unk, M, b


def dense_solve(A, psis, fs, us0):
    """Solve the composite problem by probing its (affine) residual column by
    column and a numpy dense solve."""
    unk, M, b = dense_system(A, psis, fs, us0)
    us = [u.copy() for u in us0]
    x = np.linalg.solve(M, b)
    for (a, e), v in zip(unk, x):
        us[a][e] += v
    oracle.amr_fill(A, us)
    return us
