"""Pins of the oracle's product-rule operators (Sec. 2.3): the literal strong form
div(psi C grad u) = psi C : grad grad u + grad psi . C grad u by centred
differences, with psi at nodes (the node-placed operator) or in cells averaged to
the nodes (the cell-placed update).

Each is tied to something other than itself: the node-placed form reduces on a
strip to the 1D stencil printed in Sec. 2.3; the cell-placed form reduces to the
conservative flux form, i.e. to the cell-flux operator of the solver; both are
second-order consistent with the analytic div(psi C grad u) of smooth fields in 2D
and 3D; for constant psi they coincide; and (P8 in 2D) damped Jacobi on the
node-placed form diverges next to a region where psi vanishes while on the
cell-placed form it does not.
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


def _strip(oracle, nx, bits=(1 | 2 | 4 | 8, 1 | 2 | 4 | 8, 0)):
    h = 1.0 / (nx - 1)
    return oracle.Problem(2, (nx, 3), h, 1.3, 0.5, 0.4, dirichlet=bits), h


def test_node_placed_form_reduces_to_the_printed_1d_stencil(oracle_lib):
    """psi = psi(x) at nodes, u = (u(x), 0): the x rows of the middle line are minus
    C11 times the node-placed operator printed in Sec. 2.3 and the y rows vanish."""
    oracle = oracle_lib
    nx = 21
    P, h = _strip(oracle, nx)
    x = np.arange(nx) * h
    phi = 0.2 + np.exp(np.sin(5 * x))
    ux = np.cos(3 * x) + x ** 2
    N = P.nnodes
    psi = np.tile(phi, 3)
    u = np.zeros(P.ndofs)
    u[:N] = np.tile(ux, 3)
    Ku = oracle.apply_product(P, oracle.NODE_PSI, psi, u)
    for i in range(1, nx - 1):
        printed = P.c11 * ((phi[i + 1] - phi[i - 1]) / (2 * h) * (ux[i + 1] - ux[i - 1]) / (2 * h)
                           + phi[i] * (ux[i + 1] - 2 * ux[i] + ux[i - 1]) / h ** 2)
        assert np.isclose(Ku[nx + i], -printed, rtol=1e-13, atol=1e-10)
        assert abs(Ku[N + nx + i]) <= 1e-10 * abs(printed) + 1e-9


def test_cell_placed_form_reduces_to_the_flux_form(oracle_lib):
    """psi = psi(x) in cells, u = (u(x), 0): the x rows of the middle line are the
    conservative flux form C11 [phi_{+}(u_{i+1}-u_i) - phi_{-}(u_i-u_{i-1})]/h^2 (with
    the solver's sign), the same rows the cell-flux operator gives."""
    oracle = oracle_lib
    nx = 21
    P, h = _strip(oracle, nx)
    xc = (np.arange(nx - 1) + 0.5) * h
    phic = 0.1 + np.exp(np.cos(4 * xc))
    x = np.arange(nx) * h
    ux = np.sin(2 * x) + 0.3 * x ** 3
    N = P.nnodes
    psi = np.tile(phic, 2)
    u = np.zeros(P.ndofs)
    u[:N] = np.tile(ux, 3)
    Ku = oracle.apply_product(P, oracle.CELL_PSI, psi, u)
    Kq1 = oracle.apply(P, psi, u)
    for i in range(1, nx - 1):
        flux = P.c11 * (phic[i] * (ux[i + 1] - ux[i]) - phic[i - 1] * (ux[i] - ux[i - 1])) / h ** 2
        assert np.isclose(Ku[nx + i], -flux, rtol=1e-12, atol=1e-9)
        assert np.isclose(Ku[nx + i], Kq1[nx + i], rtol=1e-12, atol=1e-9)
        assert abs(Ku[N + nx + i]) <= 1e-9


def _manufactured(dim, n, placement):
    """Max error at interior nodes of the product-rule K u against the analytic
    -div(psi C grad u) for psi = 1 + 0.5 sin(2x + y - z) and u_q = sin(k_q . x)."""
    import oracle
    h = 1.0 / (n - 1)
    nn = (n, n, n if dim == 3 else 1)
    c11, c12, c44 = 1.0, 0.6, 0.5
    P = oracle.Problem(dim, nn, h, c11, c12, c44)
    C = _cubicC(c11, c12, c44)
    kv = np.array([[1.1, 0.7, 0.9], [0.6, 1.3, 0.8], [0.9, 0.5, 1.2]])[:dim, :dim] * np.pi
    coords = np.meshgrid(*[np.arange(m) * h for m in nn[:dim]][::-1], indexing="ij")[::-1]   # x fastest
    X = [c.reshape(-1) for c in coords]
    a = np.array([2.0, 1.0, -1.0])[:dim]
    arg = sum(a[i] * X[i] for i in range(dim))
    psi_n = 1 + 0.5 * np.sin(arg)
    dpsi = [0.5 * a[i] * np.cos(arg) for i in range(dim)]
    u = np.concatenate([np.sin(sum(kv[q, i] * X[i] for i in range(dim))) for q in range(dim)])
    exact = np.zeros(P.ndofs)
    N = P.nnodes
    for p in range(dim):
        s = np.zeros(N)
        for q in range(dim):
            ph = sum(kv[q, i] * X[i] for i in range(dim))
            for aa in range(dim):
                for b in range(dim):
                    Cv = C(p, aa, q, b)
                    if Cv == 0.0:
                        continue
                    s += Cv * (dpsi[aa] * kv[q, b] * np.cos(ph) - psi_n * kv[q, aa] * kv[q, b] * np.sin(ph))
        exact[p * N:(p + 1) * N] = -s
    if placement == oracle.NODE_PSI:
        psi = psi_n
    else:
        cc = np.meshgrid(*[(np.arange(m - 1) + 0.5) * h for m in nn[:dim]][::-1], indexing="ij")[::-1]
        Xc = [c.reshape(-1) for c in cc]
        psi = 1 + 0.5 * np.sin(sum(a[i] * Xc[i] for i in range(dim)))
    Ku = oracle.apply_product(P, placement, psi, u)
    inner = np.ones(nn[::-1], dtype=bool)
    inner[(slice(1, -1),) * 0] = True
    m = np.zeros(nn[::-1], dtype=bool)
    if dim == 3:
        m[2:-2, 2:-2, 2:-2] = True
    else:
        m[:, 2:-2, 2:-2] = True
    mask = np.tile(m.reshape(-1), dim)
    return np.abs(Ku - exact)[mask].max() / np.abs(exact).max()


@pytest.mark.parametrize("dim,sizes", [(2, (17, 33, 65)), (3, (9, 17, 33))])
@pytest.mark.parametrize("which", ["node", "cell"])
def test_product_forms_are_second_order_consistent(oracle_lib, dim, sizes, which):
    placement = oracle_lib.NODE_PSI if which == "node" else oracle_lib.CELL_PSI
    errs = [_manufactured(dim, n, placement) for n in sizes]
    rates = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(3.2 < r < 4.8 for r in rates), (errs, rates)


def test_node_and_cell_placed_forms_coincide_for_constant_psi(oracle_lib):
    oracle = oracle_lib
    P = oracle.Problem(3, (7, 6, 5), 0.2, 1.0, 0.6, 0.5)
    u = W.uniform(11, P.ndofs, -1, 1)
    a = oracle.apply_product(P, oracle.NODE_PSI, np.full(P.nnodes, 0.7), u)
    b = oracle.apply_product(P, oracle.CELL_PSI, np.full(P.ncells, 0.7), u)
    assert np.allclose(a, b, rtol=1e-13, atol=1e-12)
    assert np.abs(a).max() > 1.0


def _jacobi_radius(oracle, P, placement, psi, omega=2.0 / 3.0):
    """Spectral radius of the damped-Jacobi iteration matrix of the product-rule form
    on the interior free dofs (its columns probed with unit vectors)."""
    mask = oracle.dirichlet_mask(P)
    N = P.nnodes
    nn = P.n
    interior = np.zeros(nn[::-1], dtype=bool)
    interior[..., 1:-1, 1:-1] = True
    interior = np.tile(interior.reshape(-1), P.dim) & ~mask
    idx = np.nonzero(interior)[0]
    K = np.zeros((len(idx), len(idx)))
    for c, e in enumerate(idx):
        v = np.zeros(P.ndofs)
        v[e] = 1.0
        K[:, c] = oracle.apply_product(P, placement, psi, v)[idx]
    D = oracle.diagonal_product(P, placement, psi)[idx]
    J = np.eye(len(idx)) - omega * K / D[:, None]
    return np.abs(np.linalg.eigvals(J)).max()


def test_P8_in_2d_node_placed_jacobi_diverges_cell_placed_does_not(oracle_lib):
    """Sec. 2.3 in 2D: psi vanishes (1e-6) in a disc; with psi at nodes the damped
    Jacobi iteration of the product-rule form has spectral radius far above 1 (the
    nodes at the rim of the support), with psi in cells it stays below 1."""
    oracle = oracle_lib
    n = 17
    h = 1.0 / (n - 1)
    allf = 1 | 2 | 4 | 8
    P = oracle.Problem(2, (n, n), h, 1.0, 0.4, 0.3, dirichlet=(allf, allf, 0))
    x = np.arange(n) * h
    Xn, Yn = np.meshgrid(x, x)
    xc = (np.arange(n - 1) + 0.5) * h
    Xc, Yc = np.meshgrid(xc, xc)
    void = lambda X, Y: np.hypot(X - 0.5, Y - 0.5) < 0.22
    psi_node = np.where(void(Xn, Yn), 1e-6, 1.0).reshape(-1)
    psi_cell = np.where(void(Xc, Yc), 1e-6, 1.0).reshape(-1)
    rn = _jacobi_radius(oracle, P, oracle.NODE_PSI, psi_node)
    rc = _jacobi_radius(oracle, P, oracle.CELL_PSI, psi_cell)
    assert rn > 10.0, rn
    assert rc < 1.0, rc
