"""Pins of the CPU oracle against things other than itself.

Each test ties the oracle to the paper (the cell-placed psi stencil and Jacobi
update of Sec. 2.3, the node-placed counterexample of Sec. 2.3, the material
vector space of Sec. 2.4), to closed forms (exact Q1 integrals, affine patch
solutions, manufactured solutions, Galerkin identities) or to a library routine
(numpy dense solves), so that a dropped term, a wrong sign or index or a
transposed operand in the oracle fails at least one of them.
"""
import itertools

import numpy as np
import pytest

import workloads as W

pytestmark = []


def _prob(oracle, dim, n, h=None, moduli=(1.0, 0.6, 0.5), bits=(0, 0, 0)):
    n = tuple(n)
    if h is None:
        h = 1.0 / (n[0] - 1)
    return oracle.Problem(dim, n, h, *moduli, dirichlet=bits)


def _rand_psi(P, seed, lo=1e-3):
    return W.uniform(seed, P.ncells, lo, 1.0)


# ---------------------------------------------------------------- element

def _closed_form_Ke(dim, h, c11, c12, c44):
    """Exact Q1 element stiffness from products of 1D integrals over [0,1]:
    mass int N_a N_b, stiffness int N_a' N_b', mixed int N_a' N_b, with
    a(u, v) = sum_{j,l} C_{p j q l} int d_j N_a d_l N_b  (FD scaled by h^-d)."""
    M1 = np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])
    S1 = np.array([[1.0, -1.0], [-1.0, 1.0]])
    G1 = np.array([[-0.5, -0.5], [0.5, 0.5]])      # int N_a' N_b (row a differentiated)

    def Cten(i, j, k, l):
        if i == j and k == l:
            return c11 if i == k else c12
        if i != j and ((i == k and j == l) or (i == l and j == k)):
            return c44
        return 0.0

    nc = 1 << dim
    Ke = np.zeros((nc * dim, nc * dim))
    for a in range(nc):
        for b in range(nc):
            ab = [((a >> m) & 1, (b >> m) & 1) for m in range(dim)]
            for j in range(dim):
                for l in range(dim):
                    I = 1.0
                    for m in range(dim):
                        am, bm = ab[m]
                        if m == j and m == l:
                            I *= S1[am, bm]
                        elif m == j:
                            I *= G1[am, bm]
                        elif m == l:
                            I *= G1[bm, am]
                        else:
                            I *= M1[am, bm]
                    # unit-cube integral of the physical gradients: h^(d-2); FD scale h^-d
                    I *= h ** (dim - 2) / h ** dim
                    for p in range(dim):
                        for q in range(dim):
                            Ke[a * dim + p, b * dim + q] += Cten(p, j, q, l) * I
    return Ke


@pytest.mark.parametrize("dim", [2, 3])
def test_element_matrix_closed_form(oracle_lib, dim):
    for moduli, h in [((1.0, 0.6, 0.5), 0.25), (W.iso_cubic(1.0, 0.3), 1.0 / 64), ((2.0, 0.3, 0.9), 0.1)]:
        P = _prob(oracle_lib, dim, (5,) * dim, h=h, moduli=moduli)
        Ke = oracle_lib.element_matrix(P)
        ref = _closed_form_Ke(dim, h, *moduli)
        assert np.allclose(Ke, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


def test_element_energy_of_uniform_strain(oracle_lib):
    """u = E x with symmetric E: u^T K_e u = h^-d * vol * eps:C:eps (exact)."""
    rng = np.random.default_rng(0)
    for dim in (2, 3):
        P = _prob(oracle_lib, dim, (5,) * dim, h=0.5, moduli=(1.3, 0.4, 0.7))
        Ke = oracle_lib.element_matrix(P)
        E = rng.standard_normal((dim, dim))
        E = 0.5 * (E + E.T)
        ue = np.zeros((1 << dim) * dim)
        for a in range(1 << dim):
            x = np.array([((a >> m) & 1) * P.h for m in range(dim)])
            ue[a * dim:(a + 1) * dim] = E @ x
        c11, c12, c44 = 1.3, 0.4, 0.7
        sig = np.zeros((dim, dim))
        for i in range(dim):
            for j in range(dim):
                if i == j:
                    sig[i, i] = c11 * E[i, i] + c12 * (np.trace(E) - E[i, i])
                else:
                    sig[i, j] = 2 * c44 * E[i, j]
        energy = np.sum(sig * E) * P.h ** dim
        assert np.isclose(ue @ Ke @ ue, energy / P.h ** dim, rtol=1e-13)


# ------------------------------------------------------------ P1: 1D reduction

def test_P1_reduces_to_cell_psi_stencil_of_sec_2_3(oracle_lib):
    """psi = psi(x), u = (u(x), 0): at interior nodes row x of K u equals
    -C11 * [ (phi+ - phi-)/dx (u_{i+1}-u_{i-1})/(2dx) + (phi+ + phi-)/2 (u_{i+1}-2u_i+u_{i-1})/dx^2 ],
    the operator whose Jacobi update Sec. 2.3 prints for cell-placed phi; row y is 0."""
    nx, ny = 17, 9
    h = 1.0 / (nx - 1)
    c11, c12, c44 = 1.7, 0.45, 0.6
    P = oracle_lib.Problem(2, (nx, ny), h, c11, c12, c44)
    phi_x = W.uniform(11, nx - 1, 0.0, 1.0)        # phi at x-cells i+1/2, including exact-zero-free values
    phi_x[5] = 0.0                                  # a cell where phi vanishes
    psi = np.tile(phi_x, ny - 1)
    ux = W.uniform(12, nx, -1.0, 1.0)
    N = nx * ny
    u = np.zeros(2 * N)
    u[:N] = np.tile(ux, ny)
    Ku = oracle_lib.apply(P, psi, u).reshape(2, ny, nx)
    for i in range(1, nx - 1):
        pp, pm = phi_x[i], phi_x[i - 1]
        A = ((pp - pm) / h) * ((ux[i + 1] - ux[i - 1]) / (2 * h)) + \
            0.5 * (pp + pm) * (ux[i + 1] - 2 * ux[i] + ux[i - 1]) / h ** 2
        for j in range(1, ny - 1):
            assert np.isclose(Ku[0, j, i], -c11 * A, rtol=1e-12, atol=1e-12 * c11 / h ** 2)
            assert abs(Ku[1, j, i]) <= 1e-12 * c11 / h ** 2


# ------------------------------------------------------ P2, P3, P7: invariants

@pytest.mark.parametrize("dim,n", [(2, (9, 7)), (3, (5, 6, 4))])
def test_P2_symmetry(oracle_lib, dim, n):
    P = _prob(oracle_lib, dim, n, h=0.1, moduli=W.iso_cubic(1.0, 0.3))
    psi = _rand_psi(P, 21)
    u = W.uniform(22, P.ndofs, -1, 1)
    v = W.uniform(23, P.ndofs, -1, 1)
    a = u @ oracle_lib.apply(P, psi, v)
    b = v @ oracle_lib.apply(P, psi, u)
    scale = np.abs(u) @ np.abs(oracle_lib.apply(P, psi, np.abs(v)))
    assert abs(a - b) <= 1e-13 * scale


def _rigid_modes(P):
    X, Y, Z = W.node_coords(P.dim, P.n, P.h)
    N = P.nnodes
    modes = []
    for p in range(P.dim):
        m = np.zeros(P.ndofs)
        m[p * N:(p + 1) * N] = 1.0
        modes.append(m)
    coords = [X, Y, Z]
    for (a, b) in ([(0, 1)] if P.dim == 2 else [(0, 1), (1, 2), (0, 2)]):
        m = np.zeros(P.ndofs)
        m[a * N:(a + 1) * N] = -coords[b]
        m[b * N:(b + 1) * N] = coords[a]
        modes.append(m)
    return modes


@pytest.mark.parametrize("dim,n", [(2, (9, 7)), (3, (5, 6, 4))])
def test_P3_rigid_body_null_space(oracle_lib, dim, n):
    P = _prob(oracle_lib, dim, n, h=0.1, moduli=(1.0, 0.6, 0.5))
    psi = _rand_psi(P, 31, 1e-4)
    K = oracle_lib.assemble_dense(P, psi)
    knorm = np.abs(K).max()
    for m in _rigid_modes(P):
        assert np.abs(K @ m).max() <= 1e-13 * knorm * np.abs(m).max() * 27
    # and K is positive semidefinite with exactly that null space
    ev = np.linalg.eigvalsh(K)
    nrig = 3 if dim == 2 else 6
    assert np.all(ev[nrig:] > 1e-10 * ev[-1])
    assert np.all(np.abs(ev[:nrig]) <= 1e-12 * ev[-1])


def test_P7_vector_space_linearity(oracle_lib):
    """Sec. 2.4: models form a vector space; K and the coarse average are linear in psi."""
    P = _prob(oracle_lib, 3, (9, 9, 9), moduli=(1.0, 0.6, 0.5))
    p1, p2 = _rand_psi(P, 41), _rand_psi(P, 42)
    u = W.uniform(43, P.ndofs, -1, 1)
    a, b = 0.7, -1.9
    lhs = oracle_lib.apply(P, a * p1 + b * p2, u)
    rhs = a * oracle_lib.apply(P, p1, u) + b * oracle_lib.apply(P, p2, u)
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12 * np.abs(rhs).max())
    c = oracle_lib.coarsen_psi(P, a * p1 + b * p2)
    assert np.allclose(c, a * oracle_lib.coarsen_psi(P, p1) + b * oracle_lib.coarsen_psi(P, p2), rtol=1e-13, atol=1e-15)
    # the average of a constant is that constant
    assert np.allclose(oracle_lib.coarsen_psi(P, np.full(P.ncells, 0.37)), 0.37, rtol=1e-15)


def test_coarse_psi_is_cell_mean(oracle_lib):
    P = _prob(oracle_lib, 2, (9, 9))
    psi = _rand_psi(P, 44)
    c = oracle_lib.coarsen_psi(P, psi).reshape(4, 4)
    f = psi.reshape(8, 8)
    assert np.allclose(c, 0.25 * (f[0::2, 0::2] + f[1::2, 0::2] + f[0::2, 1::2] + f[1::2, 1::2]), rtol=1e-15)


# ---------------------------------------------- P4, P5: consistency and order

@pytest.mark.parametrize("dim,n", [(2, 17), (3, 9)])
def test_P4_patch_test(oracle_lib, dim, n):
    """psi = 1 and affine Dirichlet data on every face: the discrete solution is
    the affine field itself, and K annihilates it at interior nodes."""
    nn = (n, n, n if dim == 3 else 1)
    h = 1.0 / (n - 1)
    A = np.array([[0.01, 0.004, -0.002], [-0.003, 0.02, 0.005], [0.001, -0.006, 0.015]])[:dim, :dim]
    shift = np.array([0.1, -0.2, 0.05])[:dim]
    X = W.node_coords(dim, nn, h)
    N = nn[0] * nn[1] * nn[2]
    exact = np.concatenate([sum(A[p, q] * X[q] for q in range(dim)) + shift[p] for p in range(dim)])
    allfaces = (1 << (2 * dim)) - 1
    P = oracle_lib.Problem(dim, nn, h, 1.0, 0.6, 0.5, dirichlet=(allfaces,) * dim)
    psi = np.ones(P.ncells)
    mask = oracle_lib.dirichlet_mask(P)
    u0 = np.where(mask, exact, 0.0)
    f = np.zeros(P.ndofs)
    Ku = oracle_lib.apply(P, psi, exact)
    assert np.abs(Ku[~mask]).max() <= 1e-12 / h ** 2 * np.abs(exact).max()
    res = oracle_lib.mg_solve(P, psi, f, u0, tol=1e-13, max_cycles=100)
    assert res.status == 0
    assert np.abs(res.u - exact).max() <= 1e-11


def _manufactured(dim, n, moduli):
    """u*, and f = -div(C : grad u*) from hand-differentiated closed forms."""
    c11, c12, c44 = moduli
    h = 1.0 / (n - 1)
    nn = (n, n, n if dim == 3 else 1)
    X, Y, Z = W.node_coords(dim, nn, h)
    pi = np.pi
    s, c = np.sin, np.cos
    if dim == 2:
        ux = s(pi * X) * s(pi * Y)
        uy = c(pi * X) * s(2 * pi * Y)
        # second derivatives
        ux_xx = -pi ** 2 * ux
        ux_yy = -pi ** 2 * ux
        ux_xy = pi ** 2 * c(pi * X) * c(pi * Y)
        uy_xx = -pi ** 2 * uy
        uy_yy = -4 * pi ** 2 * uy
        uy_xy = -2 * pi ** 2 * s(pi * X) * c(2 * pi * Y)
        # div sigma: x: c11 ux_xx + c12 uy_xy + c44 (ux_yy + uy_xy)
        fx = -(c11 * ux_xx + c12 * uy_xy + c44 * (ux_yy + uy_xy))
        fy = -(c11 * uy_yy + c12 * ux_xy + c44 * (uy_xx + ux_xy))
        return nn, h, np.concatenate([ux, uy]), np.concatenate([fx, fy])
    ux = s(pi * X) * s(pi * Y) * s(pi * Z)
    uy = c(pi * X) * s(pi * Y) * c(pi * Z)
    uz = s(pi * X) * c(pi * Y) * c(pi * Z)
    # all second derivatives of each component are +-pi^2 times a product of sin/cos
    d = {}
    d["ux", "xx"] = d["ux", "yy"] = d["ux", "zz"] = -pi ** 2 * ux
    d["ux", "xy"] = pi ** 2 * c(pi * X) * c(pi * Y) * s(pi * Z)
    d["ux", "xz"] = pi ** 2 * c(pi * X) * s(pi * Y) * c(pi * Z)
    d["ux", "yz"] = pi ** 2 * s(pi * X) * c(pi * Y) * c(pi * Z)
    d["uy", "xx"] = d["uy", "yy"] = d["uy", "zz"] = -pi ** 2 * uy
    d["uy", "xy"] = -pi ** 2 * s(pi * X) * c(pi * Y) * c(pi * Z)
    d["uy", "xz"] = pi ** 2 * s(pi * X) * s(pi * Y) * s(pi * Z)
    d["uy", "yz"] = -pi ** 2 * c(pi * X) * c(pi * Y) * s(pi * Z)
    d["uz", "xx"] = d["uz", "yy"] = d["uz", "zz"] = -pi ** 2 * uz
    d["uz", "xy"] = -pi ** 2 * c(pi * X) * s(pi * Y) * c(pi * Z)
    d["uz", "xz"] = -pi ** 2 * c(pi * X) * c(pi * Y) * s(pi * Z)
    d["uz", "yz"] = pi ** 2 * s(pi * X) * s(pi * Y) * s(pi * Z)

    def D(comp, a, b):
        key = "".join(sorted(a + b))
        return d["u" + comp, key]

    axes = "xyz"
    f = []
    for i in axes:          # (div sigma)_i = sum_j d_j sigma_ij
        tot = c11 * D(i, i, i)
        for j in axes:
            if j == i:
                continue
            tot = tot + c12 * D(j, i, j) + c44 * (D(i, j, j) + D(j, i, j))
        f.append(-tot)
    return nn, h, np.concatenate([ux, uy, uz]), np.concatenate(f)


@pytest.mark.parametrize("dim,sizes", [(2, (17, 33, 65)), (3, (9, 17))])
def test_P5_manufactured_second_order(oracle_lib, dim, sizes):
    moduli = (1.0, 0.6, 0.5) if dim == 3 else W.iso_cubic(1.0, 0.3)
    errs = []
    for n in sizes:
        nn, h, exact, f = _manufactured(dim, n, moduli)
        allfaces = (1 << (2 * dim)) - 1
        P = oracle_lib.Problem(dim, nn, h, *moduli, dirichlet=(allfaces,) * dim)
        mask = oracle_lib.dirichlet_mask(P)
        u0 = np.where(mask, exact, 0.0)
        res = oracle_lib.mg_solve(P, np.ones(P.ncells), f, u0, tol=1e-12, max_cycles=200)
        assert res.status == 0
        errs.append(np.abs(res.u - exact).max())
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    for r in ratios:
        assert 3.4 < r < 4.6, (errs, ratios)


# ----------------------------------------------------- transfers and Galerkin

def test_prolongation_exact_on_linears_and_R_is_scaled_transpose(oracle_lib):
    for dim, n in ((2, (17, 9)), (3, (9, 9, 17))):
        P = oracle_lib.Problem(dim, n, 0.125, 1.0, 0.6, 0.5)
        Cp = oracle_lib.coarse_problem(P)
        Xc = W.node_coords(dim, Cp.n, Cp.h)
        Xf = W.node_coords(dim, P.n, P.h)
        lin_c = np.concatenate([0.3 + 0.7 * Xc[0] - 0.2 * Xc[1] + 0.5 * Xc[2] * p for p in range(dim)])
        lin_f = np.concatenate([0.3 + 0.7 * Xf[0] - 0.2 * Xf[1] + 0.5 * Xf[2] * p for p in range(dim)])
        assert np.allclose(oracle_lib.prolong_add(P, lin_c, np.zeros(P.ndofs)), lin_f, atol=1e-14)
        # dense P and R
        Pm = np.stack([oracle_lib.prolong_add(P, e, np.zeros(P.ndofs)) for e in np.eye(Cp.ndofs)], axis=1)
        Rm = np.stack([oracle_lib.restrict(P, e) for e in np.eye(P.ndofs)], axis=1)
        assert np.allclose(Rm, Pm.T / 2 ** dim, atol=1e-15)


@pytest.mark.parametrize("dim,n", [(2, (17, 9)), (3, (9, 9, 9))])
def test_galerkin_identity_constant_psi(oracle_lib, dim, n):
    """For constant psi the rediscretised coarse operator equals R K_f P."""
    P = oracle_lib.Problem(dim, n, 0.125, 1.0, 0.6, 0.5)
    Cp = oracle_lib.coarse_problem(P)
    Kf = oracle_lib.assemble_dense(P, np.full(P.ncells, 0.8))
    Kc = oracle_lib.assemble_dense(Cp, np.full(Cp.ncells, 0.8))
    Pm = np.stack([oracle_lib.prolong_add(P, e, np.zeros(P.ndofs)) for e in np.eye(Cp.ndofs)], axis=1)
    RKP = (Pm.T / 2 ** dim) @ Kf @ Pm
    assert np.allclose(RKP, Kc, atol=1e-12 * np.abs(Kc).max())


def test_level_count_rule(oracle_lib):
    cases = {(2, (65, 65)): 5, (3, (129, 129, 129)): 6, (3, (257, 129, 129)): 6, (2, (17, 17)): 3,
             (3, (9, 9, 9)): 2, (3, (5, 5, 5)): 1}
    for (dim, n), L in cases.items():
        assert oracle_lib.num_levels(oracle_lib.Problem(dim, n, 0.1, 1, 0.5, 0.5)) == L


# ------------------------------------------------------------ smoothers

def test_jacobi_matches_dense_definition(oracle_lib):
    P = oracle_lib.Problem(3, (5, 5, 5), 0.25, 1.0, 0.6, 0.5, dirichlet=(16, 16 | 32, 16))
    psi = _rand_psi(P, 51)
    K = oracle_lib.assemble_dense(P, psi)
    mask = oracle_lib.dirichlet_mask(P)
    u = W.uniform(52, P.ndofs, -1, 1)
    f = W.uniform(53, P.ndofs, -1, 1)
    ref = u.copy()
    r = f - K @ u
    ref[~mask] += 0.6 * r[~mask] / np.diag(K)[~mask]
    assert np.allclose(oracle_lib.jacobi_sweep(P, psi, f, u, 0.6), ref, rtol=1e-13, atol=1e-13)
    assert np.allclose(oracle_lib.diagonal(P, psi), np.diag(K), rtol=1e-14)


@pytest.mark.parametrize("dim,n", [(2, (7, 6)), (3, (5, 4, 5))])
def test_multicolour_gs_matches_dense_sequential_sweep(oracle_lib, dim, n):
    """Colour classes do not couple; the sweep equals pointwise Gauss-Seidel on the
    dense matrix visiting colours in order and components x, y[, z] per node."""
    P = oracle_lib.Problem(dim, n, 0.2, 1.0, 0.6, 0.5, dirichlet=(4, 4, 4))
    psi = _rand_psi(P, 61)
    K = oracle_lib.assemble_dense(P, psi)
    mask = oracle_lib.dirichlet_mask(P)
    N = P.nnodes
    nx, ny, nz = P.n
    colour = np.array([(i & 1) + 2 * (j & 1) + (4 * (k & 1) if dim == 3 else 0)
                       for k in range(nz) for j in range(ny) for i in range(nx)])
    for c1 in range(1 << dim):
        idx = np.where(colour == c1)[0]
        for a, b in itertools.combinations(idx, 2):
            for p in range(dim):
                for q in range(dim):
                    assert K[p * N + a, q * N + b] == 0.0
    u = W.uniform(62, P.ndofs, -1, 1)
    f = W.uniform(63, P.ndofs, -1, 1)
    for desc in (False, True):
        ref = u.copy()
        order = range((1 << dim) - 1, -1, -1) if desc else range(1 << dim)
        for c1 in order:
            for node in np.where(colour == c1)[0]:
                for p in range(dim):
                    e = p * N + node
                    if mask[e]:
                        continue
                    ref[e] += (f[e] - K[e] @ ref) / K[e, e]
        got = oracle_lib.gs_sweep(P, psi, f, u, desc)
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_P8_cell_psi_jacobi_stable_node_psi_divergent(oracle_lib):
    """Sec. 2.3: with phi placed at nodes, Jacobi blows up next to a region where
    phi vanishes; with phi in cells it does not.  A 2-node-high strip with u_y held
    fixed reduces the oracle's operator to 1D."""
    nx = 33
    h = 1.0 / (nx - 1)
    c11 = 1.0
    xc = (np.arange(nx - 1) + 0.5) * h
    xn = np.arange(nx) * h
    phi_cell = np.where(np.abs(xc - 0.5) < 0.15, 0.0, 1.0)
    phi_cell = np.maximum(phi_cell, 1e-6)
    phi_node = np.maximum(np.where(np.abs(xn - 0.5) < 0.15, 0.0, 1.0), 1e-6)
    # cell-placed: oracle, u_x Dirichlet at both x ends, u_y Dirichlet everywhere
    P = oracle_lib.Problem(2, (nx, 2), h, c11, 0.3, 0.4, dirichlet=(1 | 2, 1 | 2 | 4 | 8, 0))
    K = oracle_lib.assemble_dense(P, np.tile(phi_cell, 1))
    mask = oracle_lib.dirichlet_mask(P)
    Kf = K[np.ix_(~mask, ~mask)]
    Jc = np.eye(len(Kf)) - (2.0 / 3.0) * Kf / np.diag(Kf)[:, None]
    rho_cell = np.abs(np.linalg.eigvals(Jc)).max()
    # node-placed: the product-rule stencil printed in Sec. 2.3 (A = div(phi C grad))
    A = np.zeros((nx, nx))
    for i in range(1, nx - 1):
        g = (phi_node[i + 1] - phi_node[i - 1]) / (2 * h)
        A[i, i - 1] = c11 * (-g / (2 * h) + phi_node[i] / h ** 2)
        A[i, i + 1] = c11 * (g / (2 * h) + phi_node[i] / h ** 2)
        A[i, i] = -2 * c11 * phi_node[i] / h ** 2
    An = A[1:-1, 1:-1]
    Jn = np.eye(nx - 2) - (2.0 / 3.0) * An / np.diag(An)[:, None]
    rho_node = np.abs(np.linalg.eigvals(Jn)).max()
    assert rho_cell <= 1.0 + 1e-12
    assert rho_node > 10.0


# ----------------------------------------------------- P6: MG vs direct

@pytest.mark.parametrize("smoother", ["jacobi", "gs"])
def test_P6_multigrid_matches_dense_direct(oracle_lib, smoother):
    Wk = W.plate_hole(17)
    P = oracle_lib.Problem(2, Wk.n, Wk.h, *Wk.moduli, dirichlet=Wk.dirichlet_bits())
    psi = oracle_lib.floor_psi(Wk.psi, Wk.psi_min)
    ud = oracle_lib.direct_solve(P, psi, Wk.f, Wk.u0)
    # the oracle's Cholesky against numpy's dense solve of the same free system
    K = oracle_lib.assemble_dense(P, psi)
    mask = oracle_lib.dirichlet_mask(P)
    rhs = (Wk.f - K @ Wk.u0)[~mask]
    un = Wk.u0.copy()
    un[~mask] = np.linalg.solve(K[np.ix_(~mask, ~mask)], rhs)
    assert np.allclose(ud, un, rtol=1e-12, atol=1e-14)
    res = oracle_lib.mg_solve(P, psi, Wk.f, Wk.u0, smoother=smoother, tol=1e-13, max_cycles=300)
    assert res.status == 0
    assert np.linalg.norm(res.u - ud) <= 1e-10 * np.linalg.norm(ud)


def test_mg_3d_matches_direct(oracle_lib):
    Wk = W.damage3d(9)
    P = oracle_lib.Problem(3, Wk.n, Wk.h, *Wk.moduli, dirichlet=Wk.dirichlet_bits())
    psi = oracle_lib.floor_psi(Wk.psi, Wk.psi_min)
    ud = oracle_lib.direct_solve(P, psi, Wk.f, Wk.u0)
    res = oracle_lib.mg_solve(P, psi, Wk.f, Wk.u0, tol=1e-13, max_cycles=300)
    assert res.status == 0
    assert np.linalg.norm(res.u - ud) <= 1e-9 * np.linalg.norm(ud)


# ---------------------------------------------------------- P9: gradient

def test_P9_adjoint_gradient_matches_central_differences(oracle_lib):
    Wk = W.topopt3d(9, 5, 5)
    P = oracle_lib.Problem(3, Wk.n, Wk.h, *Wk.moduli, dirichlet=Wk.dirichlet_bits())
    rho = Wk.rho
    hd = Wk.h ** 3

    def J_of(r):
        psi, _ = oracle_lib.simp(r, Wk.psi_min)
        u = oracle_lib.direct_solve(P, psi, Wk.f, Wk.u0)
        Ku = oracle_lib.apply(P, psi, u)
        return hd * (2 * Wk.f @ u - u @ Ku)    # stationary form of J = h^d f.u

    psi, dpsi = oracle_lib.simp(rho, Wk.psi_min)
    u = oracle_lib.direct_solve(P, psi, Wk.f, Wk.u0)
    mask = oracle_lib.dirichlet_mask(P)
    lam = oracle_lib.direct_solve(P, psi, np.where(mask, 0.0, hd * Wk.f), np.zeros(P.ndofs))
    g = oracle_lib.dJdpsi(P, u, lam) * dpsi
    assert np.all(oracle_lib.dJdpsi(P, u, lam) <= 1e-15)   # compliance never rises with stiffness
    cells = (W.uniform(4999, 32) * P.ncells).astype(int)
    eps = 1e-6
    for c in cells:
        rp, rm = rho.copy(), rho.copy()
        rp[c] += eps
        rm[c] -= eps
        fd = (J_of(rp) - J_of(rm)) / (2 * eps)
        assert abs(fd - g[c]) <= 1e-5 * np.abs(g).max(), (c, fd, g[c])


def test_mg_converges_on_plate_hole(oracle_lib):
    Wk = W.plate_hole(65)
    P = oracle_lib.Problem(2, Wk.n, Wk.h, *Wk.moduli, dirichlet=Wk.dirichlet_bits())
    psi = oracle_lib.floor_psi(Wk.psi, Wk.psi_min)
    res = oracle_lib.mg_solve(P, psi, Wk.f, Wk.u0, tol=1e-10, max_cycles=500)
    assert res.status == 0
    assert res.cycles < 200
    assert np.all(np.diff(res.history) < 0)


@pytest.mark.parametrize("dim,n,bits", [(2, (9, 7, 1), (1 | 8, 4, 0)), (3, (5, 6, 7), (16 | 2, 32, 1 | 4 | 8))])
def test_norm_free_is_the_2norm_over_free_dofs(oracle_lib, dim, n, bits):
    """The residual norm of the stopping rule (D6b): the Euclidean norm over the
    dofs that carry no Dirichlet condition.  The mask is built here from the face
    numbering (0:-x 1:+x 2:-y 3:+y 4:-z 5:+z) alone, and huge values planted on the
    Dirichlet dofs must not count."""
    oracle = oracle_lib
    P = _prob(oracle, dim, n, bits=bits)
    r = W.uniform(91, P.ndofs, -1.0, 1.0)
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    on_face = [i == 0, i == n[0] - 1, j == 0, j == n[1] - 1, k == 0, k == n[2] - 1]
    mask = np.zeros((dim,) + i.shape, dtype=bool)
    for p in range(dim):
        for f in range(2 * dim):
            if bits[p] >> f & 1:
                mask[p] |= on_face[f]
    mask = mask.reshape(-1)
    assert mask.any() and not mask.all()
    r[mask] = 1e6
    assert np.isclose(oracle.norm_free(P, r), np.linalg.norm(r[~mask]), rtol=1e-14, atol=0)
