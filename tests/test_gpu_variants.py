"""The operator variants of Sec. 2.3 on the GPU (sbm_apply_product,
sbm_jacobi_product) against the oracle's plain restatement, and the paper's
stability claim reproduced through the CUDA kernels (P8): damped Jacobi on the
node-placed product-rule form diverges next to a region where psi vanishes, while
on the cell-placed form, and on the solver's cell-flux operator, it does not.
"""
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

NODE, CELL = _capi.SBM_OP_PRODUCT_NODE, _capi.SBM_OP_PRODUCT_CELL


@pytest.fixture(scope="module")
def built():
    from paper_2212_02362_gb300 import build
    build.build()
    oracle.build()
    return True


def _grid(dim, n, h, moduli, bits):
    g = sbm.Grid(dim, n, h)
    g.set_moduli(sbm.SBM_CUBIC, moduli)
    faces = ["-x", "+x", "-y", "+y", "-z", "+z"][: 2 * dim]
    for p in range(dim):
        for fi, face in enumerate(faces):
            if bits[p] >> fi & 1:
                g.set_bc(face, p, sbm.SBM_DIRICHLET_FROM_U)
    return g


CASES = [(2, (37, 29, 1), (1 | 4, 2 | 8, 0)), (3, (17, 13, 11), (1 | 16, 4 | 32, 2 | 8))]


@pytest.mark.parametrize("dim,n,bits", CASES)
@pytest.mark.parametrize("variant", [NODE, CELL])
def test_product_apply_and_jacobi_parity(built, dim, n, bits, variant):
    h = 1.0 / (n[0] - 1)
    moduli = (1.0, 0.6, 0.5)
    P = oracle.Problem(dim, n, h, *moduli, dirichlet=bits)
    g = _grid(dim, n, h, moduli, bits)
    psi = W.uniform(40 + dim, P.nnodes if variant == NODE else P.ncells, 1e-3, 1.0)
    u = W.uniform(50 + dim, P.ndofs, -1, 1)
    f = W.uniform(60 + dim, P.ndofs, -1, 1)
    ref = oracle.apply_product(P, variant, psi, u)
    got = host(g.apply_product(variant, cuda(psi), cuda(u)))
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    ref = u.copy()
    for _ in range(3):
        ref = oracle.jacobi_product(P, variant, psi, f, ref, 0.6)
    got = host(g.jacobi_product(variant, cuda(psi), cuda(f), cuda(u), omega=0.6, sweeps=3))
    assert np.abs((got - u) - (ref - u)).max() <= 1e-11 * np.abs(ref - u).max()


@pytest.mark.parametrize("dim,n", [(2, 65), (3, 33)])
def test_P8_node_placed_jacobi_diverges_cell_placed_does_not(built, dim, n):
    """psi = 1e-6 inside a disc (sphere) of radius 0.22, 1 outside; homogeneous
    Dirichlet data on every face, no load, a random start: 60 damped Jacobi sweeps
    (omega = 2/3) blow up on the node-placed form and decay on the cell-placed form
    and on the solver's cell-flux operator."""
    h = 1.0 / (n - 1)
    nn = (n, n, n if dim == 3 else 1)
    allf = (1 << (2 * dim)) - 1
    bits = (allf,) * dim + (0,) * (3 - dim)
    moduli = (1.0, 0.4, 0.3)
    P = oracle.Problem(dim, nn, h, *moduli, dirichlet=bits)
    g = _grid(dim, nn, h, moduli, bits)
    node_xyz = W.node_coords(dim, nn, h)
    cell_xyz = W.cell_centres(dim, nn, h)

    def void(X):
        return np.sqrt(sum((X[a] - 0.5) ** 2 for a in range(dim))) < 0.22

    psi_node = np.where(void(node_xyz), 1e-6, 1.0).reshape(-1)
    psi_cell = np.where(void(cell_xyz), 1e-6, 1.0).reshape(-1)
    mask = oracle.dirichlet_mask(P)
    u0 = np.where(mask, 0.0, W.uniform(70, P.ndofs, -1, 1))
    f = np.zeros(P.ndofs)
    n0 = np.linalg.norm(u0)
    un = host(g.jacobi_product(NODE, cuda(psi_node), cuda(f), cuda(u0), omega=2.0 / 3.0, sweeps=60))
    uc = host(g.jacobi_product(CELL, cuda(psi_cell), cuda(f), cuda(u0), omega=2.0 / 3.0, sweeps=60))
    g.set_psi(cuda(psi_cell), 1e-6)
    g.set_source(cuda(f))
    uf = cuda(u0)
    for _ in range(60):
        uf = g.smooth(g.finest, cuda(f), uf, "jacobi", 2.0 / 3.0)
    nn_, nc_, nf_ = np.linalg.norm(un), np.linalg.norm(uc), float(torch.linalg.norm(uf))
    assert (not np.isfinite(nn_)) or nn_ > 1e6 * n0, nn_
    assert nc_ < n0 and nf_ < n0, (nc_, nf_, n0)
