"""sbm_residual_noalloc: the allocation-free residual + norm gives the oracle's
FP64 residual r = f - K u and norm (and what the grid entry point sbm_residual
gives), on two calls in a row.

The call exists for callers that cannot allocate device memory (a host program
whose device memory belongs to its own pool, code that must not trigger the
implicit synchronisation of cudaMalloc/cudaFree, a process too close to its
memory limit for a grid hierarchy).  Its scratch is a fixed device array inside
the library, so it needs no grid handle.  This file is collected last so that a
run stopping at the first failure has already run every other test, and it also
passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import workloads as W
from _sbm import cuda, gpu_grid, host, random_workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2212_02362_gb300 as sbm  # noqa: E402
from paper_2212_02362_gb300 import _capi  # noqa: E402

CASES = {
    "plate65": lambda: W.plate_hole(65),
    "damage33": lambda: W.damage3d(33),
    "ragged3d": lambda: random_workload(3, (73, 45, 21), 202),
}


@pytest.fixture(scope="module")
def built():
    from paper_2212_02362_gb300 import build
    build.build()
    oracle.build()
    return True


def _node_indexed_psi(wk):
    """Floored cell values at the node slot of their lower corner."""
    nx, ny, nz = wk.n
    ncz = nz - 1 if wk.dim == 3 else 1
    cells = np.maximum(wk.psi, wk.psi_min).reshape(ncz, ny - 1, nx - 1)
    out = np.zeros((nz, ny, nx))
    out[:ncz, : ny - 1, : nx - 1] = cells
    return out.reshape(-1)


def _noalloc(wk, psi_d, f_d, u_d, r_d):
    n = (C.c_int * 3)(*wk.n)
    mod = (C.c_double * 3)(*wk.moduli)
    bits = (C.c_uint * 3)(*wk.dirichlet_bits())
    nrm = C.c_double(-1.0)
    st = sbm.lib().sbm_residual_noalloc(wk.dim, n, wk.h, mod, bits, psi_d.data_ptr(), f_d.data_ptr(),
                                         u_d.data_ptr(), r_d.data_ptr(), C.byref(nrm), None)
    return st, nrm.value


@pytest.mark.parametrize("case", list(CASES))
def test_noalloc_residual_matches_oracle_and_grid_residual(built, case):
    wk = CASES[case]()
    P = oracle.Problem(wk.dim, wk.n, wk.h, *wk.moduli, dirichlet=wk.dirichlet_bits())
    mask = oracle.dirichlet_mask(P)
    u = wk.u0 + W.uniform(31, P.ndofs, -1e-3, 1e-3) * ~mask
    # the plain FP64 definition r = f - K u on free dofs (the oracle) ...
    r_ora = oracle.residual(P, oracle.floor_psi(wk.psi, wk.psi_min), wk.f, u)
    n_ora = oracle.norm_free(P, r_ora)
    # ... and the grid entry point, which runs the same kernel through a handle
    g = gpu_grid(wk)
    f_d, u_d = cuda(wk.f), cuda(u)
    r_grid, n_grid = g.residual(g.finest, f_d, u_d)
    r_grid = host(r_grid)
    psi_d = cuda(_node_indexed_psi(wk))
    for call in range(2):                              # two calls in a row share the scratch
        r_d = torch.full_like(u_d, float("nan"))
        st, nrm = _noalloc(wk, psi_d, f_d, u_d, r_d)
        assert st == _capi.SBM_OK, sbm.lib().sbm_last_error(None)
        r = host(r_d)
        assert np.abs(r - r_ora).max() <= 1e-12 * np.abs(r_ora).max(), call
        assert abs(nrm - n_ora) <= 1e-12 * n_ora, (call, nrm, n_ora)
        assert np.abs(r - r_grid).max() <= 1e-12 * np.abs(r_grid).max(), call
        assert abs(nrm - n_grid) <= 1e-12 * n_grid, (call, nrm, n_grid)


def test_noalloc_rejects_host_pointers(built):
    # a host buffer where device memory is required is refused before any launch
    wk = W.damage3d(17)
    P = oracle.Problem(wk.dim, wk.n, wk.h, *wk.moduli, dirichlet=wk.dirichlet_bits())
    psi_d, f_d, u_d = cuda(_node_indexed_psi(wk)), cuda(wk.f), cuda(wk.u0)
    r_h = np.zeros(P.ndofs)
    n = (C.c_int * 3)(*wk.n)
    mod = (C.c_double * 3)(*wk.moduli)
    bits = (C.c_uint * 3)(*wk.dirichlet_bits())
    nrm = C.c_double(-1.0)
    st = sbm.lib().sbm_residual_noalloc(wk.dim, n, wk.h, mod, bits, psi_d.data_ptr(), f_d.data_ptr(),
                                         u_d.data_ptr(), r_h.ctypes.data_as(C.c_void_p), C.byref(nrm), None)
    assert st == _capi.SBM_ERR_ARG
    assert b"device memory" in sbm.lib().sbm_last_error(None)
    assert np.all(r_h == 0.0) and nrm.value == -1.0
    torch.cuda.synchronize()                           # the context is still usable


def test_noalloc_rejects_grids_beyond_the_scratch(built):
    # a 4097^2 grid needs 128 x 512 stencil blocks, more than the fixed scratch holds;
    # the size check happens before any device work, so small buffers suffice here
    wk = W.plate_hole(17)
    wk.n = (4097, 4097, 1)
    wk.h = 1.0 / 4096
    tiny = torch.zeros(8, dtype=torch.float64, device="cuda")
    st, _ = _noalloc(wk, tiny, tiny, tiny, tiny)
    assert st == _capi.SBM_ERR_ARG
    assert b"fixed scratch" in sbm.lib().sbm_last_error(None)
