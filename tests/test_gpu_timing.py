"""The library's kernel timer (sbm_time_kernel), which the benchmark's roofline
figures come from: every kernel id runs on small 2D and 3D grids in both
precisions, reports a positive time and the algorithmic bytes and flops its header
states, leaves the grid usable (a solve afterwards still matches the oracle), and
rejects ids and grids it does not cover."""
import ctypes as C

import numpy as np
import pytest

import oracle
from _sbm import cuda, gpu_grid, host, oracle_problem, random_workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2212_02362_gb300 as sbm  # noqa: E402
from paper_2212_02362_gb300 import _capi  # noqa: E402


@pytest.fixture(scope="module")
def built():
    from paper_2212_02362_gb300 import build
    build.build()
    oracle.build()
    return True


def _time(g, kid, flush):
    ms, by, fl = C.c_double(), C.c_double(), C.c_double()
    st = sbm.lib().sbm_time_kernel(g._h, kid, 3, flush, C.byref(ms), C.byref(by), C.byref(fl))
    return st, ms.value, by.value, fl.value


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_every_kernel_id(built, dim, precision):
    wk = random_workload(dim, (45, 37, 21), 404)
    g = gpu_grid(wk, precision=precision)
    nodes = wk.n[0] * wk.n[1] * wk.n[2]
    word = 4 if precision == "mixed" else 8
    ids = [_capi.SBM_K_RESIDUAL64, _capi.SBM_K_JACOBI, _capi.SBM_K_RESIDUAL, _capi.SBM_K_SOURCE,
           _capi.SBM_K_TOPOPT, _capi.SBM_K_FMA64, _capi.SBM_K_FMA32]
    if dim == 2:
        ids.append(_capi.SBM_K_GS)
    for kid in ids:
        for flush in (0, 1):
            st, ms, by, fl = _time(g, kid, flush)
            assert st == _capi.SBM_OK, (kid, sbm.lib().sbm_last_error(g._h))
            assert ms > 0 and fl > 0, kid
            if kid in (_capi.SBM_K_JACOBI, _capi.SBM_K_RESIDUAL, _capi.SBM_K_GS):
                assert by == word * (3 * dim + 1) * nodes, kid
            if kid == _capi.SBM_K_GS:
                assert fl == 190.0 * nodes
    # the grid still solves to the oracle's answer after its work buffers were used
    u = cuda(wk.u0)
    info = g.solve(u, tol=1e-10)
    assert info.converged
    P = oracle_problem(wk)
    r0 = oracle.residual(P, np.maximum(wk.psi, wk.psi_min), wk.f, wk.u0)
    r = oracle.residual(P, np.maximum(wk.psi, wk.psi_min), wk.f, host(u))
    assert oracle.norm_free(P, r) <= 1e-9 * oracle.norm_free(P, r0)


def test_rejects_bad_ids_and_3d_gs(built):
    g3 = gpu_grid(random_workload(3, (17, 17, 9), 405))
    assert _time(g3, _capi.SBM_K_GS, 0)[0] == _capi.SBM_ERR_ARG
    assert _time(g3, 99, 0)[0] == _capi.SBM_ERR_ARG
    assert _time(g3, -1, 0)[0] == _capi.SBM_ERR_ARG
    ms = C.c_double()
    assert sbm.lib().sbm_time_kernel(g3._h, _capi.SBM_K_JACOBI, 0, 0, C.byref(ms), None, None) == _capi.SBM_ERR_ARG
