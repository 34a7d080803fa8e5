"""Error paths of the library, exercised without a GPU fault, a hang or real memory
pressure:
  - out of device memory, by the library's allocation cap (sbm_set_alloc_limit): a
    grid creation and a patch addition fail with SBM_ERR_OOM, free what they
    allocated, and leave the process (and an existing grid) usable;
  - a bounded wait that runs out: the grid barriers of the bottom-level inversion
    (one cooperative launch) given a one-poll limit (sbm_set_wait_limit) time out,
    every block leaves the launch, the solve returns SBM_ERR_CUDA, and the same grid
    then solves correctly with the default bound;
  - refinement boxes that are not nested or not even-cornered are refused.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from _sbm import cuda, gpu_grid, host, oracle_problem

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


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_allocation_cap_gives_oom_and_frees_the_partial_grid(built):
    wk = W.damage3d(65)
    free0 = _free_bytes()
    sbm.lib().sbm_set_alloc_limit(8 << 20)          # far below a 65^3 hierarchy
    try:
        with pytest.raises(sbm.SBMError) as e:
            sbm.Grid(3, wk.n, wk.h, precision="mixed")
        assert e.value.status == _capi.SBM_ERR_OOM
        assert b"out of memory" in sbm.lib().sbm_last_error(None)
    finally:
        sbm.lib().sbm_set_alloc_limit(0)
    assert abs(_free_bytes() - free0) <= (16 << 20)  # nothing of the failed grid is kept
    # without the cap the same grid is created and solves
    g = gpu_grid(wk, precision="mixed")
    u = cuda(wk.u0)
    assert g.solve(u, omega=wk.omega).converged


def test_allocation_cap_refuses_a_patch_and_keeps_the_grid(built):
    wk = W.voids_amr(2, 17, 1, count=2, rmin=0.1, rmax=0.2)
    g = sbm.Grid(2, wk.n, wk.h)
    g.set_moduli(sbm.SBM_CUBIC, wk.moduli)
    for face, comp, _ in wk.bcs:
        g.set_bc(face, comp, sbm.SBM_DIRICHLET_FROM_U)
    g.set_psi(cuda(wk.level_psi(0)), wk.psi_min)
    lo, hi = wk.boxes[0][:2]
    sbm.lib().sbm_set_alloc_limit(1 << 10)
    try:
        with pytest.raises(sbm.SBMError) as e:
            g.amr_add_level(lo, hi)
        assert e.value.status == _capi.SBM_ERR_OOM
    finally:
        sbm.lib().sbm_set_alloc_limit(0)
    # the grid is as before: a single-level solve works, and the patch can be added now
    u = cuda(wk.level_u0(0))
    assert g.solve(u, omega=wk.omega, smoother="gs").converged
    g.amr_add_level(lo, hi)
    g.amr_set_psi(1, cuda(wk.level_psi(1)), wk.psi_min)
    us = [cuda(wk.level_u0(a)) for a in range(2)]
    assert g.amr_solve(us, omega=wk.omega, smoother="gs").converged


def test_grid_barrier_timeout_is_reported_and_the_grid_recovers(built):
    wk = W.damage3d(17)
    g = gpu_grid(wk, precision="mixed")
    _capi.check(sbm.lib().sbm_set_wait_limit(g._h, 1), g._h)     # one poll per barrier
    with pytest.raises(sbm.SBMError) as e:
        g.solve(cuda(wk.u0), omega=wk.omega)
    assert e.value.status == _capi.SBM_ERR_CUDA
    assert b"timed out" in sbm.lib().sbm_last_error(g._h)
    x = torch.arange(10, dtype=torch.float64, device="cuda")
    assert float(x.sum()) == 45.0                                 # the context is intact
    _capi.check(sbm.lib().sbm_set_wait_limit(g._h, 0), g._h)     # the default bound
    u = cuda(wk.u0)
    info = g.solve(u, omega=wk.omega)
    assert info.converged
    P = oracle_problem(wk)
    ref = oracle.mg_solve(P, oracle.floor_psi(wk.psi, wk.psi_min), wk.f, wk.u0, omega=wk.omega, tol=1e-14,
                          max_cycles=150).u
    assert np.linalg.norm(host(u) - ref) <= 1e-8 * np.linalg.norm(ref)


def test_refinement_boxes_must_nest(built):
    wk = W.voids_amr(2, 17, 2, count=2, rmin=0.1, rmax=0.2)
    g = sbm.Grid(2, wk.n, wk.h)
    g.set_moduli(sbm.SBM_CUBIC, wk.moduli)
    g.set_psi(cuda(wk.level_psi(0)), wk.psi_min)
    bad = [((3, 4), (12, 10)),            # odd corner
           ((4, 4), (40, 10)),            # beyond the level (33 nodes)
           ((4, 4), (6, 4))]              # thinner than 2
    for lo, hi in bad:
        with pytest.raises(sbm.SBMError) as e:
            g.amr_add_level(lo, hi)
        assert e.value.status == _capi.SBM_ERR_ARG
    g.amr_add_level((4, 4), (20, 20))
    for lo, hi in [((8, 8), (60, 40)),    # leaves the parent box
                   ((10, 10), (40, 38)),  # reaches the parent's interface (needs one parent cell inside)
                   ((4, 10), (30, 30))]:  # starts outside the parent box
        with pytest.raises(sbm.SBMError) as e:
            g.amr_add_level(lo, hi)
        assert e.value.status == _capi.SBM_ERR_ARG
    g.amr_add_level((10, 10), (36, 36))   # one parent cell inside on every side
