"""Host-side pieces of bench.py (no GPU): the grid extents the refinement lines'
roofline uses for a patch coarsen to a small dense bottom level (the library refuses
a bottom level of more than 16384 dofs), for the largest finest-level patch of every
refinement workload the bench runs."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _coarsest(n):
    """Node counts after the library's coarsening rule: halve while every axis has
    an even cell count of at least 8."""
    n = list(n)
    while all((m - 1) % 2 == 0 and (m - 1) // 2 >= 4 for m in n):
        n = [(m - 1) // 2 + 1 for m in n]
    return n


def test_mg_extent_is_the_smallest_coarsenable_size():
    for m in range(2, 2000):
        e = bench.mg_extent(m)
        assert e >= m
        c = _coarsest([e])[0]
        assert 5 <= c <= 9, (m, e, c)
        # no smaller extent >= m coarsens as well
        assert all(not (5 <= _coarsest([x])[0] <= 9) for x in range(m, e)), (m, e)


def test_refinement_roofline_grids_have_small_bottom_levels():
    for name in ("voids_amr_2d", "voids_amr_2d_clustered", "voids_amr_3d", "voids_amr_3d_65",
                 "voids_amr_3d_clustered"):
        wk = bench.workload(name)
        nl = len(wk.boxes) + 1
        lmax = max(wk.level(a) for a in range(1, nl))
        for a in range(1, nl):
            if wk.level(a) != lmax:
                continue
            ns = wk.storage_shape(a)
            n = [bench.mg_extent(ns[ax]) for ax in range(wk.dim)]
            c = _coarsest(n)
            dofs = wk.dim
            for m in c:
                dofs *= m
            assert dofs <= 16384, (name, a, n, c)
