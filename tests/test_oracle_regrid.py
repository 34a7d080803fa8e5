"""Pins of the oracle's regridding (Sec. 2.2: refine where the indicator varies,
tag h |grad psi| > threshold, cluster the tags into nested boxes):

  - a straight step in psi: the tagged cells are exactly the two columns next to
    the step, and the box is their column range over the whole height (with and
    without dilation);
  - two discs far apart give two boxes, each holding every tagged cell around its
    disc; two discs close together give one box;
  - more separated blobs than the child limit: the limit holds and every tagged
    cell is still inside a box;
  - every box of a two-level regrid is valid (even corners, at least 2 thick,
    nested one parent cell inside its parent unless on the domain boundary,
    siblings two parent cells apart), checked by an independent validator.
"""
import numpy as np
import pytest

import oracle


def _base(n0):
    P = oracle.Problem(2, (n0, n0, 1), 1.0 / (n0 - 1), 1.0, 0.6, 0.5)
    return oracle.Amr(P, [])


def _cell_psi(A, a, fn):
    P = A.level_problem(a)
    o = A.origin(a)
    h = P.h
    j, i = np.meshgrid(np.arange(P.n[1] - 1), np.arange(P.n[0] - 1), indexing="ij")
    return np.ascontiguousarray(fn((i + o[0] + 0.5) * h, (j + o[1] + 0.5) * h).reshape(-1), dtype=np.float64)


def _tagged_cells(A, a, psi, thr):
    """Brute force: global cells of patch a whose centred-difference h|grad psi|
    exceeds thr (interior cells of a 2D base grid only)."""
    P = A.level_problem(a)
    nx, ny = P.n[0] - 1, P.n[1] - 1
    v = psi.reshape(ny, nx)
    out = set()
    for j in range(1, ny - 1):
        for i in range(1, nx - 1):
            gx = (v[j, i + 1] - v[j, i - 1]) / 2
            gy = (v[j + 1, i] - v[j - 1, i]) / 2
            if np.hypot(gx, gy) > thr:
                out.add((i, j))
    return out


def _valid(A, boxes, level):
    full = oracle.Amr(A.base, list(A.boxes) + [tuple(b) for b in boxes])
    for a in range(A.nlev, full.nlev):
        lo, hi, p = full.boxes[a - 1]
        N = full.global_n(a)
        for ax in range(2):
            assert lo[ax] % 2 == 0 and hi[ax] % 2 == 0 and hi[ax] - lo[ax] >= 2
            assert 0 <= lo[ax] and hi[ax] <= N[ax] - 1
            if p > 0:
                plo, phi = full.boxes[p - 1][0][ax], full.boxes[p - 1][1][ax]
                Np = full.global_n(p)[ax]
                assert (lo[ax] == 0 and plo == 0) or lo[ax] >= 2 * plo + 2
                assert (hi[ax] == N[ax] - 1 and phi == Np - 1) or hi[ax] <= 2 * phi - 2
        for b in range(A.nlev, a):
            o_lo, o_hi, _ = full.boxes[b - 1]
            assert any(lo[ax] >= o_hi[ax] + 4 or o_lo[ax] >= hi[ax] + 4 for ax in range(2))
    return full


@pytest.mark.parametrize("grow,expect", [(0, ((14, 0, 0), (18, 32, 0))), (1, ((12, 0, 0), (20, 32, 0)))])
def test_step_interface_gives_the_column_box(oracle_lib, grow, expect):
    A = _base(17)
    psi = _cell_psi(A, 0, lambda X, Y: (X > 0.5).astype(float))
    assert _tagged_cells(A, 0, psi, 0.1) == {(i, j) for i in (7, 8) for j in range(1, 15)}
    boxes = oracle.regrid_boxes(A, [psi], 1, 0.1, grow)
    assert boxes == [(expect[0], expect[1], 0)]


def _disc(cx, cy, r, w):
    return lambda X, Y: 0.5 * (1 + np.tanh((np.hypot(X - cx, Y - cy) - r) / w))


def test_separate_discs_give_separate_boxes_and_close_ones_merge(oracle_lib):
    A = _base(65)
    h = 1.0 / 64
    f1, f2 = _disc(0.25, 0.3, 0.08, 2 * h), _disc(0.72, 0.7, 0.1, 2 * h)
    psi = _cell_psi(A, 0, lambda X, Y: f1(X, Y) * f2(X, Y))
    boxes = oracle.regrid_boxes(A, [psi], 1, 0.1, 2)
    assert len(boxes) == 2
    _valid(A, boxes, 1)
    for (i, j) in _tagged_cells(A, 0, psi, 0.1):
        assert any(b[0][0] <= 2 * i and 2 * i + 2 <= b[1][0] and b[0][1] <= 2 * j and 2 * j + 2 <= b[1][1]
                   for b in boxes), (i, j)
    # the same discs moved within a few cells of each other: one box
    g1, g2 = _disc(0.4, 0.5, 0.08, 2 * h), _disc(0.62, 0.5, 0.08, 2 * h)
    psi2 = _cell_psi(A, 0, lambda X, Y: g1(X, Y) * g2(X, Y))
    assert len(oracle.regrid_boxes(A, [psi2], 1, 0.1, 2)) == 1


def test_child_limit_holds_and_covers_every_tag(oracle_lib):
    A = _base(129)
    h = 1.0 / 128
    centres = [(0.12 + 0.25 * i, 0.12 + 0.25 * j) for i in range(4) for j in range(3)]   # 12 blobs
    fs = [_disc(cx, cy, 0.04, 2 * h) for cx, cy in centres]
    psi = _cell_psi(A, 0, lambda X, Y: np.prod([f(X, Y) for f in fs], axis=0))
    boxes = oracle.regrid_boxes(A, [psi], 1, 0.1, 2, max_children=8)
    assert len(boxes) == 8
    _valid(A, boxes, 1)
    for (i, j) in _tagged_cells(A, 0, psi, 0.1):
        assert any(b[0][0] <= 2 * i and 2 * i + 2 <= b[1][0] and b[0][1] <= 2 * j and 2 * j + 2 <= b[1][1]
                   for b in boxes)


def test_two_level_regrid_is_valid(oracle_lib):
    A = _base(33)
    h0 = 1.0 / 32
    fs = [_disc(0.3, 0.3, 0.1, h0 / 2), _disc(0.72, 0.66, 0.12, h0 / 2)]
    fn = lambda X, Y: np.prod([f(X, Y) for f in fs], axis=0)
    psis = [_cell_psi(A, 0, fn)]
    b1 = oracle.regrid_boxes(A, psis, 1, 0.1, 2)
    A1 = _valid(A, b1, 1)
    psis += [_cell_psi(A1, a, fn) for a in range(1, A1.nlev)]
    b2 = oracle.regrid_boxes(A1, psis, 2, 0.1, 2)
    assert len(b2) >= 2 and {p for _, _, p in b2} == set(range(1, A1.nlev))
    _valid(A1, b2, 2)
