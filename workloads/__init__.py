"""Seeded synthetic inputs for the SBM elasticity solve.

This module holds only input generation: grids, moduli, Dirichlet faces and
values, the diffuse indicator psi (before the psi_min floor), densities and
loads.  It contains none of the solver's arithmetic (no operator, no floor, no
multigrid) and is shared by the tests, the benchmark and the smoke check, which
feed the identical arrays to the CPU oracle and to the CUDA library.

Random numbers come from splitmix64 (Steele, Lea & Flood 2014): state advances by
0x9E3779B97F4A7C15, output z -> (z ^ z>>30) * 0xBF58476D1CE4E5B9 ->
(z ^ z>>27) * 0x94D049BB133111EB -> z ^ z>>31; a uniform double is
(z >> 11) * 2^-53.  A stream is seeded with config_id * 1000 + stream_id.

Indicator recipes (the workloads of the paper's examples, Sec. 3):
  plate_hole : one circular void, psi = (1 + tanh((r - R)/(2h)))/2   (Sec. 3.1 plate with a hole)
  voids2d    : product of tanh indicators of non-overlapping random circles (Sec. 3.1 voids)
  damage3d   : psi = 1 - max_e (1 - tanh((rho_e - 1) a_min/(2h)))/2 over random
               axis-aligned ellipsoids (a damaged-region shape, Sec. 3.2)
  topopt3d   : SIMP density rho ~ U[0.05, 1], 3 neighbour-averaging passes (Sec. 3.3)
  voids3d    : product of tanh indicators of non-overlapping random spheres
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_M64 = (1 << 64) - 1


def splitmix64(seed: int, count: int) -> np.ndarray:
    """``count`` successive splitmix64 outputs of the generator seeded with ``seed``."""
    with np.errstate(over="ignore"):
        k = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed & _M64) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    u = (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return lo + (hi - lo) * u


class _Stream:
    """Sequential draws from one seeded stream."""

    def __init__(self, seed: int, size: int = 1 << 16):
        self._v = uniform(seed, size)
        self._i = 0

    def __call__(self, lo: float = 0.0, hi: float = 1.0) -> float:
        if self._i >= len(self._v):
            raise RuntimeError("random stream exhausted")
        x = self._v[self._i]
        self._i += 1
        return lo + (hi - lo) * x


def lame_from_enu(E: float, nu: float):
    """(lambda, mu) from Young's modulus and Poisson's ratio."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def iso_cubic(E: float, nu: float):
    """(c11, c12, c44) of an isotropic material: (lambda + 2 mu, lambda, mu)."""
    lam, mu = lame_from_enu(E, nu)
    return lam + 2.0 * mu, lam, mu


FACES = {"-x": 0, "+x": 1, "-y": 2, "+y": 3, "-z": 4, "+z": 5}


@dataclass
class Workload:
    name: str
    dim: int
    n: tuple                 # nodes per axis (3 entries, n[2] = 1 in 2D)
    h: float
    moduli: tuple            # (c11, c12, c44)
    bcs: list                # [(face, comp, value)] Dirichlet; "affine" handled by values
    psi: np.ndarray          # cell indicator before the floor
    psi_min: float
    f: np.ndarray            # nodal load density (packed, component-major)
    u0: np.ndarray           # initial guess carrying the Dirichlet values
    smoother: str = "jacobi"
    omega: float = 2.0 / 3.0
    precision: str = "fp64"
    rho: np.ndarray | None = None     # SIMP density when psi = p(rho)
    notes: dict = field(default_factory=dict)

    @property
    def nnodes(self):
        return self.n[0] * self.n[1] * self.n[2]

    @property
    def ncells(self):
        nz = self.n[2] - 1 if self.dim == 3 else 1
        return (self.n[0] - 1) * (self.n[1] - 1) * nz

    @property
    def ndofs(self):
        return self.dim * self.nnodes

    def dirichlet_bits(self):
        bits = [0, 0, 0]
        for face, comp, _ in self.bcs:
            bits[comp] |= 1 << FACES[face]
        return tuple(bits)


def node_coords(dim, n, h):
    """x, y, z coordinates of every node in packed order."""
    i = np.arange(n[0]) * h
    j = np.arange(n[1]) * h
    k = np.arange(n[2]) * h if dim == 3 else np.zeros(1)
    Z, Y, X = np.meshgrid(k, j, i, indexing="ij")
    return X.reshape(-1), Y.reshape(-1), Z.reshape(-1)


def cell_centres(dim, n, h):
    i = (np.arange(n[0] - 1) + 0.5) * h
    j = (np.arange(n[1] - 1) + 0.5) * h
    k = (np.arange(n[2] - 1) + 0.5) * h if dim == 3 else np.zeros(1)
    Z, Y, X = np.meshgrid(k, j, i, indexing="ij")
    return X.reshape(-1), Y.reshape(-1), Z.reshape(-1)


def initial_guess(dim, n, bcs):
    """u = 0 on free dofs and the prescribed value on Dirichlet dofs.  A face set
    later in ``bcs`` overwrites an earlier one on shared edges and corners.
    A value given as a callable is evaluated at the node coordinates."""
    N = n[0] * n[1] * n[2]
    u = np.zeros(dim * N)
    shape = (n[2], n[1], n[0])
    for face, comp, value in bcs:
        v = u[comp * N:(comp + 1) * N].reshape(shape)
        sl = {
            "-x": (slice(None), slice(None), 0), "+x": (slice(None), slice(None), n[0] - 1),
            "-y": (slice(None), 0, slice(None)), "+y": (slice(None), n[1] - 1, slice(None)),
            "-z": (0, slice(None), slice(None)), "+z": (n[2] - 1, slice(None), slice(None)),
        }[face]
        if callable(value):
            X, Y, Z = (a.reshape(shape) for a in node_coords(dim, n, 1.0))
            v[sl] = value(X[sl], Y[sl], Z[sl])
        else:
            v[sl] = value
    return u


def _tanh_step(dist, width):
    return 0.5 * (1.0 + np.tanh(dist / width))


def plate_hole(n: int = 65, radius: float = 0.2, psi_min: float = 1e-3) -> Workload:
    """2D plane strain, E=1, nu=0.3, unit square, circular void of radius 0.2 at the
    centre, bottom clamped, top u = (0, 0.01), sides traction free."""
    dim, nn, h = 2, (n, n, 1), 1.0 / (n - 1)
    x, y, _ = cell_centres(dim, nn, h)
    r = np.hypot(x - 0.5, y - 0.5)
    psi = _tanh_step(r - radius, 2.0 * h)
    bcs = [("-y", 0, 0.0), ("-y", 1, 0.0), ("+y", 0, 0.0), ("+y", 1, 0.01)]
    return Workload("plate_hole_2d", dim, nn, h, iso_cubic(1.0, 0.3), bcs, psi, psi_min,
                    np.zeros(dim * n * n), initial_guess(dim, nn, bcs))


def _random_balls(stream, count, rmin, rmax, margin, dim, max_tries=100000):
    """Rejection-sampled non-overlapping balls inside the unit box."""
    balls = []
    tries = 0
    while len(balls) < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place balls")
        r = stream(rmin, rmax)
        c = np.array([stream(r + margin, 1.0 - r - margin) for _ in range(dim)])
        if all(np.linalg.norm(c - c2) >= r + r2 + margin for c2, r2 in balls):
            balls.append((c, r))
    return balls


def voids(dim: int, n: int, count: int, rmin: float, rmax: float, width_h: float,
          seed: int, psi_min: float, margin_h: float | None = None):
    """Product of tanh indicators of ``count`` random non-overlapping voids."""
    h = 1.0 / (n - 1)
    nn = (n, n, n if dim == 3 else 1)
    st = _Stream(seed)
    balls = _random_balls(st, count, rmin, rmax, 4.0 * (margin_h if margin_h else h), dim)
    X = cell_centres(dim, nn, h)
    psi = np.ones(len(X[0]))
    for c, r in balls:
        dist = np.sqrt(sum((X[a] - c[a]) ** 2 for a in range(dim)))
        psi *= _tanh_step(dist - r, 2.0 * width_h)
    return nn, h, psi, balls


def damage3d(n: int = 129, count: int = 3, psi_min: float = 1e-4, seed: int = 3001) -> Workload:
    """3D cubic crystal (c11=1, c12=0.6, c44=0.5) with a damaged region made of
    ``count`` random ellipsoids; bottom (z=0) clamped, top u = (0, 0, 0.01)."""
    dim, nn, h = 3, (n, n, n), 1.0 / (n - 1)
    st = _Stream(seed)
    ell = []
    for _ in range(count):
        a = np.array([st(0.05, 0.2) for _ in range(3)])
        c = np.array([st(0.2, 0.8) for _ in range(3)])
        ell.append((c, a))
    X = cell_centres(dim, nn, h)
    dmg = np.zeros(len(X[0]))
    for c, a in ell:
        rho = np.sqrt(sum(((X[i] - c[i]) / a[i]) ** 2 for i in range(3)))
        d = 0.5 * (1.0 - np.tanh((rho - 1.0) * a.min() / (2.0 * h)))
        dmg = np.maximum(dmg, d)
    psi = 1.0 - dmg
    bcs = [("-z", 0, 0.0), ("-z", 1, 0.0), ("-z", 2, 0.0),
           ("+z", 0, 0.0), ("+z", 1, 0.0), ("+z", 2, 0.01)]
    return Workload("damage_3d", dim, nn, h, (1.0, 0.6, 0.5), bcs, psi, psi_min,
                    np.zeros(dim * n ** 3), initial_guess(dim, nn, bcs),
                    notes={"ellipsoids": ell})


def smooth_density(rho, ncell, passes=3):
    """Each pass replaces a cell value by the mean of itself and its existing
    face neighbours."""
    r = rho.reshape(ncell[2], ncell[1], ncell[0]).copy()
    for _ in range(passes):
        s = r.copy()
        cnt = np.ones_like(r)
        for ax in range(3):
            if r.shape[ax] < 2:
                continue
            lo = [slice(None)] * 3
            hi = [slice(None)] * 3
            lo[ax] = slice(0, -1)
            hi[ax] = slice(1, None)
            s[tuple(lo)] += r[tuple(hi)]
            cnt[tuple(lo)] += 1
            s[tuple(hi)] += r[tuple(lo)]
            cnt[tuple(hi)] += 1
        r = s / cnt
    return r.reshape(-1)


def topopt3d(nx: int = 257, ny: int = 129, nz: int = 129, psi_min: float = 1e-3,
             seed: int = 4001) -> Workload:
    """3D cantilever on [0, 2] x [0, 1] x [0, 1]: x=0 clamped, unit Gaussian load
    (sigma = 2h) in -y at the centre of the x=2 face; SIMP density rho in cells."""
    dim, nn = 3, (nx, ny, nz)
    h = 1.0 / (ny - 1)
    ncell = (nx - 1, ny - 1, nz - 1)
    rho = uniform(seed, ncell[0] * ncell[1] * ncell[2], 0.05, 1.0)
    rho = smooth_density(rho, ncell, 3)
    psi = psi_min + (1.0 - psi_min) * rho ** 3      # the recipe's stiffness field (input)
    X, Y, Z = node_coords(dim, nn, h)
    sigma = 2.0 * h
    g = np.exp(-((X - (nx - 1) * h) ** 2 + (Y - 0.5 * (ny - 1) * h) ** 2 + (Z - 0.5 * (nz - 1) * h) ** 2)
               / (2.0 * sigma ** 2))
    N = nx * ny * nz
    f = np.zeros(dim * N)
    f[N:2 * N] = -g / (h ** 3 * g.sum())           # h^3 sum f_y = -1
    bcs = [("-x", 0, 0.0), ("-x", 1, 0.0), ("-x", 2, 0.0)]
    f_masked = f.copy()
    # Isotropic nu = 0.3 Q1 elasticity has max eig(D^-1 K) ~ 3.2 > 3, so Jacobi
    # needs omega < 2/3.2; 0.5 is used.
    return Workload("topopt_3d", dim, nn, h, iso_cubic(1.0, 0.3), bcs, psi, psi_min, f_masked,
                    initial_guess(dim, nn, bcs), omega=0.5, precision="mixed", rho=rho)


@dataclass
class AmrWorkload:
    """Base grid + nested refinement patches.  ``boxes[a-1]`` is patch a: ``(lo, hi)``
    (one patch per level: parent a-1) or ``(lo, hi, parent)``, parents before their
    children.  psi is the same analytic indicator evaluated at every patch's cell
    centres; patch arrays cover the box grown by one padding node per side (cells
    outside the domain get psi = 0)."""
    name: str
    dim: int
    n: tuple
    h: float
    moduli: tuple
    bcs: list
    psi_fn: object
    psi_min: float
    boxes: list
    smoother: str = "jacobi"
    omega: float = 2.0 / 3.0
    precision: str = "fp64"
    notes: dict = field(default_factory=dict)
    affine: float = None      # Dirichlet data u_p = affine * (x_p - 1/2) instead of the bcs values

    def dirichlet_bits(self):
        bits = [0, 0, 0]
        for face, comp, _ in self.bcs:
            bits[comp] |= 1 << FACES[face]
        return tuple(bits)

    def parent(self, a):
        if a == 0:
            return -1
        b = self.boxes[a - 1]
        return b[2] if len(b) > 2 else a - 1

    def level(self, a):
        return 0 if a == 0 else self.level(self.parent(a)) + 1

    def level_h(self, a):
        return self.h / 2 ** self.level(a)

    def level_N(self, a):
        return tuple((self.n[ax] - 1) * 2 ** self.level(a) + 1 if ax < self.dim else 1 for ax in range(3))

    def storage_shape(self, a):
        """nodes per axis of patch a's storage (full grid for a = 0)"""
        if a == 0:
            return tuple(self.n)
        lo, hi = self.boxes[a - 1][0], self.boxes[a - 1][1]
        return tuple(hi[ax] - lo[ax] + 3 if ax < self.dim else 1 for ax in range(3))

    def origin(self, a):
        if a == 0:
            return (0, 0, 0)
        lo = self.boxes[a - 1][0]
        return tuple(lo[ax] - 1 if ax < self.dim else 0 for ax in range(3))

    def level_psi(self, a):
        """cell values of level a's storage (padding cells outside the domain: 0)"""
        n, o, h = self.storage_shape(a), self.origin(a), self.level_h(a)
        N = self.level_N(a)
        ncz = n[2] - 1 if self.dim == 3 else 1
        k, j, i = np.meshgrid(np.arange(ncz), np.arange(n[1] - 1), np.arange(n[0] - 1), indexing="ij")
        gi, gj, gk = i + o[0], j + o[1], k + o[2]
        X, Y, Z = (gi + 0.5) * h, (gj + 0.5) * h, ((gk + 0.5) * h if self.dim == 3 else np.zeros(gi.shape))
        v = self.psi_fn(X, Y, Z)
        inside = (gi >= 0) & (gi < N[0] - 1) & (gj >= 0) & (gj < N[1] - 1)
        if self.dim == 3:
            inside &= (gk >= 0) & (gk < N[2] - 1)
        return np.where(inside, v, 0.0).reshape(-1)

    def level_u0(self, a):
        """Dirichlet values on the level's storage nodes on the domain faces, 0 elsewhere"""
        n, o = self.storage_shape(a), self.origin(a)
        N = self.level_N(a)
        Nn = n[0] * n[1] * n[2]
        u = np.zeros(self.dim * Nn)
        k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
        g = [(i + o[0]).reshape(-1), (j + o[1]).reshape(-1), (k + o[2]).reshape(-1)]
        h = self.level_h(a)
        for face, comp, value in self.bcs:
            ax, side = FACES[face] // 2, FACES[face] % 2
            on = g[ax] == (0 if side == 0 else N[ax] - 1)
            if self.affine is not None:
                value = (self.affine * (g[comp] * h - 0.5))[on]
            u[comp * Nn:(comp + 1) * Nn][on] = value
        return u


def tag_boxes(dim, n0, psi_fn, levels, threshold=0.1, grow=2):
    """One refinement box per level: cells of level a-1 where h |grad psi| (centred
    differences of cell psi) exceeds ``threshold``, grown by ``grow`` cells, bounded
    by an even-cornered box in level-a indices, nested one parent cell inside the
    parent box unless on the domain boundary."""
    boxes = []
    h0 = 1.0 / (n0 - 1)
    for a in range(1, levels + 1):
        hp = h0 / 2 ** (a - 1)
        Np = [(n0 - 1) * 2 ** (a - 1) + 1 if ax < dim else 1 for ax in range(3)]
        nc = [Np[ax] - 1 if ax < dim else 1 for ax in range(3)]
        axes = [(np.arange(nc[ax]) + 0.5) * hp if ax < dim else np.zeros(1) for ax in range(3)]
        Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
        psi = psi_fn(X, Y, Z)
        grad = np.zeros(psi.shape)
        for ax in range(dim):
            axn = 2 - ax
            d = (np.roll(psi, -1, axn) - np.roll(psi, 1, axn)) / 2.0
            grad += d ** 2
        tag = np.sqrt(grad) > threshold
        if not tag.any():
            break
        idx = np.nonzero(tag)
        lo, hi = [0, 0, 0], [0, 0, 0]
        for ax in range(dim):
            c = idx[2 - ax]
            lo_c = max(int(c.min()) - grow, 0)
            hi_c = min(int(c.max()) + 1 + grow, nc[ax])
            lo[ax], hi[ax] = 2 * lo_c, 2 * hi_c                # parent cells -> level-a nodes
            if a > 1:
                plo, phi = boxes[-1][0][ax], boxes[-1][1][ax]
                Npa = Np[ax]
                lo[ax] = 0 if plo == 0 and lo[ax] <= 2 * plo + 2 else max(lo[ax], 2 * plo + 2)
                hi[ax] = (2 * (Npa - 1)) if phi == Npa - 1 and hi[ax] >= 2 * phi - 2 else min(hi[ax], 2 * phi - 2)
        boxes.append((tuple(lo), tuple(hi)))
    return boxes


def _apart(b1, b2, dim, gap=4):
    """Boxes (level node indices) at least ``gap`` nodes apart on some axis."""
    return any(b1[0][ax] >= b2[1][ax] + gap or b2[0][ax] >= b1[1][ax] + gap for ax in range(dim))


def _union(b1, b2, dim):
    lo = tuple(min(b1[0][ax], b2[0][ax]) if ax < dim else 0 for ax in range(3))
    hi = tuple(max(b1[1][ax], b2[1][ax]) if ax < dim else 0 for ax in range(3))
    return (lo, hi)


def _volume(b, dim):
    return int(np.prod([b[1][ax] - b[0][ax] for ax in range(dim)]))


def cluster_boxes(dim, n0, psi_fn, levels, threshold=0.1, grow=2, max_children=8):
    """Several refinement boxes per level (tagging and clustering on the host):
    inside each parent patch, the parent's cells where h |grad psi| (centred
    differences of cell psi) exceeds ``threshold`` are dilated by ``grow`` cells and
    split into connected components; each component's bounding box (even corners in
    the child level, nested one parent cell inside the parent unless on the domain
    boundary) is a child patch.  Boxes closer than two parent cells are merged into
    their bounding box, and while a parent has more than ``max_children`` the pair
    whose union adds the least volume is merged.  Returns [(lo, hi, parent)], parents
    before children."""
    from scipy import ndimage
    h0 = 1.0 / (n0 - 1)
    out = []                                      # (lo, hi, parent, level)
    parents = [(None, None, -1, 0)]              # the base grid as patch 0
    for L in range(1, levels + 1):
        hp = h0 / 2 ** (L - 1)
        Np = [(n0 - 1) * 2 ** (L - 1) + 1 if ax < dim else 1 for ax in range(3)]
        nc = [Np[ax] - 1 if ax < dim else 1 for ax in range(3)]
        axes = [(np.arange(nc[ax]) + 0.5) * hp if ax < dim else np.zeros(1) for ax in range(3)]
        Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
        psi = psi_fn(X, Y, Z)
        grad = np.zeros(psi.shape)
        for ax in range(dim):
            axn = 2 - ax
            d = (np.roll(psi, -1, axn) - np.roll(psi, 1, axn)) / 2.0
            grad += d ** 2
        tag = np.sqrt(grad) > threshold
        conn = np.ones((3, 3, 3), bool)
        if dim == 2:
            conn[0] = conn[2] = False                 # the (z, y, x) arrays of a 2D grid have one z layer
        if grow:
            tag = ndimage.binary_dilation(tag, structure=conn, iterations=grow)
        level_boxes = []
        for pidx, (plo, phi, _, plev) in enumerate(parents):
            if plev != L - 1:
                continue
            # child-level node range allowed inside this parent
            amin, amax = [0, 0, 0], [0, 0, 0]
            for ax in range(dim):
                N = 2 * (Np[ax] - 1) + 1
                if plo is None:
                    amin[ax], amax[ax] = 0, N - 1
                else:
                    amin[ax] = 0 if plo[ax] == 0 else 2 * plo[ax] + 2
                    amax[ax] = N - 1 if phi[ax] == Np[ax] - 1 else 2 * phi[ax] - 2
            sl = tuple(slice(amin[ax] // 2, amax[ax] // 2) if ax < dim else slice(0, 1) for ax in (2, 1, 0))
            sub = np.zeros(tag.shape, bool)
            sub[sl] = tag[sl]
            labels, _ = ndimage.label(sub, structure=conn)
            boxes = []
            for sls in ndimage.find_objects(labels):
                if sls is None:
                    continue
                lo, hi = [0, 0, 0], [0, 0, 0]
                for ax in range(dim):
                    sa = sls[2 - ax]
                    lo[ax] = max(2 * sa.start, amin[ax])
                    hi[ax] = min(2 * sa.stop, amax[ax])
                if all(hi[ax] - lo[ax] >= 2 for ax in range(dim)):
                    boxes.append((tuple(lo), tuple(hi)))
            changed = True
            while changed:
                changed = False
                for i in range(len(boxes)):
                    for j in range(i + 1, len(boxes)):
                        if not _apart(boxes[i], boxes[j], dim):
                            boxes[i] = _union(boxes[i], boxes[j], dim)
                            del boxes[j]
                            changed = True
                            break
                    if changed:
                        break
                if not changed and len(boxes) > max_children:
                    best = None
                    for i in range(len(boxes)):
                        for j in range(i + 1, len(boxes)):
                            u = _union(boxes[i], boxes[j], dim)
                            cost = _volume(u, dim) - _volume(boxes[i], dim) - _volume(boxes[j], dim)
                            if best is None or cost < best[0]:
                                best = (cost, i, j, u)
                    _, i, j, u = best
                    boxes[i] = u
                    del boxes[j]
                    changed = True
            for b in sorted(boxes):
                level_boxes.append((b[0], b[1], pidx, L))
        if not level_boxes:
            break
        parents = parents + level_boxes
        out.extend(level_boxes)
    return [(lo, hi, parent) for lo, hi, parent, _ in out]


def voids_amr(dim=2, n0=129, levels=3, count=8, rmin=0.03, rmax=0.10, psi_min=1e-4, seed=2001, clustered=False):
    """Random non-overlapping voids (circles / spheres), tanh width 2 h_f with h_f the
    finest spacing, refined by tag_boxes."""
    st = _Stream(seed)
    h0 = 1.0 / (n0 - 1)
    balls = _random_balls(st, count, rmin, rmax, min(4.0 * h0, 0.04), dim)
    hf = h0 / 2 ** levels

    def psi_fn(X, Y, Z):
        v = np.ones(np.shape(X))
        coords = (X, Y, Z)
        for c, r in balls:
            dist = np.sqrt(sum((coords[ax] - c[ax]) ** 2 for ax in range(dim)))
            v = v * _tanh_step(dist - r, 2.0 * hf)
        return v

    boxes = cluster_boxes(dim, n0, psi_fn, levels) if clustered else tag_boxes(dim, n0, psi_fn, levels)
    if dim == 2:
        bcs = [("-y", 0, 0.0), ("-y", 1, 0.0), ("+y", 0, 0.0), ("+y", 1, 0.01)]
        moduli = iso_cubic(1.0, 0.3)
    else:
        # triaxial loading: every component fixed on every face to the affine field
        # u = 0.01 (x - 1/2), so each face moves 0.005 outward
        bcs = [(f, p, None) for f in ("-x", "+x", "-y", "+y", "-z", "+z") for p in range(3)]
        moduli = iso_cubic(1.0, 0.25)
    n = (n0, n0, n0 if dim == 3 else 1)
    return AmrWorkload(f"voids_amr_{dim}d" + ("_clustered" if clustered else ""), dim, n, h0, moduli, bcs, psi_fn,
                       psi_min, boxes,
                       smoother="gs" if dim == 2 else "jacobi", omega=2.0 / 3.0 if dim == 2 else 0.5,
                       precision="fp64" if dim == 2 else "mixed", notes={"balls": balls},
                       affine=None if dim == 2 else 0.01)


CONFIGS = {
    "plate_hole_2d": plate_hole,
    "damage_3d": damage3d,
    "topopt_3d": topopt3d,
}
