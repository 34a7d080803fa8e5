"""ctypes front end of the plain FP64 CPU oracle (``sbm_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product path never imports it.

Every function takes and returns numpy float64 arrays in the packed layout of the
C ABI: node (i, j, k) at ``i + nx*(j + ny*k)``, component ``p`` at offset
``p*nnodes``; cell (i, j, k) at ``i + (nx-1)*(j + (ny-1)*k)``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sbm_oracle.c")
_HDR = os.path.join(_HERE, "sbm_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libsbm_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("h", C.c_double),
                ("c11", C.c_double), ("c12", C.c_double), ("c44", C.c_double),
                ("dirichlet", C.c_uint * 3)]


class _Topopt(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("alpha", "beta", "zeta", "lambda_", "lambda_rate", "V0", "mobility",
                                          "dt")]


@dataclass
class TopoptParams:
    """Parameters of the phase-field topology optimisation step (Sec. 3.3)."""
    alpha: float = 200.0
    beta: float = 0.01
    zeta: float = 0.01
    lam: float = 400.0
    lam_rate: float = 0.0
    V0: float = 0.25
    mobility: float = 1.0
    dt: float = 1e-4

    def c(self):
        return _Topopt(self.alpha, self.beta, self.zeta, self.lam, self.lam_rate, self.V0, self.mobility, self.dt)


class _Opts(C.Structure):
    _fields_ = [("nu1", C.c_int), ("nu2", C.c_int), ("omega", C.c_double),
                ("smoother", C.c_int), ("tol", C.c_double), ("max_cycles", C.c_int)]


_lib = None
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def _L():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        P = C.POINTER(_Problem)
        sig = {
            "orc_nnodes": (C.c_long, [P]),
            "orc_ncells": (C.c_long, [P]),
            "orc_is_dirichlet": (C.c_int, [P, C.c_int, C.c_int, C.c_int, C.c_int]),
            "orc_element_matrix": (None, [P, _dp]),
            "orc_apply": (None, [P, _dp, _dp, _dp]),
            "orc_residual": (None, [P, _dp, _dp, _dp, _dp]),
            "orc_diagonal": (None, [P, _dp, _dp]),
            "orc_norm_free": (C.c_double, [P, _dp]),
            "orc_jacobi_sweep": (None, [P, _dp, _dp, _dp, C.c_double]),
            "orc_gs_sweep": (None, [P, _dp, _dp, _dp, C.c_int]),
            "orc_can_coarsen": (C.c_int, [P]),
            "orc_coarse_problem": (None, [P, P]),
            "orc_coarsen_psi": (None, [P, _dp, _dp]),
            "orc_restrict": (None, [P, _dp, _dp]),
            "orc_prolong_add": (None, [P, _dp, _dp]),
            "orc_num_levels": (C.c_int, [P]),
            "orc_assemble_dense": (None, [P, _dp, _dp]),
            "orc_direct_solve": (C.c_int, [P, _dp, _dp, _dp]),
            "orc_mg_solve": (C.c_int, [P, _dp, _dp, _dp, C.POINTER(_Opts), _dp, C.POINTER(C.c_int)]),
            "orc_dJdpsi": (None, [P, _dp, _dp, _dp]),
            "orc_source_terms": (None, [P, _dp, C.c_void_p, C.c_void_p, C.c_void_p, _dp]),
            "orc_node_psi": (None, [P, _dp, _dp, _dp, _dp]),
            "orc_topopt_step": (None, [P, C.POINTER(_Topopt), C.c_int, _dp, _dp, _dp]),
            "orc_topopt_energy": (None, [P, C.POINTER(_Topopt), C.c_int, _dp, _dp]),
            "orc_apply_product": (None, [P, C.c_int, _dp, _dp, _dp]),
            "orc_diagonal_product": (None, [P, C.c_int, _dp, _dp]),
            "orc_jacobi_product": (None, [P, C.c_int, _dp, _dp, _dp, C.c_double]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


FACES = {"-x": 0, "+x": 1, "-y": 2, "+y": 3, "-z": 4, "+z": 5}


@dataclass
class Problem:
    """Grid, moduli and Dirichlet faces of one level (mirrors ``orc_problem``)."""
    dim: int
    n: tuple
    h: float
    c11: float
    c12: float
    c44: float
    dirichlet: tuple = (0, 0, 0)   # per component: bitmask over faces

    def __post_init__(self):
        n = tuple(int(v) for v in self.n)
        if self.dim == 2 and len(n) == 2:
            n = n + (1,)
        self.n = n
        self.dirichlet = tuple(int(v) for v in (tuple(self.dirichlet) + (0, 0, 0))[:3])

    @property
    def nnodes(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    @property
    def ncells(self) -> int:
        nz = (self.n[2] - 1) if self.dim == 3 else 1
        return (self.n[0] - 1) * (self.n[1] - 1) * nz

    @property
    def ndofs(self) -> int:
        return self.dim * self.nnodes

    def c(self) -> _Problem:
        p = _Problem()
        p.dim = self.dim
        p.n[:] = list(self.n)
        p.h = self.h
        p.c11, p.c12, p.c44 = self.c11, self.c12, self.c44
        p.dirichlet[:] = list(self.dirichlet)
        return p


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def element_matrix(P: Problem) -> np.ndarray:
    nd = (1 << P.dim) * P.dim
    Ke = np.zeros(nd * nd)
    _L().orc_element_matrix(C.byref(P.c()), Ke)
    return Ke.reshape(nd, nd)


def apply(P: Problem, psi, u) -> np.ndarray:
    out = np.zeros(P.ndofs)
    _L().orc_apply(C.byref(P.c()), _f64(psi), _f64(u), out)
    return out


def source_terms(P: Problem, psi, eps0=None, b=None, t=None) -> np.ndarray:
    """f of K u = f for eq. SBMLinearElasticity (see sbm_oracle.h): eigenstrain per
    cell in Voigt components, body force and diffuse traction per node; None = 0."""
    out = np.zeros(P.ndofs)
    keep = [None if a is None else _f64(a) for a in (eps0, b, t)]
    ptr = lambda a: None if a is None else a.ctypes.data_as(C.c_void_p)
    _L().orc_source_terms(C.byref(P.c()), _f64(psi), ptr(keep[0]), ptr(keep[1]), ptr(keep[2]), out)
    return out


def node_psi(P: Problem, psi):
    """(psi_n, |grad psi|_n, w_n) of source_terms at every node."""
    pn, gn, w = np.zeros(P.nnodes), np.zeros(P.nnodes), np.zeros(P.nnodes)
    _L().orc_node_psi(C.byref(P.c()), _f64(psi), pn, gn, w)
    return pn, gn, w


def topopt_step(P: Problem, T: TopoptParams, eta, u, step: int = 0) -> np.ndarray:
    """eta after one explicit step of eq. topop_evolution (see sbm_oracle.h)."""
    out = np.zeros(P.ncells)
    _L().orc_topopt_step(C.byref(P.c()), C.byref(T.c()), step, _f64(eta), _f64(u), out)
    return out


def topopt_energy(P: Problem, T: TopoptParams, eta, step: int = 0) -> np.ndarray:
    """(double-well, gradient, volume-penalty) parts of the discrete energy."""
    out = np.zeros(3)
    _L().orc_topopt_energy(C.byref(P.c()), C.byref(T.c()), step, _f64(eta), out)
    return out


def psi_of_eta(T: TopoptParams, eta) -> np.ndarray:
    """The stiffness of eq. topop_objective, psi = (eta + zeta)^2."""
    return (np.asarray(eta, dtype=np.float64) + T.zeta) ** 2


NODE_PSI, CELL_PSI = 1, 2


def apply_product(P: Problem, variant: int, psi, u) -> np.ndarray:
    """K u of the product-rule strong form (Sec. 2.3) at interior nodes, 0 on the
    faces; psi at nodes (NODE_PSI) or in cells averaged to the nodes (CELL_PSI)."""
    out = np.zeros(P.ndofs)
    _L().orc_apply_product(C.byref(P.c()), variant, _f64(psi), _f64(u), out)
    return out


def diagonal_product(P: Problem, variant: int, psi) -> np.ndarray:
    out = np.zeros(P.ndofs)
    _L().orc_diagonal_product(C.byref(P.c()), variant, _f64(psi), out)
    return out


def jacobi_product(P: Problem, variant: int, psi, f, u, omega: float) -> np.ndarray:
    out = _f64(u).copy()
    _L().orc_jacobi_product(C.byref(P.c()), variant, _f64(psi), _f64(f), out, omega)
    return out


def residual(P: Problem, psi, f, u) -> np.ndarray:
    out = np.zeros(P.ndofs)
    _L().orc_residual(C.byref(P.c()), _f64(psi), _f64(f), _f64(u), out)
    return out


def diagonal(P: Problem, psi) -> np.ndarray:
    out = np.zeros(P.ndofs)
    _L().orc_diagonal(C.byref(P.c()), _f64(psi), out)
    return out


def norm_free(P: Problem, r) -> float:
    return _L().orc_norm_free(C.byref(P.c()), _f64(r))


def dirichlet_mask(P: Problem) -> np.ndarray:
    """Boolean mask over dofs, True where the dof is Dirichlet."""
    m = np.zeros((P.dim, P.n[2], P.n[1], P.n[0]), dtype=bool)
    lib, pc = _L(), P.c()
    for p in range(P.dim):
        for k in range(P.n[2]):
            for j in range(P.n[1]):
                for i in range(P.n[0]):
                    m[p, k, j, i] = bool(lib.orc_is_dirichlet(C.byref(pc), i, j, k, p))
    return m.reshape(-1)


def jacobi_sweep(P: Problem, psi, f, u, omega: float) -> np.ndarray:
    u = _f64(u).copy()
    _L().orc_jacobi_sweep(C.byref(P.c()), _f64(psi), _f64(f), u, omega)
    return u


def gs_sweep(P: Problem, psi, f, u, descending: bool = False) -> np.ndarray:
    u = _f64(u).copy()
    _L().orc_gs_sweep(C.byref(P.c()), _f64(psi), _f64(f), u, int(descending))
    return u


def can_coarsen(P: Problem) -> bool:
    return bool(_L().orc_can_coarsen(C.byref(P.c())))


def coarse_problem(P: Problem) -> Problem:
    out = _Problem()
    _L().orc_coarse_problem(C.byref(P.c()), C.byref(out))
    return Problem(out.dim, tuple(out.n), out.h, out.c11, out.c12, out.c44, tuple(out.dirichlet))


def num_levels(P: Problem) -> int:
    return _L().orc_num_levels(C.byref(P.c()))


def coarsen_psi(P: Problem, psi) -> np.ndarray:
    out = np.zeros(coarse_problem(P).ncells)
    _L().orc_coarsen_psi(C.byref(P.c()), _f64(psi), out)
    return out


def restrict(P: Problem, r) -> np.ndarray:
    out = np.zeros(coarse_problem(P).ndofs)
    _L().orc_restrict(C.byref(P.c()), _f64(r), out)
    return out


def prolong_add(P: Problem, e_c, u) -> np.ndarray:
    u = _f64(u).copy()
    _L().orc_prolong_add(C.byref(P.c()), _f64(e_c), u)
    return u


def assemble_dense(P: Problem, psi) -> np.ndarray:
    K = np.zeros(P.ndofs * P.ndofs)
    _L().orc_assemble_dense(C.byref(P.c()), _f64(psi), K)
    return K.reshape(P.ndofs, P.ndofs)


def direct_solve(P: Problem, psi, f, u0) -> np.ndarray:
    u = _f64(u0).copy()
    st = _L().orc_direct_solve(C.byref(P.c()), _f64(psi), _f64(f), u)
    if st != 0:
        raise RuntimeError(f"orc_direct_solve status {st}")
    return u


@dataclass
class MGResult:
    u: np.ndarray
    status: int
    cycles: int
    history: np.ndarray = field(repr=False)


def mg_solve(P: Problem, psi, f, u0, *, nu1=2, nu2=2, omega=2.0 / 3.0, smoother="jacobi",
             tol=1e-10, max_cycles=500) -> MGResult:
    u = _f64(u0).copy()
    o = _Opts(nu1, nu2, omega, 1 if smoother in ("gs", "mcgs", "rbgs") else 0, tol, max_cycles)
    hist = np.full(max_cycles + 1, np.nan)
    cyc = C.c_int(0)
    st = _L().orc_mg_solve(C.byref(P.c()), _f64(psi), _f64(f), u, C.byref(o), hist, C.byref(cyc))
    return MGResult(u, st, cyc.value, hist[: cyc.value + 1])


def dJdpsi(P: Problem, u, lam) -> np.ndarray:
    out = np.zeros(P.ncells)
    _L().orc_dJdpsi(C.byref(P.c()), _f64(u), _f64(lam), out)
    return out


def floor_psi(psi, psi_min: float) -> np.ndarray:
    """psi <- max(psi, psi_min): the floor that keeps the operator definite."""
    return np.maximum(_f64(psi), psi_min)


def simp(rho, psi_min: float, q: float = 3.0):
    """SIMP stiffness map psi = psi_min + (1 - psi_min) rho^q and its derivative."""
    rho = _f64(rho)
    return psi_min + (1.0 - psi_min) * rho ** q, (1.0 - psi_min) * q * rho ** (q - 1.0)


# ------------------------------------------------------------------ BSAMR

class _Amr(C.Structure):
    _fields_ = [("base", _Problem), ("nlev", C.c_int), ("lo", (C.c_int * 3) * 65), ("hi", (C.c_int * 3) * 65),
                ("level", C.c_int * 65), ("parent", C.c_int * 65)]


_AMR_SIGS = {
    "orc_amr_level_problem": (None, [C.POINTER(_Amr), C.c_int, C.POINTER(_Problem)]),
    "orc_amr_owned": (C.c_int, [C.POINTER(_Amr), C.c_int, C.c_int, C.c_int, C.c_int]),
    "orc_amr_coarsen_psi": (None, [C.POINTER(_Amr), C.POINTER(C.POINTER(C.c_double))]),
    "orc_amr_fill": (None, [C.POINTER(_Amr), C.POINTER(C.POINTER(C.c_double))]),
    "orc_amr_residual": (None, [C.POINTER(_Amr)] + [C.POINTER(C.POINTER(C.c_double))] * 4),
    "orc_amr_residual_at": (None, [C.POINTER(_Amr)] + [C.POINTER(C.POINTER(C.c_double))] * 3 +
                            [C.c_long, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                             C.POINTER(C.c_double)]),
    "orc_amr_dJdpsi": (None, [C.POINTER(_Amr)] + [C.POINTER(C.POINTER(C.c_double))] * 3),
    "orc_amr_solve": (C.c_int, [C.POINTER(_Amr)] + [C.POINTER(C.POINTER(C.c_double))] * 3 +
                      [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)]),
}


class _AmrOpts(C.Structure):
    _fields_ = [("nu1", C.c_int), ("nu2", C.c_int), ("omega", C.c_double), ("omega_base", C.c_double),
                ("smoother_base", C.c_int), ("tol", C.c_double), ("max_cycles", C.c_int)]


def _La():
    lib = _L()
    if not getattr(lib, "_amr_ready", False):
        for name, (res, args) in _AMR_SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        lib._amr_ready = True
    return lib


@dataclass
class Amr:
    """Patch 0 = ``base`` (whole box); patch a >= 1 refines its parent by 2 on the node
    box ``boxes[a-1] = (lo, hi)`` or ``(lo, hi, parent)`` given in the node indices of
    its level (default parent a-1: one patch per level).  Parents come before their
    children.  Patch a >= 1 arrays live on the box grown by one padding node per side
    (see sbm_oracle.h)."""
    base: Problem
    boxes: list

    @property
    def nlev(self):
        return 1 + len(self.boxes)

    def parent(self, a):
        if a == 0:
            return -1
        b = self.boxes[a - 1]
        return b[2] if len(b) > 2 else a - 1

    def level(self, a):
        return 0 if a == 0 else self.level(self.parent(a)) + 1

    def c(self) -> _Amr:
        s = _Amr()
        s.base = self.base.c()
        s.nlev = self.nlev
        s.level[0], s.parent[0] = 0, -1
        for a, b in enumerate(self.boxes, start=1):
            lo, hi = b[0], b[1]
            lo3 = list(lo) + [0] * (3 - len(lo))
            hi3 = list(hi) + [0] * (3 - len(hi))
            for ax in range(3):
                s.lo[a][ax] = lo3[ax]
                s.hi[a][ax] = hi3[ax]
            s.parent[a] = self.parent(a)
            s.level[a] = self.level(a)
            assert 0 <= s.parent[a] < a
        return s

    def level_problem(self, a) -> Problem:
        out = _Problem()
        _La().orc_amr_level_problem(C.byref(self.c()), a, C.byref(out))
        return Problem(out.dim, tuple(out.n), out.h, out.c11, out.c12, out.c44, tuple(out.dirichlet))

    def origin(self, a):
        """global index (in patch a's level) of local node 0 of patch a's storage"""
        if a == 0:
            return (0, 0, 0)
        lo = list(self.boxes[a - 1][0]) + [0] * 3
        return tuple(lo[ax] - 1 if ax < self.base.dim else 0 for ax in range(3))

    def global_n(self, a):
        return tuple((self.base.n[ax] - 1) * 2 ** self.level(a) + 1 if ax < self.base.dim else 1
                     for ax in range(3))

    def owned(self, a, i, j, k=0) -> bool:
        return bool(_La().orc_amr_owned(C.byref(self.c()), a, i, j, k))


def _ptrs(arrs):
    arr = (C.POINTER(C.c_double) * len(arrs))()
    for i, a in enumerate(arrs):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
        arr[i] = a.ctypes.data_as(C.POINTER(C.c_double))
    return arr


def amr_coarsen_psi(A: Amr, psis):
    """In place: coarse cells under each patch <- mean of the fine cells."""
    _La().orc_amr_coarsen_psi(C.byref(A.c()), _ptrs(psis))
    return psis


def amr_fill(A: Amr, us):
    """In place: injection of owned fine values to covered coarse nodes, then
    ghost fill of every patch from its parent level."""
    _La().orc_amr_fill(C.byref(A.c()), _ptrs(us))
    return us


def amr_dJdpsi(A: Amr, us, lams):
    """Per-level cell gradients for the composite problem (see sbm_oracle.h)."""
    gs = [np.zeros(A.level_problem(a).ncells) for a in range(A.nlev)]
    _La().orc_amr_dJdpsi(C.byref(A.c()), _ptrs(us), _ptrs(lams), _ptrs(gs))
    return gs


def amr_residual_at(A: Amr, psis, fs, us, lev, nodes, comps):
    """Composite residual at sampled dofs: lev[s], global level node nodes[s] (3
    ints), component comps[s]; the arrays are not filled or modified."""
    lev = np.ascontiguousarray(lev, dtype=np.int32)
    nodes = np.ascontiguousarray(nodes, dtype=np.int32).reshape(-1, 3)
    comps = np.ascontiguousarray(comps, dtype=np.int32)
    r = np.zeros(len(lev))
    ip = C.POINTER(C.c_int)
    _La().orc_amr_residual_at(C.byref(A.c()), _ptrs(psis), _ptrs(fs), _ptrs(us), C.c_long(len(lev)),
                              lev.ctypes.data_as(ip), nodes.ctypes.data_as(ip), comps.ctypes.data_as(ip),
                              r.ctypes.data_as(C.POINTER(C.c_double)))
    return r


def amr_residual(A: Amr, psis, fs, us):
    """Composite residual per level (u is filled in place)."""
    rs = [np.zeros_like(u) for u in us]
    _La().orc_amr_residual(C.byref(A.c()), _ptrs(psis), _ptrs(fs), _ptrs(us), _ptrs(rs))
    return rs


def amr_solve(A: Amr, psis, fs, us, *, omega=0.5, omega_base=None, smoother_base="jacobi", nu1=2, nu2=2,
              tol=1e-14, max_cycles=200):
    """Composite solve by the oracle's correction iteration (orc_amr_solve): us
    (level arrays, initial guess with the Dirichlet values) are solved in place and
    filled.  psis must already hold the coarse means under the patches.  Returns a
    result with status, cycles and the relres history."""
    o = _AmrOpts(nu1, nu2, omega, omega if omega_base is None else omega_base,
                 1 if smoother_base in ("gs", "mcgs") else 0, tol, max_cycles)
    hist = np.zeros(max_cycles + 1)
    cyc = C.c_int()
    st = _La().orc_amr_solve(C.byref(A.c()), _ptrs(psis), _ptrs(fs), _ptrs(us), C.cast(C.byref(o), C.c_void_p),
                             hist.ctypes.data_as(C.POINTER(C.c_double)), C.byref(cyc))
    return MGResult(us, st, cyc.value, hist[: cyc.value + 1])


# ------------------------------------------------------------- regridding (Sec. 2.2)

def _apart(b1, b2, dim, gap=4):
    return any(b1[0][ax] >= b2[1][ax] + gap or b2[0][ax] >= b1[1][ax] + gap for ax in range(dim))


def _union(b1, b2, dim):
    return (tuple(min(b1[0][ax], b2[0][ax]) if ax < dim else 0 for ax in range(3)),
            tuple(max(b1[1][ax], b2[1][ax]) if ax < dim else 0 for ax in range(3)))


def _volume(b, dim):
    return int(np.prod([b[1][ax] - b[0][ax] for ax in range(dim)]))


def regrid_boxes(A: Amr, psis, level, threshold, grow, max_children=8):
    """New refinement boxes of ``level`` from the patches of level-1 of the hierarchy
    ``A`` (Sec. 2.2: refine where the indicator varies; the tagging criterion
    h |grad psi| > threshold), psis[a] = patch a's cell psi (storage layout, padding
    cells included).  Per parent patch, in patch order:
      - cells of the parent's allowed region (child nodes [amin, amax]: the whole
        level on the domain boundary, one parent cell inside the parent box
        elsewhere) are tagged where h |grad psi| > threshold, grad psi by centred
        differences of the cell values, a neighbour beyond the domain replaced by
        the cell itself (no gradient across the domain boundary);
      - the tags are dilated by ``grow`` cells (Chebyshev distance) and restricted
        to the allowed region;
      - connected components (cells sharing a face, edge or corner), in the order
        of their first cell in x-fastest order, give boxes: child nodes
        [2 c_min, 2 (c_max + 1)] clipped to [amin, amax], dropped if thinner than 2;
      - while two boxes are closer than two parent cells (4 child nodes) on every
        axis, the first such pair (i < j, in list order) becomes their union; while
        more than ``max_children`` remain, the first pair whose union adds the
        least volume is merged (and the closeness rule applied again);
      - the boxes are sorted (lo, then hi, x first).
    Returns [(lo, hi, parent)]."""
    from scipy import ndimage
    dim = A.base.dim
    out = []
    for pidx in range(A.nlev):
        if A.level(pidx) != level - 1:
            continue
        P = A.level_problem(pidx)
        o = A.origin(pidx)
        Np = A.global_n(pidx)
        ncs = [P.n[ax] - 1 if ax < dim else 1 for ax in range(3)]
        psi = np.asarray(psis[pidx], dtype=np.float64).reshape(ncs[2], ncs[1], ncs[0])
        amin, amax = [0, 0, 0], [0, 0, 0]
        for ax in range(dim):
            N = 2 * (Np[ax] - 1) + 1
            if pidx == 0:
                amin[ax], amax[ax] = 0, N - 1
            else:
                lo, hi = A.boxes[pidx - 1][0][ax], A.boxes[pidx - 1][1][ax]
                amin[ax] = 0 if lo == 0 else 2 * lo + 2
                amax[ax] = N - 1 if hi == Np[ax] - 1 else 2 * hi - 2
        # global cell index of storage cell l on axis ax: l + o[ax]; allowed cells C:
        # amin/2 <= C <= amax/2 - 1
        allowed = np.ones(psi.shape, bool)
        grids = np.meshgrid(*[np.arange(ncs[ax]) + o[ax] for ax in (2, 1, 0)], indexing="ij")
        for ax in range(dim):
            C = grids[2 - ax]
            allowed &= (C >= amin[ax] // 2) & (C <= amax[ax] // 2 - 1)
        tag = np.zeros(psi.shape, bool)
        idx = np.argwhere(allowed)
        for (k, j, i) in idx:
            g2 = 0.0
            for ax in range(dim):
                l = [i, j, k]
                up, dn = list(l), list(l)
                up[ax] += 1
                dn[ax] -= 1
                Cu, Cd = up[ax] + o[ax], dn[ax] + o[ax]
                if Cu > Np[ax] - 2:
                    up = l
                if Cd < 0:
                    dn = l
                d = (psi[up[2], up[1], up[0]] - psi[dn[2], dn[1], dn[0]]) / 2.0
                g2 += d * d
            tag[k, j, i] = np.sqrt(g2) > threshold
        conn = np.ones((3, 3, 3), bool)
        if dim == 2:
            conn[0] = conn[2] = False
        if grow:
            tag = ndimage.binary_dilation(tag, structure=conn, iterations=grow)
        tag &= allowed
        labels, _ = ndimage.label(tag, structure=conn)
        boxes = []
        for sls in ndimage.find_objects(labels):
            if sls is None:
                continue
            lo, hi = [0, 0, 0], [0, 0, 0]
            for ax in range(dim):
                sa = sls[2 - ax]
                lo[ax] = max(2 * (sa.start + o[ax]), amin[ax])
                hi[ax] = min(2 * (sa.stop + o[ax]), amax[ax])
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
        out.extend((b[0], b[1], pidx) for b in sorted(boxes))
    return out
