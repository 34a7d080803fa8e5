"""GB300-native multigrid solver for smooth-boundary-method (SBM) elasticity.

Agrawal & Runnels, "Robust, strong form mechanics on an adaptive structured
grid" (arXiv 2212.02362): the diffuse-boundary equilibrium equation
div(psi C grad u) = source (Sec. 2.1), u at nodes and psi in cells (Sec. 2.3),
solved by geometric multigrid (Sec. 2.2) with Jacobi or colour Gauss-Seidel
smoothing.  Every step runs in the CUDA kernels of ``libsbm.so``; this module
only marshals torch tensors (device memory and streams) to the C ABI declared
in ``include/sbm.h``.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import torch

from . import _capi
from ._capi import (SBM_CUBIC, SBM_DIRICHLET, SBM_DIRICHLET_FROM_U, SBM_ERR_DIVERGED, SBM_ERR_NOCONV,
                    SBM_FP64, SBM_FREE, SBM_ISO_ENU, SBM_ISO_LAME, SBM_JACOBI, SBM_MCGS, SBM_MIXED, SBM_OK,
                    SBMError)

__all__ = ["Grid", "SolveInfo", "SBMSolve", "SBMError", "SBM_FP64", "SBM_MIXED", "SBM_JACOBI", "SBM_MCGS",
           "SBM_CUBIC", "SBM_ISO_LAME", "SBM_ISO_ENU", "SBM_FREE", "SBM_DIRICHLET", "SBM_DIRICHLET_FROM_U",
           "FACES", "lib"]

FACES = {"-x": 0, "+x": 1, "-y": 2, "+y": 3, "-z": 4, "+z": 5}


def lib():
    return _capi.load()


def _ptr(t: torch.Tensor, dtype=torch.float64) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise TypeError("expected a contiguous CUDA float64 tensor")
    return t.data_ptr()


@dataclass
class SolveInfo:
    status: int
    cycles: int
    vcycles: int
    levels: int
    r0: float
    relres: float
    history: list
    solve_ms: float
    launches: int = 0

    @property
    def converged(self) -> bool:
        return self.status == SBM_OK


def make_opts(tol=1e-10, max_cycles=500, nu1=2, nu2=2, omega=2.0 / 3.0, smoother="jacobi",
              inner_cycles=1, use_graph=True, inner_rtol=0.0) -> _capi.sbm_opts:
    o = _capi.sbm_opts()
    lib().sbm_default_opts(C.byref(o))
    o.tol, o.max_cycles, o.nu1, o.nu2, o.omega = tol, max_cycles, nu1, nu2, omega
    o.smoother = SBM_MCGS if smoother in ("gs", "mcgs", "rbgs") else SBM_JACOBI
    o.inner_cycles, o.use_graph, o.inner_rtol = inner_cycles, int(bool(use_graph)), inner_rtol
    return o


class Grid:
    """One node-centred grid (2D plane strain or 3D) and its multigrid hierarchy."""

    def __init__(self, dim: int, n, h: float, precision: str = "fp64", device: int = 0, stream=None):
        n = tuple(int(v) for v in n)
        if dim == 2 and len(n) == 2:
            n = n + (1,)
        d = _capi.sbm_grid_desc()
        d.dim = dim
        d.n[:] = list(n)
        d.h = h
        d.precision = SBM_MIXED if precision == "mixed" else SBM_FP64
        d.stream = stream
        d.device = device
        self._h = C.c_void_p()
        _capi.check(lib().sbm_grid_create(C.byref(d), C.byref(self._h)), None)
        self.dim, self.n, self.h, self.precision, self.device = dim, n, h, precision, device
        nl = C.c_int()
        self._check(lib().sbm_grid_levels(self._h, C.byref(nl)))
        self.nlevels = nl.value
        self.psi_min = None
        self.psi_version = 0      # bumped whenever the grid's psi changes

    # -- bookkeeping
    def _check(self, st, allow=(SBM_OK,)):
        return _capi.check(st, self._h, allow)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().sbm_grid_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def finest(self) -> int:
        return self.nlevels - 1

    def level_shape(self, level: int):
        n = (C.c_int * 3)()
        h = C.c_double()
        self._check(lib().sbm_grid_level_shape(self._h, level, n, C.byref(h)))
        return tuple(n), h.value

    def nnodes(self, level=None):
        n, _ = self.level_shape(self.finest if level is None else level)
        return n[0] * n[1] * n[2]

    def ncells(self, level=None):
        n, _ = self.level_shape(self.finest if level is None else level)
        return (n[0] - 1) * (n[1] - 1) * ((n[2] - 1) if self.dim == 3 else 1)

    # -- set-up
    def set_psi(self, psi: torch.Tensor, psi_min: float):
        self._check(lib().sbm_set_psi(self._h, self.finest, _ptr(psi), psi_min))
        self.psi_min = psi_min
        self.psi_version += 1

    def set_density(self, rho: torch.Tensor, psi_min: float, q: float = 3.0):
        self._check(lib().sbm_set_density(self._h, self.finest, _ptr(rho), psi_min, q))
        self.psi_min = psi_min
        self.psi_version += 1

    def set_moduli(self, kind: int, params):
        arr = (C.c_double * 3)(*[float(v) for v in (list(params) + [0.0, 0.0, 0.0])[:3]])
        self._check(lib().sbm_set_moduli(self._h, kind, arr))

    def set_bc(self, face, comp: int, kind: int = SBM_DIRICHLET, value: float = 0.0):
        face = FACES[face] if isinstance(face, str) else int(face)
        self._check(lib().sbm_set_bc(self._h, face, comp, kind, value))

    def set_source(self, f: torch.Tensor):
        self._check(lib().sbm_set_source(self._h, self.finest, _ptr(f)))

    # -- solves
    def solve(self, u: torch.Tensor, raise_on_fail: bool = True, **opts) -> SolveInfo:
        o = make_opts(**opts)
        info, hist = self._info(o.max_cycles)
        st = lib().sbm_solve(self._h, _ptr(u), C.byref(o), C.byref(info))
        self._check(st, allow=(SBM_OK,) if raise_on_fail else (SBM_OK, SBM_ERR_NOCONV, SBM_ERR_DIVERGED))
        return self._to_info(info, hist)

    def adjoint(self, u: torch.Tensor, dJdu: torch.Tensor, want_rho: bool = False, **opts):
        o = make_opts(**opts)
        info, hist = self._info(o.max_cycles)
        lam = torch.empty_like(dJdu)
        g = torch.empty(self.ncells(), dtype=torch.float64, device=u.device)
        grho = torch.empty_like(g) if want_rho else None
        st = lib().sbm_adjoint(self._h, _ptr(u), _ptr(dJdu), _ptr(lam), _ptr(g),
                               _ptr(grho) if grho is not None else None, C.byref(o), C.byref(info))
        self._check(st)
        return lam, g, grho, self._to_info(info, hist)

    def _info(self, cap):
        info = _capi.sbm_info()
        hist = (C.c_double * (cap + 1))()
        info.history = C.cast(hist, C.POINTER(C.c_double))
        info.history_capacity = cap + 1
        return info, hist

    @staticmethod
    def _to_info(info, hist) -> SolveInfo:
        n = min(info.cycles + 1, info.history_capacity)
        return SolveInfo(info.status, info.cycles, info.vcycles, info.levels, info.r0, info.relres,
                         [hist[i] for i in range(n)], info.solve_ms, info.launches)

    # -- block-structured refinement
    def amr_add_level(self, lo, hi):
        """A patch one level deeper than the deepest so far; returns its number."""
        deepest = max([lv for _, _, lv, _ in getattr(self, "patches", [])], default=0)
        return self.amr_add_box(deepest + 1, lo, hi)

    def amr_add_box(self, level, lo, hi):
        """A patch of refinement level ``level`` on the node box [lo, hi]; returns its
        number (the parent is found by the library)."""
        b = _capi.sbm_box()
        b.lo[:] = (list(lo) + [0, 0, 0])[:3]
        b.hi[:] = (list(hi) + [0, 0, 0])[:3]
        idx = C.c_int(0)
        self._check(lib().sbm_amr_add_box(self._h, level, C.byref(b), C.byref(idx)))
        self.boxes = getattr(self, "boxes", []) + [(tuple(b.lo), tuple(b.hi))]
        self.patches = getattr(self, "patches", []) + [(tuple(b.lo), tuple(b.hi), level, idx.value)]
        return idx.value

    def amr_regrid(self, level, threshold=0.1, grow=2):
        """Tag and cluster a new refinement level from the grid's psi (sbm_amr_regrid);
        returns the (lo, hi, index) of the patches added."""
        n = C.c_int(0)
        first = len(getattr(self, "patches", [])) + 1
        self._check(lib().sbm_amr_regrid(self._h, level, threshold, grow, C.byref(n)))
        shape = _capi.sbm_box()
        out = []
        for a in range(first, first + n.value):
            self._check(lib().sbm_amr_get_box(self._h, a, C.byref(shape), None, None))
            lo, hi = tuple(shape.lo), tuple(shape.hi)
            self.boxes = getattr(self, "boxes", []) + [(lo, hi)]
            self.patches = getattr(self, "patches", []) + [(lo, hi, level, a)]
            out.append((lo, hi, a))
        return out

    def amr_remove_levels(self, level: int):
        """Drop the patches of refinement level >= level (sbm_amr_remove_levels)."""
        self._check(lib().sbm_amr_remove_levels(self._h, level))
        kept = [p for p in getattr(self, "patches", []) if p[2] < level]
        self.patches = [(lo, hi, lv, i + 1) for i, (lo, hi, lv, _) in enumerate(kept)]
        self.boxes = [(lo, hi) for lo, hi, _, _ in self.patches]
        self.psi_version += 1

    def amr_set_psi(self, a: int, psi: torch.Tensor, psi_min: float):
        self._check(lib().sbm_amr_set_psi(self._h, a, _ptr(psi), psi_min))
        self.psi_version += 1

    def amr_set_source(self, a: int, f: torch.Tensor):
        self._check(lib().sbm_amr_set_source(self._h, a, _ptr(f)))

    @staticmethod
    def _ptr_array(ts):
        arr = (C.c_void_p * len(ts))()
        for i, t in enumerate(ts):
            arr[i] = _ptr(t)
        return arr

    def amr_solve(self, us, raise_on_fail: bool = True, **opts) -> SolveInfo:
        """Composite solve of the patch hierarchy; us[a] = level a's nodes (base
        packed, patches on their padded boxes), in: initial guess, out: solution.
        On mixed-precision grids ``inner_cycles`` FP32 correction cycles run per
        FP64 composite residual."""
        o = make_opts(**opts)
        info, hist = self._info(o.max_cycles)
        st = lib().sbm_amr_solve(self._h, self._ptr_array(us), C.byref(o), C.byref(info))
        self._check(st, allow=(SBM_OK,) if raise_on_fail else (SBM_OK, SBM_ERR_NOCONV, SBM_ERR_DIVERGED))
        return self._to_info(info, hist)

    def amr_adjoint(self, us, dJdus, raise_on_fail: bool = True, **opts):
        """lambda (per level) of A^T lambda = dJ/du for the composite operator and
        dJ/dpsi (per level cells, packed like the psi arrays)."""
        o = make_opts(**opts)
        info, hist = self._info(o.max_cycles)
        lams = [torch.zeros_like(u) for u in us]
        grads = []
        for a in range(len(us)):
            nc = self.ncells() if a == 0 else self._patch_ncells(a)
            grads.append(torch.zeros(nc, dtype=torch.float64, device=us[0].device))
        st = lib().sbm_amr_adjoint(self._h, self._ptr_array(us), self._ptr_array(dJdus), self._ptr_array(lams),
                                   self._ptr_array(grads), C.byref(o), C.byref(info))
        self._check(st, allow=(SBM_OK,) if raise_on_fail else (SBM_OK, SBM_ERR_NOCONV, SBM_ERR_DIVERGED))
        return lams, grads, self._to_info(info, hist)

    def _patch_ncells(self, a):
        lo, hi = self.boxes[a - 1]
        n = 1
        for ax in range(self.dim):
            n *= hi[ax] - lo[ax] + 2          # padded box nodes - 1
        return n

    def amr_residual(self, us):
        rs = [torch.empty_like(u) for u in us]
        nrm = C.c_double()
        self._check(lib().sbm_amr_residual(self._h, self._ptr_array(us), self._ptr_array(rs), C.byref(nrm)))
        return rs, nrm.value

    # -- single steps of the hot path
    def apply(self, level: int, u: torch.Tensor, fp32: bool = False) -> torch.Tensor:
        out = torch.empty_like(u)
        self._check(lib().sbm_apply(self._h, level, int(fp32), _ptr(u), _ptr(out)))
        return out

    def residual(self, level: int, f: torch.Tensor, u: torch.Tensor, fp32: bool = False):
        out = torch.empty_like(u)
        nrm = C.c_double()
        self._check(lib().sbm_residual(self._h, level, int(fp32), _ptr(f), _ptr(u), _ptr(out), C.byref(nrm)))
        return out, nrm.value

    def smooth(self, level: int, f: torch.Tensor, u: torch.Tensor, smoother="jacobi", omega=2.0 / 3.0,
               descending=False, fp32=False) -> torch.Tensor:
        out = u.clone()
        sm = SBM_MCGS if smoother in ("gs", "mcgs") else SBM_JACOBI
        self._check(lib().sbm_smooth(self._h, level, int(fp32), sm, omega, int(descending), _ptr(f), _ptr(out)))
        return out

    def restrict(self, level: int, r: torch.Tensor, fp32=False) -> torch.Tensor:
        nc = self.nnodes(level - 1) * self.dim
        out = torch.empty(nc, dtype=torch.float64, device=r.device)
        self._check(lib().sbm_restrict(self._h, level, int(fp32), _ptr(r), _ptr(out)))
        return out

    def prolong_add(self, level: int, e_c: torch.Tensor, u: torch.Tensor, fp32=False) -> torch.Tensor:
        out = u.clone()
        self._check(lib().sbm_prolong_add(self._h, level, int(fp32), _ptr(e_c), _ptr(out)))
        return out

    def get_psi(self, level: int) -> torch.Tensor:
        out = torch.empty(self.ncells(level), dtype=torch.float64, device=torch.device("cuda", self.device))
        self._check(lib().sbm_get_psi(self._h, level, _ptr(out)))
        return out

    def bottom_correct(self, f: torch.Tensor, u: torch.Tensor, fp32=False) -> torch.Tensor:
        out = u.clone()
        self._check(lib().sbm_bottom_correct(self._h, int(fp32), _ptr(f), _ptr(out)))
        return out

    def source_terms(self, psi: torch.Tensor, eps0=None, b=None, t=None, level=None) -> torch.Tensor:
        """Load f of K u = f from eq. SBMLinearElasticity: per-cell eigenstrain eps0
        (Voigt slots), nodal body force b and nodal diffuse traction t (each optional);
        psi in cells of `level` (default: the finest), used as given."""
        level = self.finest if level is None else level
        out = torch.empty(self.dim * self.nnodes(level), dtype=torch.float64, device=psi.device)
        opt = lambda x: None if x is None else _ptr(x)
        self._check(lib().sbm_source_terms(self._h, level, _ptr(psi), opt(eps0), opt(b), opt(t), _ptr(out)))
        return out

    # -- phase-field topology optimisation (Sec. 3.3)
    @staticmethod
    def _topopt_params(alpha, beta, zeta, lam, lam_rate, V0, mobility, dt, psi_min):
        return _capi.sbm_topopt_params(alpha, beta, zeta, lam, lam_rate, V0, mobility, dt, psi_min)

    def topopt_step(self, eta: torch.Tensor, u: torch.Tensor, *, alpha=200.0, beta=0.01, zeta=0.01, lam=400.0,
                    lam_rate=0.0, V0=0.25, mobility=1.0, dt=1e-4, psi_min=1e-6, step=0):
        """(eta', V(eta'), compliance): one explicit step of eq. topop_evolution at u."""
        prm = self._topopt_params(alpha, beta, zeta, lam, lam_rate, V0, mobility, dt, psi_min)
        out = torch.empty_like(eta)
        vol, comp = C.c_double(), C.c_double()
        self._check(lib().sbm_topopt_step(self._h, C.byref(prm), step, _ptr(eta), _ptr(u), _ptr(out),
                                          C.byref(vol), C.byref(comp)))
        return out, vol.value, comp.value

    def topopt_run(self, eta: torch.Tensor, u: torch.Tensor, steps: int, *, alpha=200.0, beta=0.01, zeta=0.01,
                   lam=400.0, lam_rate=0.0, V0=0.25, mobility=1.0, dt=1e-4, psi_min=1e-6, raise_on_fail=True,
                   **opts):
        """The staggered loop (eta and u updated in place); returns per-step
        compliance, volume and solve cycles, and the loop's wall time in ms."""
        prm = self._topopt_params(alpha, beta, zeta, lam, lam_rate, V0, mobility, dt, psi_min)
        o = make_opts(**opts)
        cap = max(steps, 1)
        comp, vol, cyc = (C.c_double * cap)(), (C.c_double * cap)(), (C.c_int * cap)()
        info = _capi.sbm_topopt_info(0, cap, C.cast(comp, C.POINTER(C.c_double)), C.cast(vol, C.POINTER(C.c_double)),
                                     C.cast(cyc, C.POINTER(C.c_int)), 0.0)
        st = lib().sbm_topopt_run(self._h, C.byref(prm), steps, _ptr(eta), _ptr(u), C.byref(o), C.byref(info))
        self._check(st, allow=(SBM_OK,) if raise_on_fail else (SBM_OK, SBM_ERR_NOCONV, SBM_ERR_DIVERGED))
        n = info.steps
        return {"steps": n, "compliance": list(comp[:n]), "volume": list(vol[:n]), "cycles": list(cyc[:n]),
                "ms": info.ms, "status": st}

    # -- the operator variants of Sec. 2.3 (product-rule strong form)
    def apply_product(self, variant: int, psi: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
        out = torch.empty_like(u)
        self._check(lib().sbm_apply_product(self._h, variant, _ptr(psi), _ptr(u), _ptr(out)))
        return out

    def jacobi_product(self, variant: int, psi: torch.Tensor, f: torch.Tensor, u: torch.Tensor, omega=2.0 / 3.0,
                       sweeps=1) -> torch.Tensor:
        out = u.clone()
        self._check(lib().sbm_jacobi_product(self._h, variant, _ptr(psi), _ptr(f), _ptr(out), omega, sweeps))
        return out

    def dJdpsi(self, u: torch.Tensor, lam: torch.Tensor) -> torch.Tensor:
        out = torch.empty(self.ncells(), dtype=torch.float64, device=u.device)
        self._check(lib().sbm_dJdpsi(self._h, _ptr(u), _ptr(lam), _ptr(out)))
        return out


class SBMSolve(torch.autograd.Function):
    """u = solve(K(psi(rho)) u = f) with the gradient of a loss of u w.r.t. rho.

    forward(rho, grid, u0, opts): sets the SIMP stiffness psi = psi_min + (1 - psi_min)
    rho^q on the grid (grid.psi_min, grid.q), solves from u0 and returns u.
    backward: the incoming dL/du is the right-hand side of the adjoint multigrid
    solve; the fused kernel returns dL/drho = -p'(rho) lambda_c^T S_c u_c.  The
    density of the forward pass is saved with the solution: when the grid's psi
    has changed since (another forward on the same grid), backward sets it again
    before the adjoint solve.
    """

    @staticmethod
    def forward(ctx, rho, grid, u0, opts):
        rho_c = rho.detach().contiguous()
        q = getattr(grid, "q", 3.0)
        grid.set_density(rho_c, grid.psi_min, q)
        u = u0.detach().clone().contiguous()
        grid.solve(u, **(opts or {}))
        ctx.grid, ctx.opts, ctx.q, ctx.psi_min = grid, opts, q, grid.psi_min
        ctx.version = grid.psi_version
        ctx.save_for_backward(u, rho_c)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        u, rho = ctx.saved_tensors
        if ctx.grid.psi_version != ctx.version:
            ctx.grid.set_density(rho, ctx.psi_min, ctx.q)
        _, _, grho, _ = ctx.grid.adjoint(u, grad_u.contiguous(), want_rho=True, **(ctx.opts or {}))
        return grho, None, None, None
