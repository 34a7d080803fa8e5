"""Shared test helpers: build the same problem for the oracle and the CUDA library."""
import numpy as np

import oracle
import workloads as W


def oracle_problem(wk):
    return oracle.Problem(wk.dim, wk.n, wk.h, *wk.moduli, dirichlet=wk.dirichlet_bits())


def cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def gpu_grid(wk, precision="fp64", density=False, bc_values=False):
    """CUDA grid for workload ``wk``; Dirichlet values are taken from u0 unless
    ``bc_values`` (then they are written by the library from constant face values)."""
    import paper_2212_02362_gb300 as sbm
    g = sbm.Grid(wk.dim, wk.n, wk.h, precision=precision)
    g.set_moduli(sbm.SBM_CUBIC, wk.moduli)
    for face, comp, value in wk.bcs:
        if bc_values:
            g.set_bc(face, comp, sbm.SBM_DIRICHLET, float(value))
        else:
            g.set_bc(face, comp, sbm.SBM_DIRICHLET_FROM_U)
    if density and wk.rho is not None:
        g.q = 3.0
        g.psi_min = wk.psi_min
        g.set_density(cuda(wk.rho), wk.psi_min, 3.0)
    else:
        g.set_psi(cuda(wk.psi), wk.psi_min)
    g.set_source(cuda(wk.f))
    return g


def random_workload(dim, n, seed, moduli=(1.0, 0.6, 0.5), psi_lo=1e-3, bits=None):
    """A grid with uniform random psi in [psi_lo, 1], random Dirichlet data on the
    faces in ``bits`` and a random load, for step-by-step parity tests."""
    n = tuple(n) if dim == 3 else (n[0], n[1], 1)
    h = 1.0 / (n[0] - 1)
    nc = (n[0] - 1) * (n[1] - 1) * ((n[2] - 1) if dim == 3 else 1)
    psi = W.uniform(seed, nc, psi_lo, 1.0)
    N = n[0] * n[1] * n[2]
    f = W.uniform(seed + 1, dim * N, -1.0, 1.0)
    faces = ["-x", "+x", "-y", "+y", "-z", "+z"][: 2 * dim]
    if bits is None:
        bcs = [("-y" if dim == 2 else "-z", p, 0.0) for p in range(dim)] + [("+x", 0, 0.01)]
    else:
        bcs = [(faces[fi], p, 0.003 * (fi + 1) * (p + 1)) for p in range(dim) for fi in range(2 * dim)
               if bits[p] >> fi & 1]
    u0 = W.initial_guess(dim, n, bcs)
    return W.Workload(f"random{dim}d", dim, n, h, moduli, bcs, psi, psi_lo, f, u0)
