"""Write oracle-only golden records for full-size workloads (tests/golden/*.json).

Every stored value comes from the CPU oracle (oracle/), run here on the seeded
inputs of workloads/: the multigrid residual history of the FP64 solve, the
cycles it needs to reach relres 1e-10, and the solution converged to 1e-14 at a
seeded sample of dofs.  The GPU tests compare the CUDA solve with these samples.

    python tests/golden/make_golden.py damage_3d_129      # ~10 min of one CPU core
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as W  # noqa: E402

RECIPES = {
    "damage_3d_129": lambda: W.damage3d(129),
    "damage_3d_65": lambda: W.damage3d(65),
}


def make(name, nsample=4096):
    wk = RECIPES[name]()
    P = oracle.Problem(wk.dim, wk.n, wk.h, *wk.moduli, dirichlet=wk.dirichlet_bits())
    psi = oracle.floor_psi(wk.psi, wk.psi_min)
    t = time.time()
    res = oracle.mg_solve(P, psi, wk.f, wk.u0, omega=wk.omega, tol=1e-14, max_cycles=500)
    dt = time.time() - t
    hist = [float(v) for v in res.history]
    cyc10 = next(i for i, v in enumerate(hist) if v <= 1e-10)
    idx = np.unique((W.uniform(9001, nsample) * P.ndofs).astype(np.int64))
    rec = {
        "workload": name,
        "source": "oracle/sbm_oracle.c orc_mg_solve, FP64, V(2,2) damped Jacobi, "
                  f"omega={wk.omega}, written by tests/golden/make_golden.py",
        "n": list(wk.n), "h": wk.h, "moduli": list(wk.moduli), "psi_min": wk.psi_min,
        "status": res.status, "cycles_to_1e-14": res.cycles, "cycles_to_1e-10": cyc10,
        "history": hist, "oracle_seconds": dt, "seconds_per_cycle": dt / max(res.cycles, 1),
        "sample_index": idx.tolist(), "sample_u": res.u[idx].tolist(),
        "u_norm": float(np.linalg.norm(res.u)),
    }
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}_oracle.json")
    with open(out, "w") as fh:
        json.dump(rec, fh)
    print(out, res.status, res.cycles, cyc10, f"{dt:.1f}s")


if __name__ == "__main__":
    for name in sys.argv[1:] or ["damage_3d_65"]:
        make(name)
