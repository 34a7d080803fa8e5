"""Write oracle-only golden records for full-size workloads (tests/golden/*.json).

Every stored value comes from the CPU oracle (oracle/), run here on the seeded
inputs of workloads/.  A record holds, for each field the oracle computes (the
displacement u, for topology optimisation also the adjoint lambda and the
gradients dJ/dpsi, dJ/drho):
  - its values at a seeded sample of entries;
  - "sketches": its inner products with seeded random vectors w_j (entries
    uniform in [-1, 1]).  A difference e between a GPU field and the oracle field
    shows in every sketch as w_j . e, of size about |e| / sqrt(3), wherever e sits,
    so the sketches check the whole field and not only the samples;
  - its 2-norm.
plus the oracle's multigrid residual history and cycle counts.  The GPU tests
(tests/test_gpu_full_size.py) compare the CUDA results with these records, and
bench.py reports the error of its timed solve against the damage_3d records.

    python tests/golden/make_golden.py damage_3d_129      # ~4 min of one CPU core
    python tests/golden/make_golden.py topopt_3d          # ~20 min
    python tests/golden/make_golden.py voids_amr_2d       # 129^2 base + 3 levels
    python tests/golden/make_golden.py voids_amr_3d_65    # 65^3 base + 2 levels, ~6 h (400 cycles to its floor)
    python tests/golden/make_golden.py voids_amr_3d_clustered_129    # ~3 h
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

HERE = os.path.dirname(os.path.abspath(__file__))
NSKETCH = 8


def sketch_vectors(n, count=NSKETCH, seed=7100):
    """The seeded random vectors of the sketches (entries uniform in [-1, 1])."""
    return [W.uniform(seed + j, n, -1.0, 1.0) for j in range(count)]


def field_record(x, sample_seed, nsample=4096):
    idx = np.unique((W.uniform(sample_seed, nsample) * x.size).astype(np.int64))
    return {"sample_index": idx.tolist(), "sample": x[idx].tolist(),
            "sketch": [float(w @ x) for w in sketch_vectors(x.size)], "norm": float(np.linalg.norm(x))}


def _solve_to_floor(P, psi, f, u0, omega):
    """FP64 multigrid solve to relres 1e-14, or to the FP64 floor of the field (the
    rough SIMP fields stagnate near 1e-13): status 1 accepted when the history
    went below 1e-12."""
    res = oracle.mg_solve(P, psi, f, u0, omega=omega, tol=1e-14, max_cycles=150)
    hist = [float(v) for v in res.history]
    assert res.status == 0 or min(hist) <= 1e-12, (res.status, min(hist))
    return res, hist


def make_damage(name, wk):
    P = oracle.Problem(wk.dim, wk.n, wk.h, *wk.moduli, dirichlet=wk.dirichlet_bits())
    psi = oracle.floor_psi(wk.psi, wk.psi_min)
    t = time.time()
    res, hist = _solve_to_floor(P, psi, wk.f, wk.u0, wk.omega)
    dt = time.time() - t
    cyc10 = next(i for i, v in enumerate(hist) if v <= 1e-10)
    rec = {
        "workload": name,
        "source": "oracle/sbm_oracle.c orc_mg_solve, FP64, V(2,2) damped Jacobi, "
                  f"omega={wk.omega}, written by tests/golden/make_golden.py",
        "n": list(wk.n), "h": wk.h, "moduli": list(wk.moduli), "psi_min": wk.psi_min,
        "status": res.status, "cycles_to_1e-14": res.cycles, "cycles_to_1e-10": cyc10,
        "history": hist, "oracle_seconds": dt, "seconds_per_cycle": dt / max(res.cycles, 1),
        "u": field_record(res.u, 9001),
    }
    # the sample of the original record format (bench.py reads these two keys)
    rec["sample_index"] = rec["u"]["sample_index"]
    rec["sample_u"] = rec["u"]["sample"]
    rec["u_norm"] = rec["u"]["norm"]
    return rec


def make_topopt(name, wk):
    """Compliance J = h^3 f . u of the cantilever: the forward solution, the adjoint
    lambda of K lambda = dJ/du = h^3 f (homogeneous Dirichlet data), and the
    gradients dJ/dpsi_c = -lambda_c^T S_c u_c and dJ/drho = p'(rho) dJ/dpsi."""
    P = oracle.Problem(wk.dim, wk.n, wk.h, *wk.moduli, dirichlet=wk.dirichlet_bits())
    psi, dpsi = oracle.simp(wk.rho, wk.psi_min)
    t = time.time()
    res, hist = _solve_to_floor(P, psi, wk.f, wk.u0, wk.omega)
    mask = oracle.dirichlet_mask(P)
    dJdu = np.where(mask, 0.0, wk.h ** 3 * wk.f)
    adj, ahist = _solve_to_floor(P, psi, dJdu, np.zeros(P.ndofs), wk.omega)
    gpsi = oracle.dJdpsi(P, res.u, adj.u)
    dt = time.time() - t
    cyc10 = next(i for i, v in enumerate(hist) if v <= 1e-10)
    return {
        "workload": name,
        "source": "oracle/sbm_oracle.c orc_mg_solve (forward and adjoint, FP64, V(2,2) damped Jacobi, "
                  f"omega={wk.omega}) and orc_dJdpsi, written by tests/golden/make_golden.py",
        "n": list(wk.n), "h": wk.h, "moduli": list(wk.moduli), "psi_min": wk.psi_min,
        "status": res.status, "cycles": res.cycles, "cycles_to_1e-10": cyc10, "history": hist,
        "adjoint_cycles": adj.cycles, "adjoint_history": ahist, "oracle_seconds": dt,
        "compliance": float(wk.h ** 3 * wk.f @ res.u),
        "u": field_record(res.u, 9101), "lambda": field_record(adj.u, 9102),
        "dJdpsi": field_record(gpsi, 9103), "dJdrho": field_record(gpsi * dpsi, 9103),
    }


def amr_oracle(wk):
    """The oracle's composite problem for a refinement workload: levels, boxes, psi
    floored at psi_min with the coarse means under the patches."""
    P = oracle.Problem(wk.dim, wk.n, wk.h, *wk.moduli, dirichlet=wk.dirichlet_bits())
    A = oracle.Amr(P, [(b[0][:wk.dim], b[1][:wk.dim], wk.parent(a)) for a, b in enumerate(wk.boxes, start=1)])
    psis = [np.ascontiguousarray(np.maximum(wk.level_psi(a), wk.psi_min)) for a in range(A.nlev)]
    oracle.amr_coarsen_psi(A, psis)
    return A, psis


def make_amr(name, wk):
    """Composite solution of a refinement workload (no load; Dirichlet data from the
    workload's initial guess) by the oracle's correction iteration to relres 1e-14
    (or its FP64 floor).  Every level's filled storage array is recorded."""
    A, psis = amr_oracle(wk)
    fs = [np.zeros(A.level_problem(a).ndofs) for a in range(A.nlev)]
    us = [np.ascontiguousarray(wk.level_u0(a)) for a in range(A.nlev)]
    t = time.time()
    res = oracle.amr_solve(A, psis, fs, us, omega=0.5, omega_base=wk.omega,
                           smoother_base="gs" if wk.smoother in ("gs", "mcgs") else "jacobi",
                           tol=1e-14, max_cycles=400)
    dt = time.time() - t
    hist = [float(v) for v in res.history]
    assert res.status == 0 or min(hist) <= 1e-12, (res.status, min(hist))
    return {
        "workload": name,
        "source": "oracle/sbm_oracle.c orc_amr_solve (composite correction iteration, FP64) of the composite "
                  "problem of orc_amr_residual, written by tests/golden/make_golden.py",
        "n": list(wk.n), "h": wk.h, "moduli": list(wk.moduli), "psi_min": wk.psi_min,
        "boxes": [[list(b[0]), list(b[1])] + ([b[2]] if len(b) > 2 else []) for b in wk.boxes],
        "status": res.status, "cycles": res.cycles, "history": hist, "oracle_seconds": dt,
        "levels": [field_record(us[a], 9200 + a) for a in range(A.nlev)],
    }


def voids_amr_3d(n0):
    return W.voids_amr(3, n0, 2, count=16, rmin=0.04, rmax=0.12)


def voids_amr_3d_clustered(n0):
    return W.voids_amr(3, n0, 2, count=8, rmin=0.04, rmax=0.08, clustered=True)


RECIPES = {
    "damage_3d_129": (lambda: W.damage3d(129), make_damage),
    "damage_3d_65": (lambda: W.damage3d(65), make_damage),
    "topopt_3d": (lambda: W.topopt3d(), make_topopt),
    "voids_amr_2d": (lambda: W.voids_amr(2, 129, 3), make_amr),
    "voids_amr_3d_65": (lambda: voids_amr_3d(65), make_amr),
    "voids_amr_3d_33": (lambda: voids_amr_3d(33), make_amr),
    "voids_amr_2d_clustered": (lambda: W.voids_amr(2, 129, 3, clustered=True), make_amr),
    "voids_amr_3d_clustered_65": (lambda: voids_amr_3d_clustered(65), make_amr),
    "voids_amr_3d_clustered_129": (lambda: voids_amr_3d_clustered(129), make_amr),
}


def make(name):
    build, writer = RECIPES[name]
    rec = writer(name, build())
    out = os.path.join(HERE, f"{name}_oracle.json")
    with open(out, "w") as fh:
        json.dump(rec, fh)
    print(out, rec.get("status"), f"{rec['oracle_seconds']:.1f}s")


if __name__ == "__main__":
    for name in sys.argv[1:] or ["damage_3d_65"]:
        make(name)
