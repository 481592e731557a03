"""Write the stored expected values used by the full-size GPU parity tests.

Every number here comes from the CPU oracle (oracle/pf_oracle.py) on the
seeded synthetic workloads of pf_synthetic; nothing is taken from the CUDA
path.  Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402
import scipy.sparse as sp  # noqa: E402

import pf_synthetic as syn  # noqa: E402
from oracle import pf_oracle as o  # noqa: E402


def maxcut_n4096(iters=200):
    cfg, inst = syn.make_workload("maxcut_n4096")
    C = sp.csr_matrix((inst.C.vals, inst.C.colind, inst.C.rowptr), shape=(inst.n, inst.n))
    t0 = time.time()
    st, hist = o.maxcut_solve(C, inst.U0_raw[:, :cfg["p"]], cfg["degree"], iters)
    rec = {
        "workload": "maxcut_n4096",
        "source": "oracle/pf_oracle.py maxcut_solve (PFAM, Eqs. (PFAM1)-(PFAM2)), FP64 numpy",
        "n": inst.n, "p": cfg["p"], "degree": cfg["degree"], "iters": iters,
        "t": o.maxcut_step_size(C),
        "oracle_seconds": time.time() - t0,
        "obj": [h.obj for h in hist], "kkt": [h.kkt for h in hist],
        "pinf": [h.pinf for h in hist], "dinf": [h.dinf for h in hist],
        "gap": [h.gap for h in hist], "r_plus": [h.r_plus for h in hist],
        "a": [h.a for h in hist], "b": [h.b for h in hist],
        "theta_final": hist[-1].theta.tolist(),
        "lam_final_head": st.lam[:64].tolist(),
        "Z_final_samples": [[int(i), int(j), float(st.Z[i, j])] for i, j in
                            zip(*np.random.default_rng(0).integers(0, inst.n, (2, 64)))],
    }
    return rec


def completion_n400(iters=100):
    cfg, inst = syn.make_workload("completion_n400")
    p = cfg["p"]
    st, hist = o.completion_solve(inst.omega, inst.U0_raw[:, :p], cfg["mu"], cfg["t"],
                                  cfg["degree"], iters)
    st_ex, hist_ex = o.completion_solve(inst.omega, inst.U0_raw[:, :p], cfg["mu"], cfg["t"],
                                        cfg["degree"], iters, exact=True)
    return {
        "workload": "completion_n400",
        "source": "oracle/pf_oracle.py completion_solve (PFPG, Eqs. (pfpg1)-(pfpg2)) and its "
                  "full-EVD proximal-gradient counterpart, FP64 numpy",
        "n": inst.n, "p": p, "degree": cfg["degree"], "iters": iters,
        "obj": [h.obj for h in hist], "kkt": [h.kkt for h in hist],
        "r_plus": [h.r_plus for h in hist],
        "obj_full_evd": [h.obj for h in hist_ex], "kkt_full_evd": [h.kkt for h in hist_ex],
    }


# Workloads of the precision gate (tests/test_gpu_precision_gate.py): the
# optimum f* of each problem from the oracle run to a KKT residual of 1e-8.
# At a fixed point whose positive rank is below p the filtered iteration is
# the exact one (the subspace holds every positive eigenvector), so f* is
# the optimum of the convex problem itself, whatever the filter's precision.
PRECISION_MAXCUT = dict(n=2048, prob=0.01, p=64, degree=4, seed_offset=100, tol=1e-8,
                        max_iters=40000)
PRECISION_COMPLETION = dict(n=2048, rank=8, rate=0.1, p=32, degree=3, mu=0.05, t=1.0,
                            seed_offset=100, tol=1e-8, max_iters=20000)


def precision_maxcut_n2048():
    c = PRECISION_MAXCUT
    inst = syn.maxcut_instance(c["n"], c["prob"], c["p"], seed=syn.config_seed(2) + c["seed_offset"])
    C = sp.csr_matrix((inst.C.vals, inst.C.colind, inst.C.rowptr), shape=(inst.n, inst.n))
    t0 = time.time()
    st, hist = o.maxcut_solve(C, inst.U0_raw[:, :c["p"]], c["degree"], c["max_iters"],
                              tol=c["tol"])
    last = hist[-1]
    return {
        "workload": "precision_maxcut_n2048",
        "source": "oracle/pf_oracle.py maxcut_solve (PFAM, Eqs. (PFAM1)-(PFAM2)), FP64 numpy, "
                  "run to KKT <= tol",
        "config": c, "t": o.maxcut_step_size(C), "oracle_seconds": time.time() - t0,
        "iters": len(hist), "f_star": last.obj, "kkt": last.kkt, "pinf": last.pinf,
        "dinf": last.dinf, "gap": last.gap, "r_plus": last.r_plus,
        "dual_obj": float(np.sum(-st.lam / o.maxcut_step_size(C))),
        "kkt_trace": [[k + 1, h.kkt, h.obj] for k, h in enumerate(hist) if (k + 1) % 100 == 0],
    }


def precision_completion_n2048():
    c = PRECISION_COMPLETION
    inst = syn.completion_instance(c["n"], c["rank"], c["rate"], c["p"],
                                   syn.config_seed(3) + c["seed_offset"], mu=c["mu"], t=c["t"])
    t0 = time.time()
    st, hist = o.completion_solve(inst.omega, inst.U0_raw[:, :c["p"]], c["mu"], c["t"],
                                  c["degree"], c["max_iters"], tol=c["tol"])
    last = hist[-1]
    return {
        "workload": "precision_completion_n2048",
        "source": "oracle/pf_oracle.py completion_solve (PFPG, Eqs. (pfpg1)-(pfpg2)), FP64 "
                  "numpy, run to KKT <= tol",
        "config": c, "oracle_seconds": time.time() - t0, "nnz": inst.omega.nnz,
        "iters": len(hist), "f_star": last.obj, "kkt": last.kkt, "r_plus": last.r_plus,
        "kkt_trace": [[k + 1, h.kkt, h.obj] for k, h in enumerate(hist) if (k + 1) % 100 == 0],
    }


if __name__ == "__main__":
    which = sys.argv[1:] or ["maxcut_n4096", "completion_n400"]
    for name in which:
        rec = globals()[name]()
        with open(os.path.join(HERE, f"{name}_oracle.json"), "w") as f:
            json.dump(rec, f, indent=1)
        print(name, "written")
