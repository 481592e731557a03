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


if __name__ == "__main__":
    which = sys.argv[1:] or ["maxcut_n4096", "completion_n400"]
    for name in which:
        rec = globals()[name]()
        with open(os.path.join(HERE, f"{name}_oracle.json"), "w") as f:
            json.dump(rec, f, indent=1)
        print(name, "written")
