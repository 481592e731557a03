"""Full-size parity at the benchmark's configuration (max-cut SDP, n = 4096,
p = 32, degree 4, 200 PFAM iterations, dense FP64 iteration matrix), in the
launch configuration bench.py times (one CUDA-graph step replayed by
pf_solve), against stored oracle values (tests/golden/maxcut_n4096_oracle.json,
written by tests/golden/make_golden.py from oracle/ only).

Checked: the final objective (relative 1e-9), the per-iteration objectives of
a step-by-step run (relative 1e-9), the final Ritz values (1e-9 of max|theta|),
the KKT components, and 64 sampled entries of the final Z (1e-9 of max|Z|)."""
import json
import os

import numpy as np
import pytest

import pf_synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "maxcut_n4096_oracle.json")
DEV = "cuda:0"


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as f:
        return json.load(f)


def _setup(S):
    cfg, inst = syn.make_workload("maxcut_n4096")
    rp, ci, cv = S.csr_to_device(inst.C, DEV, torch.float64)
    U0 = torch.from_numpy(np.ascontiguousarray(inst.U0_raw[:, :cfg["p"]])).to(DEV)
    return cfg, rp, ci, cv, U0


def test_maxcut_n4096_graph_solve_matches_oracle(golden):
    from paper_1904_10585_gb300 import solver as S
    cfg, rp, ci, cv, U0 = _setup(S)
    with S.Context(p=cfg["p"], n_max=cfg["n"], degree=cfg["degree"],
                   stream=torch.cuda.Stream()) as ctx:
        pr = S.maxcut_problem(rp, ci, cv, U0)
        S.problem_init(ctx, pr)
        assert abs(pr.t - golden["t"]) <= 1e-14 * golden["t"]
        res = S.solve(ctx, pr, golden["iters"], 0.0)
        ctx.stream.synchronize()
        assert res.iters == golden["iters"]
        ob = golden["obj"][-1]
        assert abs(res.obj - ob) <= 1e-9 * abs(ob), (res.obj, ob)
        last = res.last
        for key in ("pinf", "gap"):
            g = golden[key][-1]
            assert abs(getattr(last, key) - g) <= 1e-8 * max(abs(g), 1e-6), key
        # dinf from the factors of X~_{k-1}, X~_k (cancellation of O(||X~||^2) terms)
        assert abs(last.dinf - golden["dinf"][-1]) <= 1e-5 * max(golden["dinf"][-1], 1e-2)
        assert last.r_plus == golden["r_plus"][-1]
        th = pr.theta.cpu().numpy()
        tg = np.array(golden["theta_final"])
        assert np.max(np.abs(th - tg)) <= 1e-9 * np.max(np.abs(tg))
        Z = pr.Z.cpu().numpy()
        zs = np.array([Z[i, j] for i, j, _ in golden["Z_final_samples"]])
        zg = np.array([v for _, _, v in golden["Z_final_samples"]])
        zmax = float(np.abs(Z).max())
        assert np.max(np.abs(zs - zg)) <= 1e-9 * zmax
        lam = pr.lam.cpu().numpy()[:64]
        assert np.max(np.abs(lam - np.array(golden["lam_final_head"]))) <= 1e-9 * np.abs(lam).max()


def test_maxcut_n4096_stepwise_objectives_match_oracle(golden):
    from paper_1904_10585_gb300 import solver as S
    cfg, rp, ci, cv, U0 = _setup(S)
    k_max = 60
    with S.Context(p=cfg["p"], n_max=cfg["n"], degree=cfg["degree"],
                   stream=torch.cuda.Stream()) as ctx:
        pr = S.maxcut_problem(rp, ci, cv, U0)
        S.problem_init(ctx, pr)
        for k in range(k_max):
            info = S.prox_step(ctx, pr)
            ob = golden["obj"][k]
            assert abs(info.obj - ob) <= 1e-9 * max(1.0, abs(ob)), (k, info.obj, ob)
            assert abs(info.a - golden["a"][k]) <= 1e-12 * abs(golden["a"][k])
            assert abs(info.b - golden["b"][k]) <= 1e-9 * max(1.0, abs(golden["b"][k]))
