"""Precision gate: solves whose filter runs in low precision, against the
optimum f* that the FP64 oracle reaches at a KKT residual of 1e-8
(tests/golden/precision_*_oracle.json, written by tests/golden/make_golden.py
from oracle/ only).

For each precision the solve must end with an FP64-evaluated relative KKT
residual <= 1e-4 and an objective within 1e-6 of f* (relative).  A KKT
residual of 1e-4 alone does not fix the objective to 1e-6 (on the max-cut
workload below the oracle's own iterate is 1.8e-6 away at the 1e-4 crossing
and 4.5e-7 at 1e-5), so the max-cut solves run to 3e-6 and the completion
solve to 1e-7, and the report gives the error at both points.

Max-cut SDP, n = 2048, Erdos-Renyi p = 0.01 with +-1 weights, p = 64,
degree 4 (the adaptive ladder may raise it to 8): the bf16 and the tf32
dense-shadow filters on the tensor cores (several passes of each TMA ring,
64-column blocks), the bf16 ladder with a tf32 rung, and the FP64 sliced path
for reference.  PSD completion, n = 2048, rank 8, 10% sampling, p = 32: the
fp32 low-rank + sparse filter with FP64 Rayleigh-Ritz."""
import json
import os

import numpy as np
import pytest

import pf_synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.join(os.path.dirname(__file__), "golden")
DEV = "cuda:0"
KKT_GATE = 1e-4
OBJ_GATE = 1e-6
SOLVE_TOL = 3e-6


def _golden(name):
    path = os.path.join(HERE, f"{name}_oracle.json")
    if not os.path.exists(path):
        pytest.skip(f"{path} not written")
    with open(path) as f:
        return json.load(f)


def _trace_solve(S, ctx, pr, tol, max_iter, every=10):
    """Solve in chunks of `every` steps (the graph path), recording the
    report at each chunk end; stops at tol."""
    trace = []
    it = 0
    while it < max_iter:
        res = S.solve(ctx, pr, every, 0.0, every)
        it += every
        trace.append((it, res.last.kkt, res.last.obj, res.last.precision, res.last.degree))
        if res.last.kkt <= tol:
            break
    return trace


PREC_NAME = {0: "fp64", 1: "tf32", 2: "bf16"}


def _report(name, trace, f_star):
    first = next((t for t in trace if t[1] <= KKT_GATE), None)
    it, kkt, obj, prec, deg = trace[-1]
    err = abs(obj - f_star) / abs(f_star)
    err_gate = abs(first[2] - f_star) / abs(f_star) if first else float("nan")
    # the ladder's rungs: (precision, degree) and the iterations each ran
    rungs, prev, start = [], None, 0
    for t in trace:
        key = (PREC_NAME.get(t[3], t[3]), t[4])
        if key != prev:
            if prev is not None:
                rungs.append(f"{prev[0]}/d{prev[1]} {start}-{t[0] - 10}")
            prev, start = key, t[0] - 10
    rungs.append(f"{prev[0]}/d{prev[1]} {start}-{it}")
    print(f"\n{name}: {it} iterations, kkt {kkt:.2e}, obj {obj:.12g}, f* {f_star:.12g}, "
          f"relative error {err:.2e}; at the KKT 1e-4 crossing (iteration "
          f"{first[0] if first else None}, {PREC_NAME.get(first[3]) if first else None}): "
          f"{err_gate:.2e}; rungs: {', '.join(rungs)}")
    return kkt, err


@pytest.fixture(scope="module")
def S():
    from paper_1904_10585_gb300 import solver
    return solver


@pytest.mark.parametrize("mode", ["bf16", "tf32", "bf16_ladder_tf32", "fp64"])
def test_maxcut_precision_gate(S, mode):
    import paper_1904_10585_gb300 as pkg
    g = _golden("precision_maxcut_n2048")
    c = g["config"]
    inst = syn.maxcut_instance(c["n"], c["prob"], c["p"], seed=syn.config_seed(2) + c["seed_offset"])
    rp, ci, v = S.csr_to_device(inst.C, DEV, torch.float64)
    U0 = torch.from_numpy(np.ascontiguousarray(inst.U0_raw[:, :c["p"]])).to(DEV)
    prec = {"bf16": pkg.PF_PREC_BF16, "tf32": pkg.PF_PREC_TF32,
            "bf16_ladder_tf32": pkg.PF_PREC_BF16, "fp64": pkg.PF_PREC_FP64}[mode]
    with S.Context(p=c["p"], n_max=c["n"], degree=c["degree"], degree_max=8,
                   adaptive=0 if mode == "fp64" else 1, precision=prec,
                   stream=torch.cuda.Stream()) as ctx:
        if mode == "fp64":
            pr = S.maxcut_problem(rp, ci, v, U0)
        else:
            lp = "tf32" if mode == "tf32" else "bf16"
            pr = S.maxcut_problem(rp, ci, v, U0, dense=False, lowprec=lp,
                                  tf32_rung=(mode == "bf16_ladder_tf32"))
        S.problem_init(ctx, pr)
        assert abs(pr.t - g["t"]) <= 1e-14 * g["t"]
        trace = _trace_solve(S, ctx, pr, SOLVE_TOL, 30000)
    kkt, err = _report(f"max-cut n={c['n']} {mode}", trace, g["f_star"])
    assert kkt <= KKT_GATE
    assert err <= OBJ_GATE, err
    if mode == "bf16_ladder_tf32":
        # the ladder passed through the tf32 rung before any FP64 step
        precs = [t[3] for t in trace]
        if pkg.PF_PREC_FP64 in precs:
            first64 = precs.index(pkg.PF_PREC_FP64)
            assert pkg.PF_PREC_TF32 in precs[:first64]


def test_completion_fp32_filter_gate(S):
    import paper_1904_10585_gb300 as pkg
    g = _golden("precision_completion_n2048")
    c = g["config"]
    inst = syn.completion_instance(c["n"], c["rank"], c["rate"], c["p"],
                                   syn.config_seed(3) + c["seed_offset"], mu=c["mu"], t=c["t"])
    rp, ci, v = S.csr_to_device(inst.omega, DEV)
    U0 = torch.from_numpy(np.ascontiguousarray(inst.U0_raw[:, :c["p"]])).to(DEV)
    with S.Context(p=c["p"], n_max=c["n"], degree=c["degree"], degree_max=c["degree"] + 3,
                   adaptive=1, precision=pkg.PF_PREC_BF16, stream=torch.cuda.Stream()) as ctx:
        pr = S.completion_problem(rp, ci, v, U0, mu=c["mu"], t=c["t"])
        S.problem_init(ctx, pr)
        trace = _trace_solve(S, ctx, pr, 1e-7, 20000)
    kkt, err = _report(f"completion n={c['n']} fp32 filter", trace, g["f_star"])
    assert kkt <= KKT_GATE
    assert err <= OBJ_GATE, err
