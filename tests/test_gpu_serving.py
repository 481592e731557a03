"""Serving loop (continuous batching): every result is the same alone and
in the mix, admission respects the HBM budget, and queued requests are
admitted while others are in flight.

The kernels' reductions are in a fixed order and requests share no device
state, so a request's arithmetic does not depend on what else is running:
results alone and in the mix must agree bitwise; the stated tolerance
(objective relative 1e-12) is a safety margin."""
import numpy as np
import pytest

import pf_synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _requests(n_req=8, seed=3):
    from paper_1904_10585_gb300.serving import Request
    mix = syn.serving_mix(n_req, seed, p=16, maxcut_n=(200, 600), completion_n=(300, 900),
                          rank=(2, 6), rate=(0.05, 0.2), maxcut_prob=0.05)
    reqs = []
    for i, m in enumerate(mix):
        inst = m["inst"]
        if m["kind"] == "maxcut":
            c = inst.C
            reqs.append(Request(i, "maxcut", m["n"], 0.0, c.rowptr, c.colind, c.vals,
                                inst.U0_raw, max_iter=40))
        else:
            c = inst.omega
            reqs.append(Request(i, "completion", m["n"], 0.0, c.rowptr, c.colind, c.vals,
                                inst.U0_raw, max_iter=30))
    return reqs


@pytest.mark.parametrize("maxcut_lowprec", [False, True])
def test_results_alone_equal_results_in_mix(maxcut_lowprec):
    from paper_1904_10585_gb300 import serving as SV
    reqs = _requests()
    kw = dict(slots=[("maxcut", 600, 3), ("completion", 900, 3)], p=16, degree=3, tol=0.0,
              chunk=5, maxcut_lowprec=maxcut_lowprec, completion_lowprec=maxcut_lowprec)
    srv = SV.Server(**kw)
    try:
        mix = {r.rid: r for r in srv.run(reqs)}
    finally:
        srv.close()
    alone = {r.rid: r for r in SV.run_alone(reqs, **dict(kw, slots=[("maxcut", 600, 1),
                                                                      ("completion", 900, 1)]))}
    assert set(mix) == set(alone) == {r.rid for r in reqs}
    for rid in mix:
        a, b = mix[rid], alone[rid]
        assert a.iters == b.iters
        assert abs(a.obj - b.obj) <= 1e-12 * max(1.0, abs(b.obj)), (rid, a.obj, b.obj)
        np.testing.assert_array_equal(a.theta, b.theta)


def test_admission_respects_budget_and_overlaps():
    from paper_1904_10585_gb300 import serving as SV
    reqs = _requests(10, seed=5)
    biggest = max(SV.problem_bytes(r.kind, r.n, r.colind.shape[0], 16, False) for r in reqs)
    budget = int(2.5 * biggest)
    srv = SV.Server(slots=[("maxcut", 600, 4), ("completion", 900, 4)], p=16, degree=3, tol=0.0,
                    chunk=5, hbm_budget=budget, maxcut_lowprec=False)
    peak = [0]
    orig = srv._admit

    def admit(slot, r, now):
        orig(slot, r, now)
        peak[0] = max(peak[0], srv.used)
    srv._admit = admit
    try:
        res = srv.run(reqs)
    finally:
        srv.close()
    assert len(res) == len(reqs)
    assert peak[0] <= budget
    # at least two requests were in flight at the same time
    spans = sorted((r.admitted, r.finished) for r in res)
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))
