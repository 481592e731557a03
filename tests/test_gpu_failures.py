"""Failure paths of the C ABI, exercised without faulting the GPU.

* A workspace larger than the device: pf_create returns PF_ERR_OOM (the
  failed cudaMalloc is not a sticky error) and a normal context still works.
* A bounded wait that runs out: pf_set_wait_limit(0) makes the tensor-core
  pipeline of the sliced dense product give up at its first wait that is not
  already satisfied.  The kernel lets its issued copies and MMAs land, frees
  its tensor memory and sets flags bit 3; pf_prox_step returns
  PF_ERR_DEVICE_TIMEOUT.  With the limit restored the same context then runs
  the problem again bitwise like a fresh context.
* A non-finite input value: PF_ERR_NAN with flags bit 2, and the context
  keeps working on clean data.
* A non-finite cost matrix is rejected by pf_problem_init (host check).
* A tolerance that is not reached: pf_solve returns PF_ERR_NOT_CONVERGED with
  the report of its last step.
"""
import ctypes

import numpy as np
import pytest

import pf_synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def pf():
    import paper_1904_10585_gb300 as pkg
    from paper_1904_10585_gb300 import solver
    return pkg, solver


def t64(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(DEV)


def raw_step(pkg, ctx, pr):
    info = pkg.pf_iter_info()
    st = pkg.raw_call("pf_prox_step", ctx.handle, ctypes.byref(pr.struct), ctypes.byref(info))
    return st, info


def test_workspace_beyond_device_memory_is_oom(pf):
    pkg, S = pf
    total = torch.cuda.get_device_properties(0).total_memory
    n_max = 200_000_000          # 4 n x 64 FP64 blocks alone: ~410 GB
    assert 4 * n_max * 64 * 8 > total
    opt = pkg.pf_options(p=64, degree=4, degree_max=4, q=1, eta=0.1, precision=0, adaptive=0,
                         p_min=8, adapt_guard=0, adapt_every=10, dense_product=0)
    out = ctypes.c_void_p()
    stream = torch.cuda.Stream()
    st = pkg.raw_call("pf_create", ctypes.byref(opt), n_max, stream.cuda_stream,
                      ctypes.byref(out))
    assert st == pkg.PF_ERR_OOM
    assert not out.value
    # the failed allocation left no error behind: a normal context works
    inst = syn.completion_instance(120, 3, 0.3, 8, seed=12)
    rp, ci, v = S.csr_to_device(inst.omega, DEV)
    with S.Context(p=8, n_max=120, degree=3, stream=stream) as ctx:
        pr = S.completion_problem(rp, ci, v, t64(inst.U0_raw), mu=0.05)
        S.problem_init(ctx, pr)
        info = S.prox_step(ctx, pr)
        assert np.isfinite(info.obj) and info.flags == 0


def _maxcut(S, n, p, seed):
    inst = syn.maxcut_instance(n, 0.04, p, seed=seed)
    rp, ci, v = S.csr_to_device(inst.C, DEV, torch.float64)
    return inst, (rp, ci, v)


def test_wait_limit_running_out_reports_device_timeout(pf):
    pkg, S = pf
    n, p, d, steps = 520, 32, 4, 3
    inst, csr = _maxcut(S, n, p, seed=7)
    stream = torch.cuda.Stream()
    with S.Context(p=p, n_max=n, degree=d, stream=stream) as ctx:
        pr = S.maxcut_problem(*csr, t64(inst.U0_raw[:, :p]))
        S.problem_init(ctx, pr)
        torch.cuda.synchronize()
        try:
            pkg.pf_set_wait_limit(0)
            st, info = raw_step(pkg, ctx, pr)
        finally:
            torch.cuda.synchronize()
            pkg.pf_set_wait_limit(2_000_000_000)
        assert st == pkg.PF_ERR_DEVICE_TIMEOUT, pkg.pf_status_string(st)
        assert info.flags & 8
        # the same context, limit restored, runs the problem from the start
        pr2 = S.maxcut_problem(*csr, t64(inst.U0_raw[:, :p]))
        S.problem_init(ctx, pr2)
        h_again = [S.prox_step(ctx, pr2) for _ in range(steps)]
    with S.Context(p=p, n_max=n, degree=d, stream=torch.cuda.Stream()) as fresh:
        pr3 = S.maxcut_problem(*csr, t64(inst.U0_raw[:, :p]))
        S.problem_init(fresh, pr3)
        h_fresh = [S.prox_step(fresh, pr3) for _ in range(steps)]
    for a, b in zip(h_again, h_fresh):
        assert a.flags == 0 and b.flags == 0
        assert a.obj == b.obj and a.kkt == b.kkt
    assert torch.equal(pr2.V, pr3.V)


def test_nan_sample_reports_nan(pf):
    pkg, S = pf
    n, p, d = 150, 8, 3
    inst = syn.completion_instance(n, 3, 0.3, p, seed=21)
    vals = inst.omega.vals.copy()
    vals[len(vals) // 2] = np.nan
    rp, ci, v_bad = S.csr_to_device(syn.CSR(n, inst.omega.rowptr, inst.omega.colind, vals), DEV)
    _, _, v_ok = S.csr_to_device(inst.omega, DEV)
    with S.Context(p=p, n_max=n, degree=d, stream=torch.cuda.Stream()) as ctx:
        pr = S.completion_problem(rp, ci, v_bad, t64(inst.U0_raw), mu=0.05)
        S.problem_init(ctx, pr)
        st, info = raw_step(pkg, ctx, pr)
        assert st == pkg.PF_ERR_NAN, pkg.pf_status_string(st)
        assert info.flags & 4
        # clean data on the same context
        pr2 = S.completion_problem(rp, ci, v_ok, t64(inst.U0_raw), mu=0.05)
        S.problem_init(ctx, pr2)
        info2 = S.prox_step(ctx, pr2)
        assert info2.flags == 0 and np.isfinite(info2.obj)


def test_nonfinite_cost_matrix_is_rejected(pf):
    pkg, S = pf
    inst, (rp, ci, v) = _maxcut(S, 100, 8, seed=3)
    v = v.clone()
    v[5] = float("inf")
    with S.Context(p=8, n_max=100, degree=3, stream=torch.cuda.Stream()) as ctx:
        pr = S.maxcut_problem(rp, ci, v, t64(inst.U0_raw[:, :8]))
        st = pkg.raw_call("pf_problem_init", ctx.handle, ctypes.byref(pr.struct))
        assert st == pkg.PF_ERR_INVALID_ARG


def test_unreached_tolerance_is_not_converged(pf):
    pkg, S = pf
    inst, csr = _maxcut(S, 200, 16, seed=4)
    with S.Context(p=16, n_max=200, degree=3, stream=torch.cuda.Stream()) as ctx:
        pr = S.maxcut_problem(*csr, t64(inst.U0_raw[:, :16]))
        S.problem_init(ctx, pr)
        res = pkg.pf_result()
        st = pkg.raw_call("pf_solve", ctx.handle, ctypes.byref(pr.struct), 5, 1e-14, 1,
                          ctypes.byref(res))
        assert st == pkg.PF_ERR_NOT_CONVERGED
        assert res.iters == 5 and res.kkt > 1e-14 and res.last.flags == 0


def test_phase_tracing_covers_the_step(pf):
    """Phase times of a traced step: every phase of a dense max-cut step is
    timed, and their sum is the step's device time (up to launch gaps)."""
    pkg, S = pf
    inst, csr = _maxcut(S, 520, 32, seed=5)
    stream = torch.cuda.Stream()
    with S.Context(p=32, n_max=520, degree=4, stream=stream) as ctx:
        pr = S.maxcut_problem(*csr, t64(inst.U0_raw[:, :32]))
        S.problem_init(ctx, pr)
        pkg.pf_set_tracing(ctx.handle, True)
        S.prox_step(ctx, pr, want_info=False)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            S.prox_step(ctx, pr, want_info=False)
            e1.record(stream)
        ph = pkg.pf_phase_times(ctx.handle)
        stream.synchronize()
        total = e0.elapsed_time(e1)
        assert all(ph[k] > 0 for k in pkg.PHASE_NAMES), ph
        assert sum(ph.values()) <= total * 1.01 + 0.01
        assert sum(ph.values()) >= 0.5 * total, (ph, total)
        # graph-replayed steps are not traced: the last traced call stays
        S.solve(ctx, pr, 3)
        assert pkg.pf_phase_times(ctx.handle) == ph
        pkg.pf_set_tracing(ctx.handle, False)
        assert all(v == 0 for v in pkg.pf_phase_times(ctx.handle).values())
