"""GPU parity of the block width rule (Sec. 4.2, reading R13) with the CPU
oracle: the active width follows r_+ + guard (rounded up to a multiple of 8,
clamped), growing from a saturated start block and shrinking to the
solution rank, while the per-iteration report matches the oracle."""
import numpy as np
import pytest
import scipy.sparse as sp

import pf_synthetic as syn
from oracle import pf_oracle as o

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def test_width_rule_nce_grows_like_the_oracle():
    from paper_1904_10585_gb300 import solver as S
    n, pmax, p0, iters = 300, 48, 16, 40
    G = syn.nce_matrix(n, "5.7", seed=31)
    full = syn.gaussian_block(n, pmax, seed=32)
    rule = o.AdaptiveWidth(guard=4, p_min=8, p_max=pmax, every=5, block=full)
    st, h_o = o.nce_solve(G, full[:, :p0], 3, iters, accel_l=2, adapt=rule)
    with S.Context(p=pmax, n_max=n, degree=3, stream=torch.cuda.Stream(), p_min=8,
                   adapt_guard=4, adapt_every=5) as ctx:
        pr = S.nce_problem(_t(G), _t(full), accel_l=2)
        S.with_width_rule(pr, _t(full), p0)
        S.problem_init(ctx, pr)
        widths, h_g = [], []
        for _ in range(iters):
            widths.append(pr.struct.p_active)
            h_g.append(S.prox_step(ctx, pr))
        ctx.stream.synchronize()
    assert widths[0] == p0 and max(widths) > p0
    for k, (a, b) in enumerate(zip(h_g, h_o)):
        assert a.r_plus == b.r_plus, k
        assert len(b.theta) == widths[k], k
        assert abs(a.obj - b.obj) <= 1e-7 * abs(b.obj), (k, a.obj, b.obj)
    assert pr.struct.p_active == st.U.shape[1]
    np.testing.assert_allclose(pr.lam.cpu().numpy(), st.x, atol=1e-6 * np.abs(st.x).max())


def test_width_rule_completion_shrinks_like_the_oracle():
    from paper_1904_10585_gb300 import solver as S
    n, r, mu, p = 80, 2, 0.1, 24
    inst = syn.completion_instance(n, r, 0.5, p, seed=13, mu=mu)
    rule = o.AdaptiveWidth(guard=4, p_min=4, p_max=p, every=10, block=inst.U0_raw)
    st, h_o = o.completion_solve(inst.omega, inst.U0_raw, mu, 1.0, 3, 80, adapt=rule)
    with S.Context(p=p, n_max=n, degree=3, stream=torch.cuda.Stream(), p_min=4,
                   adapt_guard=4, adapt_every=10) as ctx:
        rp, ci, mv = S.csr_to_device(inst.omega, DEV)
        pr = S.completion_problem(rp, ci, mv, _t(inst.U0_raw), mu=mu, t=1.0)
        S.with_width_rule(pr, _t(inst.U0_raw), p)
        S.problem_init(ctx, pr)
        h_g = [S.prox_step(ctx, pr) for _ in range(80)]
        ctx.stream.synchronize()
    for k, (a, b) in enumerate(zip(h_g, h_o)):
        assert a.r_plus == b.r_plus, k
        assert abs(a.obj - b.obj) <= 1e-8 * max(1.0, abs(b.obj)), (k, a.obj, b.obj)
    assert pr.struct.p_active == st.U.shape[1] == 8


def test_width_rule_maxcut_dense_matches_oracle():
    from paper_1904_10585_gb300 import solver as S
    n, prob, pmax, p0, iters = 256, 0.05, 32, 8, 30
    inst = syn.maxcut_instance(n, prob, pmax, seed=77)
    C = sp.csr_matrix((inst.C.vals, inst.C.colind, inst.C.rowptr), shape=(n, n))
    rule = o.AdaptiveWidth(guard=4, p_min=8, p_max=pmax, every=5, block=inst.U0_raw)
    st, h_o = o.maxcut_solve(C, inst.U0_raw[:, :p0], 3, iters, adapt=rule)
    with S.Context(p=pmax, n_max=n, degree=3, stream=torch.cuda.Stream(), p_min=8,
                   adapt_guard=4, adapt_every=5) as ctx:
        rp, ci, cv = S.csr_to_device(inst.C, DEV, torch.float64)
        pr = S.maxcut_problem(rp, ci, cv, _t(inst.U0_raw))
        S.with_width_rule(pr, _t(inst.U0_raw), p0)
        S.problem_init(ctx, pr)
        h_g = [S.prox_step(ctx, pr) for _ in range(iters)]
        ctx.stream.synchronize()
    for k, (a, b) in enumerate(zip(h_g, h_o)):
        assert a.r_plus == b.r_plus, k
        assert abs(a.obj - b.obj) <= 1e-9 * max(1.0, abs(b.obj)), (k, a.obj, b.obj)
    assert pr.struct.p_active == st.U.shape[1]


def test_width_rule_rejections():
    from paper_1904_10585_gb300 import solver as S
    from paper_1904_10585_gb300 import _binding as B
    n, p = 64, 16
    G = syn.nce_matrix(n, "5.7", seed=3)
    U0 = syn.gaussian_block(n, p, seed=4)
    with S.Context(p=p, n_max=n, degree=2, stream=torch.cuda.Stream(), adapt_guard=4) as ctx:
        pr = S.nce_problem(_t(G), _t(U0))
        with pytest.raises(B.PFError):        # no guard columns
            S.problem_init(ctx, pr)
        S.with_width_rule(pr, _t(U0), 24)     # start width above p
        with pytest.raises(B.PFError):
            S.problem_init(ctx, pr)
        S.with_width_rule(pr, _t(U0), 8)
        S.problem_init(ctx, pr)
        with pytest.raises(B.PFError):        # asynchronous steps cannot resize
            B.pf_enqueue_steps(ctx.handle, pr.struct, 1)
