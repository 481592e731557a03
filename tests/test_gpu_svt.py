"""GPU parity of polynomial-filtered SVT (Sec. 5.2.1) with the CPU oracle:
per-iteration interval, relative residual ||P_Omega(W - M)|| / ||P_Omega(M)||
(relative 1e-9), dual objective (relative 1e-9) and the count of singular
values above mu, plus the dual x after the run; then a recovery run to the
1e-4 residual with the iteration count, rank and mse of the oracle."""
import numpy as np
import pytest

import pf_synthetic as syn
from oracle import pf_oracle as o

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _problem(S, inst, p, mu, tau):
    rp, ci, mv = S.csr_to_device(inst.omega, DEV, torch.float64)
    tr = torch.from_numpy(inst.t_rowptr).to(DEV)
    tc = torch.from_numpy(inst.t_colind).to(DEV)
    tp = torch.from_numpy(inst.t_perm).to(DEV)
    U0 = torch.from_numpy(np.ascontiguousarray(inst.U0_raw[:, :p])).to(DEV)
    return S.svt_problem(rp, ci, mv, tr, tc, tp, U0, mu=mu, tau=tau)


@pytest.mark.parametrize("n,r,sr,p,d,iters", [(200, 3, 0.3, 16, 1, 40), (257, 5, 0.4, 24, 2, 30),
                                              (130, 2, 0.5, 8, 1, 25)])
def test_pfsvt_matches_oracle(n, r, sr, p, d, iters):
    from paper_1904_10585_gb300 import solver as S
    inst = syn.svt_instance(n, r, sr, p, seed=n + r)
    mu, tau = 5.0 * n, 1.2 / sr
    st, h_o = o.svt_solve(inst.omega, inst.U0_raw[:, :p], mu, tau, d, iters)
    with S.Context(p=p, n_max=n, degree=d, stream=torch.cuda.Stream()) as ctx:
        pr = _problem(S, inst, p, mu, tau)
        S.problem_init(ctx, pr)
        h_g = [S.prox_step(ctx, pr) for _ in range(iters)]
        ctx.stream.synchronize()
    for k, (a, b) in enumerate(zip(h_g, h_o)):
        assert abs(a.b - b.b) <= 1e-9 * abs(b.b), (k, a.b, b.b)
        assert a.r_plus == b.svp, k
        assert abs(a.kkt - b.rel) <= 1e-9 * max(b.rel, 1e-6), (k, a.kkt, b.rel)
        assert abs(a.obj - b.obj) <= 1e-9 * abs(b.obj), (k, a.obj, b.obj)
    np.testing.assert_allclose(pr.S.cpu().numpy(), st.x, rtol=0, atol=1e-9 * np.abs(st.x).max())


def test_pfsvt_recovers_like_the_oracle():
    from paper_1904_10585_gb300 import solver as S
    n, r, sr, p = 300, 4, 0.3, 16
    inst = syn.svt_instance(n, r, sr, p, seed=91)
    mu, tau = 5.0 * n, 1.2 / sr
    st, h_o = o.svt_solve(inst.omega, inst.U0_raw[:, :p], mu, tau, 1, 400, tol=1e-4)
    with S.Context(p=p, n_max=n, degree=1, stream=torch.cuda.Stream()) as ctx:
        pr = _problem(S, inst, p, mu, tau)
        S.problem_init(ctx, pr)
        res = S.solve(ctx, pr, 400, 1e-4, 1)
        ctx.stream.synchronize()
    assert h_o[-1].rel <= 1e-4
    assert res.iters == len(h_o) and res.last.r_plus == h_o[-1].svp == r
    x = pr.S.cpu().numpy()
    st_g = o.SVTState(x=x, U=None, theta_prev=None)
    L, s, R = o.svt_factors(inst.omega, st_g, mu, tau, 1)
    M = inst.ML @ inst.MR.T
    assert np.linalg.norm((L * s) @ R.T - M) / np.linalg.norm(M) < 1e-3
