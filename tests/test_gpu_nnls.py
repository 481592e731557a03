"""GPU parity of polynomial-filtered NNLS (accelerated proximal gradient on
the nuclear-norm regularised least-squares problem, Sec. 5.2.2) with the
CPU oracle: per-iteration interval, continuation mu, rank, relative change
and objective (relative 1e-8), and a recovery run with the oracle's
iteration count, rank and mse."""
import numpy as np
import pytest

import pf_synthetic as syn
from oracle import pf_oracle as o

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _problem(S, inst, p, mbr):
    rp, ci, mv = S.csr_to_device(inst.omega, DEV, torch.float64)
    tr = torch.from_numpy(inst.t_rowptr).to(DEV)
    tc = torch.from_numpy(inst.t_colind).to(DEV)
    tp = torch.from_numpy(inst.t_perm).to(DEV)
    U0 = torch.from_numpy(np.ascontiguousarray(inst.U0_raw[:, :p])).to(DEV)
    return S.nnls_problem(rp, ci, mv, tr, tc, tp, U0, mu_bar_rel=mbr)


@pytest.mark.parametrize("n,r,sr,p,d,iters", [(200, 3, 0.3, 16, 1, 40), (257, 4, 0.4, 24, 2, 30),
                                              (150, 2, 0.5, 32, 1, 25)])
def test_pfnnls_matches_oracle(n, r, sr, p, d, iters):
    from paper_1904_10585_gb300 import solver as S
    inst = syn.svt_instance(n, r, sr, p, seed=n + 7)
    st, h_o = o.nnls_solve(inst.omega, inst.U0_raw[:, :p], d, iters, mu_bar_rel=1e-2, cap=p - 8)
    with S.Context(p=p, n_max=n, degree=d, stream=torch.cuda.Stream()) as ctx:
        pr = _problem(S, inst, p, 1e-2)
        S.problem_init(ctx, pr)
        h_g = [S.prox_step(ctx, pr) for _ in range(iters)]
        ctx.stream.synchronize()
    for k, (a, b) in enumerate(zip(h_g, h_o)):
        # b follows the smallest Ritz value, accurate to rounding relative to the largest
        assert abs(a.b - b.b) <= 1e-8 * max(abs(b.b), b.theta[0]), (k, a.b, b.b)
        assert abs(a.dinf - b.mu) <= 1e-12 * b.mu, (k, a.dinf, b.mu)
        assert a.r_plus == b.svp, k
        # the change norm comes from ||Xn||^2 + ||X||^2 - 2<Xn, X> (factor Grams):
        # the cancellation leaves it an absolute accuracy of about 1e-12 / rel
        assert abs(a.pinf - b.rel) <= 1e-9, (k, a.pinf, b.rel)
        assert abs(a.obj - b.obj) <= 1e-8 * abs(b.obj), (k, a.obj, b.obj)


def test_pfnnls_recovers_like_the_oracle():
    from paper_1904_10585_gb300 import solver as S
    n, r, sr, p = 400, 5, 0.2, 16
    inst = syn.svt_instance(n, r, sr, p, seed=4)
    st, h_o = o.nnls_solve(inst.omega, inst.U0_raw[:, :p], 1, 300, tol=1e-4, mu_bar_rel=1e-2,
                           cap=p - 8)
    with S.Context(p=p, n_max=n, degree=1, stream=torch.cuda.Stream()) as ctx:
        pr = _problem(S, inst, p, 1e-2)
        S.problem_init(ctx, pr)
        res = S.solve(ctx, pr, 300, 1e-4, 1)
        ctx.stream.synchronize()
        fac = pr.fac.cpu().numpy()
        s = pr.fsv.cpu().numpy()[:p]
    assert res.iters == len(h_o) and res.last.r_plus == h_o[-1].svp == r
    L, R = fac[:, :p], fac[:, 2 * p:3 * p]
    M = inst.ML @ inst.MR.T
    X = (L * s) @ R.T
    Xo = (st.L * st.s) @ st.R.T
    assert np.linalg.norm(X - M) / np.linalg.norm(M) < 1e-2
    assert np.linalg.norm(X - Xo) / np.linalg.norm(Xo) < 1e-6
