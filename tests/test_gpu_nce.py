"""GPU parity of nearest correlation estimation (PFPG on the NCE dual,
Sec. 5.1) with the CPU oracle: per-iteration objective F(x_k) (relative
1e-9), gradient norm (relative 1e-8) and positive Ritz count, plus the dual
vector x after the run (1e-9 of its scale)."""
import numpy as np
import pytest

import pf_synthetic as syn
from oracle import pf_oracle as o

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("n,p,d,iters,example", [(300, 24, 3, 40, "5.7"), (257, 32, 4, 25, "5.7"),
                                                  (130, 16, 2, 30, "5.6")])
def test_nce_pfpg_matches_oracle(n, p, d, iters, example):
    from paper_1904_10585_gb300 import solver as S
    G = syn.nce_matrix(n, example, seed=n)
    U0 = syn.gaussian_block(n, p, seed=p)
    st, h_o = o.nce_solve(G, U0, d, iters)
    with S.Context(p=p, n_max=n, degree=d, stream=torch.cuda.Stream()) as ctx:
        pr = S.nce_problem(torch.from_numpy(G).to(DEV), torch.from_numpy(U0).to(DEV))
        S.problem_init(ctx, pr)
        h_g = [S.prox_step(ctx, pr) for _ in range(iters)]
        ctx.stream.synchronize()
    for k, (a, b) in enumerate(zip(h_g, h_o)):
        assert abs(a.obj - b.obj) <= 1e-9 * max(1.0, abs(b.obj)), (k, a.obj, b.obj)
        assert abs(a.pinf - b.gnorm) <= 1e-8 * max(1.0, b.gnorm), (k, a.pinf, b.gnorm)
        assert abs(a.kkt - b.rel) <= 1e-8 * max(1e-3, b.rel)
        assert a.r_plus == b.r_plus
    x = pr.lam.cpu().numpy()
    np.testing.assert_allclose(x, st.x, atol=1e-9 * np.abs(st.x).max())
