"""GPU parity of nearest correlation estimation (PFPG on the NCE dual,
Sec. 5.1) with the CPU oracle: per-iteration interval (the Lanczos lower
estimate a and b, relative 1e-9), objective F(x_k) (relative 1e-9), gradient
norm (relative 1e-8) and positive Ritz count, plus the dual vector x after
the run (1e-9 of its scale); the same with the Sec. 4.3 extrapolation."""
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
        # interval: Lanczos lower estimate and b (Sec. 4.1)
        assert abs(a.a - b.a) <= 1e-9 * abs(b.a), (k, a.a, b.a)
        assert abs(a.b - b.b) <= 1e-9 * abs(b.a), (k, a.b, b.b)
        assert abs(a.obj - b.obj) <= 1e-9 * max(1.0, abs(b.obj)), (k, a.obj, b.obj)
        assert abs(a.pinf - b.gnorm) <= 1e-8 * max(1.0, b.gnorm), (k, a.pinf, b.gnorm)
        assert abs(a.kkt - b.rel) <= 1e-8 * max(1e-3, b.rel)
        assert a.r_plus == b.r_plus
    x = pr.lam.cpu().numpy()
    np.testing.assert_allclose(x, st.x, atol=1e-9 * np.abs(st.x).max())


@pytest.mark.parametrize("n,p,d,iters,l", [(300, 24, 3, 60, 3), (211, 32, 4, 45, 5), (150, 16, 3, 30, 1)])
def test_nce_extrapolated_matches_oracle(n, p, d, iters, l):
    """Sec. 4.3 extrapolation every l + 1 steps, GPU vs oracle.  The small
    system (D^T D + 1e-10 tr I) has condition number up to ~1e10, so the
    coefficients agree only to ~1e-6 relative; the extrapolated iterate,
    which is insensitive to them along the ill-conditioned directions,
    agrees far better: objective relative 1e-7, dual x 1e-6 of its scale."""
    from paper_1904_10585_gb300 import solver as S
    G = syn.nce_matrix(n, "5.7", seed=n + 1)
    U0 = syn.gaussian_block(n, p, seed=p + 1)
    st, h_o = o.nce_solve(G, U0, d, iters, accel_l=l, accel_lam=1e-10)
    with S.Context(p=p, n_max=n, degree=d, stream=torch.cuda.Stream()) as ctx:
        pr = S.nce_problem(torch.from_numpy(G).to(DEV), torch.from_numpy(U0).to(DEV),
                           accel_l=l, accel_lam=1e-10)
        S.problem_init(ctx, pr)
        h_g = [S.prox_step(ctx, pr) for _ in range(iters)]
        ctx.stream.synchronize()
    for k, (a, b) in enumerate(zip(h_g, h_o)):
        assert abs(a.obj - b.obj) <= 1e-7 * max(1.0, abs(b.obj)), (k, a.obj, b.obj)
        assert a.r_plus == b.r_plus
    x = pr.lam.cpu().numpy()
    np.testing.assert_allclose(x, st.x, atol=1e-6 * np.abs(st.x).max())


def test_nce_extrapolation_rejects_bad_window():
    from paper_1904_10585_gb300 import solver as S
    from paper_1904_10585_gb300 import _binding as B
    n, p = 64, 8
    G = syn.nce_matrix(n, "5.7", seed=3)
    U0 = syn.gaussian_block(n, p, seed=4)
    with S.Context(p=p, n_max=n, degree=2, stream=torch.cuda.Stream()) as ctx:
        pr = S.nce_problem(torch.from_numpy(G).to(DEV), torch.from_numpy(U0).to(DEV), accel_l=3)
        pr.struct.accel_l = 7
        with pytest.raises(B.PFError):
            S.problem_init(ctx, pr)
        pr.struct.accel_l = 2
        pr.struct.hist = None
        with pytest.raises(B.PFError):
            S.problem_init(ctx, pr)


def test_nce_lanczos_breakdown_on_invariant_start():
    """G = I (n = 4): B = I maps the Lanczos start 1/sqrt(n) onto itself
    exactly, so the process ends after one step (beta_0 = 0) on both sides
    and the interval's lower end is exactly 1; p = n keeps the rest of the
    step exact (X = P_+(I) = I, F = n/2)."""
    from paper_1904_10585_gb300 import solver as S
    n = p = 4
    G = np.eye(n)
    U0 = syn.gaussian_block(n, p, seed=5)
    _, h_o = o.nce_solve(G, U0, 2, 1)
    with S.Context(p=p, n_max=n, degree=2, stream=torch.cuda.Stream()) as ctx:
        pr = S.nce_problem(torch.from_numpy(G).to(DEV), torch.from_numpy(U0).to(DEV))
        S.problem_init(ctx, pr)
        info = S.prox_step(ctx, pr)
        ctx.stream.synchronize()
    assert h_o[0].a == 1.0 and info.a == 1.0
    assert info.b == h_o[0].b
    assert info.r_plus == 4
    assert abs(info.obj - 2.0) <= 1e-12


def test_nce_planes_shared_context_matches_fresh_context():
    """The digit planes of G + Diag(x) stay with the NCE problem between
    steps, and each step re-slices only the chunks holding the diagonal.  A
    product with another dense matrix on the same context (pf_apply) takes
    the planes over; the next NCE steps must slice Z again in full.  The
    interleaved run equals, bitwise, a run on a fresh context, and the
    product equals A X within the sliced product's bound."""
    from paper_1904_10585_gb300 import solver as S
    n, p, d = 257, 32, 3
    G = syn.nce_matrix(n, "5.7", seed=3)
    U0 = syn.gaussian_block(n, p, seed=4)
    A = syn.gaussian_block(n, n, seed=5)
    X = syn.gaussian_block(n, p, seed=6)

    def run(interleave):
        with S.Context(p=p, n_max=n, degree=d, stream=torch.cuda.Stream()) as ctx:
            pr = S.nce_problem(torch.from_numpy(G).to(DEV), torch.from_numpy(U0).to(DEV))
            S.problem_init(ctx, pr)
            hist, Ys = [], []
            for k in range(12):
                hist.append(S.prox_step(ctx, pr))
                if interleave and k in (3, 7):
                    Y = torch.empty(n, p, dtype=torch.float64, device=DEV)
                    S.apply(ctx, S.dense_operator(torch.from_numpy(A).to(DEV)),
                            torch.from_numpy(X).to(DEV), Y)
                    Ys.append(Y)
            ctx.stream.synchronize()
            return hist, pr.lam.cpu().numpy(), [Y.cpu().numpy() for Y in Ys]

    h1, x1, Ys = run(True)
    h2, x2, _ = run(False)
    assert [a.obj for a in h1] == [b.obj for b in h2]
    assert np.array_equal(x1, x2)
    ref = A.astype(np.longdouble) @ X.astype(np.longdouble)
    bound = n * 2.0 ** -50 * np.abs(A).max(axis=1)[:, None] * np.abs(X).max(axis=0)[None, :]
    for Y in Ys:
        err = np.abs(Y.astype(np.longdouble) - ref).astype(np.float64)
        assert np.all(err <= bound), float(np.max(err / bound))
