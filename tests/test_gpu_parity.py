"""GPU parity: the CUDA path (called through the C ABI) against the CPU
oracle on the same seeded inputs.

Tolerances (FP64 path):
* Ritz values: |theta_gpu - theta_oracle| <= 1e-10 * max|theta| (relative to
  ||H||_2, the scale Jacobi and LAPACK both resolve eigenvalues to);
* subspaces: ||sin Theta||_2 <= 1e-8, per cluster of Ritz values whose
  relative gap is below 1e-6 (in-cluster bases are not unique);
* the orthonormal block after a filter step: elementwise 1e-9 (QR with a
  positive diagonal is unique), ||Q^T Q - I|| <= 1e-13;
* a full solve at a fixed iteration count: objective relative 1e-9.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import pf_synthetic as syn
from oracle import pf_oracle as o

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    import paper_1904_10585_gb300 as pkg
    from paper_1904_10585_gb300 import solver
    return pkg, solver


DEV = "cuda:0"


def t64(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(DEV)


def clusters(theta, rel=1e-6):
    """Group indices of descending values whose relative gap is < rel."""
    scale = max(1.0, float(np.max(np.abs(theta))))
    groups, cur = [], [0]
    for i in range(1, len(theta)):
        if abs(theta[i - 1] - theta[i]) < rel * scale:
            cur.append(i)
        else:
            groups.append(cur)
            cur = [i]
    groups.append(cur)
    return groups


def assert_ritz_parity(theta_g, V_g, theta_o, V_o, tol_theta=1e-10, tol_sin=1e-8):
    scale = max(1e-300, float(np.max(np.abs(theta_o))))
    assert np.max(np.abs(theta_g - theta_o)) <= tol_theta * scale, (theta_g, theta_o)
    for g in clusters(theta_o):
        s = o.subspace_sine(V_o[:, g], V_g[:, g])
        assert s <= tol_sin, (g, s)


def spectrum_matrix(n, p, seed, gap=1.0):
    lam = np.concatenate([np.linspace(4.0 + gap, 2.0 + gap, p), np.linspace(1.0, -3.0, n - p)])
    B, Q = syn.dense_symmetric_with_spectrum(n, lam, seed)
    return B, Q, lam


# ---------------------------------------------------------------------------
# pf_filter / pf_rayleigh_ritz on a dense operator
# ---------------------------------------------------------------------------

# dense products: 8-bit digit planes on the tensor cores (default) and FP64 FMAs
DENSE = [0, 1]


@pytest.mark.parametrize("dp", DENSE)
@pytest.mark.parametrize("n,p,d", [(300, 16, 3), (300, 32, 4), (257, 40, 2), (200, 64, 5),
                                   (130, 5, 1), (33, 33, 3), (17, 16, 2), (2, 1, 4), (150, 31, 8)])
def test_dense_filter_parity(pf, n, p, d, dp):
    pkg, S = pf
    B, Q, lam = spectrum_matrix(n, min(p, n - 1) if n > p else p, seed=n + p)
    U0 = syn.gaussian_block(n, p, seed=7)
    a, b = -3.2, 1.3
    ref = o.orth(o.cheb_filter(lambda X: B @ X, U0, a, b, d))
    with S.Context(p=p, n_max=n, degree=d, dense_product=dp) as ctx:
        Bd = t64(B)
        U = t64(U0)
        S.filter_(ctx, S.dense_operator(Bd), a, b, d, U)
        torch.cuda.synchronize()
        Ug = U.cpu().numpy()
    np.testing.assert_allclose(Ug, ref, atol=1e-9, rtol=0)
    assert np.abs(Ug.T @ Ug - np.eye(p)).max() < 1e-13


@pytest.mark.parametrize("dp", DENSE)
@pytest.mark.parametrize("n,p", [(300, 16), (300, 32), (257, 40), (200, 64), (65, 7), (17, 16)])
def test_dense_rayleigh_ritz_parity(pf, n, p, dp):
    pkg, S = pf
    B, Q, lam = spectrum_matrix(n, p, seed=3 * n + p)
    U0 = o.orth(o.cheb_filter(lambda X: B @ X, syn.gaussian_block(n, p, seed=2), -3.1, 1.5, 3))
    rr = o.rayleigh_ritz(lambda X: B @ X, U0)
    with S.Context(p=p, n_max=n, degree=3, dense_product=dp) as ctx:
        V, th, res = S.rayleigh_ritz(ctx, S.dense_operator(t64(B)), t64(U0))
        torch.cuda.synchronize()
    assert_ritz_parity(th.cpu().numpy(), V.cpu().numpy(), rr.theta, rr.V)
    np.testing.assert_allclose(res.cpu().numpy(), rr.resid, atol=1e-9 * np.abs(rr.theta).max())


def test_dense_rr_recovers_known_spectrum(pf):
    """An invariant subspace gives the exact eigenvalues (the oracle's pin,
    replayed on the GPU)."""
    pkg, S = pf
    n, p = 190, 12
    lam = np.concatenate([np.linspace(9, 3, p), np.linspace(2, -5, n - p)])
    B, Q = syn.dense_symmetric_with_spectrum(n, lam, seed=4)
    U = Q[:, :p] @ o.orth(syn.gaussian_block(p, p, seed=5))
    with S.Context(p=p, n_max=n, degree=2) as ctx:
        V, th, res = S.rayleigh_ritz(ctx, S.dense_operator(t64(B)), t64(U))
        torch.cuda.synchronize()
    np.testing.assert_allclose(th.cpu().numpy(), lam[:p], rtol=1e-12)
    assert res.max().item() < 1e-11


# ---------------------------------------------------------------------------
# low-rank + sparse operator
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,p,r,d", [(400, 16, 5, 3), (333, 40, 12, 4), (100, 64, 64, 2),
                                     (70, 8, 0, 3), (211, 44, 9, 3), (97, 20, 3, 2), (45, 5, 2, 2)])
def test_lowrank_sparse_filter_and_rr_parity(pf, n, p, r, d):
    pkg, S = pf
    inst = syn.completion_instance(n, 4, 0.2, p, seed=n + r)
    Om = o.omega_matrix(inst.omega)
    Uf = o.orth(syn.gaussian_block(n, max(r, 1), seed=9))[:, :r]
    lam_f = np.linspace(3.0, 0.5, r)
    sscale, shift = -0.7, -0.05

    def apply_B(X):
        return Uf @ (lam_f[:, None] * (Uf.T @ X)) + sscale * (Om @ X) + shift * X

    U0 = syn.gaussian_block(n, p, seed=11)
    a, ub = o.gershgorin_bounds(sscale * Om, np.full(n, shift))
    b = 0.1 * a
    ref = o.orth(o.cheb_filter(apply_B, U0, a, b, d))
    rr = o.rayleigh_ritz(apply_B, ref)
    rp, ci, vals = S.csr_to_device(inst.omega, DEV, torch.float64)
    with S.Context(p=p, n_max=n, degree=d) as ctx:
        op = S.lowrank_sparse_operator(n, t64(Uf) if r else None, t64(lam_f) if r else None,
                                       rp, ci, vals, sscale, shift)
        U = t64(U0)
        S.filter_(ctx, op, a, b, d, U)
        V, th, res = S.rayleigh_ritz(ctx, op, U)
        torch.cuda.synchronize()
    np.testing.assert_allclose(U.cpu().numpy(), ref, atol=1e-9)
    assert_ritz_parity(th.cpu().numpy(), V.cpu().numpy(), rr.theta, rr.V)


# ---------------------------------------------------------------------------
# whole solves
# ---------------------------------------------------------------------------

def _csr(c):
    return sp.csr_matrix((c.vals.astype(np.float64), c.colind, c.rowptr), shape=(c.n, c.n))


def run_maxcut_gpu(S, inst, p, d, iters, use_solve=False, dp=0):
    rp, ci, vals = S.csr_to_device(inst.C, DEV, torch.float64)
    with S.Context(p=p, n_max=inst.n, degree=d, stream=torch.cuda.Stream(),
                   dense_product=dp) as ctx:
        pr = S.maxcut_problem(rp, ci, vals, t64(inst.U0_raw[:, :p]))
        S.problem_init(ctx, pr)
        hist = []
        if use_solve:
            res = S.solve(ctx, pr, iters)
            hist.append(res.last)
        else:
            for _ in range(iters):
                hist.append(S.prox_step(ctx, pr))
        ctx.stream.synchronize()
        return pr, hist


@pytest.mark.parametrize("dp", DENSE)
@pytest.mark.parametrize("n,prob,p,d,iters", [(520, 0.04, 32, 4, 40), (300, 0.05, 16, 3, 30),
                                              (130, 0.1, 40, 4, 25)])
def test_maxcut_pfam_parity(pf, n, prob, p, d, iters, dp):
    pkg, S = pf
    inst = syn.maxcut_instance(n, prob, p, seed=n)
    C = _csr(inst.C)
    st, h_o = o.maxcut_solve(C, inst.U0_raw[:, :p], d, iters)
    pr, h_g = run_maxcut_gpu(S, inst, p, d, iters, dp=dp)
    t = o.maxcut_step_size(C)
    assert abs(pr.t - t) <= 1e-14 * t
    for k, (a, b) in enumerate(zip(h_g, h_o)):
        assert abs(a.obj - b.obj) <= 1e-9 * max(1.0, abs(b.obj)), (k, a.obj, b.obj)
        assert abs(a.a - b.a) <= 1e-12 * max(1.0, abs(b.a))
        assert abs(a.b - b.b) <= 1e-9 * max(1.0, abs(b.b))
        assert a.r_plus == b.r_plus
        assert abs(a.pinf - b.pinf) <= 1e-9 * max(1e-6, b.pinf), (k, a.pinf, b.pinf)
        assert abs(a.gap - b.gap) <= 1e-9 * max(1e-3, b.gap) + 1e-12, (k, a.gap, b.gap)
        if dp == 0:
            # the sliced update takes dinf from the factors of X~_{k-1} and
            # X~_k: the cancellation of O(||X~||^2) terms leaves a relative
            # error of about u ||X~||^2 / ||Z_k - Z_{k+1}||^2
            assert abs(a.dinf - b.dinf) <= 1e-5 * max(1e-2, b.dinf), (k, a.dinf, b.dinf)
        else:
            assert abs(a.dinf - b.dinf) <= 1e-7 * max(1e-3, b.dinf), (k, a.dinf, b.dinf)
        assert a.kkt == max(a.pinf, a.dinf, a.gap)
    # saturation flag (bit 4): r_+ >= p - 2 on each of the last 20 steps
    run = 0
    for k, b in enumerate(h_o):
        run = run + 1 if b.r_plus >= p - 2 else 0
        assert bool(h_g[k].flags & 16) == (run >= 20), (k, run, h_g[k].flags)
    th = pr.theta.cpu().numpy()
    assert np.max(np.abs(th - h_o[-1].theta)) <= 1e-9 * np.max(np.abs(h_o[-1].theta))
    Zg = pr.Z.cpu().numpy()
    np.testing.assert_allclose(Zg, st.Z, atol=1e-9 * np.abs(st.Z).max())
    np.testing.assert_allclose(pr.lam.cpu().numpy(), st.lam, atol=1e-9 * np.abs(st.lam).max())


def test_maxcut_graph_solve_matches_steps_bitwise(pf):
    pkg, S = pf
    inst = syn.maxcut_instance(260, 0.05, 16, seed=1)
    pr1, h1 = run_maxcut_gpu(S, inst, 16, 3, 15)
    pr2, h2 = run_maxcut_gpu(S, inst, 16, 3, 15, use_solve=True)
    assert torch.equal(pr1.Z, pr2.Z) and torch.equal(pr1.U, pr2.U)
    assert h1[-1].obj == h2[-1].obj and h1[-1].kkt == h2[-1].kkt


def test_maxcut_deterministic(pf):
    pkg, S = pf
    inst = syn.maxcut_instance(300, 0.05, 32, seed=2)
    a, _ = run_maxcut_gpu(S, inst, 32, 4, 10)
    b, _ = run_maxcut_gpu(S, inst, 32, 4, 10)
    assert torch.equal(a.Z, b.Z) and torch.equal(a.theta, b.theta)


def run_completion_gpu(S, inst, p, d, iters, mu, t=1.0, mirror=False):
    rp, ci, vals = S.csr_to_device(inst.omega, DEV)
    mir = (torch.from_numpy(S.mirror_map(inst.omega.rowptr, inst.omega.colind)).to(DEV)
           if mirror else None)
    with S.Context(p=p, n_max=inst.n, degree=d, stream=torch.cuda.Stream()) as ctx:
        pr = S.completion_problem(rp, ci, vals, t64(inst.U0_raw[:, :p]), mu=mu, t=t, mirror=mir)
        S.problem_init(ctx, pr)
        hist = [S.prox_step(ctx, pr) for _ in range(iters)]
        ctx.stream.synchronize()
        return pr, hist


# mirror: the sampled residual formed on the upper triangle of the symmetric
# pattern and mirrored (with the Gershgorin row bounds from a second pass)
@pytest.mark.parametrize("mirror", [False, True])
@pytest.mark.parametrize("n,rank,rate,p,d,iters", [(400, 8, 0.2, 16, 3, 100), (333, 5, 0.1, 40, 4, 30),
                                                   (90, 2, 0.5, 8, 3, 40), (1000, 6, 0.06, 33, 3, 12)])
def test_completion_pfpg_parity(pf, n, rank, rate, p, d, iters, mirror):
    pkg, S = pf
    if n == 400:
        cfg, inst = syn.make_workload("completion_n400")
    else:
        inst = syn.completion_instance(n, rank, rate, p, seed=n)
    mu = 0.05
    st, h_o = o.completion_solve(inst.omega, inst.U0_raw[:, :p], mu, 1.0, d, iters)
    pr, h_g = run_completion_gpu(S, inst, p, d, iters, mu, mirror=mirror)
    for k, (a, b) in enumerate(zip(h_g, h_o)):
        assert abs(a.obj - b.obj) <= 1e-9 * max(1.0, abs(b.obj)), (k, a.obj, b.obj)
        assert a.r_plus == b.r_plus
        assert abs(a.kkt - b.kkt) <= 1e-6 * max(1e-4, b.kkt), (k, a.kkt, b.kkt)
    Xg = (pr.V.cpu().numpy() * np.maximum(pr.theta.cpu().numpy(), 0)) @ pr.V.cpu().numpy().T
    Xo = (st.V * st.w) @ st.V.T
    np.testing.assert_allclose(Xg, Xo, atol=1e-9 * max(1.0, np.abs(Xo).max()))


def test_completion_wrong_mirror_map_is_rejected(pf):
    """A map that does not send (i, j) to (j, i) fails pf_problem_init (the
    device check reads in-range indices only)."""
    import ctypes
    pkg, S = pf
    inst = syn.completion_instance(120, 3, 0.3, 8, seed=5)
    rp, ci, vals = S.csr_to_device(inst.omega, DEV)
    nnz = ci.numel()
    good = S.mirror_map(inst.omega.rowptr, inst.omega.colind)
    for bad in (np.arange(nnz, dtype=np.int32), np.roll(good, 1),
                np.where(np.arange(nnz) == 7, nnz + 5, good).astype(np.int32)):
        with S.Context(p=8, n_max=120, degree=3, stream=torch.cuda.Stream()) as ctx:
            pr = S.completion_problem(rp, ci, vals, t64(inst.U0_raw[:, :8]), mu=0.05,
                                      mirror=torch.from_numpy(bad).to(DEV))
            st = pkg.raw_call("pf_problem_init", ctx.handle, ctypes.byref(pr.struct))
            assert st == pkg.PF_ERR_INVALID_ARG
    with S.Context(p=8, n_max=120, degree=3, stream=torch.cuda.Stream()) as ctx:
        pr = S.completion_problem(rp, ci, vals, t64(inst.U0_raw[:, :8]), mu=0.05,
                                  mirror=torch.from_numpy(good).to(DEV))
        S.problem_init(ctx, pr)
        assert S.prox_step(ctx, pr).flags == 0


# ---------------------------------------------------------------------------
# error paths (host-side validation; nothing here can fault the GPU)
# ---------------------------------------------------------------------------

def test_invalid_arguments_are_rejected(pf):
    pkg, S = pf
    B = pkg
    assert B.raw_call("pf_create", None, 10, None, None) == B.PF_ERR_INVALID_ARG
    with pytest.raises(B.PFError):
        S.Context(p=65, n_max=100, degree=3)
    with pytest.raises(B.PFError):
        S.Context(p=8, n_max=4, degree=3)
    with pytest.raises(B.PFError) as ei:
        S.Context(p=8, n_max=100, degree=3, precision=B.PF_PREC_BF16 + 7)
    with S.Context(p=8, n_max=100, degree=3) as ctx:
        A = torch.zeros(100, 100, dtype=torch.float64, device=DEV)
        U = torch.zeros(100, 8, dtype=torch.float64, device=DEV)
        with pytest.raises(B.PFError) as ei:
            S.filter_(ctx, S.dense_operator(A), 1.0, 0.0, 3, U)   # a >= b
        assert ei.value.status == B.PF_ERR_INVALID_ARG
        big = torch.zeros(101, 101, dtype=torch.float64, device=DEV)
        with pytest.raises(B.PFError):
            S.filter_(ctx, S.dense_operator(big), -1.0, 0.0, 3, U)  # n > n_max
        with pytest.raises(B.PFError):
            S.filter_(ctx, S.dense_operator(A), -1.0, 0.0, 0, U)    # degree 0


def test_rank_deficient_block_reports_shift_or_breakdown(pf):
    """A block with repeated columns cannot be orthonormalised: the Cholesky
    pivot collapses, the shifted pass is taken and the report says so; the
    call returns normally (no fault, no hang)."""
    pkg, S = pf
    n, p = 120, 8
    B, Q, lam = spectrum_matrix(n, p, seed=8)
    U0 = syn.gaussian_block(n, p, seed=3)
    U0[:, 5] = U0[:, 4]
    with S.Context(p=p, n_max=n, degree=2) as ctx:
        U = t64(U0)
        S.filter_(ctx, S.dense_operator(t64(B)), -3.5, 1.0, 2, U)
        info = pkg.pf_get_info(ctx.handle)
        assert info.flags & 1
        assert torch.isfinite(U).all()
