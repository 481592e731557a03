"""Pins of the CPU oracle against facts fixed by the paper and by mathematics,
never against the oracle itself: closed forms, invariants, special cases that
reduce to textbook formulas, brute force on tiny inputs and the paper's error
bound.  Each pin is chosen so that a plausible mistake in the oracle (a
swapped interval map, a wrong first recurrence step, a sign error in the prox,
a transposed projection) fails at least one of them; ``test_planted_*``
plants such mistakes in the oracle and checks that a pin catches them."""
import itertools
import math

import numpy as np
import pytest
import scipy.sparse as sp
from numpy.polynomial import chebyshev as npcheb

import pf_synthetic as syn
from oracle import pf_oracle as o


def diag_apply(x):
    return lambda Y: x[:, None] * Y


def T_closed(d, x):
    """Independent closed form of T_d: cos/cosh branches, with the sign
    (-1)^d on x < -1 (Eq. (cheb) rewritten with arccosh)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    m = np.abs(x) <= 1
    out[m] = np.cos(d * np.arccos(x[m]))
    hi = x > 1
    out[hi] = np.cosh(d * np.arccosh(x[hi]))
    lo = x < -1
    out[lo] = (-1) ** d * np.cosh(d * np.arccosh(-x[lo]))
    return out


# --------------------------------------------------------------------------
# Chebyshev filter (Sec. 2.1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("d", [0, 1, 2, 3, 4, 7, 8])
def test_closed_form_T_matches_numpy_chebval(d):
    x = np.linspace(-3, 3, 1001)
    coef = np.zeros(d + 1)
    coef[d] = 1
    ref = npcheb.chebval(x, coef)
    np.testing.assert_allclose(o.chebyshev_T(d, x), ref, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(T_closed(d, x), ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("d", [1, 2, 3, 4, 6, 8])
def test_filter_on_diagonal_matrix_is_T_d_of_mapped_eigenvalues(d):
    a, b = -2.5, 0.7
    x = np.linspace(-3.0, 9.0, 37)
    Y = o.cheb_filter(diag_apply(x), np.eye(x.size), a, b, d)
    mapped = (x - (a + b) / 2) / ((b - a) / 2)
    ref = T_closed(d, mapped)
    np.testing.assert_allclose(np.diag(Y), ref, rtol=1e-13, atol=1e-13)
    assert np.abs(Y - np.diag(np.diag(Y))).max() == 0.0
    # damped inside [a, b], amplified outside
    inside = (x >= a) & (x <= b)
    assert np.all(np.abs(np.diag(Y)[inside]) <= 1 + 1e-12)


@pytest.mark.parametrize("d", [1, 2, 3, 5, 8])
def test_chebyshev_growth_lemma(d):
    """Lemma (cheb-est): T_d(+-(1+eps)) >= 2^{d min(sqrt(eps),1) - 1}."""
    eps = np.logspace(-6, 2, 200)
    for sgn in (1.0, -1.0):
        x = sgn * (1 + eps)
        # evaluate through the oracle's filter on a diagonal matrix, a=-1, b=1
        Y = o.cheb_filter(diag_apply(x), np.ones((x.size, 1)), -1.0, 1.0, d)[:, 0]
        bound = 2.0 ** (d * np.minimum(np.sqrt(eps), 1.0) - 1.0)
        assert np.all(np.abs(Y) >= bound * (1 - 1e-12))


def test_filter_known_spectrum():
    n, p, d = 60, 5, 4
    lam = np.concatenate([np.linspace(5, 3, p), np.linspace(1.0, -4.0, n - p)])
    B, Q = syn.dense_symmetric_with_spectrum(n, lam, seed=3)
    U = syn.gaussian_block(n, p, seed=4)
    a, b = -4.0, 1.2
    Y = o.cheb_filter(lambda X: B @ X, U, a, b, d)
    coef = np.zeros(d + 1)
    coef[d] = 1
    rho = npcheb.chebval((lam - (a + b) / 2) / ((b - a) / 2), coef)
    ref = Q @ (rho[:, None] * (Q.T @ U))
    np.testing.assert_allclose(Y, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_contraction_bound_one_step():
    """sin Theta(V_p, orth(rho(B)U)) <= eta tan Theta(V_p, U) with
    eta = max_{i>p}|rho(l_i)| / min_{i<=p}|rho(l_i)| (Eq. (err-oi))."""
    n, p = 80, 6
    lam = np.concatenate([np.linspace(4, 2.5, p), np.linspace(1.5, -3, n - p)])
    B, Q = syn.dense_symmetric_with_spectrum(n, lam, seed=11)
    Vp = Q[:, :p]
    for seed, d in itertools.product([1, 2, 3], [2, 4, 6]):
        U = o.orth(syn.gaussian_block(n, p, seed=seed))
        a, b = -3.0, 1.6
        Up = o.orth(o.cheb_filter(lambda X: B @ X, U, a, b, d))
        rho = np.abs(o.chebyshev_T(d, (lam - (a + b) / 2) / ((b - a) / 2)))
        eta = rho[p:].max() / rho[:p].min()
        s0 = o.subspace_sine(Vp, U)
        tan0 = s0 / math.sqrt(1 - s0 * s0)
        assert o.subspace_sine(Vp, Up) <= eta * tan0 * (1 + 1e-8) + 1e-14


# --------------------------------------------------------------------------
# orth and Rayleigh-Ritz
# --------------------------------------------------------------------------

def classical_gram_schmidt(Y):
    n, p = Y.shape
    Q = np.zeros_like(Y)
    for j in range(p):
        v = Y[:, j].copy()
        for i in range(j):
            v -= (Q[:, i] @ Y[:, j]) * Q[:, i]
        Q[:, j] = v / math.sqrt(v @ v)
    return Q


def test_orth_is_unique_positive_diagonal_qr():
    Y = syn.gaussian_block(9, 4, seed=5)
    Q = o.orth(Y)
    np.testing.assert_allclose(Q, classical_gram_schmidt(Y), atol=1e-12)
    R = Q.T @ Y
    assert np.allclose(np.tril(R, -1), 0, atol=1e-12)
    assert np.all(np.diag(R) > 0)
    np.testing.assert_allclose(Q.T @ Q, np.eye(4), atol=1e-14)


def test_rr_recovers_invariant_subspace_exactly():
    n, p = 50, 7
    lam = np.concatenate([np.array([9, 8, 7.5, 6, 5, 4, 3.0]), np.linspace(2, -6, n - p)])
    B, Q = syn.dense_symmetric_with_spectrum(n, lam, seed=8)
    R = o.orth(syn.gaussian_block(p, p, seed=9))
    U = Q[:, :p] @ R                          # an orthonormal basis of the invariant subspace
    rr = o.rayleigh_ritz(lambda X: B @ X, U)
    np.testing.assert_allclose(rr.theta, lam[:p], rtol=1e-13)
    assert rr.resid.max() < 1e-12
    assert o.subspace_sine(rr.V, Q[:, :p]) < 1e-12
    # each Ritz vector is an eigenvector: compare projectors one by one
    for i in range(p):
        Pi = np.outer(rr.V[:, i], rr.V[:, i])
        np.testing.assert_allclose(Pi, np.outer(Q[:, i], Q[:, i]), atol=1e-12)


def test_rr_tiny_brute_force_2x2_and_3x3():
    # 2x2 closed form
    A = np.array([[2.0, 0.7], [0.7, -1.0]])
    rr = o.rayleigh_ritz(lambda X: A @ X, np.eye(2))
    m, h = (A[0, 0] + A[1, 1]) / 2, math.hypot((A[0, 0] - A[1, 1]) / 2, A[0, 1])
    np.testing.assert_allclose(rr.theta, [m + h, m - h], rtol=1e-14)
    # 3x3: roots of the characteristic polynomial written out
    A = np.array([[1.0, 2.0, -0.5], [2.0, 0.3, 0.1], [-0.5, 0.1, -2.0]])
    tr = np.trace(A)
    minors = sum(A[i, i] * A[j, j] - A[i, j] * A[j, i] for i in range(3) for j in range(i + 1, 3))
    det = (A[0, 0] * (A[1, 1] * A[2, 2] - A[1, 2] * A[2, 1])
           - A[0, 1] * (A[1, 0] * A[2, 2] - A[1, 2] * A[2, 0])
           + A[0, 2] * (A[1, 0] * A[2, 1] - A[1, 1] * A[2, 0]))
    roots = np.sort(np.roots([1.0, -tr, minors, -det]).real)[::-1]
    rr = o.rayleigh_ritz(lambda X: A @ X, np.eye(3))
    np.testing.assert_allclose(rr.theta, roots, rtol=1e-12)


def test_subspace_sine_known_angle():
    for phi in [0.0, 0.1, 0.7, 1.4, math.pi / 2]:
        X = np.array([[1.0], [0.0]])
        Y = np.array([[math.cos(phi)], [math.sin(phi)]])
        assert abs(o.subspace_sine(X, Y) - abs(math.sin(phi))) < 1e-12


def test_psd_projection_properties():
    Z = syn.gaussian_block(12, 12, seed=2)
    Z = Z + Z.T
    P = o.psd_part(Z)
    np.testing.assert_allclose(o.psd_part(P), P, atol=1e-12)           # idempotent
    assert np.linalg.eigvalsh(P).min() > -1e-12                        # PSD
    assert np.linalg.eigvalsh(Z - P).max() < 1e-12                     # remainder NSD
    assert abs(np.sum(P * (Z - P))) < 1e-10                            # complementary
    d = np.array([3.0, -1.0, 0.5, -2.0])
    np.testing.assert_allclose(o.psd_part(np.diag(d)), np.diag(np.maximum(d, 0)), atol=1e-15)


# --------------------------------------------------------------------------
# Interval bounds
# --------------------------------------------------------------------------

def test_gershgorin_lower_bound_is_rigorous_for_psd_plus_sparse():
    n = 70
    inst = syn.maxcut_instance(n, 0.2, 4, seed=21)
    C = sp.csr_matrix((inst.C.vals, inst.C.colind, inst.C.rowptr), shape=(n, n))
    rng = np.random.default_rng(0)
    for _ in range(5):
        lam = rng.standard_normal(n)
        t = 0.3
        G = rng.standard_normal((n, 5))
        Z = G @ G.T - t * C.toarray() - np.diag(lam)
        a, ub = o.gershgorin_bounds(-t * C, -lam)
        assert a <= np.linalg.eigvalsh(Z).min() + 1e-12
        assert ub >= np.linalg.eigvalsh(-t * C.toarray() - np.diag(lam)).max() - 1e-12


# --------------------------------------------------------------------------
# Max-cut SDP via DRS / PFAM (Sec. 2.3)
# --------------------------------------------------------------------------

def test_prox_G_minus_sign_satisfies_its_kkt():
    rng = np.random.default_rng(1)
    n, t = 6, 0.7
    Y = rng.standard_normal((n, n)); Y = Y + Y.T
    C = rng.standard_normal((n, n)); C = C + C.T
    X = o.prox_G_maxcut(Y, C, t)
    np.testing.assert_allclose(np.diag(X), 1.0, atol=1e-15)
    # stationarity of <C,X> + ||X-Y||^2/(2t) on {diag X = 1}: X - Y + tC is diagonal
    R = X - Y + t * C
    np.testing.assert_allclose(R - np.diag(np.diag(R)), 0.0, atol=1e-14)
    f = lambda W: np.sum(C * W) + np.sum((W - Y) ** 2) / (2 * t)  # noqa: E731
    for _ in range(20):
        D = rng.standard_normal((n, n)); D = D + D.T; np.fill_diagonal(D, 0.0)
        assert f(X + 1e-3 * D) > f(X)


def _csr(inst_C):
    return sp.csr_matrix((inst_C.vals, inst_C.colind, inst_C.rowptr), shape=(inst_C.n, inst_C.n))


def test_maxcut_complete_graph_closed_form():
    """K_n, unit weights: min <C,X> = -n^2/4, attained at X = (nI - J)/(n-1)."""
    n = 8
    i, j = np.triu_indices(n, 1)
    C = _csr(syn.maxcut_cost_from_edges(n, i, j, np.ones(i.size)))
    U0 = syn.gaussian_block(n, n, seed=1)
    for exact in (True, False):
        st, hist = o.maxcut_solve(C, U0, 4, 400, exact=exact, tol=1e-10)
        assert abs(hist[-1].obj + n * n / 4) < 1e-6 * n * n
        assert hist[-1].kkt < 1e-6


def test_maxcut_bipartite_value_is_total_weight():
    """Connected bipartite graph with positive weights: the SDP value is the
    total weight (rank-1 optimum), reached by PFAM with a small block."""
    rng = np.random.default_rng(3)
    n1, n2 = 12, 14
    edges = [(a, n1 + b) for a in range(n1) for b in range(n2) if rng.random() < 0.4]
    edges += [(a, n1 + (a % n2)) for a in range(n1)] + [((b % n1), n1 + b) for b in range(n2)]
    edges = sorted(set(edges))
    i = np.array([e[0] for e in edges]); j = np.array([e[1] for e in edges])
    w = rng.uniform(0.5, 2.0, i.size)
    C = _csr(syn.maxcut_cost_from_edges(n1 + n2, i, j, w))
    U0 = syn.gaussian_block(n1 + n2, 4, seed=2)
    st, hist = o.maxcut_solve(C, U0, 4, 3000, tol=1e-9)
    assert abs(hist[-1].obj + w.sum()) < 1e-5 * w.sum()


def test_maxcut_relaxation_bound_brute_force():
    """n = 10: the SDP minimum is <= min over x in {+-1}^n of x^T C x."""
    n = 10
    inst = syn.maxcut_instance(n, 0.6, n, seed=5)
    C = _csr(inst.C)
    Cd = C.toarray()
    best = min(np.array(x) @ Cd @ np.array(x) for x in itertools.product([-1.0, 1.0], repeat=n))
    st, hist = o.maxcut_solve(C, inst.U0_raw, 4, 5000, exact=True, tol=1e-8)
    assert hist[-1].kkt < 1e-6
    assert hist[-1].obj <= best + 1e-6


def test_maxcut_pf_with_full_block_equals_exact_drs():
    n = 24
    inst = syn.maxcut_instance(n, 0.3, n, seed=6)
    C = _csr(inst.C)
    _, h_pf = o.maxcut_solve(C, inst.U0_raw, 3, 40)
    _, h_ex = o.maxcut_solve(C, inst.U0_raw, 3, 40, exact=True)
    for a, b in zip(h_pf, h_ex):
        assert abs(a.obj - b.obj) <= 1e-9 * max(1.0, abs(b.obj))


def test_maxcut_dual_residual_identity():
    """C - Diag(y) - S = (Z_k - Z_{k+1})/t for y = -lambda/t, S = (X~ - Z_k)/t."""
    n = 30
    inst = syn.maxcut_instance(n, 0.3, 8, seed=7)
    C = _csr(inst.C)
    t = o.maxcut_step_size(C)
    st = o.maxcut_init(C, inst.U0_raw, t)
    for _ in range(5):
        Zk = st.Z
        st, info = o.maxcut_pfam_step(C, st, t, 4)
        alt = np.linalg.norm(Zk - st.Z) / (t * (1 + np.linalg.norm(C.toarray())))
        assert abs(alt - info.dinf) <= 1e-10 * max(1.0, alt)


# --------------------------------------------------------------------------
# PSD completion via PFPG
# --------------------------------------------------------------------------

def test_completion_full_sampling_closed_form():
    """Omega = all entries, t = 1: the PG fixed point is P_+(M - mu I), whose
    eigenvalues are (sigma_i(G)^2 - mu)_+ (an SVD route independent of EVD)."""
    n, r, mu = 40, 3, 0.05
    inst = syn.completion_instance(n, r, 1.0, r + 5, seed=12, mu=mu)
    st_ex, h_ex = o.completion_solve(inst.omega, inst.U0_raw, mu, 1.0, 3, 3, exact=True)
    st_pf, h_pf = o.completion_solve(inst.omega, inst.U0_raw, mu, 1.0, 3, 60)
    Gs = inst.G.astype(np.float32).astype(np.float64)  # M values are stored in float32
    M = inst.omega.to_dense()
    Uo, s, _ = np.linalg.svd(inst.G, full_matrices=False)
    lam_ref = np.maximum(np.linalg.eigvalsh(M)[::-1][:r] - mu, 0)
    np.testing.assert_allclose(np.sort(lam_ref), np.sort(np.maximum(s ** 2 - mu, 0)), rtol=1e-6)
    Xref = o.psd_part(M - mu * np.eye(n))
    for st in (st_ex, st_pf):
        X = (st.V * st.w) @ st.V.T
        np.testing.assert_allclose(X, Xref, atol=1e-10)
    del Gs, Uo


def test_completion_objective_decreases_and_recovers_low_rank():
    """Noiseless rank-2 M, half the entries seen, small mu: the iterates
    settle on rank 2 and X approaches M (the recovery regime of Sec. 5.2)."""
    n, r = 80, 2
    inst = syn.completion_instance(n, r, 0.5, 8, seed=13, mu=1e-2)
    st, hist = o.completion_solve(inst.omega, inst.U0_raw, 1e-2, 1.0, 3, 300)
    objs = np.array([h.obj for h in hist])
    assert objs[-1] < objs[5]
    assert hist[-1].r_plus == r and hist[-1].kkt < 1e-5
    M = inst.G @ inst.G.T
    X = (st.V * st.w) @ st.V.T
    assert np.linalg.norm(X - M) / np.linalg.norm(M) < 5e-3


def test_completion_kkt_factor_formula_matches_dense():
    rng = np.random.default_rng(4)
    V1 = o.orth(rng.standard_normal((30, 4))); w1 = rng.uniform(0, 2, 4)
    V2 = o.orth(rng.standard_normal((30, 3))); w2 = rng.uniform(0, 2, 3)
    dense = np.linalg.norm((V1 * w1) @ V1.T - (V2 * w2) @ V2.T)
    assert abs(o._lowrank_fro_diff(V1, w1, V2, w2) - dense) < 1e-12


# --------------------------------------------------------------------------
# Interval rule of Sec. 4.1 (reading R4) and the max-cut step (reading R6),
# against values computed by hand from the printed formulas
# --------------------------------------------------------------------------

def test_choose_b_r_largest_rule_hand_values():
    """b = (1 - eta) lambda_r_prev + eta a with lambda_r_prev the smallest of
    the previous Ritz values: a = -4, previous values {5, 2, 1}, eta = 0.1
    gives 0.9 * 1 + 0.1 * (-4) = 0.5; eta = 0.2 gives 0.8 - 0.8 = 0."""
    th = np.array([5.0, 2.0, 1.0])
    assert o.choose_b(-4.0, th, ub=100.0, eta=0.1) == pytest.approx(0.5, abs=1e-15)
    assert o.choose_b(-4.0, th, ub=100.0, eta=0.2) == pytest.approx(0.0, abs=1e-15)
    # the estimate is the smallest previous value wherever it sits in the array
    assert o.choose_b(-4.0, np.array([1.0, 5.0, 2.0]), ub=100.0) == pytest.approx(0.5, abs=1e-15)
    # the upper Gershgorin bound plays no part once Ritz values exist
    assert o.choose_b(-4.0, th, ub=-1e9) == o.choose_b(-4.0, th, ub=1e9)


def test_choose_b_first_step_hand_values():
    """No previous Ritz values: the all-positive rule b = eta a for a < 0
    (a = -4: b = -0.4); for a >= 0 the interval keeps (1 - eta) of the way to
    the upper bound (a = 2, ub = 12: b = 2 + 0.9 * 10 = 11)."""
    assert o.choose_b(-4.0, None, ub=12.0) == pytest.approx(-0.4, abs=1e-15)
    assert o.choose_b(-4.0, None, ub=12.0, eta=0.2) == pytest.approx(-0.8, abs=1e-15)
    assert o.choose_b(2.0, None, ub=12.0) == pytest.approx(11.0, abs=1e-14)
    assert o.choose_b(0.0, None, ub=12.0) == pytest.approx(10.8, abs=1e-14)


def test_choose_b_gap_guard_hand_values():
    """b - a is kept >= 1e-3 max(1, |a|): a = -4 with a previous smallest Ritz
    value of -4 gives b = -4 -> -4 + 0.004; a = -0.5 with -0.5 gives
    -0.5 + 0.001; a gap already wide enough is left alone."""
    assert o.choose_b(-4.0, np.array([-4.0]), ub=0.0) == pytest.approx(-3.996, abs=1e-15)
    assert o.choose_b(-0.5, np.array([-0.5]), ub=0.0) == pytest.approx(-0.499, abs=1e-15)
    # -3.9 is 0.09 above a = -4 after the rule (0.9 * -3.9 + 0.1 * -4 = -3.91)
    assert o.choose_b(-4.0, np.array([-3.9]), ub=0.0) == pytest.approx(-3.91, abs=1e-14)


def test_maxcut_step_size_hand_value():
    """t = 10 sqrt(n)/||C||_F with C = -L/4.  Path 1-2-3 with weights +1
    and -1: D = diag(1, 0, -1), L = D - W has six entries of magnitude 1 and
    a zero middle diagonal, so ||C||_F = sqrt(6)/4 and
    t = 10 sqrt(3) * 4/sqrt(6) = 20 sqrt(2)."""
    L = np.array([[1.0, -1.0, 0.0], [-1.0, 0.0, 1.0], [0.0, 1.0, -1.0]])
    C = sp.csr_matrix(-L / 4.0)
    assert o.maxcut_step_size(C) == pytest.approx(20.0 * math.sqrt(2.0), rel=1e-15)
    # one edge of weight 1 on four vertices (two isolated): ||C||_F = 1/2,
    # t = 10 * 2 / (1/2) = 40
    C4 = sp.csr_matrix(([-0.25, 0.25, 0.25, -0.25], ([0, 0, 1, 1], [0, 1, 0, 1])), shape=(4, 4))
    assert o.maxcut_step_size(C4) == pytest.approx(40.0, rel=1e-15)
    # the synthetic generator's cost matrix: ||C||_F from its definition
    inst = syn.maxcut_instance(60, 0.2, 4, seed=5)
    Cs = sp.csr_matrix((inst.C.vals, inst.C.colind, inst.C.rowptr), shape=(60, 60))
    ref = 10.0 * math.sqrt(60) / math.sqrt(float(np.sum(inst.C.vals.astype(np.float64) ** 2)))
    assert o.maxcut_step_size(Cs) == pytest.approx(ref, rel=1e-14)


@pytest.mark.parametrize("mutation", ["swap_eta", "theta_max", "first_step_sign", "no_guard"])
def test_planted_interval_mistakes_are_caught(monkeypatch, mutation):
    def bad(a, theta_prev, ub, eta=o.ETA):
        if theta_prev is None:
            if mutation == "first_step_sign":
                b = -eta * a if a < 0 else a + (1.0 - eta) * (ub - a)
            else:
                b = eta * a if a < 0 else a + (1.0 - eta) * (ub - a)
        elif mutation == "swap_eta":
            b = eta * float(np.min(theta_prev)) + (1.0 - eta) * a
        elif mutation == "theta_max":
            b = (1.0 - eta) * float(np.max(theta_prev)) + eta * a
        else:
            b = (1.0 - eta) * float(np.min(theta_prev)) + eta * a
        if mutation != "no_guard":
            gap = 1e-3 * max(1.0, abs(a))
            if b - a < gap:
                b = a + gap
        return b
    monkeypatch.setattr(o, "choose_b", bad)
    with pytest.raises(AssertionError):
        test_choose_b_r_largest_rule_hand_values()
        test_choose_b_first_step_hand_values()
        test_choose_b_gap_guard_hand_values()


def test_planted_step_size_mistakes_are_caught(monkeypatch):
    for bad in (lambda C: 10.0 * C.shape[0] / float(sp.linalg.norm(C, "fro")),
                lambda C: math.sqrt(C.shape[0]) / float(sp.linalg.norm(C, "fro")),
                lambda C: 10.0 * math.sqrt(C.shape[0]) / float(sp.linalg.norm(C, "fro")) ** 2):
        monkeypatch.setattr(o, "maxcut_step_size", bad)
        with pytest.raises(AssertionError):
            test_maxcut_step_size_hand_value()


# --------------------------------------------------------------------------
# Planted mistakes: each must be caught by a pin above
# --------------------------------------------------------------------------

def test_planted_swapped_interval_map_is_caught(monkeypatch):
    """The printed (garbled) recurrence coefficients c0=2/(b-a), c1=(a+b)/(a-b)
    used as 'centre, half-width' must fail the closed-form pin."""
    monkeypatch.setattr(o, "interval_map", lambda a, b: (2 / (b - a), (a + b) / (a - b)))
    with pytest.raises(AssertionError):
        test_filter_on_diagonal_matrix_is_T_d_of_mapped_eigenvalues(3)


def test_planted_plus_sign_prox_is_caught(monkeypatch):
    def bad(Y, C, t):
        W = Y + t * C
        return W - np.diag(np.diag(W) - 1.0)
    monkeypatch.setattr(o, "prox_G_maxcut", bad)
    with pytest.raises(AssertionError):
        test_prox_G_minus_sign_satisfies_its_kkt()


def test_planted_first_step_factor_is_caught(monkeypatch):
    orig = o.cheb_filter

    def bad(apply_B, U, a, b, d):
        c, e = o.interval_map(a, b)
        Yp = np.array(U, dtype=np.float64)
        if d == 0:
            return Yp
        Y = 2.0 * (apply_B(Yp) - c * Yp) / e        # wrong: first step uses 2/e
        for _ in range(1, d):
            Yp, Y = Y, 2.0 * (apply_B(Y) - c * Y) / e - Yp
        return Y
    monkeypatch.setattr(o, "cheb_filter", bad)
    with pytest.raises(AssertionError):
        test_filter_on_diagonal_matrix_is_T_d_of_mapped_eigenvalues(2)
    monkeypatch.setattr(o, "cheb_filter", orig)


def test_planted_transposed_projection_is_caught(monkeypatch):
    def bad_rr(apply_B, Q):
        W = apply_B(Q)
        H = W.T @ W                                   # wrong: not Q^T B Q
        lam, Yv = np.linalg.eigh(0.5 * (H + H.T))
        order = np.argsort(-lam)
        return o.RitzPairs(lam[order], Q @ Yv[:, order], np.zeros(Q.shape[1]), H)
    monkeypatch.setattr(o, "rayleigh_ritz", bad_rr)
    with pytest.raises(AssertionError):
        test_rr_recovers_invariant_subspace_exactly()


# --------------------------------------------------------------------------
# Input generator sanity (shapes, symmetry, sampling rates, reproducibility)
# --------------------------------------------------------------------------

def test_synthetic_inputs_laws():
    cfg, inst = syn.make_workload("completion_n400")
    A = inst.omega.to_dense()
    assert np.array_equal(A != 0, (A != 0).T)
    frac = inst.omega.nnz / (400 * 400)
    assert 0.18 < frac < 0.22
    cfg2, inst2 = syn.make_workload("completion_n400")
    assert np.array_equal(inst.omega.colind, inst2.omega.colind)
    assert np.array_equal(inst.U0_raw, inst2.U0_raw)
    mc = syn.maxcut_instance(500, 0.05, 8, seed=1)
    Cd = mc.C.to_dense()
    np.testing.assert_allclose(Cd, Cd.T)
    np.testing.assert_allclose(Cd.sum(axis=1), 0.0, atol=1e-12)     # Laplacian rows sum to 0
    off = Cd[~np.eye(500, dtype=bool)]
    assert set(np.unique(off[off != 0]).tolist()) <= {-0.25, 0.25}
    assert abs(mc.n_edges / (500 * 499 / 2) - 0.05) < 0.01


# --------------------------------------------------------------------------
# Nearest correlation estimation (Sec. 5.1)
# --------------------------------------------------------------------------

def test_nce_gradient_matches_finite_differences_of_the_dual():
    """grad F(x) = diag(P_+(G + Diag x)) - 1 (Eq. (NCE-gradient)) against
    central differences of F computed from eigenvalues only."""
    n = 12
    G = syn.nce_matrix(n, "5.7", seed=3)
    x = np.random.default_rng(0).uniform(-2, 0, n)
    st = o.NCEState(x=x, U=np.eye(n), theta_prev=None)
    _, info = o.nce_step(G, st, 3, exact=True)
    lam, V = np.linalg.eigh(G + np.diag(x))
    g_ref = np.array([(o.nce_objective(G, x + 1e-6 * e) - o.nce_objective(G, x - 1e-6 * e)) / 2e-6
                      for e in np.eye(n)])
    pos = lam > 0
    g_oracle = np.sum((V[:, pos] ** 2) * lam[pos], axis=1) - 1.0
    np.testing.assert_allclose(g_oracle, g_ref, atol=1e-6)
    assert abs(info.gnorm - np.linalg.norm(g_ref)) < 1e-6


def test_nce_closed_forms():
    """A correlation matrix is its own nearest correlation matrix (x* = 0 is
    a fixed point); for G = 2I the answer is I with x* = -1."""
    n = 20
    Y = syn.gaussian_block(n, 4, seed=1)
    Cm = Y @ Y.T
    d = np.sqrt(np.diag(Cm))
    Cm = Cm / np.outer(d, d)                      # PSD with unit diagonal
    st = o.NCEState(x=np.zeros(n), U=syn.gaussian_block(n, n, seed=2), theta_prev=None)
    st2, info = o.nce_step(Cm, st, 3, exact=True)
    assert info.gnorm < 1e-12 and np.abs(st2.x).max() < 1e-12
    st, hist = o.nce_solve(2.0 * np.eye(n), syn.gaussian_block(n, n, seed=3), 3, 50, exact=True)
    np.testing.assert_allclose(st.x, -1.0, atol=1e-12)


def test_nce_pf_with_full_block_equals_gradient_method():
    n = 30
    G = syn.nce_matrix(n, "5.7", seed=4)
    U0 = syn.gaussian_block(n, n, seed=5)
    _, h_pf = o.nce_solve(G, U0, 3, 30)
    _, h_ex = o.nce_solve(G, U0, 3, 30, exact=True)
    for a, b in zip(h_pf, h_ex):
        assert abs(a.obj - b.obj) <= 1e-9 * max(1.0, abs(b.obj))
        assert abs(a.gnorm - b.gnorm) <= 1e-8 * max(1.0, b.gnorm)


def test_nce_pf_converges_on_example_5_7_law():
    """PFPG with a 24-wide block reaches the gradient method's objective on a
    small Example-5.7-law matrix (few positive eigenvalues at the solution)."""
    n = 80
    G = syn.nce_matrix(n, "5.7", seed=6)
    _, h_ex = o.nce_solve(G, syn.gaussian_block(n, n, seed=7), 3, 1500, exact=True, tol=1e-5)
    _, h_pf = o.nce_solve(G, syn.gaussian_block(n, 24, seed=7), 3, 1500, tol=1e-5)
    assert h_pf[-1].rel <= 1e-5 and h_ex[-1].rel <= 1e-5
    assert abs(h_pf[-1].obj - h_ex[-1].obj) <= 1e-7 * abs(h_ex[-1].obj)


def test_rna_coefficients_solve_the_constrained_quadratic():
    """c = argmin_{1^T c = 1} c^T (U^T U + lam I) c (Sec. 4.3): 1^T c = 1 and
    the KKT condition (U^T U + lam I) c = nu 1; on points of a linear
    fixed-point iteration x+ = A x + b with l + 1 >= dim, the combination
    recovers the fixed point (the classical extrapolation property)."""
    rng = np.random.default_rng(2)
    pts = [rng.standard_normal(7) for _ in range(5)]
    x, c = o.rna_combination(pts, 1e-6)
    assert abs(c.sum() - 1.0) < 1e-14
    X = np.stack(pts, axis=1)
    U = X[:, 1:] - X[:, :-1]
    M = U.T @ U + 1e-6 * np.trace(U.T @ U) * np.eye(4)
    r = M @ c
    np.testing.assert_allclose(r, r.mean() * np.ones(4), rtol=1e-9)
    d = 3
    A = np.diag([0.9, -0.5, 0.3])
    bvec = np.array([1.0, 2.0, -1.0])
    xs = [np.zeros(d)]
    for _ in range(d + 1):
        xs.append(A @ xs[-1] + bvec)
    xf, _ = o.rna_combination(xs, 0.0)
    np.testing.assert_allclose(xf, np.linalg.solve(np.eye(d) - A, bvec), atol=1e-10)


def test_nce_accelerated_reaches_same_optimum_much_faster():
    n = 120
    G = syn.nce_matrix(n, "5.7", seed=8)
    U0 = syn.gaussian_block(n, 24, seed=9)
    _, h_plain = o.nce_solve(G, U0, 3, 3000, tol=1e-7)
    _, h_acc = o.nce_solve(G, U0, 3, 3000, tol=1e-7, accel_l=3)
    assert h_acc[-1].rel <= 1e-7 and h_plain[-1].rel <= 1e-7
    assert len(h_acc) * 4 < len(h_plain)
    assert abs(h_acc[-1].obj - h_plain[-1].obj) <= 1e-9 * abs(h_plain[-1].obj)


def _sym_with_spectrum(lam, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((len(lam), len(lam))))
    return (Q * lam) @ Q.T


def test_lanczos_estimate_brackets_an_eigenvalue_and_interlaces():
    """Sec. 4.1 Lanczos estimate of lambda_min: the Ritz value theta is >=
    lambda_min (Cauchy interlacing) and an eigenvalue of B lies in
    [theta - r, theta + r] with r the residual bound; on a matrix with a
    separated bottom eigenvalue 12 steps find it to 1e-6."""
    for seed in range(4):
        rng = np.random.default_rng(seed)
        lam = np.sort(rng.uniform(-3, 5, 60))
        B = _sym_with_spectrum(lam, 10 + seed)
        lo, th = o.lanczos_lower_estimate(lambda v: B @ v, 60, 12)
        assert th >= lam[0] - 1e-12
        r = th - lo
        assert r >= 0
        assert np.min(np.abs(lam - th)) <= r + 1e-12
    lam = np.concatenate([[-10.0], np.linspace(0.0, 1.0, 79)])
    B = _sym_with_spectrum(lam, 3)
    lo, th = o.lanczos_lower_estimate(lambda v: B @ v, 80, 12)
    assert abs(th - (-10.0)) < 1e-6 and lo <= -10.0 + 1e-9


def test_lanczos_full_krylov_space_is_exact():
    """k = n steps from a start vector with components along every
    eigenvector span the whole space: theta = lambda_min and the residual
    bound vanishes (to rounding); an invariant start (B = c I) stops after
    one step with the exact value."""
    lam = np.array([-2.5, -1.0, 0.25, 0.5, 3.0, 7.0])
    B = _sym_with_spectrum(lam, 5)
    lo, th = o.lanczos_lower_estimate(lambda v: B @ v, 6, 6)
    assert abs(th - lam[0]) < 1e-10 and abs(lo - lam[0]) < 1e-8
    lo, th = o.lanczos_lower_estimate(lambda v: 3.0 * v, 9, 12)
    assert lo == th == pytest.approx(3.0, abs=1e-15)


def test_lanczos_planted_sign_error_is_caught():
    """A recurrence with +beta q_{j-1} instead of -beta q_{j-1} no longer
    produces the Lanczos tridiagonal: its theta misses lambda_min."""
    lam = np.array([-2.5, -1.0, 0.25, 0.5, 3.0, 7.0])
    B = _sym_with_spectrum(lam, 5)

    def wrong(n, k):
        q = np.full(n, 1.0 / np.sqrt(n)); qp = np.zeros(n); bp = 0.0; al = []; be = []
        for _ in range(k):
            w = B @ q + bp * qp
            a = q @ w; w = w - a * q; al.append(a); bj = np.linalg.norm(w); be.append(bj)
            qp, q, bp = q, w / bj, bj
        T = np.diag(al) + np.diag(be[:-1], 1) + np.diag(be[:-1], -1)
        return np.linalg.eigvalsh(T)[0]

    assert abs(wrong(6, 6) - lam[0]) > 1e-3


def test_adaptive_width_rule_and_resize():
    """Sec. 4.2 width rule (reading R13): r_+ + guard rounded up to a multiple
    of 8 and clamped; growth appends the guard block's columns of the same
    index and repeats the smallest Ritz value; shrinking drops only
    columns with non-positive Ritz values."""
    n = 30
    block = np.arange(n * 24, dtype=float).reshape(n, 24)
    rule = o.AdaptiveWidth(guard=4, p_min=8, p_max=24, every=5, block=block)
    assert [rule.width(r) for r in (0, 3, 4, 5, 12, 13, 30)] == [8, 8, 8, 16, 16, 24, 24]
    U = np.ones((n, 8))
    th = np.array([5.0, 4.0, 3.0, 2.0, 1.0, 0.5, 0.25, 0.125])
    U2, th2 = o.adapt_width(U, th, 8, rule)
    assert U2.shape == (n, 16) and np.array_equal(U2[:, 8:], block[:, 8:16])
    assert np.array_equal(U2[:, :8], U) and np.all(th2[8:] == 0.125)
    th3 = np.concatenate([[3.0, 2.0], -np.arange(1.0, 15.0)])
    U3, th3b = o.adapt_width(U2, th3, 2, rule)
    assert U3.shape == (n, 8) and np.array_equal(U3, U2[:, :8]) and np.array_equal(th3b, th3[:8])
    with pytest.raises(AssertionError):
        o.adapt_width(U2, np.ones(16), 2, rule)


def test_adaptive_width_nce_grows_from_a_saturated_block():
    """Example 5.7 at n = 120 keeps about a dozen positive eigenvalues: a
    start block of 8 is saturated.  With the width rule it grows and
    reaches the optimum of a fixed 32-wide block (same objective, same
    positive count), ending at ceil8(r_+ + guard)."""
    n = 120
    G = syn.nce_matrix(n, "5.7", seed=8)
    full = syn.gaussian_block(n, 32, seed=9)
    _, h_fix = o.nce_solve(G, full, 3, 3000, tol=1e-7, accel_l=2)
    rule = o.AdaptiveWidth(guard=4, p_min=8, p_max=32, every=5, block=full)
    st, h_ad = o.nce_solve(G, full[:, :8], 3, 3000, tol=1e-7, accel_l=2, adapt=rule)
    assert h_fix[-1].rel <= 1e-7 and h_ad[-1].rel <= 1e-7
    assert abs(h_ad[-1].obj - h_fix[-1].obj) <= 1e-9 * abs(h_fix[-1].obj)
    assert h_ad[-1].r_plus == h_fix[-1].r_plus
    assert h_ad[0].r_plus == 8 and st.U.shape[1] in (rule.width(h_ad[-2].r_plus), rule.width(h_ad[-1].r_plus))


def test_adaptive_width_completion_shrinks_to_the_solution_rank():
    """Rank-2 completion (mu = 0.1) started 24 wide: the positive count falls
    to 2, the block shrinks to 8 (2 + 4 guards), and the solve reaches the
    optimum of the fixed 24-wide solve (objective to 1e-9)."""
    n, r, mu = 80, 2, 0.1
    inst = syn.completion_instance(n, r, 0.5, 24, seed=13, mu=mu)
    rule = o.AdaptiveWidth(guard=4, p_min=4, p_max=24, every=10, block=inst.U0_raw)
    st, hist = o.completion_solve(inst.omega, inst.U0_raw, mu, 1.0, 3, 300, adapt=rule, tol=1e-9)
    _, hist_fix = o.completion_solve(inst.omega, inst.U0_raw, mu, 1.0, 3, 300, tol=1e-9)
    assert st.U.shape[1] == 8
    assert hist[-1].r_plus == r and hist[-1].kkt <= 1e-9 and hist_fix[-1].kkt <= 1e-9
    assert abs(hist[-1].obj - hist_fix[-1].obj) <= 1e-9 * abs(hist_fix[-1].obj)


def _svt_F(omega, x, mu):
    n = omega.n
    Y = sp.csr_matrix((x, omega.colind, omega.rowptr), shape=(n, n)).toarray()
    s = np.linalg.svd(Y, compute_uv=False)
    return 0.5 * float(np.sum(np.maximum(s - mu, 0.0) ** 2)) - float(omega.vals @ x)


def test_svt_step_is_a_gradient_step_on_the_dual():
    """Eq. (ANM-dual): F(x) = 1/2||shrink_mu(A*(x))||^2 - b^T x has gradient
    A(shrink_mu(A*(x))) - b, so the SVT update x + tau (b - A(W)) is
    x - tau grad F.  Checked against central differences of F computed
    from singular values alone (no shrink code involved)."""
    n = 24
    I = syn.svt_instance(n, 2, 0.5, n, seed=4)
    rng = np.random.default_rng(1)
    x = 3.0 * I.omega.vals * (1 + 0.1 * rng.standard_normal(I.omega.nnz))
    mu, tau = 0.8, 0.7
    st = o.SVTState(x=x.copy(), U=I.U0_raw, theta_prev=None)
    st2, info = o.svt_step(I.omega, st, mu, tau, 1, exact=True)
    grad = -(st2.x - x) / tau
    for k in range(3):
        d = rng.standard_normal(I.omega.nnz)
        eps = 1e-6
        fd = (_svt_F(I.omega, x + eps * d, mu) - _svt_F(I.omega, x - eps * d, mu)) / (2 * eps)
        assert abs(fd - grad @ d) <= 1e-5 * max(1.0, abs(fd))
    assert abs(info.obj - _svt_F(I.omega, x, mu)) <= 1e-10 * abs(info.obj)


def test_shrink_is_the_nuclear_norm_prox():
    """shrink_mu(X) minimises mu||W||_* + 1/2||W - X||^2: its value is below
    that of random perturbations, and on a diagonal matrix it soft-thresholds
    the absolute diagonal."""
    rng = np.random.default_rng(2)
    X = rng.standard_normal((7, 7)) * 3
    mu = 2.0
    W = o.shrink(X, mu)
    f = lambda V: mu * np.linalg.svd(V, compute_uv=False).sum() + 0.5 * np.sum((V - X) ** 2)  # noqa: E731
    for _ in range(20):
        assert f(W) <= f(W + 1e-3 * rng.standard_normal((7, 7))) + 1e-12
    D = np.diag([5.0, -3.0, 1.0, -0.5])
    np.testing.assert_allclose(o.shrink(D, 2.0), np.diag([3.0, -1.0, 0.0, 0.0]), atol=1e-14)


def test_pfsvt_full_block_is_exact_svt():
    """p = n: the filtered block spans everything, so one PFSVT step equals
    the exact SVT step (Sec. 5.2.1)."""
    n = 30
    I = syn.svt_instance(n, 2, 0.4, n, seed=6)
    mu, tau = 5.0, 1.2 / 0.4
    st = o.svt_init(I.omega, I.U0_raw, tau)
    for _ in range(3):
        st, _ = o.svt_step(I.omega, st, mu, tau, 1, exact=True)
    a, ia = o.svt_step(I.omega, st, mu, tau, 1, exact=True)
    b, ib = o.svt_step(I.omega, st, mu, tau, 1)
    np.testing.assert_allclose(b.x, a.x, rtol=0, atol=1e-9 * np.abs(a.x).max())
    assert ia.svp == ib.svp and abs(ia.rel - ib.rel) < 1e-10


def test_svt_and_pfsvt_recover_a_low_rank_matrix():
    """Example MC (rank 2, n = 100, SR = 0.5, mu = 5n, tau = 1.2/SR): SVT
    reaches the 1e-4 residual with the right rank and mse near 1e-4, and
    PFSVT with degree 1 takes the same number of iterations (Table 5.x
    reports iter/svp/mse equal across SVT and PFSVT)."""
    n, r, sr = 100, 2, 0.5
    I = syn.svt_instance(n, r, sr, 8, seed=3)
    mu, tau = 5 * n, 1.2 / sr
    st_e, h_e = o.svt_solve(I.omega, I.U0_raw, mu, tau, 1, 500, exact=True, tol=1e-4)
    st_p, h_p = o.svt_solve(I.omega, I.U0_raw, mu, tau, 1, 500, tol=1e-4)
    assert h_e[-1].rel <= 1e-4 and h_p[-1].rel <= 1e-4
    assert h_e[-1].svp == h_p[-1].svp == r
    assert abs(len(h_e) - len(h_p)) <= 2
    M = I.ML @ I.MR.T
    L, s, R = o.svt_factors(I.omega, st_p, mu, tau, 1)
    assert np.linalg.norm((L * s) @ R.T - M) / np.linalg.norm(M) < 1e-3


def test_nnls_converges_to_the_prox_gradient_fixed_point():
    """With mu held fixed (no continuation) accelerated proximal gradient
    converges to the minimiser of mu||X||_* + 1/2||P_Omega(X) - b||^2, the
    fixed point X = shrink_mu(X - A*(A(X) - b)) (Sec. 5.2.2); the gradient and
    the prox are recomputed here densely from the definitions."""
    n = 40
    I = syn.svt_instance(n, 2, 0.5, n, seed=5)
    mu = 0.5
    st, hist = o.nnls_solve(I.omega, I.U0_raw, 1, 3000, exact=True, tol=1e-12, mu0=mu,
                            mu_bar_rel=1.0)
    X = (st.L * st.s) @ st.R.T
    mask = np.zeros((n, n))
    rows = I.omega.row_of_entries()
    mask[rows, I.omega.colind] = 1.0
    Md = np.zeros((n, n))
    Md[rows, I.omega.colind] = I.omega.vals
    G = X - (mask * X - Md)
    assert np.linalg.norm(o.shrink(G, mu) - X) <= 1e-8 * np.linalg.norm(X)
    # and it beats nearby points on the objective
    f = lambda Z: mu * np.linalg.svd(Z, compute_uv=False).sum() + 0.5 * np.sum((mask * Z - Md) ** 2)  # noqa: E731
    rng = np.random.default_rng(0)
    for _ in range(10):
        assert f(X) <= f(X + 1e-4 * rng.standard_normal((n, n))) + 1e-12


def test_pfnnls_full_block_is_exact_nnls():
    n = 30
    I = syn.svt_instance(n, 2, 0.5, n, seed=6)
    _, h_e = o.nnls_solve(I.omega, I.U0_raw, 1, 12, exact=True, mu_bar_rel=1e-2)
    _, h_p = o.nnls_solve(I.omega, I.U0_raw, 1, 12, mu_bar_rel=1e-2)
    for a, b in zip(h_e, h_p):
        assert a.svp == b.svp and abs(a.obj - b.obj) <= 1e-9 * abs(a.obj)
        assert abs(a.rel - b.rel) <= 1e-8 * max(a.rel, 1e-3)


def test_pfnnls_capped_matches_capped_nnls_and_recovers():
    """Reading R15 (at most p - 8 pairs): exact NNLS and PFNNLS (degree 1)
    reach the 1e-4 change with the same rank and nearly the same iterate, and
    recover the rank-5 matrix (Tables 5.x report equal iter/svp/mse)."""
    n, r, sr, p = 400, 5, 0.2, 16
    I = syn.svt_instance(n, r, sr, p, seed=4)
    M = I.ML @ I.MR.T
    out = []
    for exact in (True, False):
        st, h = o.nnls_solve(I.omega, I.U0_raw, 1, 300, exact=exact, tol=1e-4, mu_bar_rel=1e-2,
                             cap=p - 8)
        out.append((len(h), h[-1].svp, (st.L * st.s) @ st.R.T))
    assert out[0][1] == out[1][1] == r and abs(out[0][0] - out[1][0]) <= 5
    for _, _, X in out:
        assert np.linalg.norm(X - M) / np.linalg.norm(M) < 1e-2
    assert np.linalg.norm(out[0][2] - out[1][2]) / np.linalg.norm(out[0][2]) < 1e-3
