"""Plain, slow FP64 CPU oracle of the polynomial-filtered subspace extraction.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this module: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path (no kernels, headers, helpers or constants); its
only common ground with the CUDA path is the seeded input module
``pf_synthetic``, which holds none of the method's arithmetic.

Everything here is float64 numpy.  Library primitives (a matmul, a sparse
matmul, a QR factorisation, a symmetric eigendecomposition) serve as single
steps; there is no blocking, fusion or reordering beyond what the paper's
definitions state, so each function can be read against the paper by eye.

Citations are to the paper "Low-rank Matrix Optimization Using
Polynomial-filtered Subspace Extraction":

* Chebyshev polynomial T_d ............................ Sec. 2.1, Eq. (cheb)
* interval map rho(t) = T_d((t-(a+b)/2)/((b-a)/2)) ..... Sec. 2.1, Eq. (cheb-linear-map)
* three-term recurrence (mapped variable) .............. Sec. 4 (commented recurrence)
* filtered subspace update U+ = orth(rho(A) U) .......... Sec. 2.1, Eq. (subspace-update)
* projection P_S and Rayleigh-Ritz H = V^T X V .......... Sec. 2.2, Eq. (RR)
* PFPG ................................................. Sec. 2.2, Eqs. (pfpg1)-(pfpg2)
* DRS / PFAM for the standard SDP ...................... Sec. 2.3, Eqs. (PFAM1)-(PFAM2)
* choice of [a, b] ..................................... Sec. 4.1
* principal angles ..................................... Sec. 3.1, Definition of Theta
* Chebyshev growth lemma ............................... Sec. 3.1, Lemma (cheb-est)

Readings taken where the paper is silent or garbled (each also listed in the
design notes):

R1  The commented recurrence in Sec. 4 prints the mapped variable as
    c0 + c1*t with c0 = 2/(b-a), c1 = (a+b)/(a-b); the coefficients are
    swapped.  The oracle uses the map of Eq. (cheb-linear-map),
    x = (t - c)/e with c = (a+b)/2, e = (b-a)/2.
R2  The prox of G in Sec. 2.3 prints "+ tC"; from the prox definition applied
    to G = 1{AX=b} + <C,X> the sign is minus:
    prox_tG(Y) = (Y - tC) - A*(AA*)^{-1}(A(Y - tC) - b).
R3  orth is the thin QR factor Q with positive diagonal R (unique for a full
    rank block), as "a single QR decomposition" (Sec. 2.1).
R4  a = a rigorous lower bound of lambda_min: the Gershgorin bound of the
    sparse/diagonal part of the iteration matrix; the remaining part is PSD
    (X_k for completion, X~ for max-cut), so by Weyl's inequality the bound
    holds for the whole matrix.  b = (1-eta) theta_min_prev + eta a with
    eta = 0.1 (the "r largest" rule of Sec. 4.1 with the previous smallest
    Ritz value as the estimate); on the first iteration b = eta a when a < 0
    (the "all positive" rule), else b = a + (1-eta)(ub - a) with ub the
    Gershgorin upper bound.  If b - a < 1e-3 max(1,|a|), b is moved up to
    a + 1e-3 max(1,|a|) so the map stays finite.
R5  Ritz values are sorted descending (the paper's eigenvalue order, Sec. 1
    Notation); Ritz vectors are compared per cluster of equal values, so the
    sign and in-cluster basis carry no meaning.
R6  Max-cut: Z^0 = 0 gives X~ = 0 for any U, so the iteration starts at
    Z^1 = I - t offdiag(C) (the exact DRS image of Z^0 = 0).  The step is
    fixed at t = 10 sqrt(n)/||C||_F: sqrt(n)/||C||_F balances ||b|| = sqrt(n)
    against ||C||_F, and the factor 10 keeps the iterates' positive rank low
    (it converged fastest of 0.1..100 times that balance on seeded graphs).
R7  Max-cut KKT: y = -lambda/t, S = (X~ - Z_k)/t;
    pinf = ||diag X~ - 1||_2/(1+sqrt n);
    dinf = ||C - Diag(y) - S||_F/(1+||C||_F) = ||Z_k - Z_{k+1}||_F/(t(1+||C||_F));
    gap  = |<C,X~> - 1^T y|/(1+|<C,X~>|+|1^T y|); kkt = max of the three.
R9  The block carried to the next filter is the Ritz basis V~ = QY, the
    output "U <- QV" of the commented CheSE algorithm (Sec. 2.1); it spans the
    same subspace as the orthonormal Q (the warm start U^k of Eqs. (pfpg2),
    (PFAM2)), so the filtered subspace is unchanged in exact arithmetic.
R8  PSD completion, min_{X psd} 1/2||P_Omega(X-M)||^2 + mu tr X, PG step
    X+ = P_+(X - t P_Omega(X - M) - t mu I) (the symmetric analogue of the
    NNLS/SVT tests of Sec. 5.2); X^0 = 0; each iteration filters the current
    iteration matrix B_k = X_k - tS_k - t mu I before its Rayleigh-Ritz step
    (Eq. (pfpg2) shifted by one index, so U^0 is filtered before first use);
    kkt = ||X_k - X_{k+1}||_F/(1 + ||X_k||_F + ||t S_k||_F);
    objective f_k = 1/2||S_k||^2 + mu sum(max(theta,0)) at X_k.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional

import numpy as np
import scipy.sparse as sp

ETA = 0.1

# ---------------------------------------------------------------------------
# Chebyshev polynomials (Sec. 2.1)
# ---------------------------------------------------------------------------


def chebyshev_T(d: int, t):
    """T_d(t) from the closed form, Eq. (cheb):
    cos(d arccos t) on |t| <= 1, 1/2((t - sqrt(t^2-1))^d + (t + sqrt(t^2-1))^d) outside."""
    t = np.asarray(t, dtype=np.float64)
    out = np.empty_like(t)
    inside = np.abs(t) <= 1.0
    out[inside] = np.cos(d * np.arccos(t[inside]))
    to = t[~inside]
    s = np.sqrt(to * to - 1.0)
    out[~inside] = 0.5 * ((to - s) ** d + (to + s) ** d)
    return out


def interval_map(a: float, b: float):
    """Centre c and half-width e of [a, b]; x = (t - c)/e maps [a, b] to [-1, 1],
    Eq. (cheb-linear-map)."""
    return 0.5 * (a + b), 0.5 * (b - a)


def cheb_filter(apply_B: Callable[[np.ndarray], np.ndarray], U: np.ndarray,
                a: float, b: float, d: int) -> np.ndarray:
    """rho(B) U with rho(t) = T_d((t-c)/e), Eqs. (cheb-linear-map) and (cheb),
    evaluated by the Chebyshev three-term recurrence in the mapped variable
    x = (B - cI)/e (reading R1):
        Y_0 = U,  Y_1 = x Y_0,  Y_{j+1} = 2 x Y_j - Y_{j-1}."""
    c, e = interval_map(a, b)
    Y_prev = np.array(U, dtype=np.float64)
    if d == 0:
        return Y_prev
    Y = (apply_B(Y_prev) - c * Y_prev) / e
    for _ in range(1, d):
        Y_next = 2.0 * (apply_B(Y) - c * Y) / e - Y_prev
        Y_prev, Y = Y, Y_next
    return Y


# ---------------------------------------------------------------------------
# orth and Rayleigh-Ritz (Sec. 2.1 Eq. (subspace-update), Sec. 2.2 Eq. (RR))
# ---------------------------------------------------------------------------


def orth(Y: np.ndarray) -> np.ndarray:
    """Thin QR factor with positive diagonal R (reading R3)."""
    Q, R = np.linalg.qr(np.asarray(Y, dtype=np.float64), mode="reduced")
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s


@dataclasses.dataclass
class RitzPairs:
    theta: np.ndarray   # p Ritz values, descending
    V: np.ndarray       # n x p Ritz vectors  V~ = Q Y
    resid: np.ndarray   # ||B v_i - theta_i v_i||_2
    H: np.ndarray       # projected matrix Q^T B Q (symmetrised)


def rayleigh_ritz(apply_B, Q: np.ndarray) -> RitzPairs:
    """H = Q^T B Q, H = Y Lambda Y^T, V~ = Q Y (Sec. 2.2, Eq. (RR))."""
    W = apply_B(Q)
    H = Q.T @ W
    H = 0.5 * (H + H.T)
    lam, Yv = np.linalg.eigh(H)
    order = np.argsort(-lam, kind="stable")
    theta = lam[order]
    Yv = Yv[:, order]
    V = Q @ Yv
    R = W @ Yv - V * theta
    return RitzPairs(theta, V, np.linalg.norm(R, axis=0), H)


def subspace_sine(X: np.ndarray, Y: np.ndarray) -> float:
    """||sin Theta(X, Y)||_2 for orthonormal X, Y of equal width.  The
    singular values of X^T Y are cos Theta (Sec. 3.1 definition); the sines are
    the singular values of (I - X X^T) Y, which is the form used here because
    it keeps small angles accurate (1 - cos^2 cancels)."""
    if Y.shape[1] == 0:
        return 0.0
    R = Y - X @ (X.T @ Y)
    return float(np.linalg.norm(R, 2))


def psd_part(B: np.ndarray) -> np.ndarray:
    """P_+(B), the projection onto the PSD cone by a full EVD."""
    lam, V = np.linalg.eigh(0.5 * (B + B.T))
    return (V * np.maximum(lam, 0.0)) @ V.T


# ---------------------------------------------------------------------------
# Interval choice (Sec. 4.1, reading R4)
# ---------------------------------------------------------------------------


def gershgorin_bounds(S: sp.csr_matrix, diag_shift: np.ndarray):
    """Lower/upper Gershgorin bounds of the symmetric matrix S + Diag(diag_shift)."""
    S = sp.csr_matrix(S)
    d = S.diagonal() + diag_shift
    off = np.asarray(abs(S).sum(axis=1)).ravel() - np.abs(S.diagonal())
    return float(np.min(d - off)), float(np.max(d + off))


def choose_b(a: float, theta_prev: Optional[np.ndarray], ub: float, eta: float = ETA) -> float:
    if theta_prev is None:
        b = eta * a if a < 0 else a + (1.0 - eta) * (ub - a)
    else:
        b = (1.0 - eta) * float(np.min(theta_prev)) + eta * a
    gap = 1e-3 * max(1.0, abs(a))
    if b - a < gap:
        b = a + gap
    return b


# ---------------------------------------------------------------------------
# Block width (Sec. 4.2): when all positive eigenpairs are wanted, the number
# of positive Ritz values of the previous iteration estimates the dimension,
# and guard vectors are added.  Reading R13: after every `every`-th step the
# width becomes min(p_max, max(p_min, r_+ + guard)) rounded up to a multiple
# of `mult`; shrinking keeps the leading columns (the Ritz basis is sorted by
# decreasing Ritz value, so only columns with non-positive Ritz values are
# dropped), growing appends the same-index columns of a caller-drawn random
# block and repeats the smallest previous Ritz value for them (the iterate,
# held as factors of its positive part, is unchanged either way).
# ---------------------------------------------------------------------------


@dataclasses.dataclass
class AdaptiveWidth:
    guard: int
    p_min: int
    p_max: int
    every: int
    block: np.ndarray          # n x p_max random columns for growth
    mult: int = 8

    def width(self, r_plus: int) -> int:
        want = r_plus + self.guard
        want = ((want + self.mult - 1) // self.mult) * self.mult
        return int(min(self.p_max, max(self.p_min, want)))


def adapt_width(U: np.ndarray, theta_prev: np.ndarray, r_plus: int, rule: AdaptiveWidth):
    p = U.shape[1]
    p_new = rule.width(r_plus)
    if p_new < p:
        assert np.all(theta_prev[p_new:] <= 0.0), "would drop a positive Ritz pair"
        return U[:, :p_new].copy(), theta_prev[:p_new].copy()
    if p_new > p:
        U = np.hstack([U, rule.block[:, p:p_new]])
        theta_prev = np.concatenate([theta_prev, np.full(p_new - p, theta_prev[-1])])
    return U, theta_prev


# ---------------------------------------------------------------------------
# Max-cut SDP by PFAM / DRS (Sec. 2.3)
# ---------------------------------------------------------------------------


def prox_G_maxcut(Y: np.ndarray, C: np.ndarray, t: float) -> np.ndarray:
    """prox_tG(Y) for G = 1{diag X = 1} + <C, X> (reading R2, minus sign):
    A = diag, A* = Diag, AA* = I, b = 1."""
    W = Y - t * C
    return W - np.diag(np.diag(W) - 1.0)


@dataclasses.dataclass
class MaxCutState:
    Z: np.ndarray                       # dense iteration matrix
    U: np.ndarray                       # n x p block (warm start)
    lam: np.ndarray                     # lambda of the step that produced Z
    theta_prev: Optional[np.ndarray]    # Ritz values of the previous RR
    Xt_V: Optional[np.ndarray] = None   # factors of X~ of the previous step
    Xt_theta: Optional[np.ndarray] = None


@dataclasses.dataclass
class MaxCutInfo:
    a: float
    b: float
    obj: float
    pinf: float
    dinf: float
    gap: float
    kkt: float
    r_plus: int
    theta: np.ndarray


def maxcut_step_size(C: sp.csr_matrix) -> float:
    """t = 10 sqrt(n)/||C||_F (reading R6)."""
    return 10.0 * math.sqrt(C.shape[0]) / float(sp.linalg.norm(C, "fro"))


def maxcut_init(C: sp.csr_matrix, U0_raw: np.ndarray, t: float) -> MaxCutState:
    """Z^1 = prox_tG(2 P_+(Z^0) - Z^0) - P_+(Z^0) + Z^0 with Z^0 = 0, i.e. the
    exact DRS image of Z^0 = 0 (reading R6)."""
    n = C.shape[0]
    Cd = C.toarray()
    Z1 = prox_G_maxcut(np.zeros((n, n)), Cd, t)
    lam = np.diag(-t * Cd) - 1.0
    return MaxCutState(Z=Z1, U=np.array(U0_raw, dtype=np.float64), lam=lam, theta_prev=None)


def _maxcut_kkt(C: sp.csr_matrix, Cd: np.ndarray, Xt: np.ndarray, Z: np.ndarray,
                Z_next: np.ndarray, lam: np.ndarray, t: float):
    n = Z.shape[0]
    y = -lam / t
    Cnorm = float(np.linalg.norm(Cd))
    pobj = float(np.sum(Cd * Xt))
    dobj = float(np.sum(y))
    pinf = float(np.linalg.norm(np.diag(Xt) - 1.0)) / (1.0 + math.sqrt(n))
    S = (Xt - Z) / t
    dinf = float(np.linalg.norm(Cd - np.diag(y) - S)) / (1.0 + Cnorm)
    gap = abs(pobj - dobj) / (1.0 + abs(pobj) + abs(dobj))
    return pobj, pinf, dinf, gap


def maxcut_pfam_step(C: sp.csr_matrix, st: MaxCutState, t: float, degree: int,
                     exact: bool = False, eta: float = ETA):
    """One PFAM iteration, Eqs. (PFAM1)-(PFAM2), in the order
    filter (PFAM2 for the current Z) -> Rayleigh-Ritz -> DRS update (PFAM1).
    With ``exact`` the filter/RR pair is replaced by a full EVD (plain DRS)."""
    Cd = C.toarray()
    Z = st.Z
    n = Z.shape[0]
    apply_Z = lambda X: Z @ X  # noqa: E731
    # [a, b] from the sparse part -tC - Diag(lam) of Z = X~ - tC - Diag(lam)
    a, ub_sp = gershgorin_bounds(-t * C, -st.lam)
    ub = ub_sp + (float(np.max(st.Xt_theta)) if st.Xt_theta is not None and st.Xt_theta.size else 0.0)
    ub = max(ub, 0.0)
    b = choose_b(a, st.theta_prev, ub, eta)
    if exact:
        lamZ, VZ = np.linalg.eigh(Z)
        order = np.argsort(-lamZ, kind="stable")
        theta, V = lamZ[order], VZ[:, order]
        U = st.U
    else:
        U = orth(cheb_filter(apply_Z, st.U, a, b, degree))
        rr = rayleigh_ritz(apply_Z, U)
        theta, V = rr.theta, rr.V
    pos = theta > 0
    Xt = (V[:, pos] * theta[pos]) @ V[:, pos].T               # P_+(P_U(Z))
    lam = np.diag(2.0 * Xt - Z - t * Cd) - 1.0
    Z_next = prox_G_maxcut(2.0 * Xt - Z, Cd, t) - Xt + Z       # T_DRS, Eq. (PFAM1)
    pobj, pinf, dinf, gap = _maxcut_kkt(C, Cd, Xt, Z, Z_next, lam, t)
    info = MaxCutInfo(a, b, pobj, pinf, dinf, gap, max(pinf, dinf, gap), int(pos.sum()), theta)
    # the extracted block carried to the next filter is the Ritz basis V~ = Q Y
    # (the output U <- QV of the commented CheSE algorithm, Sec. 2.1); it spans
    # the same subspace as Q
    new = MaxCutState(Z=Z_next, U=V if not exact else U, lam=lam, theta_prev=theta,
                      Xt_V=V[:, pos], Xt_theta=theta[pos])
    return new, info


def maxcut_solve(C: sp.csr_matrix, U0_raw: np.ndarray, degree: int, iters: int,
                 t: Optional[float] = None, exact: bool = False, tol: float = 0.0,
                 adapt: Optional[AdaptiveWidth] = None):
    t = maxcut_step_size(C) if t is None else t
    st = maxcut_init(C, U0_raw, t)
    hist = []
    for k in range(iters):
        st, info = maxcut_pfam_step(C, st, t, degree, exact=exact)
        hist.append(info)
        if tol > 0 and info.kkt <= tol:
            break
        if adapt is not None and (k + 1) % adapt.every == 0:
            st.U, st.theta_prev = adapt_width(st.U, st.theta_prev, info.r_plus, adapt)
    return st, hist


# ---------------------------------------------------------------------------
# PSD completion by PFPG (Sec. 2.2, reading R8)
# ---------------------------------------------------------------------------


@dataclasses.dataclass
class CompletionState:
    V: np.ndarray                       # n x r+ factor of X_k, X_k = V diag(w) V^T
    w: np.ndarray                       # r+ nonnegative weights
    U: np.ndarray                       # n x p warm-start block
    theta_prev: Optional[np.ndarray]


@dataclasses.dataclass
class CompletionInfo:
    a: float
    b: float
    obj: float
    kkt: float
    r_plus: int
    theta: np.ndarray


def omega_matrix(omega) -> sp.csr_matrix:
    return sp.csr_matrix((omega.vals.astype(np.float64), omega.colind, omega.rowptr),
                         shape=(omega.n, omega.n))


def sampled_residual(Om: sp.csr_matrix, V: np.ndarray, w: np.ndarray) -> sp.csr_matrix:
    """S = P_Omega(X - M) with X = V diag(w) V^T, entry by entry on Omega."""
    coo = Om.tocoo()
    if V.shape[1]:
        x = np.einsum("ij,ij->i", V[coo.row] * w, V[coo.col])
    else:
        x = np.zeros(coo.nnz)
    return sp.csr_matrix((x - coo.data, (coo.row, coo.col)), shape=Om.shape)


def completion_init(n: int, U0_raw: np.ndarray) -> CompletionState:
    return CompletionState(V=np.zeros((n, 0)), w=np.zeros(0), U=np.array(U0_raw, dtype=np.float64),
                           theta_prev=None)


def _lowrank_fro_diff(V1, w1, V2, w2) -> float:
    """||V1 diag(w1) V1^T - V2 diag(w2) V2^T||_F from the factors."""
    def tr(Va, wa, Vb, wb):
        if Va.shape[1] == 0 or Vb.shape[1] == 0:
            return 0.0
        M = Va.T @ Vb
        return float(np.sum((wa[:, None] * M) * (M * wb[None, :])))
    v = tr(V1, w1, V1, w1) - 2.0 * tr(V1, w1, V2, w2) + tr(V2, w2, V2, w2)
    return math.sqrt(max(v, 0.0))


def completion_pfpg_step(Om: sp.csr_matrix, st: CompletionState, mu: float, t: float,
                         degree: int, exact: bool = False, eta: float = ETA):
    """One PFPG iteration (Eqs. (pfpg1)-(pfpg2), reading R8)."""
    n = Om.shape[0]
    S = sampled_residual(Om, st.V, st.w)
    V, w = st.V, st.w

    def apply_B(Y):
        XY = V @ (w[:, None] * (V.T @ Y)) if V.shape[1] else np.zeros_like(Y)
        return XY - t * (S @ Y) - t * mu * Y

    a, ub_sp = gershgorin_bounds(-t * S, np.full(n, -t * mu))
    ub = max(ub_sp + (float(np.max(w)) if w.size else 0.0), 0.0)
    b = choose_b(a, st.theta_prev, ub, eta)
    if exact:
        Bd = (V * w) @ V.T - t * S.toarray() - t * mu * np.eye(n)
        lamB, VB = np.linalg.eigh(0.5 * (Bd + Bd.T))
        order = np.argsort(-lamB, kind="stable")
        theta, Vr = lamB[order], VB[:, order]
        U = st.U
    else:
        U = orth(cheb_filter(apply_B, st.U, a, b, degree))
        rr = rayleigh_ritz(apply_B, U)
        theta, Vr = rr.theta, rr.V
    pos = theta > 0
    V_next, w_next = Vr[:, pos], theta[pos]
    Snorm = float(sp.linalg.norm(S, "fro"))
    Xnorm = float(np.linalg.norm(w))
    kkt = _lowrank_fro_diff(V, w, V_next, w_next) / (1.0 + Xnorm + t * Snorm)
    obj = 0.5 * Snorm ** 2 + mu * float(np.sum(w))
    info = CompletionInfo(a, b, obj, kkt, int(pos.sum()), theta)
    return CompletionState(V=V_next, w=w_next, U=Vr if not exact else U, theta_prev=theta), info


def completion_solve(omega, U0_raw, mu: float, t: float, degree: int, iters: int,
                     exact: bool = False, tol: float = 0.0,
                     adapt: Optional[AdaptiveWidth] = None):
    Om = omega_matrix(omega)
    st = completion_init(omega.n, U0_raw)
    hist = []
    for k in range(iters):
        st, info = completion_pfpg_step(Om, st, mu, t, degree, exact=exact)
        hist.append(info)
        if tol > 0 and info.kkt <= tol:
            break
        if adapt is not None and (k + 1) % adapt.every == 0:
            st.U, st.theta_prev = adapt_width(st.U, st.theta_prev, info.r_plus, adapt)
    return st, hist


# ---------------------------------------------------------------------------
# Nearest correlation estimation by PFPG on the dual (Sec. 5.1)
# ---------------------------------------------------------------------------
#
# min_x F(x) = 1/2 ||P_+(G + Diag(x))||_F^2 - 1^T x  (the dual of the NCE
# problem, Eq. (NCE-dual)), grad F(x) = diag(P_+(G + Diag(x))) - 1
# (Eq. (NCE-gradient)); the gradient method takes x+ = x - tau grad F(x).
# PFPG replaces P_+ by the projection onto the positive Ritz pairs of the
# filtered subspace.  Readings: tau = 1 (grad F is 1-Lipschitz); x^0 =
# 1 - diag(G) (as in Sec. 5.1); the interval uses reading R4 with the lower
# end a from a LANCZOS_STEPS-step Lanczos run on G + Diag(x) (Sec. 4.1 names
# Lanczos for estimating the smallest eigenvalue; a Gershgorin bound of a
# dense matrix is some sqrt(n) times too loose), a = theta_min - residual
# bound, with full reorthogonalisation (without it the process loses
# orthogonality once the dominant Ritz value has converged, which it does in
# a step or two for these G, and the small end drifts with rounding),
# refreshed every iteration; the Gershgorin upper bound stays as the
# upper bound; the reported residual is ||grad F(x_k)|| / ||grad F(x_0)||.
# Reading R11 (acceleration, Sec. 4.3): windows of l + 2 iterates (the NCE
# workload takes l = 2), lam = 1e-10 tr(U^T U); after a combination the
# iteration restarts from it.


@dataclasses.dataclass
class NCEState:
    x: np.ndarray
    U: np.ndarray
    theta_prev: Optional[np.ndarray]
    g0: Optional[float] = None


@dataclasses.dataclass
class NCEInfo:
    a: float
    b: float
    obj: float
    gnorm: float
    rel: float
    r_plus: int
    theta: np.ndarray


LANCZOS_STEPS = 12


def lanczos_lower_estimate(matvec, n: int, k: int = LANCZOS_STEPS):
    """k steps of the symmetric Lanczos process from q_0 = 1/sqrt(n), with
    full reorthogonalisation (classical Gram-Schmidt against every basis
    vector, the form ARPACK-style Lanczos codes use):
        y = B q_j - beta_{j-1} q_{j-1},  c = Q_j^T y,  alpha_j = c_j,
        w = y - Q_j c,  beta_j = ||w||,  q_{j+1} = w / beta_j,
    Q_j = [q_0, ..., q_j].  With (theta, s) the smallest eigenpair of the
    tridiagonal T (alpha on the diagonal, beta beside it), some eigenvalue of
    B lies within beta_{k-1} |s_{k-1}| of theta, and theta >= lambda_min(B)
    (interlacing).  Returns (theta - beta_{k-1}|s_{k-1}|, theta).  A zero
    beta ends the process early (an invariant subspace: exact)."""
    Q = np.zeros((n, min(k, n)))
    q = np.full(n, 1.0 / np.sqrt(n))
    beta_prev = 0.0
    alpha, beta = [], []
    for j in range(min(k, n)):
        Q[:, j] = q
        y = matvec(q)
        if j > 0:
            y = y - beta_prev * Q[:, j - 1]
        c = Q[:, :j + 1].T @ y
        alpha.append(float(c[j]))
        w = y - Q[:, :j + 1] @ c
        bj = float(np.linalg.norm(w))
        beta.append(bj)
        if bj == 0.0:
            break
        q, beta_prev = w / bj, bj
    m = len(alpha)
    T = np.diag(alpha) + np.diag(beta[:m - 1], 1) + np.diag(beta[:m - 1], -1)
    th, S = np.linalg.eigh(T)
    return float(th[0] - beta[m - 1] * abs(S[m - 1, 0])), float(th[0])


def nce_objective(G: np.ndarray, x: np.ndarray) -> float:
    lam = np.linalg.eigvalsh(G + np.diag(x))
    return 0.5 * float(np.sum(np.maximum(lam, 0.0) ** 2)) - float(np.sum(x))


def nce_init(G: np.ndarray, U0_raw: np.ndarray) -> NCEState:
    return NCEState(x=1.0 - np.diag(G).copy(), U=np.array(U0_raw, dtype=np.float64),
                    theta_prev=None)


def nce_step(G: np.ndarray, st: NCEState, degree: int, tau: float = 1.0, exact: bool = False,
             eta: float = ETA):
    """One (polynomial-filtered) gradient step on the NCE dual."""
    B = G + np.diag(st.x)
    off = np.sum(np.abs(B), axis=1) - np.abs(np.diag(B))
    ub = float(np.max(np.diag(B) + off))
    a, _ = lanczos_lower_estimate(lambda v: B @ v, B.shape[0])
    b = choose_b(a, st.theta_prev, max(ub, 0.0), eta)
    if exact:
        lam, VB = np.linalg.eigh(B)
        order = np.argsort(-lam, kind="stable")
        theta, V = lam[order], VB[:, order]
        U = st.U
    else:
        U = orth(cheb_filter(lambda X: B @ X, st.U, a, b, degree))
        rr = rayleigh_ritz(lambda X: B @ X, U)
        theta, V = rr.theta, rr.V
        U = V
    pos = theta > 0
    dX = np.sum((V[:, pos] ** 2) * theta[pos], axis=1)        # diag(P_+(B)) from the Ritz pairs
    g = dX - 1.0
    gnorm = float(np.linalg.norm(g))
    g0 = gnorm if st.g0 is None else st.g0
    obj = 0.5 * float(np.sum(theta[pos] ** 2)) - float(np.sum(st.x))
    info = NCEInfo(a, b, obj, gnorm, gnorm / g0 if g0 > 0 else 0.0, int(pos.sum()), theta)
    return NCEState(x=st.x - tau * g, U=U, theta_prev=theta, g0=g0), info


def rna_combination(points, lam_rel: float):
    """Extrapolation of Sec. 4.3 (regularized nonlinear acceleration): with
    U = [x_1 - x_0, ..., x_{l+1} - x_l] (l+2 points), the coefficients
    c = argmin_{1^T c = 1} c^T (U^T U + lam I) c are (U^T U + lam I)^{-1} 1
    normalised to sum 1, and the new point is sum_{i=0}^{l} c_i x_i.
    Reading R11: lam = lam_rel * tr(U^T U)."""
    X = np.stack(points, axis=1)
    U = X[:, 1:] - X[:, :-1]
    M = U.T @ U
    M = M + lam_rel * np.trace(M) * np.eye(M.shape[0])
    z = np.linalg.solve(M, np.ones(M.shape[0]))
    c = z / np.sum(z)
    return X[:, :-1] @ c, c


def nce_solve(G, U0_raw, degree: int, iters: int, exact: bool = False, tol: float = 0.0,
              accel_l: int = 0, accel_lam: float = 1e-10,
              adapt: Optional[AdaptiveWidth] = None):
    """Filtered (or exact) gradient method on the NCE dual; with accel_l > 0
    every l+2 iterates are combined by rna_combination and the iteration
    restarts from the combination (Sec. 4.3)."""
    st = nce_init(G, U0_raw)
    hist = []
    window = [st.x.copy()]
    for k in range(iters):
        st, info = nce_step(G, st, degree, exact=exact)
        hist.append(info)
        if tol > 0 and info.rel <= tol:
            break
        if adapt is not None and (k + 1) % adapt.every == 0:
            st.U, st.theta_prev = adapt_width(st.U, st.theta_prev, info.r_plus, adapt)
        if accel_l > 0:
            window.append(st.x.copy())
            if len(window) == accel_l + 2:
                st.x, _ = rna_combination(window, accel_lam)
                window = [st.x.copy()]
    return st, hist


# ---------------------------------------------------------------------------
# Nuclear-norm matrix completion by SVT and its polynomial-filtered form
# PFSVT (Sec. 5.2.1, Eq. (svt))
# ---------------------------------------------------------------------------
#
# min ||X||_* + 1/(2 mu) ||X||_F^2 s.t. P_Omega(X) = P_Omega(M) is solved on
# its dual F(x) = 1/2 ||shrink_mu(A*(x))||_F^2 - b^T x (Eq. (ANM-dual)) by the
# SVT iteration W = shrink_mu(A*(x)), x <- x + tau (b - A(W)), a gradient step
# on F.  A*(x) is the sparse matrix Y with the values x on Omega.  PFSVT takes
# the singular pairs of Y from a subspace filtered on Y^T Y (Sec. 5.2.1:
# extraction from A^T A), then a Rayleigh-Ritz step on the projected Gram
# matrix: B = Y Q, B^T B = Wr diag(theta) Wr^T, sigma = sqrt(theta), right
# vectors Q Wr, left vectors B Wr / sigma.
# Readings (R14): square M (the paper's tests have m = n); x starts at
# tau P_Omega(M), the exact result of the first iteration from x = 0 (W = 0
# there); the interval on Y^T Y >= 0 is a = 0 with reading R4 for b and the
# bound ||Y||_1 ||Y||_inf >= sigma_max^2 as upper bound; mu = 5 n and
# tau = 1.2 / SR as in the SVT reference the paper cites; the reported
# residual is ||P_Omega(W - M)||_F / ||P_Omega(M)||_F, the stopping rule of
# that reference; the block carried forward is the Ritz basis Q Wr.


def shrink(X: np.ndarray, mu: float) -> np.ndarray:
    """Singular value soft-thresholding U diag((sigma - mu)_+) V^T (dense)."""
    Ud, s, Vt = np.linalg.svd(X, full_matrices=False)
    return (Ud * np.maximum(s - mu, 0.0)) @ Vt


@dataclasses.dataclass
class SVTState:
    x: np.ndarray                       # dual variable on Omega (row-major entry order)
    U: np.ndarray                       # n x p warm-start block (right singular subspace)
    theta_prev: Optional[np.ndarray]


@dataclasses.dataclass
class SVTInfo:
    a: float
    b: float
    obj: float                          # F(x) at the step's x
    rel: float                          # ||P_Omega(W - M)|| / ||P_Omega(M)||
    svp: int                            # singular values above mu
    theta: np.ndarray                   # Ritz values of Y^T Y (sigma^2), descending


def svt_pattern(omega) -> sp.csr_matrix:
    return sp.csr_matrix((np.ones(omega.nnz), omega.colind, omega.rowptr),
                         shape=(omega.n, omega.n))


def svt_init(omega, U0_raw: np.ndarray, tau: float) -> SVTState:
    return SVTState(x=tau * omega.vals.astype(np.float64), U=np.array(U0_raw, dtype=np.float64),
                    theta_prev=None)


def svt_step(omega, st: SVTState, mu: float, tau: float, degree: int, exact: bool = False,
             eta: float = ETA):
    n = omega.n
    m_vals = omega.vals.astype(np.float64)
    Y = sp.csr_matrix((st.x, omega.colind, omega.rowptr), shape=(n, n))
    absY = abs(Y)
    ub = float(np.max(np.asarray(absY.sum(axis=0)))) * float(np.max(np.asarray(absY.sum(axis=1))))
    a = 0.0
    b = choose_b(a, st.theta_prev, ub, eta)
    rows = omega.row_of_entries()
    if exact:
        Ud, s, Vt = np.linalg.svd(Y.toarray())
        theta = s ** 2
        Vr, Lr = Vt.T, Ud * s
        U_next = st.U
    else:
        Q = orth(cheb_filter(lambda Z: Y.T @ (Y @ Z), st.U, a, b, degree))
        Bm = Y @ Q
        H = Bm.T @ Bm
        H = 0.5 * (H + H.T)
        lam, Wr = np.linalg.eigh(H)
        order = np.argsort(-lam, kind="stable")
        theta, Wr = lam[order], Wr[:, order]
        Vr, Lr = Q @ Wr, Bm @ Wr
        U_next = Vr
    sigma = np.sqrt(np.maximum(theta, 0.0))
    keep = sigma > mu
    scale = np.zeros_like(sigma)
    scale[keep] = (sigma[keep] - mu) / sigma[keep]
    w = np.einsum("el,el->e", Lr[rows][:, keep] * scale[keep], Vr[omega.colind][:, keep])
    resid = m_vals - w
    rel = float(np.linalg.norm(resid) / np.linalg.norm(m_vals))
    obj = 0.5 * float(np.sum((sigma[keep] - mu) ** 2)) - float(m_vals @ st.x)
    info = SVTInfo(a, b, obj, rel, int(keep.sum()), theta)
    return SVTState(x=st.x + tau * resid, U=U_next, theta_prev=theta), info


def svt_factors(omega, st: SVTState, mu: float, tau: float, degree: int):
    """Factors (L, s, R) of the primal iterate W = L diag(s) R^T that the
    next step would form (for recovery checks)."""
    n = omega.n
    Y = sp.csr_matrix((st.x, omega.colind, omega.rowptr), shape=(n, n))
    Ud, s, Vt = np.linalg.svd(Y.toarray())
    keep = s > mu
    return Ud[:, keep], s[keep] - mu, Vt[keep].T


def svt_solve(omega, U0_raw, mu: float, tau: float, degree: int, iters: int,
              exact: bool = False, tol: float = 0.0, adapt: Optional[AdaptiveWidth] = None):
    st = svt_init(omega, U0_raw, tau)
    hist = []
    for k in range(iters):
        st, info = svt_step(omega, st, mu, tau, degree, exact=exact)
        hist.append(info)
        if tol > 0 and info.rel <= tol:
            break
        if adapt is not None and (k + 1) % adapt.every == 0:
            st.U, st.theta_prev = adapt_width(st.U, st.theta_prev, info.svp, adapt)
    return st, hist


# ---------------------------------------------------------------------------
# Nuclear-norm regularised least squares by accelerated proximal gradient and
# its polynomial-filtered form PFNNLS (Sec. 5.2.2, Eq. (NMM-penalized))
# ---------------------------------------------------------------------------
#
# min mu ||X||_* + 1/2 ||A(X) - b||^2 (the paper's ||X||_* + 1/(2mu)||A(X)-b||^2
# scaled by mu), A = P_Omega, by the accelerated proximal gradient method of
# the NNLS reference the paper uses: Y = (1 + beta) X^k - beta X^{k-1} with
# beta = (t_{k-1} - 1)/t_k, G = Y - A*(A(Y) - b) (step 1/L, L = ||A||^2 = 1),
# X^{k+1} = shrink_mu(G), t_{k+1} = (1 + sqrt(1 + 4 t_k^2))/2.  G is the
# matrix beta_1 U^k V^k^T - beta_2 U^{k-1} V^{k-1}^T - beta_3 G^k of Sec. 5.2.2
# (low rank plus sparse); PFNNLS takes its singular pairs from a subspace
# filtered on G^T G, as PFSVT does.  Readings (R15): continuation
# mu_{k+1} = max(0.7 mu_k, mu_bar) from mu_0 = 0.1 ||P_Omega(M)||_1-inf bound
# (sqrt(||.||_1 ||.||_inf) >= sigma_max) to mu_bar = 1e-4 mu_0, as in that
# reference for noiseless data; X^0 = X^{-1} = 0, t_0 = t_{-1} = 1; the
# iterate is kept as orthonormal factors X = L diag(s) R^T; the reported
# change is ||X^{k+1} - X^k||_F / max(1, ||X^{k+1}||_F) and the objective is
# that of X^k with the step's mu; the interval on G^T G takes a = 0, b by
# reading R4 and the upper bound ((1+beta) max s^k + beta max s^{k-1}
# + sqrt(||A*(r)||_1 ||A*(r)||_inf))^2.


@dataclasses.dataclass
class NNLSState:
    L: np.ndarray                       # n x r_k left factor of X^k (orthonormal columns)
    s: np.ndarray                       # r_k shrunk singular values
    R: np.ndarray                       # n x r_k right factor
    Lp: np.ndarray
    sp_: np.ndarray
    Rp: np.ndarray
    t: float
    t_prev: float
    mu: float
    U: np.ndarray                       # n x p warm-start block
    theta_prev: Optional[np.ndarray]


@dataclasses.dataclass
class NNLSInfo:
    a: float
    b: float
    obj: float
    rel: float                          # ||X^{k+1} - X^k|| / max(1, ||X^{k+1}||)
    svp: int
    mu: float
    theta: np.ndarray


def _abs_bound(omega, vals) -> float:
    n = omega.n
    Rm = sp.csr_matrix((np.abs(vals), omega.colind, omega.rowptr), shape=(n, n))
    return math.sqrt(float(np.max(np.asarray(Rm.sum(axis=1)))) *
                     float(np.max(np.asarray(Rm.sum(axis=0)))))


def nnls_init(omega, U0_raw: np.ndarray, mu0: Optional[float] = None) -> NNLSState:
    n = omega.n
    z = np.zeros((n, 0))
    mu0 = 0.1 * _abs_bound(omega, omega.vals.astype(np.float64)) if mu0 is None else mu0
    return NNLSState(L=z, s=np.zeros(0), R=z, Lp=z, sp_=np.zeros(0), Rp=z, t=1.0, t_prev=1.0,
                     mu=mu0, U=np.array(U0_raw, dtype=np.float64), theta_prev=None)


def _sampled(omega, L, s, R):
    rows = omega.row_of_entries()
    if s.size == 0:
        return np.zeros(omega.nnz)
    return np.einsum("el,el->e", L[rows] * s, R[omega.colind])


def _factor_fro_diff(L1, s1, R1, L2, s2, R2) -> float:
    """||L1 S1 R1^T - L2 S2 R2^T||_F from p x p Grams (orthonormal factors)."""
    cross = float(np.sum((s1[:, None] * (L1.T @ L2) * s2[None, :]) * (R1.T @ R2)))
    return math.sqrt(max(float(s1 @ s1) + float(s2 @ s2) - 2.0 * cross, 0.0))


def nnls_step(omega, st: NNLSState, degree: int, mu_bar: float, exact: bool = False,
              eta: float = ETA, cap: Optional[int] = None):
    n = omega.n
    m_vals = omega.vals.astype(np.float64)
    beta = (st.t_prev - 1.0) / st.t
    x_now = _sampled(omega, st.L, st.s, st.R)
    x_prev = _sampled(omega, st.Lp, st.sp_, st.Rp)
    r = (1.0 + beta) * x_now - beta * x_prev - m_vals          # A(Y) - b
    Rsp = sp.csr_matrix((r, omega.colind, omega.rowptr), shape=(n, n))
    cL, cP = (1.0 + beta) * st.s, beta * st.sp_

    def apply_G(Z):
        out = -(Rsp @ Z)
        if st.s.size:
            out = out + st.L @ (cL[:, None] * (st.R.T @ Z))
        if st.sp_.size:
            out = out - st.Lp @ (cP[:, None] * (st.Rp.T @ Z))
        return out

    def apply_Gt(Z):
        out = -(Rsp.T @ Z)
        if st.s.size:
            out = out + st.R @ (cL[:, None] * (st.L.T @ Z))
        if st.sp_.size:
            out = out - st.Rp @ (cP[:, None] * (st.Lp.T @ Z))
        return out

    lr = (float(np.max(cL)) if cL.size else 0.0) + (float(np.max(cP)) if cP.size else 0.0)
    ub = (lr + _abs_bound(omega, r)) ** 2
    a = 0.0
    b = choose_b(a, st.theta_prev, ub, eta)
    mu = st.mu
    if exact:
        Gd = apply_G(np.eye(n))
        Ud, sig, Vt = np.linalg.svd(Gd)
        theta = sig ** 2
        Rr, Bw = Vt.T, Ud * sig
        U_next = st.U
    else:
        Q = orth(cheb_filter(lambda Z: apply_Gt(apply_G(Z)), st.U, a, b, degree))
        Bm = apply_G(Q)
        H = Bm.T @ Bm
        lam, Wr = np.linalg.eigh(0.5 * (H + H.T))
        order = np.argsort(-lam, kind="stable")
        theta, Wr = lam[order], Wr[:, order]
        Rr, Bw = Q @ Wr, Bm @ Wr
        U_next = Rr
    sigma = np.sqrt(np.maximum(theta, 0.0))
    keep = sigma > mu
    if cap is not None:
        keep[cap:] = False                     # at most `cap` pairs (reading R15)
    L_new = Bw[:, keep] / sigma[keep]
    s_new = sigma[keep] - mu
    R_new = Rr[:, keep]
    rel = _factor_fro_diff(L_new, s_new, R_new, st.L, st.s, st.R) / max(
        1.0, float(np.linalg.norm(s_new)))
    obj = mu * float(np.sum(st.s)) + 0.5 * float(np.sum((x_now - m_vals) ** 2))
    info = NNLSInfo(a, b, obj, rel, int(keep.sum()), mu, theta)
    t_next = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * st.t * st.t))
    new = NNLSState(L=L_new, s=s_new, R=R_new, Lp=st.L, sp_=st.s, Rp=st.R, t=t_next,
                    t_prev=st.t, mu=max(0.7 * mu, mu_bar), U=U_next, theta_prev=theta)
    return new, info


def nnls_solve(omega, U0_raw, degree: int, iters: int, exact: bool = False, tol: float = 0.0,
               mu0: Optional[float] = None, mu_bar_rel: float = 1e-4, cap: Optional[int] = None):
    st = nnls_init(omega, U0_raw, mu0)
    mu_bar = mu_bar_rel * st.mu
    hist = []
    for _ in range(iters):
        st, info = nnls_step(omega, st, degree, mu_bar, exact=exact, cap=cap)
        hist.append(info)
        if tol > 0 and info.mu <= mu_bar and info.rel <= tol:
            break
    return st, hist
