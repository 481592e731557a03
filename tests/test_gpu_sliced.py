"""The sliced dense product (int8 digit planes of A, fp16 planes of X, fp16
MMAs on the tensor cores, exact fp32 level sums, int64 fold) against an
extended-precision reference.

Bound.  With rowmax_i = max_k |A_ik| and colmax_j = max_k |X_kj|, each term
A_ik X_kj of the sum carries at most
  * 2^-54 rowmax_i colmax_j from rounding A and X to their digit planes
    (each entry to within 2^(e - 56), e its row's / chunk's exponent with
    max < 2^e <= 2 max),
  * 24 * 2^-56 rowmax_i colmax_j from the dropped pairs of digit planes
    (six pairs of weight 2^(eA + eX - 56) at the first dropped level),
and each 128-wide chunk at most 2^-48 rowmax_i colmax_j from the int64 fold,
so |Y_ij - (A X)_ij| <= n 2^-50 rowmax_i colmax_j.  An FP64 dot product's
worst-case bound is n 2^-53 sum_k |A_ik X_kj|, the same order.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
SLICED, FP64 = 0, 1


@pytest.fixture(scope="module")
def S():
    from paper_1904_10585_gb300 import solver
    return solver


def t64(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(DEV)


def wide_range(n, p, seed, span_a=30, span_x=20):
    """A with rows scaled by 2^U(-span_a, span_a), X with columns scaled by
    2^U(-span_x, span_x); a zero row and a zero column where there is room."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) * np.exp2(rng.uniform(-span_a, span_a, n))[:, None]
    X = rng.standard_normal((n, p)) * np.exp2(rng.uniform(-span_x, span_x, p))[None, :]
    if n > 3:
        A[n // 2] = 0.0
    if p > 2:
        X[:, p // 2] = 0.0
    return A, X


def reference(A, X, rows=None):
    Ar = A if rows is None else A[rows]
    return Ar.astype(np.longdouble) @ X.astype(np.longdouble)


def check_bound(Y, A, X, rows=None):
    n = A.shape[0]
    Ar = A if rows is None else A[rows]
    Yr = Y if rows is None else Y[rows]
    ref = reference(A, X, rows)
    bound = n * 2.0 ** -50 * np.abs(Ar).max(axis=1)[:, None] * np.abs(X).max(axis=0)[None, :]
    err = np.abs(Yr.astype(np.longdouble) - ref).astype(np.float64)
    assert np.all(err <= bound), float(np.max(err / np.maximum(bound, 1e-300)))
    return err, ref


def gpu_apply(S, A, X, dp, ctx=None):
    n, p = X.shape
    own = ctx is None
    if own:
        ctx = S.Context(p=p, n_max=n, degree=1, dense_product=dp)
    try:
        Y = torch.empty(n, p, dtype=torch.float64, device=DEV)
        S.apply(ctx, S.dense_operator(t64(A)), t64(X), Y)
        torch.cuda.synchronize()
        return Y.cpu().numpy()
    finally:
        if own:
            ctx.close()


@pytest.mark.parametrize("n,p", [(2, 1), (17, 16), (64, 5), (130, 33), (300, 40), (513, 64),
                                 (1000, 32)])
def test_sliced_product_within_bound(S, n, p):
    A, X = wide_range(n, p, seed=n + p)
    Y = gpu_apply(S, A, X, SLICED)
    err, ref = check_bound(Y, A, X)
    # the FP64 FMA product on the same data, for scale: the sliced error is
    # of the same order
    Y64 = gpu_apply(S, A, X, FP64)
    err64 = np.abs(Y64.astype(np.longdouble) - ref).astype(np.float64)
    scale = np.abs(A).max(axis=1)[:, None] * np.abs(X).max(axis=0)[None, :]
    with np.errstate(invalid="ignore", divide="ignore"):
        rel_s = np.nanmax(np.where(scale > 0, err / scale, 0.0))
        rel_d = np.nanmax(np.where(scale > 0, err64 / scale, 0.0))
    assert rel_s <= 32 * rel_d + n * 2.0 ** -56, (rel_s, rel_d)


@pytest.mark.parametrize("n,p", [(2000, 48), (4100, 32), (5000, 64), (9000, 16)])
def test_sliced_product_large_sampled_rows(S, n, p):
    """Several K splits per row block (the last CTA of each row block sums
    the partials); checked on sampled rows."""
    A, X = wide_range(n, p, seed=n, span_a=8, span_x=8)
    Y = gpu_apply(S, A, X, SLICED)
    rows = np.random.default_rng(1).choice(n, 64, replace=False)
    check_bound(Y, A, X, rows)


def test_sliced_product_reuses_context_across_sizes(S):
    """One context, sizes 1000 -> 300 -> 1000: digit planes and arrival
    tickets are reused (the tickets must return to zero after each launch)."""
    p = 24
    with S.Context(p=p, n_max=1000, degree=1, dense_product=SLICED) as ctx:
        for n, seed in [(1000, 1), (300, 2), (1000, 3)]:
            A, X = wide_range(n, p, seed=seed)
            check_bound(gpu_apply(S, A, X, SLICED, ctx=ctx), A, X)


def test_sliced_product_deterministic(S):
    A, X = wide_range(777, 40, seed=5)
    assert np.array_equal(gpu_apply(S, A, X, SLICED), gpu_apply(S, A, X, SLICED))


def test_sliced_product_exact_on_small_integers(S):
    """Entries that are small integers are their own first digit plane: the
    product is exact (every level sum is an exact fp32 integer)."""
    rng = np.random.default_rng(3)
    n, p = 640, 32
    A = rng.integers(-100, 101, (n, n)).astype(np.float64)
    X = rng.integers(-100, 101, (n, p)).astype(np.float64)
    Y = gpu_apply(S, A, X, SLICED)
    assert np.array_equal(Y, A @ X)


def test_sliced_product_propagates_non_finite(S):
    n, p = 300, 8
    A, X = wide_range(n, p, seed=9, span_a=2, span_x=2)
    A[3, 5] = np.nan
    X[7, 2] = np.inf
    Y = gpu_apply(S, A, X, SLICED)
    assert np.isnan(Y[3]).all()
    assert not np.isfinite(Y[:, 2]).any()
    mask = np.ones_like(Y, dtype=bool)
    mask[3] = False
    mask[:, 2] = False
    assert np.isfinite(Y[mask]).all()
