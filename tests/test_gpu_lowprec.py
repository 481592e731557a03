"""Low-precision (tcgen05) dense filter: the tensor-core product and the
bf16/tf32 filter against plain PyTorch references of the same operation.

* product: Y = s * (A_lp X_lp) with A_lp = A/s in bf16 (or fp32 read as tf32)
  and X_lp the block rounded the same way; reference = float64 matmul of the
  identically rounded bf16 inputs (exact products, so only the kernel's fp32
  accumulation order differs): |Y - ref| <= 1e-5 * max|ref|.  For tf32 the
  hardware's input rounding is not emulated; the bound is the tf32 unit
  roundoff: |Y - ref| <= 4e-3 * max|ref| against the unrounded fp64 product.
* filter: the bf16 filter step against an fp32 PyTorch emulation of the same
  recurrence (bf16 operands each step, fp32 recurrence, CholQR2 in fp64),
  elementwise 2e-3; and the subspace it spans against the FP64 oracle's,
  within the bf16 floor.
"""
import numpy as np
import pytest

import pf_synthetic as syn
from oracle import pf_oracle as o

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def S():
    import paper_1904_10585_gb300  # noqa: F401
    from paper_1904_10585_gb300 import solver
    return solver


def lp_operator(S, A_lp, scale):
    return S.dense_operator(None, A_lp=A_lp, lp_scale=scale)


def to_lp(M, dtype):
    """Copy M into a low-precision matrix whose row pitch is a multiple of 16
    bytes (the tensor-map rule), returned as an n x n view."""
    n = M.shape[0]
    align = 16 // torch.tensor([], dtype=dtype).element_size()
    ld = ((n + align - 1) // align) * align
    out = torch.zeros(n, ld, dtype=dtype, device=DEV)
    out[:, :n] = M.to(DEV).to(dtype)
    return out[:, :n]


def sym_matrix(n, seed):
    g = torch.Generator().manual_seed(seed)
    A = torch.randn(n, n, generator=g, dtype=torch.float64)
    return (A + A.T) / 2


@pytest.mark.parametrize("n,p", [(256, 64), (300, 16), (1000, 32), (513, 40), (129, 48), (2048, 64)])
def test_bf16_product_matches_fp32_reference(S, n, p):
    import paper_1904_10585_gb300 as B
    A = sym_matrix(n, n + p)
    s = float(A.abs().max())
    A_lp = to_lp(A / s, torch.bfloat16)
    X = torch.randn(n, p, dtype=torch.float64, generator=torch.Generator().manual_seed(p)).to(DEV)
    Y = torch.empty(n, p, dtype=torch.float64, device=DEV)
    with S.Context(p=p, n_max=n, degree=1, precision=B.PF_PREC_BF16) as ctx:
        S.apply(ctx, lp_operator(S, A_lp, s), X, Y)
        torch.cuda.synchronize()
    ref = s * (A_lp.double() @ X.to(torch.float32).to(torch.bfloat16).double())
    err = (Y - ref).abs().max().item()
    assert err <= 1e-5 * ref.abs().max().item(), err


@pytest.mark.parametrize("n,p", [(256, 32), (300, 64), (777, 16)])
def test_tf32_product_within_tf32_roundoff(S, n, p):
    import paper_1904_10585_gb300 as B
    A = sym_matrix(n, 3 * n)
    s = float(A.abs().max())
    A_lp = to_lp(A / s, torch.float32)
    X = torch.randn(n, p, dtype=torch.float64, generator=torch.Generator().manual_seed(1)).to(DEV)
    Y = torch.empty(n, p, dtype=torch.float64, device=DEV)
    with S.Context(p=p, n_max=n, degree=1, precision=B.PF_PREC_TF32) as ctx:
        S.apply(ctx, lp_operator(S, A_lp, s), X, Y)
        torch.cuda.synchronize()
    ref = A.to(DEV) @ X
    err = (Y - ref).abs().max().item()
    assert err <= 4e-3 * ref.abs().max().item(), err


def emulate_bf16_filter(A_lp, s, U, a, b, d):
    """Plain PyTorch reference of the bf16 filter step: fp32 recurrence with
    the block rounded to bf16 before every product, then QR with a positive
    diagonal in fp64."""
    c, e = (a + b) / 2, (b - a) / 2
    Af = A_lp.float()
    Y0 = U.float()
    Y1 = (s * (Af @ Y0.to(torch.bfloat16).float()) - c * Y0) / e
    prev, cur = Y0, Y1
    for _ in range(1, d):
        nxt = 2 * (s * (Af @ cur.to(torch.bfloat16).float()) - c * cur) / e - prev
        prev, cur = cur, nxt
    Q, R = torch.linalg.qr(cur.double())
    return Q * torch.sign(torch.diagonal(R))


@pytest.mark.parametrize("n,p,d", [(512, 32, 4), (700, 64, 3), (300, 16, 6)])
def test_bf16_filter_matches_emulation_and_oracle_subspace(S, n, p, d):
    import paper_1904_10585_gb300 as B
    lam = np.concatenate([np.linspace(6.0, 4.0, p), np.linspace(1.0, -3.0, n - p)])
    Bm, Qm = syn.dense_symmetric_with_spectrum(n, lam, seed=n)
    U0 = syn.gaussian_block(n, p, seed=p)
    a, b = -3.2, 1.4
    s = float(np.abs(Bm).max())
    A_lp = to_lp(torch.from_numpy(Bm / s), torch.bfloat16)
    U = torch.from_numpy(U0).to(DEV)
    with S.Context(p=p, n_max=n, degree=d, precision=B.PF_PREC_BF16) as ctx:
        S.filter_(ctx, lp_operator(S, A_lp, s), a, b, d, U)
        info = B.pf_get_info(ctx.handle)
        torch.cuda.synchronize()
    assert not (info.flags & 8), "device wait timed out"
    ref = emulate_bf16_filter(A_lp, s, torch.from_numpy(U0).to(DEV), a, b, d)
    assert (U - ref).abs().max().item() <= 2e-3
    exact = o.orth(o.cheb_filter(lambda X: Bm @ X, U0, a, b, d))
    Ug = U.cpu().numpy()
    assert o.subspace_sine(exact, Ug) <= 0.05
    # the filter helps: the block captures far more of the top-p eigenspace
    # than the random start block (||Q_p^T U||_F^2 is about p^2/n for it)
    before = np.linalg.norm(Qm[:, :p].T @ o.orth(U0))
    after = np.linalg.norm(Qm[:, :p].T @ Ug)
    assert after > 2.0 * before, (after, before)


def test_lowprec_operator_validation(S):
    import paper_1904_10585_gb300 as B
    n, p = 64, 16
    with S.Context(p=p, n_max=n, degree=2, precision=B.PF_PREC_BF16) as ctx:
        A_lp = to_lp(torch.zeros(n, n), torch.bfloat16)
        U = torch.randn(n, p, dtype=torch.float64, device=DEV)
        bad = lp_operator(S, A_lp, 0.0)          # scale must be positive
        with pytest.raises(B.PFError):
            S.filter_(ctx, bad, -1.0, 0.0, 2, U)
        odd = torch.zeros(n, n + 1, dtype=torch.bfloat16, device=DEV)[:, :n]
        with pytest.raises(B.PFError):           # row pitch not a multiple of 16 bytes
            S.filter_(ctx, lp_operator(S, odd, 1.0), -1.0, 0.0, 2, U)


@pytest.mark.parametrize("n,p,r,d", [(400, 16, 5, 3), (333, 40, 12, 4), (1000, 64, 20, 2)])
def test_fp32_lowrank_sparse_filter_tracks_fp64(S, n, p, r, d):
    """A bf16 context filters a low-rank + sparse operator with fp32 products
    (CUDA cores) and FP64 CholQR2: the block agrees with the FP64 oracle's
    filter to fp32 accuracy (elementwise 2e-5 relative to the block's scale)."""
    import paper_1904_10585_gb300 as B
    inst = syn.completion_instance(n, 4, 0.2, p, seed=n + r)
    Om = o.omega_matrix(inst.omega)
    Uf = o.orth(syn.gaussian_block(n, max(r, 1), seed=9))[:, :r]
    lam_f = np.linspace(3.0, 0.5, r)
    sscale, shift = -0.7, -0.05

    def apply_B(X):
        return Uf @ (lam_f[:, None] * (Uf.T @ X)) + sscale * (Om @ X) + shift * X

    U0 = syn.gaussian_block(n, p, seed=11)
    a, _ = o.gershgorin_bounds(sscale * Om, np.full(n, shift))
    b = 0.1 * a
    ref = o.orth(o.cheb_filter(apply_B, U0, a, b, d))
    rp, ci, vals = S.csr_to_device(inst.omega, DEV, torch.float64)
    with S.Context(p=p, n_max=n, degree=d, precision=B.PF_PREC_BF16) as ctx:
        op = S.lowrank_sparse_operator(n, torch.from_numpy(Uf).to(DEV),
                                       torch.from_numpy(lam_f).to(DEV), rp, ci, vals, sscale, shift)
        U = torch.from_numpy(U0).to(DEV)
        S.filter_(ctx, op, a, b, d, U)
        torch.cuda.synchronize()
    err = np.abs(U.cpu().numpy() - ref).max()
    assert err <= 2e-5 * np.abs(ref).max(), err
