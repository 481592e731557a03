"""The allocation-free dense product pf_apply_dense_noalloc against the
context-based pf_apply on the same inputs.

pf_apply_dense_noalloc serves callers that cannot allocate device memory
(no pf_ctx to own a workspace, a memory manager that owns all device memory,
or a path that must not pay for cudaMalloc): its split-K partial sums live in
a fixed array inside the library.  It must give the same product as the
workspace path, within the FP64 tolerance of the parity tests, on two calls
in a row (the second call finds the first call's leftovers in the shared
array).  This file sorts last so that a stop-at-first-failure run has
already run every other test; it also passes alone in a fresh process."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _sym(n, seed):
    g = torch.Generator(device=DEV).manual_seed(seed)
    A = torch.randn(n, n, generator=g, dtype=torch.float64, device=DEV)
    return (A + A.T) / 2


# The array holds 2 Mi doubles.  For (8192, 32) and (16384, 64) the split
# count the workspace path would use does not fit (room for 8 and 2 splits of
# n x p partial sums), so these cases run the capped-split branch.
@pytest.mark.parametrize("n,p", [(300, 16), (4096, 32), (1000, 40), (2048, 64), (8192, 32),
                                 (16384, 64)])
def test_noalloc_product_matches_workspace_product_twice(n, p):
    import paper_1904_10585_gb300 as B
    from paper_1904_10585_gb300 import solver as S
    stream = torch.cuda.Stream()
    with S.Context(p=p, n_max=n, degree=1, stream=stream) as ctx:
        for call in range(2):
            A = _sym(n, 10 * n + p + call)
            X = torch.randn(n, p, dtype=torch.float64,
                            generator=torch.Generator().manual_seed(call)).to(DEV)
            Y_ref = torch.empty_like(X)
            Y = torch.full_like(X, float("nan"))
            with torch.cuda.stream(stream):
                S.apply(ctx, S.dense_operator(A), X, Y_ref)
                B.pf_apply_dense_noalloc(A.data_ptr(), A.stride(0), X.data_ptr(), X.stride(0),
                                         Y.data_ptr(), Y.stride(0), n, p, stream.cuda_stream)
            stream.synchronize()
            # independent FP64 reference: the plain host product A @ X
            Y_np = A.cpu().numpy() @ X.cpu().numpy()
            scale = float(np.abs(Y_np).max())
            err_np = float(np.abs(Y.cpu().numpy() - Y_np).max())
            assert np.isfinite(err_np) and err_np <= 1e-12 * scale, (call, err_np, scale)
            # and the library's own context product on the same inputs
            err = (Y - Y_ref).abs().max().item()
            assert np.isfinite(err) and err <= 1e-12 * scale, (call, err, scale)
            del A


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import paper_1904_10585_gb300 as B
    n, p = 40000, 64                     # n * p = 2,560,000 > 2 Mi doubles
    # host-side check: no device memory is touched for a rejected call
    st = B.raw_call("pf_apply_dense_noalloc", 16, n, 16, p, 32, p, n, p, None)
    assert st == B.PF_ERR_INVALID_ARG
