"""PyTorch-facing helpers around the C ABI: they hold device tensors (memory
and streams are PyTorch's) and fill the pf_* structs with their pointers.
No arithmetic of the method happens here."""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
import torch

from . import _binding as B


def _ptr(t: Optional[torch.Tensor]) -> int:
    if t is None:
        return 0
    if not t.is_cuda:
        raise ValueError("libpf takes device tensors; got a host tensor")
    if not t.is_contiguous() and t.dim() == 1:
        raise ValueError("vectors must be contiguous")
    return t.data_ptr()


def _ld(t: torch.Tensor) -> int:
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("blocks must be row-major 2-D tensors with unit column stride")
    return t.stride(0)


class Context:
    """Owns one pf_ctx (workspace only) bound to a CUDA stream."""

    def __init__(self, p: int, n_max: int, degree: int, eta: float = 0.1,
                 precision: int = B.PF_PREC_FP64, stream: Optional[torch.cuda.Stream] = None,
                 degree_max: int = 0, adaptive: int = 0, p_min: int = 0, adapt_guard: int = 0,
                 adapt_every: int = 10, dense_product: int = B.PF_DENSE_SLICED):
        """p is the (maximum) block width; adapt_guard > 0 turns on the block
        width rule of Sec. 4.2 (width r_+ + adapt_guard, rounded up to a
        multiple of 8, in [p_min, p], after every adapt_every-th step).
        dense_product selects the arithmetic of FP64 dense products: bf16
        digit planes on the tensor cores (PF_DENSE_SLICED, FP64-accurate) or
        FP64 FMAs on the CUDA cores (PF_DENSE_FP64)."""
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.opt = B.pf_options(p=p, degree=degree, degree_max=degree_max or degree, q=1,
                                eta=eta, precision=precision, adaptive=adaptive,
                                p_min=p_min or min(8, p), adapt_guard=adapt_guard,
                                adapt_every=adapt_every, dense_product=dense_product)
        self.p = p
        self.n_max = n_max
        self.handle = B.pf_create(self.opt, n_max, self.stream.cuda_stream)

    def close(self):
        if self.handle:
            B.pf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _keep(op, *tensors):
    """Hold references to the tensors whose device pointers a struct carries,
    so the caching allocator cannot recycle them while the struct is in use."""
    op._keep = [t for t in tensors if t is not None]
    return op


def dense_operator(A: torch.Tensor, A_lp: Optional[torch.Tensor] = None,
                   lp_scale: float = 0.0) -> B.pf_operator:
    assert A is None or (A.dtype == torch.float64 and A.shape[0] == A.shape[1])
    n = A.shape[0] if A is not None else A_lp.shape[0]
    op = B.pf_operator(kind=B.PF_OP_DENSE, n=n, A=_ptr(A), lda=_ld(A) if A is not None else n)
    if A_lp is not None:
        op.A_lp = _ptr(A_lp)
        op.lda_lp = _ld(A_lp)
        op.lp_scale = lp_scale
    return _keep(op, A, A_lp)


def lowrank_sparse_operator(n: int, Uf: Optional[torch.Tensor], lam: Optional[torch.Tensor],
                            rowptr: Optional[torch.Tensor], colind: Optional[torch.Tensor],
                            vals: Optional[torch.Tensor], sparse_scale: float, shift: float
                            ) -> B.pf_operator:
    r = 0 if Uf is None else Uf.shape[1]
    op = B.pf_operator(kind=B.PF_OP_LOWRANK_SPARSE, n=n,
                       Uf=_ptr(Uf), lduf=(_ld(Uf) if Uf is not None else 0), lam=_ptr(lam), r=r,
                       rowptr=_ptr(rowptr), colind=_ptr(colind), vals=_ptr(vals),
                       nnz=0 if vals is None else vals.numel(),
                       sparse_scale=sparse_scale, shift=shift)
    return _keep(op, Uf, lam, rowptr, colind, vals)


def filter_(ctx: Context, op: B.pf_operator, a: float, b: float, degree: int,
            U: torch.Tensor) -> None:
    B.pf_filter(ctx.handle, op, a, b, degree, _ptr(U), _ld(U))


def apply(ctx: Context, op: B.pf_operator, X: torch.Tensor, Y: torch.Tensor) -> None:
    B.pf_apply(ctx.handle, op, _ptr(X), _ld(X), _ptr(Y), _ld(Y))


def rayleigh_ritz(ctx: Context, op: B.pf_operator, Q: torch.Tensor):
    n, p = Q.shape
    V = torch.empty_like(Q)
    theta = torch.empty(p, dtype=torch.float64, device=Q.device)
    resid = torch.empty(p, dtype=torch.float64, device=Q.device)
    B.pf_rayleigh_ritz(ctx.handle, op, _ptr(Q), _ld(Q), _ptr(V), _ld(V), _ptr(theta), _ptr(resid))
    return V, theta, resid


@dataclasses.dataclass
class Problem:
    """Device-resident data and state of one solve (caller-owned buffers)."""

    kind: int
    n: int
    rowptr: torch.Tensor
    colind: torch.Tensor
    vals: torch.Tensor
    U: torch.Tensor
    V: torch.Tensor
    theta: torch.Tensor
    Z: Optional[torch.Tensor] = None
    Z_lp: Optional[torch.Tensor] = None
    lam: Optional[torch.Tensor] = None
    S: Optional[torch.Tensor] = None
    t: float = 0.0
    mu: float = 0.0
    hist: Optional[torch.Tensor] = None
    accel_l: int = 0
    accel_lam: float = 0.0
    t_pattern: Optional[tuple] = None      # SVT, NNLS: transposed pattern (rowptr, colind, perm)
    fac: Optional[torch.Tensor] = None     # NNLS: [L | Lp | R | Rp], n x 4p
    fsv: Optional[torch.Tensor] = None     # NNLS: [s | sp]
    rank_cap: int = 0
    guard: Optional[torch.Tensor] = None   # n x p random columns for width growth
    Z_tf32: Optional[torch.Tensor] = None  # max-cut, bf16 context: fp32 shadow of the tf32 rung
    mirror: Optional[torch.Tensor] = None  # completion, symmetric pattern: entry -> transposed entry
    p_active: int = 0                      # start width (0: the context's p)
    struct: Optional[B.pf_problem] = None

    def make_struct(self) -> B.pf_problem:
        s = B.pf_problem(kind=self.kind, n=self.n, rowptr=_ptr(self.rowptr),
                         colind=_ptr(self.colind),
                         nnz=self.colind.numel() if self.colind is not None else 0,
                         t=self.t, mu=self.mu,
                         U=_ptr(self.U), ldu=_ld(self.U), V=_ptr(self.V), ldv=_ld(self.V),
                         theta=_ptr(self.theta), p_active=self.p_active)
        if self.guard is not None:
            s.guard = _ptr(self.guard)
            s.ldg = _ld(self.guard)
        if self.kind == B.PF_PROBLEM_NCE:
            s.Z = _ptr(self.Z)
            s.ldz = _ld(self.Z)
            s.lam = _ptr(self.lam)
            if self.hist is not None:
                s.hist = _ptr(self.hist)
                s.accel_l = self.accel_l
                s.accel_lam = self.accel_lam
            self.struct = s
            return s
        if self.kind in (B.PF_PROBLEM_SVT, B.PF_PROBLEM_NNLS):
            s.vals_f64 = _ptr(self.vals)
            s.S = _ptr(self.S)
            tr, tc, tp = self.t_pattern
            s.t_rowptr, s.t_colind, s.t_perm = _ptr(tr), _ptr(tc), _ptr(tp)
            if self.kind == B.PF_PROBLEM_NNLS:
                s.fac, s.ldfac, s.fsv = _ptr(self.fac), _ld(self.fac), _ptr(self.fsv)
                s.rank_cap = self.rank_cap
            self.struct = s
            return s
        if self.kind == B.PF_PROBLEM_MAXCUT:
            s.vals_f64 = _ptr(self.vals)
            if self.Z is not None:
                s.Z = _ptr(self.Z)
                s.ldz = _ld(self.Z)
            if self.Z_lp is not None:
                s.Z_lp = _ptr(self.Z_lp)
                s.ldz_lp = _ld(self.Z_lp)
            if self.Z_tf32 is not None:
                s.Z_tf32 = _ptr(self.Z_tf32)
                s.ldz_tf32 = _ld(self.Z_tf32)
            s.lam = _ptr(self.lam)
            if self.S is not None:
                s.S = _ptr(self.S)
        else:
            s.vals_f32 = _ptr(self.vals)
            s.S = _ptr(self.S)
            if self.mirror is not None:
                s.t_perm = _ptr(self.mirror)
        self.struct = s
        return s


def with_width_rule(pr: Problem, guard: torch.Tensor, p_start: int) -> Problem:
    """Attach guard columns (n x p device block, the context's p) and the
    start width for the block width rule; the problem's U must be n x p with
    the start block in its first p_start columns."""
    pr.guard = guard
    pr.p_active = p_start
    pr.make_struct()
    return pr


def maxcut_problem(rowptr, colind, vals, U0: torch.Tensor, t: float = 0.0, dense: bool = True,
                   lowprec: Optional[str] = None, tf32_rung: bool = False) -> Problem:
    """Max-cut SDP with cost C (CSR, float64 values incl. every diagonal
    entry); U0 is the n x p start block (copied).

    dense=True keeps the FP64 iteration matrix Z (n x n); dense=False applies
    Z = X~ - tC - Diag(lam) in structured form.  lowprec="bf16"/"tf32" adds the
    dense low-precision shadow the tensor-core filter reads (use with a
    context of the same precision); tf32_rung with lowprec="bf16" adds the
    fp32 shadow that the adaptive ladder's tf32 rung reads."""
    n, p = U0.shape
    dev = U0.device
    Z_lp = None
    Z_tf32 = None
    if lowprec is not None:
        dt = torch.bfloat16 if lowprec == "bf16" else torch.float32
        align = 8 if lowprec == "bf16" else 4
        ld = ((n + align - 1) // align) * align
        Z_lp = torch.empty(n, ld, dtype=dt, device=dev)[:, :n]
        if tf32_rung and lowprec == "bf16":
            ld4 = ((n + 3) // 4) * 4
            Z_tf32 = torch.empty(n, ld4, dtype=torch.float32, device=dev)[:, :n]
    pr = Problem(kind=B.PF_PROBLEM_MAXCUT, n=n, rowptr=rowptr, colind=colind, vals=vals,
                 U=U0.clone(), V=torch.zeros(n, p, dtype=torch.float64, device=dev),
                 theta=torch.zeros(p, dtype=torch.float64, device=dev),
                 Z=torch.empty(n, n, dtype=torch.float64, device=dev) if dense else None,
                 Z_lp=Z_lp,
                 lam=torch.empty(n, dtype=torch.float64, device=dev),
                 S=(torch.empty(colind.numel(), dtype=torch.float64, device=dev)
                    if (not dense or lowprec is not None) else None), t=t, Z_tf32=Z_tf32)
    pr.make_struct()
    return pr


def nce_problem(G: torch.Tensor, U0: torch.Tensor, tau: float = 1.0, accel_l: int = 0,
                accel_lam: float = 1e-10) -> Problem:
    """Nearest correlation estimation for the symmetric G (copied: the copy
    becomes the iteration matrix G + Diag(x)); lam holds the dual x.
    accel_l > 0 turns on the extrapolation of Sec. 4.3 over windows of
    accel_l + 2 iterates (regulariser accel_lam * tr(D^T D))."""
    n, p = U0.shape
    dev = U0.device
    pr = Problem(kind=B.PF_PROBLEM_NCE, n=n, rowptr=None, colind=None, vals=None,
                 U=U0.clone(), V=torch.zeros(n, p, dtype=torch.float64, device=dev),
                 theta=torch.zeros(p, dtype=torch.float64, device=dev),
                 Z=G.clone().contiguous(), lam=torch.empty(n, dtype=torch.float64, device=dev),
                 t=tau, accel_l=accel_l, accel_lam=accel_lam,
                 hist=(torch.zeros(accel_l + 2, n, dtype=torch.float64, device=dev)
                       if accel_l > 0 else None))
    pr.make_struct()
    return pr


def svt_problem(rowptr, colind, mvals_f64, t_rowptr, t_colind, t_perm, U0: torch.Tensor,
                mu: float, tau: float) -> Problem:
    """Nuclear-norm matrix completion by PFSVT: M on Omega (row-major CSR,
    float64 values) with the transposed pattern; S holds the dual x."""
    n, p = U0.shape
    dev = U0.device
    pr = Problem(kind=B.PF_PROBLEM_SVT, n=n, rowptr=rowptr, colind=colind, vals=mvals_f64,
                 U=U0.clone(), V=torch.zeros(n, p, dtype=torch.float64, device=dev),
                 theta=torch.zeros(p, dtype=torch.float64, device=dev),
                 S=torch.empty(colind.numel(), dtype=torch.float64, device=dev), t=tau, mu=mu)
    pr.t_pattern = (t_rowptr, t_colind, t_perm)
    pr.make_struct()
    return pr


def nnls_problem(rowptr, colind, mvals_f64, t_rowptr, t_colind, t_perm, U0: torch.Tensor,
                 mu_bar_rel: float = 1e-2, mu0: float = 0.0, rank_cap: int = 0) -> Problem:
    """Nuclear-norm regularised least squares by PFNNLS (accelerated proximal
    gradient with continuation to mu_bar = mu_bar_rel mu_0)."""
    n, p = U0.shape
    dev = U0.device
    pr = Problem(kind=B.PF_PROBLEM_NNLS, n=n, rowptr=rowptr, colind=colind, vals=mvals_f64,
                 U=U0.clone(), V=torch.zeros(n, p, dtype=torch.float64, device=dev),
                 theta=torch.zeros(p, dtype=torch.float64, device=dev),
                 S=torch.empty(colind.numel(), dtype=torch.float64, device=dev), t=mu0,
                 mu=mu_bar_rel)
    pr.t_pattern = (t_rowptr, t_colind, t_perm)
    pr.fac = torch.zeros(n, 4 * p, dtype=torch.float64, device=dev)
    pr.fsv = torch.zeros(2 * p, dtype=torch.float64, device=dev)
    pr.rank_cap = rank_cap
    pr.make_struct()
    return pr


def completion_problem(rowptr, colind, mvals_f32, U0: torch.Tensor, mu: float, t: float = 1.0,
                       mirror: Optional[torch.Tensor] = None) -> Problem:
    """mirror (optional, int32 device tensor of nnz): for a symmetric sampling
    pattern, the index of each entry's transposed entry (mirror_map); the
    library then forms the sampled residual on the upper triangle only."""
    n, p = U0.shape
    dev = U0.device
    pr = Problem(kind=B.PF_PROBLEM_COMPLETION, n=n, rowptr=rowptr, colind=colind, vals=mvals_f32,
                 U=U0.clone(), V=torch.zeros(n, p, dtype=torch.float64, device=dev),
                 theta=torch.zeros(p, dtype=torch.float64, device=dev),
                 S=torch.empty(colind.numel(), dtype=torch.float64, device=dev), t=t, mu=mu,
                 mirror=mirror)
    pr.make_struct()
    return pr


def mirror_map(rowptr: np.ndarray, colind: np.ndarray) -> np.ndarray:
    """The transposed-entry map of a symmetric CSR pattern (host arrays):
    entry e = (i, j) -> the index of (j, i).  Entries in (column, row) order
    are the transposed CSR, which for a symmetric pattern has the same
    positions, so the k-th of them is the mirror of entry k."""
    n = len(rowptr) - 1
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    order = np.argsort(colind.astype(np.int64) * n + rows, kind="stable")
    return order.astype(np.int32)


def problem_init(ctx: Context, pr: Problem) -> None:
    B.pf_problem_init(ctx.handle, pr.struct)
    pr.t = pr.struct.t


def prox_step(ctx: Context, pr: Problem, want_info: bool = True):
    return B.pf_prox_step(ctx.handle, pr.struct, want_info)


def solve(ctx: Context, pr: Problem, max_iter: int, tol: float = 0.0, check_every: int = 10):
    return B.pf_solve(ctx.handle, pr.struct, max_iter, tol, check_every)


def csr_to_device(csr, device, vals_dtype=None):
    """Copy a pf_synthetic.CSR to the device (int32 indices)."""
    rp = torch.from_numpy(csr.rowptr).to(device=device, dtype=torch.int32)
    ci = torch.from_numpy(csr.colind).to(device=device, dtype=torch.int32)
    v = torch.from_numpy(csr.vals)
    if vals_dtype is not None:
        v = v.to(vals_dtype)
    return rp, ci, v.to(device)
