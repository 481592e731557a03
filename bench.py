"""Benchmark of the polynomial-filtered subspace extraction on GB300.

One step = one whole solve of the workload through the hot path (interval,
Chebyshev filter, CholQR2, Rayleigh-Ritz, prox/DRS update, KKT report) from a
fresh initial state, run until the relative KKT residual is <= 1e-4 (checked
every 10 iterations; a cap of ``max_iters`` iterations bounds it).  Default
workload ``completion_n50000``, the largest configuration of the metric on
one GPU: PSD matrix completion by PFPG, n = 50000, rank-20 ground truth, 1%
symmetric uniform sampling (about 25M entries), p = 40, degree 4, the
iteration matrix applied as low-rank + sparse.  ``--workload maxcut_n4096``
is the max-cut SDP of an Erdos-Renyi graph (n = 4096, edge probability
0.01, weights +-1) solved by PFAM with a dense FP64 iteration matrix, p = 32,
degree 4.

Metric: solves/s at KKT 1e-4 (whole job), with p50/p99 solve latency; the
filter's product is reported against its roofline (the metric's "filter
GB/s vs roofline", on the method's bytes), and the device time of every
phase of the step is measured with CUDA events over one traced solve.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs as replicas (torchrun, one process per GPU, no data-path
collective): every rank solves its own copy of the workload, value = all
solves / max-over-ranks time.  ``--impl reference`` times the CPU oracle on
this host's cores (a bounded sample of each solve).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import pf_synthetic as syn  # noqa: E402

WORKLOAD = "completion_n50000"
TOL = 1e-4
CHECK_EVERY = 10
FP64_PEAK_TFLOPS = 1.25        # GB300 FP64 nominal (no measured FP64 peak is provided)
FP64_CUBLAS_MEASURED = 1.09    # torch float64 matmul 16384x16384x64 on this pool (context)
HBM_PEAK_GBS = 6773.2          # measured STREAM-style copy on the GB300s
# DRAM bytes (read + written) per launch of the roofline kernel, from an ncu
# capture of the current kernel (None where no capture of it exists), keyed
# by workload and dense-product mode: k_oz_product<32> at n = 4096, p = 32
# read 120.02 MB and wrote 3.57 MB (7.4 bytes an entry of the iteration
# matrix); k_lrsp_apply<5> at n = 50000 (25.0M entries, p = 40) read
# 364.6 MB and wrote 16.0 MB (the FP64 residual values and int32 indices,
# 12 bytes an entry, and the blocks)
NCU_TRAFFIC_BYTES = {
    ("maxcut_n4096", "sliced"): 123.58e6,
    ("completion_n50000", "sliced"): 380.6e6,
}
# Iterations the default workload's solve takes to reach KKT 1e-4 on the GPU;
# the oracle follows the same trajectory (parity of every iteration), so the
# reference arm scales its sampled iterations to this count.
ITERS_TO_TOL = {"maxcut_n4096": 2740, "completion_n50000": 750}
SLICED_NOTE = ("7 int8 digit planes of Z (bytes in HBM, widened to fp16 in shared memory) and 7 "
               "fp16 planes of X on tcgen05 (TMA, TMEM), level sums exact in fp32, "
               "int64 fold, FP64 recurrence epilogue: an FP64-accurate product")

CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    """nvidia-smi sampling during the timed region (200 ms period)."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={CLOCK_FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle, bounded samples
# ---------------------------------------------------------------------------

def max_over_ranks(values, pg, device=None):
    """Element-wise max of per-rank timings over the process group (the whole
    job is as slow as its slowest replica); identity on a single process."""
    import torch
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    if pg is not None:
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return [float(x) for x in t]


def cpu_model() -> str:
    """Model name of the host CPU (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class WorkloadSpec:
    """Host-side description of one configuration (no GPU needed): the seeded
    inputs, the oracle sample used by the CPU baseline and the config dict."""

    def __init__(self, name):
        self.name = name
        self.cfg, self.inst = syn.make_workload(name)
        c = self.cfg
        self.n, self.p, self.d, self.iters = c["n"], c["p"], c["degree"], c["iters"]
        # solves run to the tolerance, capped at max_iters (the configured
        # iteration count where no cap is given)
        self.max_iters = c.get("max_iters", c["iters"])
        self.kind = c["kind"]
        self.lowprec = "bf16" if name.endswith("lowprec") else None
        self.structured = name.endswith("structured")
        self.sliced = True   # dense FP64 products as int8 digit planes on the tensor cores

    def dense_f64(self):
        """The step applies a dense FP64 iteration matrix."""
        return self.kind == "nce" or (self.kind == "maxcut" and not self.lowprec
                                      and not self.structured)

    def nnz(self):
        if self.kind == "nce":
            return self.n * self.n
        if self.kind in ("svt", "nnls"):
            return self.inst.omega.nnz
        return self.inst.C.nnz if self.kind == "maxcut" else self.inst.omega.nnz

    def oracle_sample(self, iters_sample):
        """Seconds the oracle takes for the initial state + iters_sample iterations."""
        import scipy.sparse as sp
        from oracle import pf_oracle as o
        t0 = time.perf_counter()
        if self.kind == "nce":
            o.nce_solve(self.inst.G, self.inst.U0_raw[:, :self.p], self.d, iters_sample,
                        accel_l=self.cfg.get("accel_l", 0))
        elif self.kind == "svt":
            o.svt_solve(self.inst.omega, self.inst.U0_raw[:, :self.p], *self.svt_params(),
                        self.d, iters_sample)
        elif self.kind == "nnls":
            o.nnls_solve(self.inst.omega, self.inst.U0_raw[:, :self.p], self.d, iters_sample,
                         mu_bar_rel=self.cfg["mu_bar_rel"], cap=self.p - 8)
        elif self.kind == "maxcut":
            inst = self.inst
            C = sp.csr_matrix((inst.C.vals, inst.C.colind, inst.C.rowptr), shape=(inst.n, inst.n))
            t = o.maxcut_step_size(C)
            st = o.maxcut_init(C, inst.U0_raw[:, :self.p], t)
            for _ in range(iters_sample):
                st, _ = o.maxcut_pfam_step(C, st, t, self.d)
        else:
            Om = o.omega_matrix(self.inst.omega)
            st = o.completion_init(self.n, self.inst.U0_raw[:, :self.p])
            for _ in range(iters_sample):
                st, _ = o.completion_pfpg_step(Om, st, self.cfg["mu"], self.cfg["t"], self.d)
        return time.perf_counter() - t0

    def svt_params(self):
        """(mu, tau) of the SVT reference: mu = 5 n, tau = 1.2 / SR."""
        return 5.0 * self.n, 1.2 / self.cfg["sr"]

    def tol(self):
        return 1e-7 if self.kind == "nce" else TOL

    def sample_iters(self):
        return min(self.iters, {"maxcut_n4096": 15, "maxcut_n4096_structured": 15,
                                "completion_n400": 100, "nce_n4000": 10,
                                "svt_n5000": 20, "nnls_n10000": 15,
                                "completion_n50000": 2}.get(self.name, 1))

    def config(self):
        c = self.cfg
        d = {"workload": self.name, "n": c["n"], "p": c["p"], "degree": c["degree"],
             "tol_kkt": self.tol(), "max_iters": self.max_iters,
             "configured_iters": c["iters"],
             "stopping": (f"each solve runs until its KKT residual is <= {self.tol():g} "
                          f"(checked every {CHECK_EVERY} iterations), at most "
                          f"{self.max_iters} iterations")}
        if self.kind == "nnls":
            d["problem"] = ("nuclear-norm regularised least squares, PFNNLS (Sec. 5.2.2): "
                            "accelerated proximal gradient, filter on G^T G, FP64")
            d["matrix"] = (f"Example MC: M = M_L M_R^T rank {c['rank']}, Bernoulli sampling "
                           f"SR {c['sr']}, continuation to mu_bar = {c['mu_bar_rel']} mu_0, "
                           f"rank cap p - 8")
            d["tol"] = "relative change ||X_k+1 - X_k|| / max(1, ||X_k+1||) 1e-4 at mu_bar"
            d["nnz"] = int(self.nnz())
            bytes_z = self.nnz() * 16
        elif self.kind == "svt":
            mu, tau = self.svt_params()
            d["problem"] = ("nuclear-norm matrix completion, PFSVT (Sec. 5.2.1): filter on Y^T Y "
                            "by two CSR SpMMs per product, FP64")
            d["matrix"] = (f"Example MC: M = M_L M_R^T rank {c['rank']}, Bernoulli sampling "
                           f"SR {c['sr']}, mu = 5n = {mu:g}, tau = 1.2/SR = {tau:g}")
            d["tol"] = "relative residual ||P_Omega(X - M)|| / ||P_Omega(M)|| 1e-4"
            d["nnz"] = int(self.nnz())
            bytes_z = self.nnz() * 16
        elif self.kind == "nce":
            d["problem"] = ("nearest correlation estimation, PFPG on the dual (dense FP64 "
                            "G + Diag(x))")
            d["matrix"] = f"Example {c['example']} law (off-diagonal uniform, unit diagonal)"
            d["tol"] = "relative gradient norm 1e-7 (the paper's stopping rule)"
            if c.get("accel_l"):
                d["extrapolation"] = (f"Sec. 4.3 over windows of {c['accel_l'] + 2} iterates, "
                                      "lambda 1e-10 tr(D^T D)")
            bytes_z = self.n * self.n * 8
            d["dense_product"] = SLICED_NOTE if self.sliced else "FP64 FMAs on the CUDA cores"
        elif self.kind == "maxcut":
            if self.structured:
                d["problem"] = ("max-cut SDP (PFAM, structured FP64 iteration matrix "
                                "Z = X~ - tC - Diag(lam), never formed)")
            elif self.lowprec:
                d["problem"] = ("max-cut SDP (PFAM, bf16 dense shadow filter on tcgen05, "
                                "structured FP64 Rayleigh-Ritz)")
            else:
                d["problem"] = "max-cut SDP (PFAM, dense FP64 iteration matrix)"
                d["dense_product"] = SLICED_NOTE if self.sliced else "FP64 FMAs on the CUDA cores"
            d["graph"] = f"Erdos-Renyi p={c['prob']}, weights +-1"
            bytes_z = (self.nnz() * 16 if self.structured
                       else self.n * self.n * (2 if self.lowprec else 8))
        else:
            d["problem"] = "PSD matrix completion (PFPG, low-rank + sparse FP64 operator)"
            d["sampling"] = f"symmetric uniform {c['rate']}, rank {c['rank']}, mu {c['mu']}"
            d["nnz"] = int(self.nnz())
            bytes_z = self.nnz() * 16
        d["l2"] = ("inputs larger than L2 (129 MB): iteration matrix %.0f MB" % (bytes_z / 1e6)
                   if bytes_z > 129e6 else
                   "working set fits L2 (%.1f MB); L2 not flushed between solves" % (bytes_z / 1e6))
        return d


def run_reference(args):
    world, rank, local = dist_setup()
    if rank != 0:
        return 0
    W = WorkloadSpec(args.workload)
    iters_sample = 2 if W.name == "maxcut_n4096" else max(1, W.sample_iters() // 10)
    iters_solve = ITERS_TO_TOL.get(W.name, W.iters)
    for _ in range(args.warmup):
        W.oracle_sample(iters_sample)
    times = [W.oracle_sample(iters_sample) for _ in range(args.steps)]
    per_solve = [tt * iters_solve / iters_sample for tt in times]
    value = len(per_solve) / sum(per_solve)
    sample = (f"initial state + {iters_sample} iterations per step, scaled to one "
              f"{iters_solve}-iteration solve (the iterations to KKT {W.tol():g})")
    line = {
        "impl": "reference", "metric": "solves/s", "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.mean(per_solve), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": W.config(),
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": host_cores(),
                         "cpu_model": cpu_model(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def sparse_bytes(nnz, n, p, r):
    """The method's bytes of one low-rank + sparse application (the CSR
    product of the completion / SVT / NNLS operators): each entry's column
    index and FP32-sized value (8 B), the row pointers, the n x r factor and
    the n x p block read in FP64, the n x p result written in FP64."""
    return 8.0 * nnz + 4.0 * (n + 1) + 8.0 * n * (r + p) + 8.0 * n * p


class Workload(WorkloadSpec):
    """Device side of a configuration: problem buffers and the dominant
    kernel's operator."""

    def __init__(self, name, dev, S, B):
        import torch
        super().__init__(name)
        self.dev, self.S, self.B = dev, S, B
        self.U0 = torch.from_numpy(np.ascontiguousarray(self.inst.U0_raw[:, :self.p])).to(dev)
        if self.kind == "nce":
            self.G = torch.from_numpy(self.inst.G).to(dev)
        elif self.kind in ("svt", "nnls"):
            self.rp, self.ci, self.cv = S.csr_to_device(self.inst.omega, dev, torch.float64)
            self.tr = torch.from_numpy(self.inst.t_rowptr).to(dev)
            self.tc = torch.from_numpy(self.inst.t_colind).to(dev)
            self.tp = torch.from_numpy(self.inst.t_perm).to(dev)
        elif self.kind == "maxcut":
            self.rp, self.ci, self.cv = S.csr_to_device(self.inst.C, dev, torch.float64)
        else:
            self.rp, self.ci, self.cv = S.csr_to_device(self.inst.omega, dev)
            # the sampling pattern is symmetric: the residual is formed on its
            # upper triangle and mirrored through this map
            self.mir = torch.from_numpy(S.mirror_map(self.inst.omega.rowptr,
                                                     self.inst.omega.colind)).to(dev)

    def inputs(self):
        """Device tensors holding this workload's inputs (copied from the host
        in the end-to-end measurement), start block last."""
        if self.kind == "nce":
            return [self.G, self.U0]
        if self.kind in ("svt", "nnls"):
            return [self.rp, self.ci, self.cv, self.tr, self.tc, self.tp, self.U0]
        if self.kind == "completion":
            return [self.rp, self.ci, self.cv, self.mir, self.U0]
        return [self.rp, self.ci, self.cv, self.U0]

    def problem_from(self, tensors):
        if self.kind == "nce":
            return self.S.nce_problem(tensors[0], tensors[1], accel_l=self.cfg.get("accel_l", 0))
        if self.kind == "svt":
            return self.S.svt_problem(*tensors, *self.svt_params())
        if self.kind == "nnls":
            return self.S.nnls_problem(*tensors, mu_bar_rel=self.cfg["mu_bar_rel"])
        if self.kind == "completion":
            return self.problem(tensors[0], tensors[1], tensors[2], tensors[4], mirror=tensors[3])
        return self.problem(*tensors)

    def precision(self):
        return self.B.PF_PREC_BF16 if self.lowprec == "bf16" else self.B.PF_PREC_FP64

    def problem(self, rp=None, ci=None, cv=None, U0=None, mirror=None):
        S = self.S
        if self.kind == "nce":
            return S.nce_problem(self.G, self.U0 if U0 is None else U0,
                                 accel_l=self.cfg.get("accel_l", 0))
        if self.kind == "svt":
            return S.svt_problem(self.rp, self.ci, self.cv, self.tr, self.tc, self.tp,
                                 self.U0 if U0 is None else U0, *self.svt_params())
        if self.kind == "nnls":
            return S.nnls_problem(self.rp, self.ci, self.cv, self.tr, self.tc, self.tp,
                                  self.U0 if U0 is None else U0,
                                  mu_bar_rel=self.cfg["mu_bar_rel"])
        rp = self.rp if rp is None else rp
        ci = self.ci if ci is None else ci
        cv = self.cv if cv is None else cv
        U0 = self.U0 if U0 is None else U0
        if self.kind == "maxcut":
            if self.lowprec or self.structured:
                return S.maxcut_problem(rp, ci, cv, U0, dense=False, lowprec=self.lowprec)
            return S.maxcut_problem(rp, ci, cv, U0)
        return S.completion_problem(rp, ci, cv, U0, mu=self.cfg["mu"], t=self.cfg["t"],
                                    mirror=self.mir if mirror is None else mirror)

    def kernel_op(self, pr):
        """(operator, description, bound, work per launch, unit) of the dominant kernel."""
        import torch
        S, B, n, p = self.S, self.B, self.n, self.p
        if self.kind == "nnls":
            # G X: CSR SpMM of the residual plus the rank-2p low-rank part
            # (the same kernel and work as the step's products)
            ones = torch.ones(2 * p, dtype=torch.float64, device=pr.fac.device)
            self._keep = ones
            op = S.lowrank_sparse_operator(n, pr.fac[:, :2 * p], ones, self.rp, self.ci, pr.S,
                                           -1.0, 0.0)
            nnz = self.ci.numel()
            return (op, "k_split_pairs4 + k_lrsp_apply (G X: CSR SpMM + rank-2p low-rank)", "hbm",
                    sparse_bytes(nnz, n, p, 2 * p), "GB/s")
        if self.kind == "svt":
            # Y X with Y = A*(x): the plain CSR product of the filter and the
            # Ritz step (the transposed product k_svt_spmm does the same work)
            op = S.lowrank_sparse_operator(n, None, None, self.rp, self.ci, pr.S, 1.0, 0.0)
            nnz = self.ci.numel()
            return (op, "k_split_pairs4 + k_lrsp_apply (Y X, CSR SpMM)", "hbm",
                    sparse_bytes(nnz, n, p, 0), "GB/s")
        if self.dense_f64() and self.sliced:
            # the method's bytes: the FP64 iteration matrix read once, X and
            # Y_prev read and Y_next written in FP64 (the digit planes the
            # kernel moves instead are its representation, reported beside)
            return (S.dense_operator(pr.Z),
                    "k_oz_product + k_oz_finish (Y = Z X from int8 digit planes x7 on tcgen05, "
                    "recurrence epilogue)", "hbm",
                    8.0 * n * n + 24.0 * n * p, "GB/s")
        if self.kind == "nce":
            return (S.dense_operator(pr.Z),
                    "k_gemm_f64_splitk + k_combine (Y = (G + Diag x) X, dense FP64 filter product)",
                    "alu", 2.0 * n * n * p, "TFLOP/s")
        if self.kind == "maxcut" and self.structured:
            # the structured product Z X = X~ X - tC X - lam o X (one SpMM + low-rank)
            th = pr.theta.clamp(min=0)
            Sv = torch.empty_like(pr.S)
            Sv.copy_(-pr.t * self.cv)
            self._keep = (th, Sv)
            op = S.lowrank_sparse_operator(n, pr.V, th, self.rp, self.ci, Sv, 1.0, 0.0)
            nnz = self.ci.numel()
            return (op, "k_split_pairs4 + k_lrsp_apply (structured Z X: CSR SpMM + low-rank)",
                    "hbm", sparse_bytes(nnz, n, p, p), "GB/s")
        if self.kind == "maxcut" and not self.lowprec:
            return (S.dense_operator(pr.Z),
                    "k_gemm_f64_splitk + k_combine (Y = Z X, dense FP64 filter product)",
                    "alu", 2.0 * n * n * p, "TFLOP/s")
        if self.kind == "maxcut":
            op = S.dense_operator(None, A_lp=pr.Z_lp, lp_scale=1.0)
            nbytes = 2.0 * n * n + n * p * (4 + 2)
            return (op, "k_tc_filter<64,bf16> (tcgen05 bf16 filter product, TMA + TMEM)", "hbm",
                    nbytes, "GB/s")
        # completion: Y = X_k X - t S X - t mu X with X_k = V diag(max(theta,0)) V^T
        th = pr.theta.clamp(min=0)
        self._keep = th
        op = S.lowrank_sparse_operator(n, pr.V, th, self.rp, self.ci, pr.S, -self.cfg["t"],
                                       -self.cfg["t"] * self.cfg["mu"])
        nnz = self.ci.numel()
        return (op, "k_split_pairs4 + k_lrsp_apply (fused CSR SpMM + low-rank, FP64-accurate "
                "Dot2 sums on the FP32 pipe)", "hbm", sparse_bytes(nnz, n, p, p), "GB/s")


def run_ours(args):
    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    import paper_1904_10585_gb300 as pkg
    from paper_1904_10585_gb300 import solver as S

    W = Workload(args.workload, dev, S, pkg)
    n, p, d, iters = W.n, W.p, W.d, W.iters
    stream = torch.cuda.Stream(device=dev)
    W.sliced = args.dense_product == "sliced"
    ctx = S.Context(p=p, n_max=n, degree=d, stream=stream, precision=W.precision(),
                    dense_product=pkg.PF_DENSE_SLICED if W.sliced else pkg.PF_DENSE_FP64)
    pr = W.problem()

    def solve_once(problem):
        problem.U.copy_(W.U0)           # fresh start block (on the library stream below)
        if W.kind == "nce":
            problem.Z.copy_(W.G)        # the iteration matrix starts from G again
        S.problem_init(ctx, problem)
        return S.solve(ctx, problem, W.max_iters, W.tol(), CHECK_EVERY)

    # launch counting (non-graph calls): init + one step
    with torch.cuda.stream(stream):
        c0 = pkg.pf_kernel_launch_count()
        pr.U.copy_(W.U0)
        if W.kind == "nce":
            pr.Z.copy_(W.G)
        S.problem_init(ctx, pr)
        c1 = pkg.pf_kernel_launch_count()
        S.prox_step(ctx, pr, want_info=False)
        c2 = pkg.pf_kernel_launch_count()
    init_launches, step_launches = c1 - c0, c2 - c1
    if args.profile:
        # short run for profiler captures: --profile-iters more non-graph
        # iterations (skip the first ones in the profiler to see steady state)
        with torch.cuda.stream(stream):
            for _ in range(args.profile_iters):
                S.prox_step(ctx, pr, want_info=False)
        stream.synchronize()
        print(json.dumps({"profile_run": args.workload, "launches_per_iteration": step_launches}))
        ctx.close()
        return 0

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            solve_once(pr)
    stream.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    results = []
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        for k in range(args.steps):
            results.append(solve_once(pr))
            ev[k + 1].record(stream)
    stream.synchronize()
    torch.cuda.synchronize(dev)
    if pg:
        pg.barrier()
    clocks = sampler.stop()
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[args.steps])
    iters_run = [int(r.iters) for r in results]
    gpu_launches = sum(init_launches + it * step_launches for it in iters_run)

    # device time per phase over one whole solve, stepped outside the graph
    # with the library's phase events (the same kernels the graph replays)
    phase_ms = {k: 0.0 for k in pkg.PHASE_NAMES}
    traced_iters = 0
    pkg.pf_set_tracing(ctx.handle, True)
    with torch.cuda.stream(stream):
        pr.U.copy_(W.U0)
        if W.kind == "nce":
            pr.Z.copy_(W.G)
        S.problem_init(ctx, pr)
        cap = min(W.max_iters, int(np.max(iters_run)))
        for k in range(cap):
            info = S.prox_step(ctx, pr, want_info=(k + 1) % CHECK_EVERY == 0)
            for name, v in pkg.pf_phase_times(ctx.handle).items():
                phase_ms[name] += v
            traced_iters += 1
            if info is not None and info.kkt <= W.tol():
                break
    pkg.pf_set_tracing(ctx.handle, False)
    phase_total = sum(phase_ms.values())
    phases = {"iterations": traced_iters,
              "ms_per_iteration": {k: v / max(1, traced_iters) for k, v in phase_ms.items()},
              "share": {k: (v / phase_total if phase_total > 0 else 0.0)
                        for k, v in phase_ms.items()},
              "how": "CUDA events at the phase boundaries of one solve stepped outside the "
                     "graph (pf_set_tracing / pf_phase_times)"}
    dominant_phase = max(phase_ms, key=phase_ms.get)

    # the filter's product, timed with CUDA events on the library stream over
    # R launches of the same operator on the state left by the solves above
    R = 20
    op, kname, bound, work, unit = W.kernel_op(pr)
    X = pr.U.clone()
    Y = torch.empty_like(X)

    def timed(fn, reps):
        with torch.cuda.stream(stream):
            for _ in range(3):
                fn()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1) / reps

    if W.lowprec or (W.sliced and W.dense_f64()):
        # the tensor-core product alone: a degree-5 filter minus a degree-1
        # filter on the same block is exactly four product launches (the
        # operand preparation and CholQR2 cancel)
        info = pkg.pf_get_info(ctx.handle)
        a_int, b_int = info.a, info.b
        Ub = pr.U.clone()

        def filt(deg):
            return lambda: (X.copy_(Ub), S.filter_(ctx, op, a_int, b_int, deg, X))
        apply_ms = (timed(filt(5), R) - timed(filt(1), R)) / 4.0
    else:
        apply_ms = timed(lambda: S.apply(ctx, op, X, Y), R)
    if unit == "TFLOP/s":
        achieved = work / (apply_ms * 1e-3) / 1e12
        peak, peak_src = FP64_PEAK_TFLOPS, ("recipe nominal FP64 1.25 TFLOP/s (no measured FP64 peak; "
                                            f"cuBLAS DGEMM reached {FP64_CUBLAS_MEASURED} on this pool)")
    else:
        achieved = work / (apply_ms * 1e-3) / 1e9
        peak, peak_src = HBM_PEAK_GBS, "measured HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"

    # end to end through the public API: host (pinned) inputs copied in and the
    # solution factors read back inside the timed region
    h_in = [t.cpu().pin_memory() for t in W.inputs()]
    d_in = [torch.empty_like(t) for t in W.inputs()]
    h_V = torch.empty((n, p), dtype=torch.float64).pin_memory()
    h_th = torch.empty((p,), dtype=torch.float64).pin_memory()
    pe = W.problem_from(d_in)
    h2d = sum(t.numel() * t.element_size() for t in h_in)
    d2h = h_V.numel() * 8 + h_th.numel() * 8
    e2e_steps = max(1, min(args.steps, 3))

    def e2e_once():
        for hd, dd in zip(h_in, d_in):
            dd.copy_(hd, non_blocking=True)
        pe.U.copy_(d_in[-1])
        if W.kind == "nce":
            pe.Z.copy_(d_in[0])
        S.problem_init(ctx, pe)
        S.solve(ctx, pe, W.max_iters, W.tol(), CHECK_EVERY)
        h_V.copy_(pe.V, non_blocking=True)
        h_th.copy_(pe.theta, non_blocking=True)
        stream.synchronize()

    with torch.cuda.stream(stream):
        e2e_once()                      # warm-up (captures this problem's graph)
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for _ in range(e2e_steps):
            e2e_once()
    e2e_s = time.perf_counter() - t0

    # max over ranks
    total_ms, e2e_s = max_over_ranks([total_ms, e2e_s], pg, dev)
    value = world * args.steps / (total_ms * 1e-3)
    e2e_value = world * e2e_steps / e2e_s

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle takes the same iterations as the GPU solve (parity), so
        # its per-iteration time is scaled to the iterations the solves ran
        iters_sample = W.sample_iters()
        secs = W.oracle_sample(iters_sample)
        it_solve = float(np.mean(iters_run))
        cpu = {"value": 1.0 / (secs * it_solve / iters_sample), "unit": "solves/s",
               "cores": host_cores(), "cpu_model": cpu_model(), "kind": "oracle",
               "sample": f"initial state + {iters_sample} iterations of the same workload "
                         f"({secs:.1f} s), scaled to one {it_solve:.0f}-iteration solve (the "
                         f"iterations the timed GPU solves ran)"}

    last = results[-1].last
    line = {
        "metric": "solves/s", "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": ("bf16+f64" if W.lowprec else
                  "f16x7->f64" if (W.sliced and W.dense_f64()) else "f64"),
        "data": "synthetic",
        "config": W.config(),
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                       "p99": float(np.percentile(step_ms, 99))},
        "solve": {"iters": iters_run[-1], "kkt": float(last.kkt), "obj": float(last.obj),
                  "pinf": float(last.pinf), "dinf": float(last.dinf), "gap": float(last.gap),
                  "r_plus": int(last.r_plus), "reached_tol": bool(last.kkt <= W.tol()),
                  "jacobi_sweeps_last": int(last.jacobi_sweeps)},
        "roofline": {"kernel": kname, "bound": bound, "achieved": achieved, "peak": peak,
                     "unit": unit, "frac": achieved / peak,
                     "traffic": NCU_TRAFFIC_BYTES.get((args.workload, args.dense_product)),
                     "work_per_launch": work, "avg_launch_ms": apply_ms, "peak_source": peak_src,
                     "note": ("the metric's filter product; work = the method's algorithmic "
                              "bytes (FP64 iteration matrix and blocks)")},
        "phases": phases,
        "dominant_phase": dominant_phase,
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps},
        "gpu_launches": gpu_launches,
        "launches_per_iteration": step_launches,
    }
    if W.sliced and W.dense_f64():
        # what the sliced product moves: 7 int8 digit planes of Z (7 bytes an
        # entry), the fp16 planes of X read and of the next block written, and
        # the FP64 blocks
        line["roofline"]["representation_bytes_per_launch"] = 7.0 * n * n + 52.0 * n * p
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if pg:
        pg.destroy_process_group()
    return 0


def run_serving(args):
    """Serving mix (continuous batching): saturation throughput with every
    request queued at t = 0, latency percentiles under Poisson arrivals at 0.8x
    that rate, and the plain baseline (the same requests one at a time through
    the FP64 path: dense FP64 Z for max-cut, FP64 operator for completion)."""
    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_1904_10585_gb300 as pkg
    from paper_1904_10585_gb300 import serving as SV
    from paper_1904_10585_gb300 import solver as S

    N = args.serving_requests
    p, degree = 32, 4
    mc_n, cp_n = (512, 4096), (2000, 16000)
    mix = syn.serving_mix(N, syn.config_seed(4) + rank, p=p, maxcut_n=mc_n, completion_n=cp_n,
                          rank=(5, 20), rate=(0.01, 0.10), maxcut_prob=0.01)
    reqs = []
    for i, m in enumerate(mix):
        inst = m["inst"]
        c = inst.C if m["kind"] == "maxcut" else inst.omega
        # every request runs to KKT 1e-4 (the caps only bound a runaway)
        reqs.append(SV.Request(i, m["kind"], m["n"], 0.0, c.rowptr, c.colind, c.vals,
                               inst.U0_raw, max_iter=8000 if m["kind"] == "maxcut" else 4000))
    SV.Server.prepare(reqs)
    slots = [("maxcut", mc_n[1], 8), ("completion", cp_n[1], 8)]
    budget = 16 << 30
    srv = SV.Server(slots, p=p, degree=degree, tol=TOL, chunk=10, hbm_budget=budget,
                    maxcut_lowprec=True, completion_lowprec=True, device=dev)
    # warm-up: two small requests of each kind
    warm = sorted(reqs, key=lambda r: r.n)[:4]
    srv.run([dataclasses_replace(r, arrival=0.0, max_iter=20) for r in warm])
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local)
    sampler.start()
    t0 = time.perf_counter()
    res_sat = srv.run([dataclasses_replace(r, arrival=0.0) for r in reqs])
    makespan = time.perf_counter() - t0
    clocks = sampler.stop()
    sat_rate = N / makespan
    arrivals = syn.poisson_arrivals(N, 0.8 * sat_rate, syn.config_seed(4) + 100 + rank)
    res_p = srv.run([dataclasses_replace(r, arrival=float(a)) for r, a in zip(reqs, arrivals)])
    p50, p99 = SV.latency_percentiles(res_p)
    sp50, sp99 = SV.latency_percentiles(res_sat)
    srv.close()

    # plain baselines: one request at a time, FP64 path -- with FP64 FMAs
    # (the plain method) and with the FP64-accurate sliced tensor-core products
    def one_at_a_time(dense_product):
        stream = torch.cuda.Stream(device=dev)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ctxs = {}
        for r in reqs:
            key = r.kind
            if key not in ctxs:
                ctxs[key] = S.Context(p=p, n_max=(mc_n[1] if key == "maxcut" else cp_n[1]),
                                      degree=degree, stream=stream,
                                      dense_product=dense_product)
            ctx = ctxs[key]
            with torch.cuda.stream(stream):
                rp = r.pinned["rowptr"].to(dev, non_blocking=True)
                ci = r.pinned["colind"].to(dev, non_blocking=True)
                vv = r.pinned["vals"].to(dev, non_blocking=True)
                U0 = r.pinned["U0"].to(dev, non_blocking=True)
                if r.kind == "maxcut":
                    pr = S.maxcut_problem(rp, ci, vv, U0)
                else:
                    pr = S.completion_problem(rp, ci, vv, U0, mu=r.mu, t=r.t)
                S.problem_init(ctx, pr)
                S.solve(ctx, pr, r.max_iter, TOL, 10)
                pr.V.to("cpu")
        stream.synchronize()
        secs = time.perf_counter() - t0
        for c in ctxs.values():
            c.close()
        return secs

    plain_s = one_at_a_time(pkg.PF_DENSE_FP64)
    sliced_s = one_at_a_time(pkg.PF_DENSE_SLICED)
    plain_rate = N / plain_s
    kkts = np.array([r.kkt for r in res_sat])
    line = {
        "metric": "solves/s", "value": sat_rate, "unit": "solves/s", "n_gpus": world,
        "steps": 1, "warmup": 1, "ms_per_step": makespan * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f64", "data": "synthetic",
        "config": {"workload": "serving_mix", "requests": N, "maxcut_n": mc_n,
                   "completion_n": cp_n, "rank": [5, 20], "sampling": [0.01, 0.10], "p": p,
                   "degree": degree, "slots": slots, "hbm_budget_bytes": budget,
                   "maxcut_filter": "bf16 dense shadow on tcgen05 + FP64 structured RR",
                   "completion_filter": "fp32 low-rank + sparse products + FP64 RR",
                   "l2": "requests' matrices mostly exceed L2; not flushed between requests"},
        "latency_s": {"poisson_0.8x_p50": p50, "poisson_0.8x_p99": p99,
                      "saturation_p50": sp50, "saturation_p99": sp99},
        "plain_one_at_a_time_fp64": {"value": plain_rate, "seconds": plain_s,
                                     "dense_product": "FP64 FMAs on the CUDA cores",
                                     "speedup_of_serving": sat_rate / plain_rate},
        "one_at_a_time_fp64_sliced": {"value": N / sliced_s, "seconds": sliced_s,
                                      "dense_product": "FP64-accurate int8 digit planes on "
                                                       "tcgen05",
                                      "speedup_of_serving": sat_rate * sliced_s / N},
        "kkt_reached_fraction": float(np.mean(kkts <= TOL)),
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def dataclasses_replace(obj, **kw):
    import dataclasses
    return dataclasses.replace(obj, **kw)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(syn.WORKLOADS) + ["serving_mix"])
    ap.add_argument("--serving-requests", type=int, default=48)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--dense-product", default="sliced", choices=["sliced", "fp64"],
                    help="dense FP64 products: int8 digit planes on the tensor cores (FP64-"
                         "accurate) or FP64 FMAs on the CUDA cores")
    ap.add_argument("--profile", action="store_true",
                    help="short run for profiler captures (init + 1 + --profile-iters "
                         "iterations, no timing)")
    ap.add_argument("--profile-iters", type=int, default=3)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving_mix":
        return run_serving(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
