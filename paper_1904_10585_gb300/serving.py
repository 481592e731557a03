"""Request loop serving many polynomial-filtered solves on one GPU
(continuous batching).

Requests of different kinds and sizes arrive over time.  Each admitted
request owns a slot: a pre-created pf_ctx (workspace only) bound to its own
CUDA stream, plus the request's resident device state (warm-started block U,
Ritz factors, duals, iteration matrix) allocated when it is admitted.  A slot
advances its solve in chunks of `chunk` steps: one pf_enqueue_steps call
(replays of the request's captured step graph) followed by pf_report_async
into pinned host memory and an event, all without a host synchronisation,
so the steps of different requests overlap on the device.  The loop admits
queued requests (first come, first served, skipping ones that do not fit)
whenever a slot of the right class is free and the request's device
footprint fits the HBM budget, and retires a request when its KKT residual
reaches the tolerance or its iteration cap is hit (copying its factors to
the host).

Everything numeric runs in libpf's kernels; this module only schedules.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import time
from typing import List, Optional

import numpy as np
import torch

from . import _binding as B
from . import solver as S


@dataclasses.dataclass
class Request:
    rid: int
    kind: str                 # "maxcut" | "completion"
    n: int
    arrival: float            # seconds after the start of the run
    rowptr: np.ndarray
    colind: np.ndarray
    vals: np.ndarray          # C values (float64) or sampled M values (float32)
    U0: np.ndarray            # n x p start block
    max_iter: int = 200
    mu: float = 0.05
    t: float = 1.0
    # host copies in page-locked memory (filled by Server.prepare)
    pinned: Optional[dict] = None


@dataclasses.dataclass
class Result:
    rid: int
    kind: str
    n: int
    arrival: float
    admitted: float
    finished: float
    iters: int
    kkt: float
    obj: float
    r_plus: int
    theta: np.ndarray
    V: np.ndarray

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class _Slot:
    def __init__(self, kind: str, p: int, n_max: int, degree: int, precision: int, dev,
                 degree_max: int = 0):
        self.kind, self.p, self.n_max, self.precision = kind, p, n_max, precision
        self.stream = torch.cuda.Stream(device=dev)
        # a low-precision slot climbs the adaptive ladder (to FP64 when its
        # filter's precision floor stalls the KKT residual)
        adaptive = 1 if precision != B.PF_PREC_FP64 else 0
        self.ctx = S.Context(p=p, n_max=n_max, degree=degree, precision=precision,
                             stream=self.stream, adaptive=adaptive,
                             degree_max=degree_max or degree)
        self.info_buf = torch.empty(ctypes.sizeof(B.pf_iter_info), dtype=torch.uint8).pin_memory()
        self.info = B.pf_iter_info.from_address(self.info_buf.data_ptr())
        self.event = torch.cuda.Event()
        self.req: Optional[Request] = None
        self.prob: Optional[S.Problem] = None
        self.bytes = 0
        self.admitted = 0.0
        self.steps = 0

    def close(self):
        self.ctx.close()


def problem_bytes(kind: str, n: int, nnz: int, p: int, lowprec: bool) -> int:
    """Device bytes a request's resident state occupies (its CSR input, the
    blocks and vectors, and the iteration matrix where there is one)."""
    blocks = 2 * n * p * 8 + p * 8
    csr = (n + 1) * 4 + nnz * 4
    if kind == "maxcut":
        z = n * (((n + 7) // 8) * 8) * 2 if lowprec else n * n * 8
        return blocks + csr + nnz * 8 + nnz * 8 + n * 8 + z
    return blocks + csr + nnz * 4 + nnz * 8


class Server:
    """Continuous-batching loop over a fixed pool of slots.

    slots: list of (kind, n_max, count); p, degree and the per-kind precision
    are shared.  hbm_budget bounds the summed footprint of admitted requests."""

    def __init__(self, slots, p=32, degree=4, tol=1e-4, chunk=10, hbm_budget=16 << 30,
                 maxcut_lowprec=True, completion_lowprec=False, device=None):
        self.dev = device or torch.device("cuda", torch.cuda.current_device())
        self.p, self.degree, self.tol, self.chunk = p, degree, tol, chunk
        self.budget = int(hbm_budget)
        self.maxcut_lowprec = maxcut_lowprec
        self.completion_lowprec = completion_lowprec
        self.slots: List[_Slot] = []
        for kind, n_max, count in slots:
            lp = maxcut_lowprec if kind == "maxcut" else completion_lowprec
            prec = B.PF_PREC_BF16 if lp else B.PF_PREC_FP64
            for _ in range(count):
                self.slots.append(_Slot(kind, p, n_max, degree, prec, self.dev))
        self.used = 0

    def close(self):
        for s in self.slots:
            s.close()

    @staticmethod
    def prepare(requests: List[Request]):
        """Page-locked host copies of every request's inputs (outside timing)."""
        for r in requests:
            r.pinned = {
                "rowptr": torch.from_numpy(r.rowptr.astype(np.int32)).pin_memory(),
                "colind": torch.from_numpy(r.colind.astype(np.int32)).pin_memory(),
                "vals": torch.from_numpy(r.vals).pin_memory(),
                "U0": torch.from_numpy(np.ascontiguousarray(r.U0)).pin_memory(),
            }

    def footprint(self, r: Request) -> int:
        return problem_bytes(r.kind, r.n, r.colind.shape[0], self.p,
                             r.kind == "maxcut" and self.maxcut_lowprec)

    # -- slot life cycle ------------------------------------------------------
    def _admit(self, slot: _Slot, r: Request, now: float):
        dev = self.dev
        with torch.cuda.stream(slot.stream):
            pin = r.pinned
            rp = pin["rowptr"].to(dev, non_blocking=True)
            ci = pin["colind"].to(dev, non_blocking=True)
            vv = pin["vals"].to(dev, non_blocking=True)
            U0 = pin["U0"].to(dev, non_blocking=True)
            if r.kind == "maxcut":
                lp = "bf16" if self.maxcut_lowprec else None
                pr = S.maxcut_problem(rp, ci, vv, U0, dense=False, lowprec=lp)
            else:
                pr = S.completion_problem(rp, ci, vv, U0, mu=r.mu, t=r.t)
            pr._keep_inputs = (rp, ci, vv, U0)
            S.problem_init(slot.ctx, pr)
        slot.req, slot.prob = r, pr
        slot.bytes = self.footprint(r)
        self.used += slot.bytes
        slot.admitted = now
        slot.steps = 0
        self._advance(slot)

    def _advance(self, slot: _Slot, kkt: Optional[float] = None):
        r = slot.req
        if kkt is not None and math.isfinite(kkt):
            B.pf_ladder_update(slot.ctx.handle, slot.prob.struct, kkt)
        k = min(self.chunk, r.max_iter - slot.steps)
        B.pf_enqueue_steps(slot.ctx.handle, slot.prob.struct, k)
        slot.steps += k
        B.pf_report_async(slot.ctx.handle, slot.info_buf.data_ptr())
        slot.event.record(slot.stream)

    def _retire(self, slot: _Slot, now: float) -> Result:
        r, pr, info = slot.req, slot.prob, slot.info
        with torch.cuda.stream(slot.stream):
            V = pr.V.to("cpu", non_blocking=True)
            th = pr.theta.to("cpu", non_blocking=True)
        slot.stream.synchronize()
        res = Result(rid=r.rid, kind=r.kind, n=r.n, arrival=r.arrival, admitted=slot.admitted,
                     finished=now, iters=slot.steps, kkt=float(info.kkt), obj=float(info.obj),
                     r_plus=int(info.r_plus), theta=th.numpy().copy(), V=V.numpy())
        self.used -= slot.bytes
        slot.req, slot.prob, slot.bytes = None, None, 0
        return res

    # -- the loop -------------------------------------------------------------
    def run(self, requests: List[Request]) -> List[Result]:
        for r in requests:
            if r.pinned is None:
                self.prepare([r])
            if not any(s.kind == r.kind and s.n_max >= r.n for s in self.slots):
                raise ValueError(f"request {r.rid}: no slot class holds {r.kind} n={r.n}")
            if self.footprint(r) > self.budget:
                raise ValueError(f"request {r.rid} needs more than the HBM budget")
        pending = sorted(requests, key=lambda q: q.arrival)
        queue: List[Request] = []
        results: List[Result] = []
        t0 = time.perf_counter()
        while pending or queue or any(s.req is not None for s in self.slots):
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                queue.append(pending.pop(0))
            progressed = False
            # admission (first come, first served; a request that does not fit
            # waits, later ones may pass it)
            for r in list(queue):
                need = self.footprint(r)
                if self.used + need > self.budget:
                    continue
                slot = next((s for s in self.slots if s.req is None and s.kind == r.kind
                             and s.n_max >= r.n), None)
                if slot is None:
                    continue
                queue.remove(r)
                self._admit(slot, r, time.perf_counter() - t0)
                progressed = True
            # progress of the requests in flight
            for slot in self.slots:
                if slot.req is None or not slot.event.query():
                    continue
                progressed = True
                info = slot.info
                if info.flags & 8:
                    raise RuntimeError(f"request {slot.req.rid}: a device wait timed out")
                done = (self.tol > 0 and info.kkt <= self.tol) or slot.steps >= slot.req.max_iter
                if done:
                    results.append(self._retire(slot, time.perf_counter() - t0))
                else:
                    self._advance(slot, float(info.kkt))
            if not progressed:
                time.sleep(20e-6)
        return results


def run_alone(requests: List[Request], **server_kw) -> List[Result]:
    """Each request on an otherwise idle server, one after another (the
    'alone' side of the alone-vs-mix comparison)."""
    out = []
    for r in requests:
        r2 = dataclasses.replace(r, arrival=0.0)
        srv = Server(**server_kw)
        try:
            out.extend(srv.run([r2]))
        finally:
            srv.close()
    return out


def latency_percentiles(results: List[Result]):
    lat = np.array([r.latency for r in results])
    return float(np.percentile(lat, 50)), float(np.percentile(lat, 99))
