"""Serving loop for streams of independent IPM solve requests (one GPU).

A request is one normal-equations system (A, theta, b, block partition) plus
follow-up scalings theta_1..theta_f.  It is served as: setup (S = A Theta A^T
+ rho I), factor (filter, correction, levels, block IC(0)), solve, then per
follow-up a device-side value update (sdsl_update_diag) and a solve with the
kept preconditioner -- the matrix, the factors and the Krylov state stay
resident in HBM for the request's lifetime (preconditioner reuse, Sec. 3.4).

Continuous batching: requests are admitted as they arrive, whenever a slot
and enough HBM are free; every admitted request prepares its solves (setup,
factor, value updates) on its own CUDA stream in its own worker thread.  In
batched mode (the default) each ready solve is handed to one batching
thread, which runs all the solves ready at that moment together through
sdsl_batch_solve -- the blocks of every request in the same launches, each
request's result that of its solve alone -- and solves that become ready
meanwhile join the next batch.  Without batching, each worker solves on its
own stream and the requests' kernels merely overlap.  The C-ABI calls
release the GIL (ctypes), so the workers block on the device, not on each
other.

Admission by free HBM: the budget is the device's free memory at start
(minus a reserve); a request is charged an upper-bound estimate of its
device footprint (from the column counts of A) at admission, and its
measured footprint (the handle's peak device bytes after its first
factorization, plus its buffers) from then until it completes.  The
queue is first-come first-served with backfill: when the head does not fit
the remaining budget, a later request that fits may start.

The scheduling logic (Scheduler) is separate from the device work (an
executor callable), so it can be exercised without a GPU.
"""
from __future__ import annotations

import dataclasses
import queue
import threading
import time
from typing import Callable, List, Optional, Sequence

import numpy as np


# --------------------------------------------------------------------------- requests and results

@dataclasses.dataclass
class SolveRecord:
    start_s: float        # wall time the solve (or setup+factor+solve) was issued, from stream start
    done_s: float         # wall time its result was on the host
    iters: int
    status: int
    rel_res: float
    x: Optional[np.ndarray] = None
    rebuilt: int = 0      # 1 if the preconditioner was rebuilt for this solve (reuse rule)


@dataclasses.dataclass
class RequestResult:
    index: int
    arrival_s: float
    admitted_s: float
    done_s: float
    m: int
    solves: List[SolveRecord]

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


def footprint_bytes(A, factor_prec: int = 32) -> int:
    """Upper bound of a request's device memory: A and A^T, S (at most
    sum_j c_j^2 + m entries for column counts c_j), the filtered copy, the
    factors and their level tiles, and the Krylov vectors."""
    m, n = A.nrows, A.ncols
    cc = np.bincount(A.col, minlength=n).astype(np.int64)
    nnz_s = int((cc * cc).sum()) + m
    nnz_a = int(A.nnz)
    fac = 4 if factor_prec == 32 else 8
    b = 2 * (12 * nnz_a + 8 * (max(m, n) + 1))      # A, A^T (CSR)
    b += 12 * nnz_s + 8 * (m + 1)                    # S
    b += 12 * nnz_s + 8 * (m + 1)                    # filtered, corrected P
    b += (8 + fac) * nnz_s                           # factor values (both precisions)
    b += (2 + fac) * nnz_s + 64 * m                  # staged level tiles of both directions
    b += 16 * 8 * max(m, n)                          # vectors (x, r, z, p, q, u, b, ...)
    return int(1.25 * b) + (8 << 20)


# --------------------------------------------------------------------------- scheduler (host logic only)

class Scheduler:
    """Admission of requests into slots under a memory budget.

    `run(arrivals, costs, execute)` releases request i at arrivals[i]
    (seconds from start), admits it when a slot is free and costs[i] fits the
    remaining budget (FCFS with backfill), and calls execute(i, slot) in the
    slot's worker thread.  Returns (admit_times, done_times, max_concurrency).
    """

    def __init__(self, slots: int, budget_bytes: int, clock: Callable[[], float] = time.perf_counter):
        if slots < 1:
            raise ValueError("slots must be >= 1")
        self.slots = slots
        self.budget = int(budget_bytes)
        self.clock = clock

    def recharge(self, i: int, cost: int) -> None:
        """Replace request i's charge (admission estimate) by a measured one
        while it runs; a lower charge frees budget for the queue at once."""
        cv, state, costs = self._cv, self._state, self._costs
        with cv:
            state["used"] += int(cost) - costs[i]
            costs[i] = int(cost)
            cv.notify_all()

    def run(self, arrivals: Sequence[float], costs: Sequence[int],
            execute: Callable[[int, int], None]) -> tuple:
        n = len(arrivals)
        if any(c > self.budget for c in costs):
            raise ValueError("a request exceeds the whole memory budget")
        costs = [int(c) for c in costs]
        order = sorted(range(n), key=lambda i: (arrivals[i], i))
        cv = threading.Condition()
        queue: List[int] = []          # arrived, not admitted (arrival order)
        free_slots = list(range(self.slots))
        state = {"used": 0, "running": 0, "max_running": 0, "error": None, "arrived": 0}
        self._cv, self._state, self._costs = cv, state, costs
        self.charged = []  # (time, budget in use) right after each admission
        admit = [0.0] * n
        done = [0.0] * n
        t0 = self.clock()

        def worker(i: int, slot: int):
            try:
                execute(i, slot)
            except BaseException as e:  # noqa: BLE001 -- reported to the caller after the run
                with cv:
                    state["error"] = state["error"] or e
            finally:
                with cv:
                    done[i] = self.clock() - t0
                    state["used"] -= costs[i]
                    state["running"] -= 1
                    free_slots.append(slot)
                    cv.notify_all()

        threads = []
        k = 0
        with cv:
            while True:
                now = self.clock() - t0
                while k < n and arrivals[order[k]] <= now:
                    queue.append(order[k])
                    k += 1
                # admit in FCFS order, letting later requests that fit pass a blocked head
                started = True
                while started and queue and free_slots and state["error"] is None:
                    started = False
                    for qi, i in enumerate(queue):
                        if state["used"] + costs[i] <= self.budget:
                            queue.pop(qi)
                            slot = free_slots.pop(0)
                            state["used"] += costs[i]
                            self.charged.append((self.clock() - t0, state["used"]))
                            state["running"] += 1
                            state["max_running"] = max(state["max_running"], state["running"])
                            admit[i] = self.clock() - t0
                            th = threading.Thread(target=worker, args=(i, slot), daemon=True)
                            threads.append(th)
                            th.start()
                            started = True
                            break
                if state["error"] is not None or (k == n and not queue and state["running"] == 0):
                    break
                wait = None
                if k < n:
                    wait = max(0.0, arrivals[order[k]] - (self.clock() - t0))
                cv.wait(timeout=wait if wait is not None else 0.5)
        for th in threads:
            th.join()
        if state["error"] is not None:
            raise state["error"]
        return admit, done, state["max_running"]


# --------------------------------------------------------------------------- GPU executor

class _Batcher:
    """Continuous batching of the workers' solves: one thread keeps a batch
    (sdsl_batch_*) running; a solve that becomes ready joins it between graph
    launches, and a finished solve leaves it and wakes its worker at once.  A
    handle that does not fit the batch's kernel shape is solved alone."""

    def __init__(self, sdsl, max_batch: int, graph_iters: int):
        self.sdsl = sdsl
        self.max_batch = max_batch
        self.graph_iters = graph_iters
        self.q: "queue.Queue" = queue.Queue()
        self.sizes: List[int] = []
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()

    def solve(self, h, b, x):
        item = {"h": h, "b": b, "x": x, "done": threading.Event(), "st": None, "err": None}
        self.q.put(item)
        item["done"].wait()
        if item["err"] is not None:
            raise item["err"]
        return item["st"]

    def close(self):
        self.q.put(None)
        self.thread.join()

    @staticmethod
    def _finish(item, st=None, err=None):
        item["st"], item["err"] = st, err
        item["done"].set()

    def _loop(self):
        sdsl = self.sdsl
        B = sdsl.sdsl_batch_create(self.graph_iters)
        running = {}  # handle value -> waiting item
        closing = False
        try:
            while True:
                new = []
                if not running and not closing:
                    new.append(self.q.get())  # idle: wait for work
                while True:
                    try:
                        new.append(self.q.get_nowait())
                    except queue.Empty:
                        break
                for item in new:
                    if item is None:
                        closing = True
                        continue
                    h = item["h"]
                    hv = h.value if hasattr(h, "value") else h
                    if len(running) >= self.max_batch:
                        self.q.put(item)  # full: next round
                        continue
                    try:
                        sdsl.sdsl_batch_add(B, h, item["b"], item["x"])
                        running[hv] = item
                    except sdsl.SdslError:
                        try:  # does not fit the batch: alone
                            st = sdsl.sdsl_solve(h, item["b"], item["x"],
                                                 allow=(sdsl.ERR_NOT_CONVERGED, sdsl.ERR_BREAKDOWN))
                            self._finish(item, st=st)
                        except Exception as e:  # noqa: BLE001 -- handed to the waiting worker
                            self._finish(item, err=e)
                if not running:
                    if closing:
                        return
                    continue
                self.sizes.append(len(running))
                try:
                    out = sdsl.sdsl_batch_step(B, max_graphs=1, cap=len(running))
                except Exception as e:  # noqa: BLE001 -- every member's worker gets it
                    for item in running.values():
                        self._finish(item, err=e)
                    running.clear()
                    continue
                for hv, st in out:
                    self._finish(running.pop(hv), st=st)
        finally:
            sdsl.sdsl_batch_free(B)


class GpuServer:
    """Serves NormalProblem requests on one GPU through the C ABI."""

    def __init__(self, slots: int = 8, factor_prec: int = 32, device: int = 0, reserve_frac: float = 0.1,
                 budget_bytes: Optional[int] = None, keep_x: bool = False, graph_iters: int = 16,
                 batch: bool = True, max_batch: int = 16, batchers: int = 1):
        import torch

        from . import sdsl

        sdsl.load()
        self.torch = torch
        self.sdsl = sdsl
        self.dev = torch.device("cuda", device)
        torch.cuda.set_device(self.dev)
        if budget_bytes is None:
            free, _ = torch.cuda.mem_get_info(self.dev)
            budget_bytes = int(free * (1.0 - reserve_frac))
        self.budget = budget_bytes
        self.slots = slots
        self.factor_prec = factor_prec
        self.keep_x = keep_x
        self.graph_iters = graph_iters
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(slots)]
        self.batch = batch
        self.max_batch = max_batch
        self.n_batchers = max(1, batchers)
        self._batchers: List[_Batcher] = []

    def _serve_one(self, req, stream, t0: float, slot: int = 0,
                   recharge: Optional[Callable[[int], None]] = None) -> List[SolveRecord]:
        torch, sdsl = self.torch, self.sdsl
        prob = req.problem
        A = prob.A
        recs: List[SolveRecord] = []
        with torch.cuda.stream(stream):
            host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
                    for a in (A.rowptr, A.col, A.val, prob.theta, prob.b)]
            d_rp, d_ci, d_v, d_th, d_b = [a.to(self.dev, non_blocking=True) for a in host]
            d_x = torch.empty_like(d_b)
            o, keep = sdsl.options_for(prob, factor_prec=self.factor_prec, graph_iters=self.graph_iters,
                                       stream=stream.cuda_stream)
            if self.batch:  # one kernel shape for every request, so that their solves batch
                o.sweep_slots = 2
                o.spmv_form = 3
            start = time.perf_counter() - t0
            h = sdsl.sdsl_setup(o, A.nrows, A.ncols, d_rp, d_ci, d_v, d_th)
            try:
                sdsl.sdsl_factor(h)
                if recharge is not None:
                    # the request's measured footprint replaces the estimate:
                    # the handle's peak (temporaries of setup and factor
                    # included) plus the input and solution buffers
                    info = sdsl.sdsl_get_info(h)
                    inputs = sum(t.numel() * t.element_size() for t in (d_rp, d_ci, d_v, d_th, d_b, d_x))
                    recharge(int(1.1 * (info.peak_device_bytes + inputs)) + (8 << 20))
                thetas = [None] + list(req.followups)
                for k, th in enumerate(thetas):
                    if th is not None:
                        start = time.perf_counter() - t0
                        d_th.copy_(torch.from_numpy(th).pin_memory(), non_blocking=True)
                        sdsl.sdsl_update_diag(h, d_th)
                    if self._batchers:  # each slot feeds one batcher (batches overlap like streams)
                        st = self._batchers[slot % len(self._batchers)].solve(h, d_b, d_x)
                    else:
                        st = sdsl.sdsl_solve(h, d_b, d_x, allow=(sdsl.ERR_NOT_CONVERGED, sdsl.ERR_BREAKDOWN))
                    x = d_x.cpu().numpy() if self.keep_x else None
                    stream.synchronize()
                    recs.append(SolveRecord(start, time.perf_counter() - t0, int(st.iters), int(st.status),
                                            float(st.rel_res_true), x, int(st.rebuilt)))
            finally:
                sdsl.sdsl_free(h)
        return recs

    def serve(self, requests: Sequence, arrivals: Optional[Sequence[float]] = None,
              costs: Optional[Sequence[int]] = None) -> tuple:
        """Serve `requests` (workloads.Request) released at `arrivals` (seconds
        from start; default: their own arrival times).  Returns (results,
        summary)."""
        n = len(requests)
        arrivals = [r.arrival_s for r in requests] if arrivals is None else list(arrivals)
        costs = [footprint_bytes(r.problem.A, self.factor_prec) for r in requests] if costs is None else list(costs)
        recs: List[Optional[List[SolveRecord]]] = [None] * n
        t0_box = {}

        def execute(i: int, slot: int):
            recs[i] = self._serve_one(requests[i], self.streams[slot], t0_box["t0"], slot,
                                      recharge=lambda c: sched.recharge(i, c))

        sched = Scheduler(self.slots, self.budget)
        self.scheduler = sched
        self._batchers = ([_Batcher(self.sdsl, self.max_batch, self.graph_iters) for _ in range(self.n_batchers)]
                          if self.batch else [])
        t0_box["t0"] = time.perf_counter()
        try:
            admit, done, maxc = sched.run(arrivals, costs, execute)
        finally:
            sizes = []
            for b in self._batchers:
                b.close()
                sizes += b.sizes
            self._batchers = []
        results = [RequestResult(i, arrivals[i], admit[i], recs[i][-1].done_s, requests[i].problem.A.nrows, recs[i])
                   for i in range(n)]
        summ = summarize(results, maxc)
        if sizes:  # requests running together, sampled at every graph launch
            summ["batch_steps"] = len(sizes)
            summ["mean_batch"] = round(float(np.mean(sizes)), 2)
            summ["max_batch"] = int(max(sizes))
        return results, summ


def serve_sequential(requests: Sequence, factor_prec: int = 64, device: int = 0, keep_x: bool = False,
                     arrivals: Optional[Sequence[float]] = None) -> tuple:
    """Baseline: one request at a time in arrival order on the default
    stream, plain FP64 factors (no overlap between requests)."""
    srv = GpuServer(slots=1, factor_prec=factor_prec, device=device, keep_x=keep_x, batch=False)
    return srv.serve(requests, arrivals=arrivals, costs=[0] * len(requests))


def summarize(results: Sequence[RequestResult], max_concurrency: int = 1) -> dict:
    lat = np.array([r.latency_s for r in results])
    solve_lat = np.array([s.done_s - s.start_s for r in results for s in r.solves])
    nsolves = sum(len(r.solves) for r in results)
    nconv = sum(1 for r in results for s in r.solves if s.status == 0)
    t_first = min(r.arrival_s for r in results)
    t_last = max(r.done_s for r in results)
    span = max(t_last - t_first, 1e-9)
    return {
        "requests": len(results), "solves": nsolves, "span_s": round(span, 3),
        "solves_per_s": round(nsolves / span, 3), "requests_per_s": round(len(results) / span, 3),
        "converged_solves": nconv, "converged_solves_per_s": round(nconv / span, 3),
        "latency_p50_s": round(float(np.percentile(lat, 50)), 4),
        "latency_p99_s": round(float(np.percentile(lat, 99)), 4),
        "solve_latency_p50_s": round(float(np.percentile(solve_lat, 50)), 4),
        "solve_latency_p99_s": round(float(np.percentile(solve_lat, 99)), 4),
        "unconverged_solves": int(sum(1 for r in results for s in r.solves if s.status != 0)),
        "max_concurrency": int(max_concurrency),
    }
