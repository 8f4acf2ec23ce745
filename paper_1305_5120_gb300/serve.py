"""Continuous-batching server for sequences of generalized eigenproblems on one GPU.

Each admitted sequence (one k-point's chain of SCF problems, Section 2) runs in a solver
slot: a persistent host worker thread with its own CUDA stream and chfsi context, so the
sequence's Ritz block and filter bounds stay on the device between its steps (Algorithm 1
Require: the previous eigenvectors and eigenvalues).  Work of different slots overlaps on
the device.  A waiting sequence is admitted as soon as a slot is free and the library's
memory estimate for its size fits the remaining HBM budget; its step l + 1 is issued when
step l completes (the SCF dependence).  Latency of a solve = its completion time minus the
time the step became ready (arrival for step 0, completion of the previous step after).

The library does all the computing; this module only moves host inputs to the device,
sequences calls and keeps time.
"""
from __future__ import annotations

import dataclasses
import queue
import threading
import time
from typing import Callable, List, Optional

import numpy as np

from . import chfsi


@dataclasses.dataclass
class SequenceRequest:
    seq_id: int
    arrival: float                     # seconds after the start of run()
    n: int
    nev: int
    nex: int
    steps: int
    make_step: Callable[[int], tuple]  # l -> (H, S or None): mathematical orientation, numpy or torch
    tol: float = 1e-10
    degree: int = 20
    X0: Optional[np.ndarray] = None


@dataclasses.dataclass
class SolveRecord:
    seq_id: int
    step: int
    status: int
    evals: np.ndarray
    X: Optional[np.ndarray]
    ready: float        # when the step became ready (arrival, or the previous step's completion)
    start: float        # when its solve was issued
    done: float
    slot: int
    info: dict

    @property
    def latency(self) -> float:
        return self.done - self.ready


class Server:
    def __init__(self, device: int = 0, slots: int = 4, hbm_budget: Optional[int] = None,
                 keep_vectors: bool = False, **params):
        import torch
        self.device = device
        self.slots = slots
        self.params = params
        self.keep_vectors = keep_vectors
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info(device)
            hbm_budget = int(0.8 * free)
        self.hbm_budget = hbm_budget

    def _worker(self, slot: int, work: "queue.Queue", done: "queue.Queue", t0: float):
        import torch
        torch.cuda.set_device(self.device)
        stream = torch.cuda.Stream(self.device)
        ctx = None
        with torch.cuda.stream(stream):
            while True:
                req = work.get()
                if req is None:
                    break
                if ctx is None:
                    ctx = chfsi.Context(device=self.device, stream=stream, **self.params)
                evals = torch.empty(req.nev, dtype=torch.float64, device="cuda")
                X = torch.empty((req.nev, req.n), dtype=torch.complex128, device="cuda")
                ready = req.arrival
                for l in range(req.steps):
                    start = time.perf_counter() - t0
                    H, S = req.make_step(l)
                    Hd = chfsi.colmajor(H)
                    Sd = chfsi.colmajor(S) if S is not None else None
                    if l == 0:
                        X0 = chfsi.colmajor(req.X0) if req.X0 is not None else None
                        st, ev, Xo, info = ctx.solve(Hd, Sd, req.n, req.nev, req.nex, X0, req.tol, req.degree, evals, X)
                    else:
                        st, ev, Xo, info = ctx.next_in_sequence(Hd, Sd, evals, X)
                    stream.synchronize()
                    now = time.perf_counter() - t0
                    rec = SolveRecord(req.seq_id, l, st, ev.cpu().numpy(),
                                      chfsi.to_numpy(Xo) if self.keep_vectors else None,
                                      ready, start, now, slot, info.as_dict())
                    done.put(("solve", rec))
                    ready = now
                    if st not in (0,):
                        break
                done.put(("finished", req))
        if ctx is not None:
            ctx.close()

    def run(self, requests: List[SequenceRequest], realtime: bool = True) -> List[SolveRecord]:
        """Serve all requests; returns one record per solve (in completion order)."""
        pending = sorted(requests, key=lambda r: r.arrival)
        need = {r.seq_id: chfsi.workspace_bytes(r.n, r.nev, r.nex, self.params.get("precision", 1))
                for r in pending}
        for r in pending:
            if need[r.seq_id] > self.hbm_budget:
                raise ValueError(f"sequence {r.seq_id} needs {need[r.seq_id]} B > budget {self.hbm_budget}")
        work = [queue.Queue() for _ in range(self.slots)]
        done: "queue.Queue" = queue.Queue()
        t0 = time.perf_counter()
        threads = [threading.Thread(target=self._worker, args=(i, work[i], done, t0), daemon=True)
                   for i in range(self.slots)]
        for t in threads:
            t.start()
        free_slots = list(range(self.slots))
        busy = {}                       # seq_id -> slot
        used = 0
        records: List[SolveRecord] = []
        waiting: List[SequenceRequest] = []
        remaining = len(pending)
        while remaining:
            now = time.perf_counter() - t0
            while pending and (pending[0].arrival <= now or not realtime):
                waiting.append(pending.pop(0))
            # admit in arrival order while a slot and the memory budget allow
            progressed = True
            while progressed and waiting and free_slots:
                progressed = False
                for i, r in enumerate(waiting):
                    if used + need[r.seq_id] <= self.hbm_budget:
                        slot = free_slots.pop(0)
                        busy[r.seq_id] = slot
                        used += need[r.seq_id]
                        work[slot].put(r)
                        waiting.pop(i)
                        progressed = True
                        break
            timeout = 0.002
            if pending and realtime:
                timeout = max(0.0005, min(0.05, pending[0].arrival - (time.perf_counter() - t0)))
            try:
                kind, obj = done.get(timeout=timeout)
            except queue.Empty:
                continue
            if kind == "solve":
                records.append(obj)
            else:
                slot = busy.pop(obj.seq_id)
                used -= need[obj.seq_id]
                free_slots.append(slot)
                remaining -= 1
        for q in work:
            q.put(None)
        for t in threads:
            t.join()
        return records


def latency_summary(records: List[SolveRecord]) -> dict:
    lat = np.array([r.latency for r in records])
    span = max(r.done for r in records) - min(r.ready for r in records)
    return {"solves": len(records), "eigenproblems_per_s": len(records) / span if span > 0 else None,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "failed": int(sum(1 for r in records if r.status != 0))}
