"""Continuous-batching request server for many-shot sampling of Clifford circuits.

A request carries a circuit (gate layers ending with a Z-measurement of every
qubit) and a shot count. Serving a request means: upload its gate records,
run it single-shot on a device-resident tableau (the reference record of
Sec. 5), and draw its shots with Pauli frames (Sec. 5, Alg. 9) -- all through
the C ABI of libqs. The paper has no server; this loop is the serving pattern
built around its method:

  * admission: requests wait in arrival order and the head is admitted when a
    slot is free and its device footprint (tableau in both layouts, frames,
    record, gate records) fits the remaining device-memory budget;
  * continuous batching: every slot is a host worker with its own CUDA stream,
    so requests admitted while others are on the GPU run concurrently and their
    kernels overlap on the device; a request finishing frees its slot and its
    memory for the next one. Small requests (under 1,024 qubits, no noise
    channels) that wait together are served together: when a slot admits one,
    it also takes the small requests queued right behind it (in arrival order,
    within the memory budget, up to max_batch) and runs them as one batch --
    all their reference shots in one persistent launch (qs_batch_run) and all
    their shots in one sampling launch (qs_batch_sample);
  * results do not depend on the mix: each request owns its tableau and its
    coins and frames are keyed by (seed, shot, index), so a request's record is
    bit-identical alone and among others.

The scheduling core (`Scheduler`) is independent of the GPU and is tested on
the CPU with a fake executor.
"""
from __future__ import annotations

import threading
import time
from collections import deque
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional

import numpy as np


@dataclass
class Request:
    rid: int
    arrival_s: float
    circuit: object          # workloads.circuits.Circuit
    shots: int
    seed: int


@dataclass
class Result:
    rid: int
    n: int
    shots: int
    arrival_s: float
    admit_s: float
    done_s: float
    footprint: int
    record: Optional[np.ndarray] = None      # single-shot reference record (M bytes)
    samples: Optional[np.ndarray] = None     # (M, ceil(shots/64)) uint64

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


def footprint_bytes(n: int, n_gates: int, n_meas: int, shots: int) -> int:
    """Device bytes one request holds while it is served."""
    from . import qs
    ow = (shots + 63) // 64
    fw = (ow + 3) // 4 * 4
    return (qs.qs_sim_required_bytes(n) + 2 * n * fw * 8 + max(n_meas, 1) * ow * 8
            + 2 * max(n_meas, 1) * ow * 8 + n_gates * 8 + n_meas * 4 + 3 * 4096)


class Scheduler:
    """FIFO admission by slots and a byte budget, with worker threads.

    execute(request, slot) -> Result does the work of one request; it is
    called on the slot's worker thread. The head of the queue waits until a
    slot is free and its footprint fits (no overtaking, so no starvation).
    """

    def __init__(self, slots: int, budget_bytes: int, footprint: Callable[[Request], int],
                 execute: Callable[[Request, int, float, int], Result],
                 execute_batch: Optional[Callable] = None,
                 batchable: Optional[Callable[[Request], bool]] = None, max_batch: int = 64):
        self.slots = slots
        self.budget = budget_bytes
        self.footprint = footprint
        self.execute = execute
        # execute_batch(requests, slot, admit_s, footprints) -> [Result]; requests
        # for which batchable() holds are grouped when they wait together
        self.execute_batch = execute_batch
        self.batchable = batchable
        self.max_batch = max_batch
        self.batches = 0          # batches of two or more requests run
        self.batched_requests = 0
        self.cv = threading.Condition()
        self.pending: deque = deque()
        self.in_use = 0
        self.peak_in_use = 0
        self.active = 0
        self.peak_active = 0
        self.closed = False
        self.results: List[Result] = []
        self.errors: List[BaseException] = []
        self.t0 = 0.0

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def _worker(self, slot: int):
        while True:
            with self.cv:
                while True:
                    if self.pending:
                        req = self.pending[0]
                        fp = self.footprint(req)
                        if fp > self.budget:
                            self.pending.popleft()
                            self.errors.append(MemoryError(
                                f"request {req.rid} needs {fp} bytes, budget {self.budget}"))
                            self.cv.notify_all()
                            continue
                        if self.in_use + fp <= self.budget:
                            self.pending.popleft()
                            self.in_use += fp
                            group, fps = [req], [fp]
                            # small requests queued right behind join the head's batch
                            if self.execute_batch is not None and self.batchable(req):
                                while (self.pending and len(group) < self.max_batch
                                       and self.batchable(self.pending[0])):
                                    f2 = self.footprint(self.pending[0])
                                    if self.in_use + f2 > self.budget:
                                        break
                                    group.append(self.pending.popleft())
                                    fps.append(f2)
                                    self.in_use += f2
                            self.peak_in_use = max(self.peak_in_use, self.in_use)
                            self.active += len(group)
                            self.peak_active = max(self.peak_active, self.active)
                            admit = self.now()
                            break
                    elif self.closed:
                        return
                    self.cv.wait()
            try:
                if len(group) > 1:
                    results = self.execute_batch(group, slot, admit, fps)
                    with self.cv:
                        self.batches += 1
                        self.batched_requests += len(group)
                else:
                    results = [self.execute(req, slot, admit, fp)]
                done = self.now()
                for res in results:
                    res.done_s = done
                with self.cv:
                    self.results.extend(results)
            except BaseException as e:  # reported to the caller of run()
                with self.cv:
                    self.errors.append(e)
            finally:
                with self.cv:
                    self.in_use -= sum(fps)
                    self.active -= len(group)
                    self.cv.notify_all()

    def run(self, requests: List[Request], realtime: bool = True) -> List[Result]:
        """Feeds requests at their arrival times (seconds from the start) and
        returns the results in completion order."""
        self.t0 = time.perf_counter()
        workers = [threading.Thread(target=self._worker, args=(s,), daemon=True)
                   for s in range(self.slots)]
        for w in workers:
            w.start()
        for req in sorted(requests, key=lambda r: r.arrival_s):
            if realtime:
                delay = req.arrival_s - self.now()
                if delay > 0:
                    time.sleep(delay)
            with self.cv:
                self.pending.append(req)
                self.cv.notify_all()
        with self.cv:
            self.closed = True
            self.cv.notify_all()
        for w in workers:
            w.join()
        if self.errors:
            raise self.errors[0]
        return self.results


class GpuExecutor:
    """Serves one request on one slot: its own stream, device-resident tableau
    and frames, all work through the C ABI."""

    def __init__(self, slots: int, device: str = "cuda", keep_samples: bool = True):
        import torch
        from . import qs
        self.torch = torch
        self.qs = qs
        self.device = torch.device(device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]
        self.keep_samples = keep_samples

    def footprint(self, req: Request) -> int:
        c = req.circuit
        return footprint_bytes(c.n, c.n_gates, c.n_measurements, req.shots)

    @staticmethod
    def batchable(req: Request) -> bool:
        """Small noiseless circuits run in the batch's persistent kernel."""
        c = req.circuit
        return c.n < 1024 and not any(op[0] == "noise" for op in c.ops)

    def execute_batch(self, reqs: List[Request], slot: int, admit_s: float, fps) -> List[Result]:
        """Serves requests together: reference shots in one persistent launch
        (qs_batch_run), shots in one sampling launch (qs_batch_sample); the
        coins are keyed (seed, 0) and the frames by seed + 1, as for a request
        served alone, so the results are the same."""
        torch, qs = self.torch, self.qs
        stream = self.streams[slot]
        with torch.cuda.device(self.device), torch.cuda.stream(stream):
            b = qs.Batch([r.circuit for r in reqs], [r.seed for r in reqs], device=str(self.device),
                         stream=stream)
            b.run()
            outs = b.sample([r.shots for r in reqs], [r.seed + 1 for r in reqs])
            samples = []
            for o in outs:
                h = None
                if self.keep_samples and o is not None:
                    h = torch.empty(tuple(o.shape), dtype=torch.int64, pin_memory=True)
                    h.copy_(o, non_blocking=True)
                samples.append(h)
            b.sync()
            records = [b.record(i) for i in range(len(reqs))]
            stream.synchronize()
            b.close()
        return [Result(r.rid, r.circuit.n, r.shots, r.arrival_s, admit_s, 0.0, f, rec,
                       s.numpy().view(np.uint64) if s is not None else None)
                for r, f, rec, s in zip(reqs, fps, records, samples)]

    def __call__(self, req: Request, slot: int, admit_s: float, fp: int) -> Result:
        torch, qs = self.torch, self.qs
        c = req.circuit
        stream = self.streams[slot]
        with torch.cuda.device(self.device), torch.cuda.stream(stream):
            sim = qs.Simulator(c.n, device=str(self.device), stream=stream)
            packed = qs.qs_pack_layers(c.n, c.gates, c.layer_ptr)
            host = torch.from_numpy(packed.view(np.int32)).pin_memory()
            gates = host.to(self.device, non_blocking=True)
            lp = np.asarray(c.layer_ptr, np.int64)
            qlists = []
            for op in c.ops:
                if op[0] == "layers":
                    qs.qs_sim_apply_layers_dev(sim.sim, gates.data_ptr(), lp, op[1], op[2])
                elif op[0] == "noise":
                    qs.qs_sim_noise(sim.sim, op[1], op[2], op[3])
                else:
                    q = torch.from_numpy(np.asarray(op[1], np.uint32).view(np.int32)).pin_memory()
                    qd = q.to(self.device, non_blocking=True)
                    qlists.append((q, qd))
                    qs.qs_sim_measure_dev(sim.sim, qd.data_ptr(), qd.numel(), req.seed, 0)
            M = sim.num_measurements
            ow = (req.shots + 63) // 64
            out = torch.empty((max(M, 1), ow), dtype=torch.int64, device=self.device)
            fb = qs.qs_sim_sample_required_bytes(sim.sim, req.shots)
            fws = torch.empty(fb, dtype=torch.uint8, device=self.device)
            qs.qs_sim_sample(sim.sim, req.shots, req.seed + 1, out.data_ptr(), M * ow,
                             fws.data_ptr(), fb)
            samples = None
            if self.keep_samples:  # to pinned host memory (the caching host allocator reuses it)
                samples = torch.empty((M, ow), dtype=torch.int64, pin_memory=True)
                samples.copy_(out[:M], non_blocking=True)
            record = sim.record()  # syncs the slot's stream and checks the device flags
            stream.synchronize()
            sim.close()
        return Result(req.rid, c.n, req.shots, req.arrival_s, admit_s, 0.0, fp, record,
                      samples.numpy().view(np.uint64) if samples is not None else None)


def summarize(results: List[Result], makespan_s: float) -> Dict[str, float]:
    lat = np.array([r.latency_s for r in results])
    shots = sum(r.shots for r in results)
    return {"requests": len(results),
            "p50_latency_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_latency_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "mean_latency_s": float(lat.mean()) if len(lat) else None,
            "shots_per_s": shots / makespan_s if makespan_s > 0 else None,
            "makespan_s": makespan_s}


def serve(requests: List[Request], slots: int = 8, budget_bytes: int = 64 << 30,
          device: str = "cuda", keep_samples: bool = True, realtime: bool = True,
          batching: bool = True, max_batch: int = 64):
    """Runs the request stream; returns (results sorted by id, summary, scheduler stats)."""
    ex = GpuExecutor(slots, device, keep_samples)
    sch = Scheduler(slots, budget_bytes, ex.footprint, ex,
                    execute_batch=ex.execute_batch if batching else None,
                    batchable=ex.batchable, max_batch=max_batch)
    t = time.perf_counter()
    res = sch.run(requests, realtime=realtime)
    makespan = time.perf_counter() - t
    stats = {"peak_active": sch.peak_active, "peak_bytes": sch.peak_in_use,
             "budget_bytes": budget_bytes, "slots": slots, "batches": sch.batches,
             "batched_requests": sch.batched_requests}
    return sorted(res, key=lambda r: r.rid), summarize(res, makespan), stats
