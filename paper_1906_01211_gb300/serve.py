"""Continuous-batching server for polarization solves of uneven sizes.

Requests (isolated clusters or small periodic boxes, any size) arrive at any
time. The server keeps ``n_slots`` workers, each bound to its own CUDA stream
and owning reusable solver contexts (one per PME grid size, plus one for
clusters). A request is admitted as soon as a slot is free AND its estimated
device memory fits into the budget next to the requests already running, so
new requests join while others are still iterating and their kernels overlap
on the device (one stream per running request). Per request the whole path
runs in the CUDA library: neighbour lists (periodic) or all-pairs tiles
(clusters), permanent field, PCG solve, energy.

State kept on the device between requests:
  * every slot context keeps its buffers, neighbour lists and cuFFT plans, so
    a request of the same grid size reuses them (no allocation);
  * the last converged dipoles of each request ``key`` (byte budget, least
    recently used evicted) warm-start the next solve of that key.

Failures stay per request: an invalid input, a request larger than the whole
memory budget or a cancelled request gets an error result; the other requests
and the slots continue. A worker that dies is reported by ``health()``.

Host-side scheduling only; the paper has no serving counterpart (its
throughput runs are many MPI ranks on one system).
"""
from __future__ import annotations

import collections
import math
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from .synth import System, small_box_settings


@dataclass
class Result:
    rid: int
    ok: bool
    error: str | None = None
    mu: np.ndarray | None = None
    energy: float | None = None
    iters: int = 0
    rms_debye: float = 0.0
    t_submit: float = 0.0
    t_start: float = 0.0
    t_done: float = 0.0
    slot: int = -1
    warm_start: bool = False

    @property
    def latency(self) -> float:
        return self.t_done - self.t_submit


@dataclass
class _Req:
    rid: int
    system: System
    key: str | None
    est_bytes: int
    t_submit: float
    done: threading.Event = field(default_factory=threading.Event)
    result: Result | None = None


def box_settings(L: float):
    """Cutoff, beta and grid of a periodic request box (capped cutoff below L/2)."""
    return small_box_settings(L)


def estimate_bytes(system: System, precision: str) -> int:
    """Device memory one request needs beyond the reusable context buffers."""
    n = system.n
    per_atom = 1200
    if system.box is None:
        return n * per_atom + 16 * 32 * n
    rc, beta, K = box_settings(system.box)
    density = n / system.box ** 3
    half = int(n * 2.0 * math.pi / 3.0 * rc ** 3 * density) + 1024
    per_pair = 16 + 48 + (48 if precision == "mixed" else 96) + 24
    grid = K ** 3 * (8 + 8 + 4 + 4) + K * K * (K // 2 + 1) * (16 + 8 + 8 + 4)
    return n * per_atom + half * per_pair + grid


class _Slot:
    def __init__(self, server: "Server", index: int):
        self.server = server
        self.index = index
        self.stream = server._create_stream()
        self.periodic = {}  # K -> Polarization
        self.cluster = None
        self.alive = True
        self.thread = threading.Thread(target=self._run, name=f"amp-slot-{index}", daemon=True)

    def solver_for(self, system: System):
        from .amoebapol import Config, Polarization
        srv = self.server
        if system.box is None:
            cfg = Config(box=0.0, tol_debye=srv.tol, max_iter=srv.max_iter, precision=srv.precision)
            if self.cluster is None:
                self.cluster = Polarization(cfg, self.stream)
            return self.cluster
        rc, beta, K = box_settings(system.box)
        cfg = Config(box=system.box, cutoff=rc, ewald_beta=beta, pme_grid=K, tol_debye=srv.tol,
                     max_iter=srv.max_iter, precision=srv.precision)
        p = self.periodic.get(K)
        if p is None:
            p = Polarization(cfg, self.stream)
            self.periodic[K] = p
        else:
            p.reconfigure(cfg)
        return p

    def _run(self):
        srv = self.server
        srv._bind_thread()
        req = None
        try:
            while True:
                req = srv._next(self)
                if req is None:
                    return
                res = Result(rid=req.rid, ok=False, t_submit=req.t_submit, t_start=time.perf_counter(),
                             slot=self.index)
                try:
                    srv._execute(self, req, res)
                    res.ok = True
                except Exception as exc:  # noqa: BLE001 - reported per request
                    res.error = f"{type(exc).__name__}: {exc}"
                res.t_done = time.perf_counter()
                srv._finish(req, res)
                req = None
        except BaseException as exc:
            # the worker is gone: fail its request, release its memory, let the
            # other slots carry on; health() reports the dead slot
            self.alive = False
            if req is not None:
                srv._finish(req, Result(req.rid, False, error=f"worker died: {type(exc).__name__}",
                                        t_submit=req.t_submit, t_done=time.perf_counter(), slot=self.index))


class Server:
    """Continuous batching of polarization solves on one GPU (see module doc)."""

    def __init__(self, n_slots: int = 4, mem_budget_bytes: int = 8 << 30, precision: str = "mixed",
                 tol_debye: float = 1e-5, max_iter: int = 100, device: int = 0,
                 resident_budget_bytes: int = 256 << 20):
        self.device = device
        self._bind_thread()
        self.precision = precision
        self.tol = tol_debye
        self.max_iter = max_iter
        self.budget = int(mem_budget_bytes)
        self.resident_budget = int(resident_budget_bytes)
        self._cv = threading.Condition()
        self._queue: collections.deque[_Req] = collections.deque()
        self._reqs: dict[int, _Req] = {}
        self._in_use = 0
        self._running = 0
        self._next_id = 0
        self._closing = False
        self._done = 0
        self._failed = 0
        self._resident: collections.OrderedDict[str, object] = collections.OrderedDict()
        self._resident_bytes = 0
        self._slots = [_Slot(self, k) for k in range(n_slots)]
        for s in self._slots:
            s.thread.start()

    # ---------------------------------------------------------------- client side
    def submit(self, system: System, key: str | None = None) -> int:
        est = estimate_bytes(system, self.precision)
        with self._cv:
            if self._closing:
                raise RuntimeError("server is closed")
            rid = self._next_id
            self._next_id += 1
            req = _Req(rid, system, key, est, time.perf_counter())
            self._reqs[rid] = req
            if est > self.budget:
                self._finish_locked(req, Result(rid, False, error="request exceeds the memory budget",
                                                t_submit=req.t_submit, t_done=req.t_submit))
            else:
                self._queue.append(req)
                self._cv.notify_all()
        return rid

    def result(self, rid: int, timeout: float | None = None) -> Result:
        req = self._reqs[rid]
        if not req.done.wait(timeout):
            raise TimeoutError(f"request {rid} not finished")
        return req.result

    def poll(self, rid: int) -> Result | None:
        req = self._reqs[rid]
        return req.result if req.done.is_set() else None

    def cancel(self, rid: int) -> bool:
        """Cancel a request that has not started; returns False once it runs."""
        with self._cv:
            req = self._reqs[rid]
            if req in self._queue:
                self._queue.remove(req)
                self._finish_locked(req, Result(rid, False, error="cancelled", t_submit=req.t_submit,
                                                t_done=time.perf_counter()))
                return True
            return False

    def stats(self) -> dict:
        with self._cv:
            return {"queued": len(self._queue), "running": self._running, "done": self._done,
                    "failed": self._failed, "bytes_in_use": self._in_use, "budget": self.budget,
                    "resident_keys": len(self._resident), "resident_bytes": self._resident_bytes}

    def health(self) -> dict:
        return {f"slot{s.index}": s.alive and s.thread.is_alive() for s in self._slots}

    def close(self):
        with self._cv:
            self._closing = True
            self._cv.notify_all()
        for s in self._slots:
            s.thread.join()
        for s in self._slots:
            for p in list(s.periodic.values()) + ([s.cluster] if s.cluster else []):
                p.close()
        self._resident.clear()

    # ---------------------------------------------------------------- device side
    def _create_stream(self):
        import torch
        return torch.cuda.Stream(device=self.device)

    def _bind_thread(self):
        import torch
        torch.cuda.set_device(self.device)

    def _execute(self, slot: _Slot, req: _Req, res: Result):
        """Run one request on the slot's stream: lists/tiles, E0, PCG, energy."""
        import torch
        with torch.cuda.stream(slot.stream):
            p = slot.solver_for(req.system)
            p.set_synthetic(req.system)
            E0 = p.permanent_field()
            guess = self._resident_get(req.key, req.system.n)
            mu, it, rms = p.solve(E0, mu=guess)
            U = p.energy(mu, E0)
            self._resident_put(req.key, mu)
            res.mu = mu.cpu().numpy()
        res.energy, res.iters, res.rms_debye = U, it, rms
        res.warm_start = guess is not None

    # ---------------------------------------------------------------- slot side
    def _next(self, slot: _Slot):
        with self._cv:
            while True:
                if self._queue:
                    head = self._queue[0]
                    if self._in_use + head.est_bytes <= self.budget or self._running == 0:
                        self._queue.popleft()
                        self._in_use += head.est_bytes
                        self._running += 1
                        return head
                elif self._closing:
                    return None
                self._cv.wait()

    def _finish(self, req: _Req, res: Result):
        with self._cv:
            self._in_use -= req.est_bytes
            self._running -= 1
            self._finish_locked(req, res)
            self._cv.notify_all()

    def _finish_locked(self, req: _Req, res: Result):
        req.result = res
        if res.ok:
            self._done += 1
        else:
            self._failed += 1
        req.done.set()

    def _resident_get(self, key, n):
        if key is None:
            return None
        with self._cv:
            mu = self._resident.get(key)
            if mu is None or mu.shape[0] != n:
                return None
            self._resident.move_to_end(key)
            return mu.clone()

    def _resident_put(self, key, mu):
        if key is None:
            return
        nbytes = mu.numel() * mu.element_size()
        with self._cv:
            old = self._resident.pop(key, None)
            if old is not None:
                self._resident_bytes -= old.numel() * old.element_size()
            while self._resident and self._resident_bytes + nbytes > self.resident_budget:
                _, ev = self._resident.popitem(last=False)
                self._resident_bytes -= ev.numel() * ev.element_size()
            if nbytes <= self.resident_budget:
                self._resident[key] = mu.detach().clone()
                self._resident_bytes += nbytes


def request_stream(n_requests: int, seed: int = 4, min_waters: int = 64, max_waters: int = 4096):
    """Synthetic request mix: sizes log-uniform in waters, half clusters, half
    periodic boxes at 0.0334 waters per cubic Angstrom (seeded)."""
    from .synth import density_box_edge, make_waters
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.floor(np.exp(rng.uniform(math.log(min_waters), math.log(max_waters), n_requests))).astype(int)
    kinds = rng.random(n_requests) < 0.5
    out = []
    for k, (nw, is_cluster) in enumerate(zip(sizes, kinds)):
        L = density_box_edge(int(nw))
        out.append(make_waters(int(nw), L, seed * 1_000_003 + k, periodic=not is_cluster))
    return out


def percentile(xs, p):
    xs = sorted(xs)
    if not xs:
        return float("nan")
    k = min(len(xs) - 1, max(0, int(math.ceil(p / 100.0 * len(xs))) - 1))
    return xs[k]
