"""Continuous-batching server for polarization solves of uneven sizes.

A thin binding of the native server in libamoebapol (amp_server_* in
include/amoebapol.h): argument marshalling only. The scheduling, admission
by memory, the context pool, the batched engine for small clusters
(persistent kernels over a device work queue, per-request PCG state on the
device) and the worker streams all run in the library.

Requests (isolated clusters or small periodic boxes, any size) arrive at any
time; each is admitted as soon as memory and a place free up and runs beside
the requests already in flight. Small clusters without a key share the
batched engine; the other requests run on worker streams through the
single-system calls, on contexts pooled by PME grid size. Dipoles of keyed
requests stay on the device and warm-start the next solve of that key.
Failures stay per request (invalid input, a request larger than the memory
budget); the server and the other requests go on.

The paper has no serving counterpart (its throughput runs are many MPI ranks
on one system, Section "Parallel performance").
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .synth import System

PATHS = ("batched", "worker")


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
    path: str = ""
    warm_start: bool = False

    @property
    def latency(self) -> float:
        return self.t_done - self.t_submit

    @property
    def service(self) -> float:
        return self.t_done - self.t_start


class Server:
    """The native server (see the module doc). precision "mixed" or "fp64";
    clusters of at most batch_max_atoms atoms use the batched engine
    (0 disables it); n_workers worker streams take the other requests."""

    def __init__(self, n_workers: int = 4, mem_budget_bytes: int = 16 << 30, precision: str = "mixed",
                 tol_debye: float = 1e-5, max_iter: int = 100, device: int = 0, batch_max_atoms: int = 3072,
                 batch_arena_atoms: int = 1 << 19, batch_max_requests: int = 1024,
                 resident_budget_bytes: int = 256 << 20):
        from . import amoebapol as ap
        self._ap = ap
        cfg = ap.amp_server_config(n_workers=int(n_workers), mem_budget_bytes=int(mem_budget_bytes),
                                   precision=ap.AMP_MIXED if precision == "mixed" else ap.AMP_FP64,
                                   tol_debye=float(tol_debye), max_iter=int(max_iter),
                                   batch_max_atoms=int(batch_max_atoms),
                                   batch_arena_atoms=int(max(batch_arena_atoms, batch_max_atoms)),
                                   batch_max_requests=int(batch_max_requests),
                                   resident_bytes=int(resident_budget_bytes))
        self._h = ap.amp_server_create(cfg, device)
        self._n = {}

    def submit(self, system: System, key: str | None = None, cutoff: float = 0.0, beta: float = 0.0,
               grid: int = 0) -> int:
        """Queue one request; its host arrays are copied before this returns."""
        f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)  # noqa: E731
        box = 0.0 if system.box is None else float(system.box)
        rid = self._ap.amp_server_submit(self._h, system.n, box, cutoff, beta, grid, f64(system.xyz), f64(system.q),
                                         f64(system.dip), f64(system.quad), f64(system.alpha), f64(system.thole),
                                         np.ascontiguousarray(system.mol, dtype=np.int32), key)
        self._n[rid] = system.n
        return rid

    def _result(self, rid: int, code: int, mu: np.ndarray, rec) -> Result:
        ap = self._ap
        self._n.pop(rid, None)
        ok = code == ap.AMP_OK
        return Result(rid=rid, ok=ok, error=None if ok else (rec.error.decode() or f"error {code}"),
                      mu=mu if ok else None, energy=rec.energy, iters=rec.iters, rms_debye=rec.rms_debye,
                      t_submit=rec.t_submit, t_start=rec.t_start, t_done=rec.t_done,
                      path=PATHS[rec.path] if rec.path in (0, 1) else "", warm_start=bool(rec.warm_start))

    def result(self, rid: int, timeout: float | None = None) -> Result:
        """Wait for a request (without limit, or up to timeout seconds)."""
        ap = self._ap
        mu = np.zeros((self._n[rid], 3))
        rec = ap.amp_server_result()
        code = ap.amp_server_wait(self._h, rid, -1.0 if timeout is None else float(timeout), mu.ctypes.data, rec)
        if code == ap.AMP_PENDING:
            raise TimeoutError(f"request {rid} not finished")
        return self._result(rid, code, mu, rec)

    def poll(self, rid: int) -> Result | None:
        ap = self._ap
        mu = np.zeros((self._n[rid], 3))
        rec = ap.amp_server_result()
        code = ap.amp_server_poll(self._h, rid, mu.ctypes.data, rec)
        if code == ap.AMP_PENDING:
            return None
        return self._result(rid, code, mu, rec)

    def stats(self) -> dict:
        c = self._ap.amp_server_stats(self._h)
        return {name: getattr(c, name) for name, _ in c._fields_}

    def close(self):
        if self._h is not None:
            self._ap.amp_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


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
