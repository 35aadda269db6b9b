#!/usr/bin/env python
"""Benchmark of the AMOEBA polarization solve on one GB300 (or N replicas).

A step is one pass of the whole hot path on the 23,556-atom water box (the
DHFR-sized workload, float64, PCG to 1e-5 Debye): cell + neighbour lists,
per-pair tensors, permanent field (real + PME + self), the PCG solve (each
iteration one T*mu = real + PME + self) and the polarization energy.

value = unique pairs x T*mu applications in the step / step time  (pairs/s)
ms_per_step = step_ms = time of the whole step, positions to energy (the
energy is written on the device and read back after the timed steps);
solve_ms = amp_solve_induced alone, from the permanent field to the converged
dipoles. e2e: the same step with the inputs copied from pinned host memory
(one packed buffer, one copy) and mu and the energy copied back, every step. The mixed-precision step on the same box and the 96,000-atom box
(float64 and mixed) are reported beside it with their errors against the
oracle's stored solutions (tests/golden).

Multi-GPU: independent replicas (one per rank, same workload, no data-path
collective), weak scaling; a barrier and a max over ranks bracket the timing.

--impl reference times the CPU oracle (float64 numpy) on the host cores: each
step applies T once to the same workload (real + PME + self), a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "T·μ pairs/s & solve ms, FP64 vs mixed @1e-5 D RMS; serving p50/p99"
UNIT = "pairs/s"
# The headline path's arithmetic: per-pair terms, T*mu and its PME chain in
# double-float (a value is the unevaluated sum of two floats), the permanent
# field and the PCG vectors, dot products and scalars in float64.
DTYPE = "f32x2+f64"
DTYPE_NOTE = ("double-float (hi + lo float32 pairs, ~48-bit significand) for the pair terms, T*mu and its PME "
              "spreading, FFTs and gather; float64 for the permanent field E0 and the PCG vectors, dot products "
              "and scalars")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--workload", default="water-23556")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-md", action="store_true", help="skip the list-reuse trajectory measurement")
    ap.add_argument("--no-large", action="store_true", help="skip the 96,000-atom box (float64 and mixed)")
    ap.add_argument("--no-multipole", action="store_true", help="skip the permanent-multipole energy measurement")
    ap.add_argument("--multipole-only", action="store_true",
                    help="time only the permanent-multipole energy call on the workload and print it")
    ap.add_argument("--serving", action="store_true",
                    help="only the serving measurement (request stream, rates) as its own JSON line")
    ap.add_argument("--batch-only", action="store_true",
                    help="only the batched engine: the stream's small clusters, all submitted at once")
    ap.add_argument("--cluster-only", type=int, default=0, metavar="WATERS",
                    help="only single-system solves of one isolated water cluster of this many waters "
                         "(the workers' largest requests), mixed and float64")
    ap.add_argument("--requests", type=int, default=10000)
    ap.add_argument("--workers", type=int, default=6, help="serving: context workers beside the batched engine")
    ap.add_argument("--rates", default="1,2", help="serving: arrival rates as multiples of the float64 capacity")
    ap.add_argument("--rates-capacity", default="0.5,0.8",
                    help="serving: arrival rates as multiples of the server's measured capacity")
    return ap.parse_args()


# ------------------------------------------------------------------ serving

def run_md_reuse(solver, sysm, dev, dev_in, stream, flush, frames: int = 24, skin: float = 1.0,
                 speed: float = 0.01, seed: int = 9, order: int = 2):
    """An MD-like trajectory: every atom moves at a constant random velocity,
    N(0, speed) Angstrom per axis per frame (frames generated on the device
    before timing). Each frame: new positions, permanent field, solve, energy.
    Timed three times on the same frames: amp_set_system on every frame with a
    cold start; with a list skin (amp_update_positions, amp_set_system when an
    atom has moved more than skin/2) and a cold start; the same with the ASPC
    warm start of the given order."""
    import torch
    g = torch.Generator(device=dev).manual_seed(seed)
    x0 = dev_in[0]
    vel = torch.randn(tuple(x0.shape), generator=g, device=dev, dtype=torch.float64) * speed
    traj = x0.unsqueeze(0) + vel.unsqueeze(0) * torch.arange(1, frames + 1, device=dev,
                                                              dtype=torch.float64).view(-1, 1, 1)
    rest = dev_in[1:]
    E0 = torch.empty_like(x0)
    U_dev = torch.empty(1, dtype=torch.float64, device=dev)

    def run(p, reuse, predict):
        p.set_system(x0, *rest)
        rebuilds, ms, its = 0, [], []
        for f in range(frames):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if not (reuse and p.update_positions(traj[f])):
                p.set_system(traj[f], *rest)
                rebuilds += 1
            p.permanent_field(out=E0)
            mu, it, rms = p.solve(E0, predict=predict)
            p.energy_on_device(mu, E0, U_dev)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            its.append(it)
        return ms, rebuilds, its, mu

    p = solver("fp64")
    ms_full, _, it_full, mu_full = run(p, False, False)
    p.set_list_skin(skin)
    run(p, True, False)  # warm the reuse path (candidate buffers)
    ms_reuse, rebuilds, it_reuse, _ = run(p, True, False)
    p.set_predictor(order)
    ms_pred, rebuilds_p, it_pred, mu_pred = run(p, True, True)
    p.close()
    d = (mu_pred - mu_full).double()
    return {"frames": frames, "skin_angstrom": skin, "speed_angstrom_per_frame": speed,
            "ms_per_step_rebuild_every_frame": statistics.mean(ms_full),
            "mean_iters_cold": statistics.mean(it_full),
            "ms_per_step_list_reuse": statistics.mean(ms_reuse), "list_rebuilds": rebuilds,
            "ms_per_step_list_reuse_aspc": statistics.mean(ms_pred), "aspc_order": order,
            "mean_iters_aspc": statistics.mean(it_pred), "list_rebuilds_aspc": rebuilds_p,
            "last_frame_mu_rms_diff_debye": float(4.8032047 * torch.sqrt((d * d).sum() / d.shape[0]))}


def run_multipole(solver, dev_in, stream, flush, reps: int = 10):
    """Permanent-multipole energy with forces and moment gradients
    (amp_multipole_energy) on the bench system: list build by amp_set_system
    once, then `reps` calls, each timed with CUDA events on the context's
    stream and including the energy's readback to the host."""
    import torch
    from paper_1906_01211_gb300.amoebapol import amp_multipole_energy
    p = solver("fp64")
    p.set_system(*dev_in)
    n = dev_in[0].shape[0]
    outs = [torch.empty(sh, dtype=torch.float64, device=dev_in[0].device) for sh in ((n, 3), (n,), (n, 3), (n, 6))]
    ptrs = [t.data_ptr() for t in outs]
    for _ in range(3):
        U = amp_multipole_energy(p.ctx, *ptrs)
    ms = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        U = amp_multipole_energy(p.ctx, *ptrs)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    pairs = p.pair_count()
    p.close()
    return {"ms_per_call": statistics.mean(ms), "ms_min": min(ms), "U_kcal_mol": U, "unique_pairs": pairs,
            "outputs": "U, F, dU/dq, dU/dd, dU/dTheta (float64)"}


def run_serving(n_requests: int, workers: int, rates_vs_fp64, rates_vs_capacity, baseline_requests: int = 2000,
                warm: int = 60):
    """The native server (amp_server_*) on a seeded Poisson stream of solve
    requests (sizes log-uniform 64..4096 waters, half clusters, half periodic
    boxes; mixed precision, 1e-5 D), against one-at-a-time float64 solves.

    1. one-at-a-time float64 (one worker, no batched engine, each request
       submitted after the previous one finished) on the first
       baseline_requests of the stream: its throughput is the float64
       capacity, its latency the service time alone;
    2. the server saturated (all requests submitted at once): its capacity;
    3. Poisson arrivals at multiples of the server's capacity and of the
       float64 capacity: throughput, p50 and p99 latency (submission to
       result), mean iterations, and which path served the requests.
    Warm-up requests (one per PME grid size the stream needs, the largest
    box of each, and a few clusters) run first on every server, so that the
    context pool is built before the timed stream."""
    import numpy as np
    from paper_1906_01211_gb300.serve import Server, percentile, request_stream
    reqs = request_stream(n_requests + warm, seed=4)
    warm_reqs, reqs = reqs[:warm], reqs[warm:]
    # the largest periodic box per grid size, so that every pooled context is sized once
    by_grid = {}
    for r in reqs:
        if r.box is not None:
            from paper_1906_01211_gb300.synth import small_box_settings
            K = small_box_settings(r.box)[2]
            if K not in by_grid or r.n > by_grid[K].n:
                by_grid[K] = r
    warm_set = list(by_grid.values()) + warm_reqs

    def warm_up(srv):
        ids = [srv.submit(s) for s in warm_set]
        for i in ids:
            r = srv.result(i)
            if not r.ok:
                raise RuntimeError(r.error)

    base = Server(n_workers=1, precision="fp64", tol_debye=1e-5, batch_max_atoms=0)
    warm_up(base)
    sample = reqs[:baseline_requests]
    service = []
    t0 = time.perf_counter()
    for s in sample:
        r = base.result(base.submit(s))
        if not r.ok:
            raise RuntimeError(r.error)
        service.append(r.t_done - r.t_submit)
    cap64 = len(sample) / (time.perf_counter() - t0)
    base.close()
    out = {"requests": len(reqs), "workers": workers, "precision": "mixed", "tol_debye": 1e-5,
           "one_at_a_time_fp64": {"requests": len(sample), "throughput_per_s": cap64,
                                  "p50_ms": 1e3 * percentile(service, 50), "p99_ms": 1e3 * percentile(service, 99)},
           "rates": []}

    def stream(srv, lam, gaps):
        t_start = time.perf_counter()
        t_next = t_start
        ids = []
        for s, g in zip(reqs, gaps):
            if lam is not None:
                t_next += g
                dt = t_next - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
            ids.append(srv.submit(s))
        res = [srv.result(i) for i in ids]
        wall = time.perf_counter() - t_start
        bad = [r.error for r in res if not r.ok]
        if bad:
            raise RuntimeError(bad[0])
        lat = [r.latency for r in res]
        paths = {p: sum(1 for r in res if r.path == p) for p in ("batched", "worker")}
        return {"throughput_per_s": len(res) / wall, "p50_ms": 1e3 * percentile(lat, 50),
                "p99_ms": 1e3 * percentile(lat, 99), "mean_iters": float(np.mean([r.iters for r in res])),
                "served_by": paths}

    srv = Server(n_workers=workers, precision="mixed", tol_debye=1e-5)
    warm_up(srv)
    sat = stream(srv, None, [0.0] * len(reqs))
    cap = sat["throughput_per_s"]
    out["saturated"] = sat
    out["batch_launches"] = srv.stats()["batch_launches"]
    rng = np.random.Generator(np.random.PCG64(44))
    for label, f, ref in [("capacity", f, cap) for f in rates_vs_capacity] + \
                         [("fp64_capacity", f, cap64) for f in rates_vs_fp64]:
        lam = f * ref
        res = stream(srv, lam, rng.exponential(1.0 / lam, len(reqs)))
        res.update({"arrival_per_s": lam, "rate_vs": label, "factor": f})
        out["rates"].append(res)
    srv.close()
    return out


def run_cluster_only(n_waters: int, steps: int, warmup: int, seed: int = 5):
    """One isolated water cluster (all pairs, no Ewald) solved through the
    single-system calls, as the server's workers solve clusters too large for
    the batched engine: per precision the whole solve (set_system, permanent
    field, PCG to 1e-5 D with the mixed path's float64 check) with a host
    clock around it, and T*v alone with CUDA events (all-pairs interactions
    per second, n (n - 1) per application)."""
    import numpy as np
    import torch
    from paper_1906_01211_gb300 import amoebapol as ap
    from paper_1906_01211_gb300.synth import density_box_edge, make_waters
    s = make_waters(n_waters, density_box_edge(n_waters), seed, periodic=False)
    stream = torch.cuda.current_stream()
    out = {"n_atoms": s.n}
    for prec in ("mixed", "fp64"):
        p = ap.Polarization(ap.Config(box=0.0, tol_debye=1e-5, precision=prec), stream)
        ms, its = [], []
        for k in range(warmup + steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            p.set_synthetic(s)
            E0 = p.permanent_field()
            mu, it, rms = p.solve(E0)
            torch.cuda.synchronize()
            if k >= warmup:
                ms.append((time.perf_counter() - t0) * 1e3)
                its.append(it)
        v = torch.randn(s.n, 3, dtype=torch.float64, device="cuda", generator=torch.Generator(
            device="cuda").manual_seed(seed)) * 0.1
        p.apply_T(v)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            p.apply_T(v)
        e1.record(stream)
        e1.synchronize()
        t_ms = e0.elapsed_time(e1) / steps
        out[prec] = {"solve_ms_median": float(np.median(ms)), "iters": its[-1], "apply_T_ms": t_ms,
                     "pair_terms_per_s": s.n * (s.n - 1) / (t_ms / 1e3)}
        p.close()
    return out


def run_batch_only(n_requests: int, max_waters: int = 1024):
    """The batched engine alone: the stream's clusters of at most max_waters
    waters, submitted at once (after a warm-up of 32), solved to 1e-5 D in
    mixed precision. Reports solves/s and the all-pairs interactions per
    second of the pair phase (n (n - 1) per operator application)."""
    from paper_1906_01211_gb300.serve import Server, request_stream
    reqs = [s for s in request_stream(4 * n_requests, seed=4) if s.box is None and s.n <= 3 * max_waters]
    warm, reqs = reqs[:32], reqs[32:32 + n_requests]
    with Server(n_workers=1, precision="mixed", tol_debye=1e-5) as srv:
        for i in [srv.submit(s) for s in warm]:
            srv.result(i)
        l0 = srv.stats()["batch_launches"]
        t0 = time.perf_counter()
        ids = [srv.submit(s) for s in reqs]
        res = [srv.result(i) for i in ids]
        wall = time.perf_counter() - t0
        launches = srv.stats()["batch_launches"] - l0
    bad = [r.error for r in res if not r.ok or r.path != "batched"]
    if bad:
        raise RuntimeError(bad[0])
    pair_terms = sum(s.n * (s.n - 1) * (r.iters + 2) for s, r in zip(reqs, res))
    return {"requests": len(reqs), "waters_max": max_waters, "solves_per_s": len(reqs) / wall, "wall_s": wall,
            "kernel_launches": launches, "mean_iters": sum(r.iters for r in res) / len(res),
            "pair_terms_per_s": pair_terms / wall,
            "note": "pair terms = n (n - 1) per T*v application (iterations + the initial residual + the "
                    "float64 check), E0 not counted"}


def max_over_ranks(t_ms: float, world: int, device) -> float:
    """The largest of every rank's time (t_ms itself on one rank): the job
    takes as long as its slowest replica."""
    if world <= 1:
        return t_ms
    import torch
    tt = torch.tensor([t_ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
    return float(tt.item())


def whole_job_rate(units_per_rank: float, world: int, t_ms: float) -> float:
    """Units per second of the whole job: every rank processes the same
    units (weak scaling, independent replicas) in at most t_ms."""
    return world * units_per_rank / (t_ms / 1e3)


class Staging:
    """A step's input arrays in one pinned host buffer and one device buffer,
    each array at a 256-byte offset: the end-to-end loop moves them with one
    host-to-device copy per step (one copy-engine transfer instead of one per
    array). ``views`` are the device arrays (fixed views of the device buffer);
    ``nbytes`` is what one upload copies."""

    def __init__(self, arrays, dev):
        import torch
        offs, o = [], 0
        for a in arrays:
            offs.append(o)
            o += (a.nbytes + 255) // 256 * 256
        self.nbytes = o
        self.host = torch.empty(o, dtype=torch.uint8).pin_memory()
        self.dev = torch.empty(o, dtype=torch.uint8, device=dev)
        self.views = []
        for a, off in zip(arrays, offs):
            t = torch.from_numpy(a)
            self.host[off:off + a.nbytes].copy_(t.reshape(-1).view(torch.uint8))
            self.views.append(self.dev[off:off + a.nbytes].view(t.dtype).view(t.shape))
        self.dev.copy_(self.host)

    def upload(self):
        self.dev.copy_(self.host, non_blocking=True)
        return self.views


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


# ------------------------------------------------------------------ oracle side

def cpu_model() -> str:
    """The host CPU's model name (lscpu), for the baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def _oracle_worker(conn, workload_name: str, part: int, parts: int):
    """One process of the oracle pool. With one part it computes the whole
    T*mu. With several, part 0 computes the reciprocal and self terms and part
    k >= 1 the real-space terms of every (parts-1)-th unique pair from k-1 on
    (the oracle's own PairTerms and dipole_field_real on that subset of the
    pair list). Receives mu, sends its partial T*mu."""
    import numpy as np
    from oracle import Setup
    from oracle.pairs import pairs_for
    from oracle.pme import PmeGrid, dipole_field_recip, self_field
    from oracle.realspace import PairTerms, dipole_field_real
    from paper_1906_01211_gb300.synth import WORKLOADS
    w = WORKLOADS[workload_name]
    sysm = w.system()
    st = Setup(box=w.L, cutoff=w.cutoff, beta=w.beta, grid=w.grid, order=w.order)
    i, j, r = pairs_for(sysm.xyz, st)
    terms = None
    if parts == 1 or part > 0:
        sel = slice(0, None, 1) if parts == 1 else slice(part - 1, None, parts - 1)
        terms = PairTerms(sysm, st, i[sel], j[sel], r[sel])
    grid = PmeGrid(sysm.xyz, st.box, st.grid, st.order, st.beta) if part == 0 else None
    conn.send(len(i))
    while True:
        mu = conn.recv()
        if mu is None:
            break
        t = np.zeros_like(mu)
        if terms is not None:
            t = t + dipole_field_real(sysm, st, mu, terms)
        if grid is not None:
            t = t + dipole_field_recip(sysm, st, mu, grid) + self_field(st, mu)
        conn.send(t)
    conn.close()


class OraclePool:
    """The float64 numpy oracle's T*mu split over `procs` processes, each
    single-threaded (started with spawn, so it is safe beside CUDA): the
    harness divides the pair list and sums the partial fields; every term is
    the oracle's own code."""

    def __init__(self, workload_name: str, procs: int):
        import multiprocessing as mp
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[var] = "1"
        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for k in range(procs):
            a, b = ctx.Pipe()
            pr = ctx.Process(target=_oracle_worker, args=(b, workload_name, k, procs), daemon=True)
            pr.start()
            self.conns.append(a)
            self.procs.append(pr)
        self.n_pairs = [c.recv() for c in self.conns][0]

    def apply_T(self, mu):
        for c in self.conns:
            c.send(mu)
        out = None
        for c in self.conns:
            t = c.recv()
            out = t if out is None else out + t
        return out

    def close(self):
        for c in self.conns:
            try:
                c.send(None)
            except Exception:
                pass
        for pr in self.procs:
            pr.join(timeout=10)


def oracle_sample(workload, steps: int, warmup: int, procs: int = 1):
    """Time T*mu applications (real + PME + self, float64 numpy oracle) on the
    workload, one per step, on `procs` single-threaded host processes."""
    import numpy as np
    t0 = time.perf_counter()
    pool = OraclePool(workload.name, procs)
    t_build = time.perf_counter() - t0
    try:
        mu = np.random.default_rng(0).normal(size=(3 * workload.n_waters, 3)) * 0.1
        for _ in range(warmup):
            pool.apply_T(mu)
        times = []
        for _ in range(steps):
            t0 = time.perf_counter()
            pool.apply_T(mu)
            times.append(time.perf_counter() - t0)
    finally:
        pool.close()
    return pool.n_pairs, times, t_build


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baselines(workload, steps_one: int = 2, steps_all: int = 8):
    """The oracle's T*mu pairs/s on one host core and on every host core."""
    cores = host_cores()
    model = cpu_model()
    pairs, t1, b1 = oracle_sample(workload, steps_one, 0, 1)
    out = {"value": pairs * len(t1) / sum(t1), "unit": UNIT, "cores": 1, "kind": "oracle",
           "cpu_model": model, "host_cores": cores,
           "sample": f"{len(t1)} T*mu applications (real+PME+self) of the float64 numpy oracle on "
                     f"{workload.name}, one single-threaded process; geometry terms built once "
                     f"({b1:.1f} s, untimed)"}
    if cores > 1:
        pairs, ta, ba = oracle_sample(workload, steps_all, 1, cores)
        out["all_cores"] = {"value": pairs * len(ta) / sum(ta), "unit": UNIT, "cores": cores,
                            "sample": f"{len(ta)} T*mu applications after one warm-up on {cores} "
                                      f"single-threaded processes: the reciprocal and self terms in one, the "
                                      f"real-space pair list split over the others, partial fields summed by "
                                      f"the harness"}
    return out


def oracle_multipole_sample(workload, pairs_sample: int = 200_000):
    """The CPU oracle's permanent-multipole energy and gradients on the
    workload, timed on a bounded sample: the real-space pair terms of the
    first `pairs_sample` unique pairs (scaled to all pairs) plus one full
    reciprocal evaluation."""
    from oracle import Setup
    from oracle.multipole import real_space, reciprocal
    from oracle.pairs import periodic_pairs
    w = workload
    sysm = w.system()
    st = Setup(box=w.L, cutoff=w.cutoff, beta=w.beta, grid=w.grid, order=w.order)
    i, j, r = periodic_pairs(sysm.xyz, st.box, st.cutoff)
    p = min(pairs_sample, len(i))
    t0 = time.perf_counter()
    real_space(sysm, st, (i[:p], j[:p], r[:p]))
    t_real = time.perf_counter() - t0
    t0 = time.perf_counter()
    reciprocal(sysm, st)
    t_rec = time.perf_counter() - t0
    est = t_real * len(i) / p + t_rec
    return {"ms_per_call": 1e3 * est, "cores": 1, "kind": "oracle",
            "sample": f"real-space pair terms of {p} of {len(i)} unique pairs ({t_real:.1f} s, scaled to all "
                      f"pairs) + one reciprocal evaluation ({t_rec:.1f} s) of the float64 numpy oracle on {w.name}"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_1906_01211_gb300.synth import WORKLOADS
    w = WORKLOADS[args.workload]
    cores = host_cores()
    pairs, times, t_build = oracle_sample(w, args.steps, args.warmup, cores)
    total = sum(times)
    value = pairs * len(times) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w.name, "n_atoms": 3 * w.n_waters, "box": w.L,
                                        "pme_grid": w.grid, "cutoff": w.cutoff, "beta": w.beta},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
                         "sample": f"{len(times)} T*mu applications (real+PME+self) on {w.name} on {cores} "
                                   f"single-threaded processes (reciprocal and self terms in one, the "
                                   f"real-space pair list split over the others); operator geometry built "
                                   f"once ({t_build:.1f} s, untimed)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ rooflines

# Canonical float64 work of one unique pair in the pair build (tensor + both
# permanent fields): the arithmetic of the formulas, each of erfc, the two
# exp, sqrt and 1/r counted as one operation (their internal polynomials are
# not algorithmic work).
PAIR_BUILD_FLOPS = 130
# The pair build runs in double-float on the float32 pipe; one float64
# operation of the formulas costs about DF_FP32_PER_FP64 float32 operations
# (the df_* helpers: a double-float multiply-add is one multiply, three fused
# multiply-adds and about nine adds).
DF_FP32_PER_FP64 = 13
# DRAM traffic (read + write) per launch of k_t_real_df on water-23556, from
# one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of the
# current kernel (empty until the current kernel has been captured).
T_REAL_TRAFFIC = {"water-23556": 68.4e6}
# kernels launched by one amp_polarization_energy_noalloc call (block partials, final sum)
NOALLOC_ENERGY_LAUNCHES = 2


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def kernel_rooflines(phases, n_pairs, n_atoms, workload=None, K=0):
    """Roofline entries from the live phase timers (one kernel per phase).

    real-space T*v (k_t_real_df): bound "hbm". achieved = the algorithmic
    bytes of one T*mu, 80 B per atom (float64 position, dipole, damping
    factor and output field) + 4 B per unique pair (a half-list index),
    divided by the kernel's average launch time; peak = MEASURED_PEAKS.json
    hbm_gbs. This kernel does not recompute the damped radial terms: it
    streams the tensor's two scalars stored per directed entry (16 B) with
    the neighbour index (4 B), rebuilds r from the positions, and reads
    132 B per atom (positions and v as hi/lo floats, v and the output in
    float64, the row start), 8x the algorithmic bytes at water-23556; those
    bytes are reported as stored_tensor_bytes with their own fraction, and
    the DRAM traffic measured by ncu as traffic.
    pair build (k_pair_build_df): bound "alu" on the float32 pipe, which runs
    it in double-float; achieved = PAIR_BUILD_FLOPS float64 operations per
    unique pair / launch time, peak = the float32 pipe's rate divided by
    DF_FP32_PER_FP64 (152 SMs x 128 lanes x 2 flop x max SM clock / 13), the
    float64-equivalent rate of double-float arithmetic on this GPU.
    """
    peaks = measured_peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    df_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12 / DF_FP32_PER_FP64
    hbm = peaks.get("hbm_gbs")
    peak = hbm if hbm else 6800.0
    steps_seen = max(1, phases["pair"][1])
    out = []
    ms, cnt = phases["t_real"]
    if cnt:
        per = ms / cnt
        nbytes = 80 * n_atoms + 4 * n_pairs
        stored = (16 + 4) * 2 * n_pairs + 132 * n_atoms
        ach = nbytes / (per / 1e3) / 1e9
        ach_stored = stored / (per / 1e3) / 1e9
        out.append({"kernel": "k_t_real_df (real-space T*v, double-float)", "bound": "hbm", "achieved": ach,
                    "peak": peak, "unit": "GB/s", "frac": ach / peak,
                    "traffic": T_REAL_TRAFFIC.get(workload), "algorithmic_bytes": nbytes,
                    "stored_tensor_bytes": stored, "achieved_stored": ach_stored, "frac_stored": ach_stored / peak,
                    "launch_ms": per, "ms_per_step": ms / steps_seen,
                    "peak_source": "measured" if hbm else "fallback"})
    # the reciprocal chain of one T*mu and the cell search, from their
    # sub-phase timers: bytes each must move at least once (grids of K^3
    # points, per-atom weights), against the HBM copy rate; their working
    # sets (2 MB grids at K = 64) sit in the 129 MB L2, so these fractions
    # say how far from a streaming bound the latency-bound steps are
    if K:
        nh = K * K * (K // 2 + 1)
        for key, kern, nbytes in (
                ("t_spread", "k_spread_dipoles_fx (dipole spreading, fixed point)", 8 * K ** 3 + 288 * n_atoms),
                ("t_fft", "k_fft_plane_fwd + k_fft_x_conv + k_fft_plane_inv (double-float, 3 passes)",
                 16 * K ** 3 + 72 * nh),
                ("t_gather", "k_gather_field_df (field gather, double-float)", 8 * K ** 3 + 288 * n_atoms),
                ("list_search", "k_neighbours<2> (cell search, owned neighbours into slab rows)", 16 * n_atoms + 4 * n_pairs)):
            ms, cnt = phases.get(key, (0.0, 0))
            if cnt:
                per = ms / cnt
                ach = nbytes / (per / 1e3) / 1e9
                out.append({"kernel": kern, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                            "frac": ach / peak, "traffic": None, "algorithmic_bytes": nbytes, "launch_ms": per,
                            "ms_per_step": ms / steps_seen, "peak_source": "measured" if hbm else "fallback"})
    ms, cnt = phases["pair"]
    if cnt:
        per = ms / cnt
        ach = PAIR_BUILD_FLOPS * n_pairs / (per / 1e3) / 1e12
        out.append({"kernel": "k_pair_build_df (tensors + permanent fields per unique pair, double-float)",
                    "bound": "alu", "achieved": ach, "peak": df_peak, "unit": "TFLOP/s", "frac": ach / df_peak,
                    "traffic": None, "launch_ms": per, "ms_per_step": ms / steps_seen,
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock / 13 (double-float cost)"})
    return out


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(gpu_index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ precision runs

def load_oracle_solution(name: str):
    """The oracle's stored solutions of a box (tests/golden, written by
    make_oracle_solutions.py), or None."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", name.replace("-", "") + "_oracle.npz")
    if not os.path.exists(path):
        return None
    return np.load(path)


def oracle_errors(mu, U, gold):
    """Errors of a GPU solution (mu on the device, U) against the oracle's
    solutions of the box: the run to the box's tolerance and the converged one."""
    import numpy as np
    m = mu.double().cpu().numpy()
    out = {}
    for key, mkey, ukey in (("vs_oracle_at_tol", "mu_tol", "U_tol"), ("vs_oracle_converged", "mu", "U")):
        d = m - gold[mkey]
        out[key] = {"rms_debye": float(4.8032047 * np.sqrt((d * d).sum() / d.shape[0])),
                    "max_atom_debye": float(4.8032047 * np.linalg.norm(d, axis=1).max()),
                    "energy_rel": abs(U / float(gold[ukey]) - 1.0)}
    out["oracle_iters"] = {"at_tol": int(gold["iters_tol"]), "converged": int(gold["iters"]),
                           "converged_tol_debye": float(gold["tol_debye"])}
    return out


def precision_run(ap, w, precision, dev_in, stream, flush, warmup, steps, mu_ref=None, U_ref=None, gold=None):
    """Whole steps (set_system, permanent field, solve, energy) of workload w
    in one precision, timed with CUDA events on the context's stream: step_ms
    per step and solve_ms from the permanent field to the converged dipoles
    (amp_solve_induced); phase times on three more steps with the library's
    timers. Errors against a reference solution and the oracle's stored ones."""
    import torch
    p = ap.Polarization(ap.Config(box=w.L, cutoff=w.cutoff, ewald_beta=w.beta, pme_grid=w.grid,
                                  tol_debye=w.tol_debye, precision=precision), stream)
    step_ms, solve_ms = [], []
    U_dev = torch.empty(1, dtype=torch.float64, device=dev_in[0].device)
    for k in range(warmup + steps):
        flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        p.set_system(*dev_in)
        E0 = p.permanent_field()
        ev[1].record(stream)
        mu, it, rms = p.solve(E0)
        ev[2].record(stream)
        p.energy_on_device(mu, E0, U_dev)
        ev[3].record(stream)
        ev[3].synchronize()
        if k >= warmup:
            step_ms.append(ev[0].elapsed_time(ev[3]))
            solve_ms.append(ev[1].elapsed_time(ev[2]))
    torch.cuda.synchronize()
    U = float(U_dev.item())
    p.profile(True)
    for _ in range(3):
        flush.zero_()
        p.set_system(*dev_in)
        E0p = p.permanent_field()
        mup, _, _ = p.solve(E0p)
        p.energy_on_device(mup, E0p, U_dev)
    torch.cuda.synchronize()
    phases = p.profile_read()
    p.profile(False)
    n_pairs = p.pair_count()
    out = {"precision": precision, "step_ms": statistics.mean(step_ms), "solve_ms": statistics.mean(solve_ms),
           "iters": it, "fp64_checks": p.last_solve_stats()[1], "unique_pairs": n_pairs,
           "tmu_pairs_per_s_in_solve": n_pairs * (it + (1 if precision == "mixed" else 0)) /
           (statistics.mean(solve_ms) / 1e3),
           "phase_ms_per_step": {k: round(v[0] / 3, 4) for k, v in phases.items()}}
    if mu_ref is not None:
        d = (mu - mu_ref).double()
        out["rms_vs_fp64_gpu_debye"] = float(4.8032047 * torch.sqrt((d * d).sum() / d.shape[0]))
        out["energy_rel_vs_fp64_gpu"] = abs(U / U_ref - 1.0)
    if gold is not None:
        out.update(oracle_errors(mu, U, gold))
    p.close()
    return out, mu, U


def run_large_box(ap, dev, stream, flush):
    """The 96,000-atom box at its own tolerance (1e-5 D): float64 and mixed
    whole steps, each against the oracle's stored solutions."""
    import numpy as np
    import torch
    from paper_1906_01211_gb300.synth import WATER_96000
    w = WATER_96000
    sysm = w.system()
    host = [np.ascontiguousarray(a) for a in
            (sysm.xyz, sysm.q, sysm.dip, sysm.quad, sysm.alpha, sysm.thole, sysm.mol.astype(np.int32))]
    dev_in = [torch.from_numpy(a).to(dev) for a in host]
    gold = load_oracle_solution(w.name)
    f64, mu64, U64 = precision_run(ap, w, "fp64", dev_in, stream, flush, 2, 3, gold=gold)
    mix, _, _ = precision_run(ap, w, "mixed", dev_in, stream, flush, 2, 3, mu_ref=mu64, U_ref=U64, gold=gold)
    return {"workload": w.name, "n_atoms": sysm.n, "box": w.L, "pme_grid": w.grid, "tol_debye": w.tol_debye,
            "fp64": f64, "mixed": mix, "mixed_solve_speedup_vs_fp64": f64["solve_ms"] / mix["solve_ms"]}


# ------------------------------------------------------------------ GPU side

def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    rank, world, local = dist_env()
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    if args.cluster_only:
        if rank == 0:
            print(json.dumps({"config": {"workload": f"isolated water cluster, {args.cluster_only} waters"},
                              "cluster_solve": run_cluster_only(args.cluster_only, args.steps, args.warmup)}),
                  flush=True)
        return
    if args.batch_only:
        if rank == 0:
            print(json.dumps({"config": {"workload": "small water clusters of the request stream"},
                              "batched_engine": run_batch_only(min(args.requests, 2000))}), flush=True)
        return
    if args.serving:
        if rank == 0:
            sv = run_serving(args.requests, args.workers, [float(x) for x in args.rates.split(",")],
                             [float(x) for x in args.rates_capacity.split(",")])
            print(json.dumps({"metric": "serving solves/s and p50/p99 latency", "unit": "solves/s",
                              "value": sv["saturated"]["throughput_per_s"], "higher_is_better": True,
                              "dtype": "f32+f64", "data": "synthetic",
                              "config": {"workload": "water request stream (64..4096 waters, half clusters)"},
                              "serving": sv}), flush=True)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1906_01211_gb300 import amoebapol as ap
    from paper_1906_01211_gb300.synth import WORKLOADS

    w = WORKLOADS[args.workload]
    sysm = w.system()
    n = sysm.n
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    def solver(precision):
        return ap.Polarization(ap.Config(box=w.L, cutoff=w.cutoff, ewald_beta=w.beta, pme_grid=w.grid,
                                         tol_debye=w.tol_debye, precision=precision), stream)

    host = [np.ascontiguousarray(a) for a in
            (sysm.xyz, sysm.q, sysm.dip, sysm.quad, sysm.alpha, sysm.thole, sysm.mol.astype(np.int32))]
    staging = Staging(host, dev)
    dev_in = [t.clone() for t in staging.views]
    h2d_bytes = staging.nbytes
    E0 = torch.empty((n, 3), dtype=torch.float64, device=dev)
    U_dev = torch.empty(1, dtype=torch.float64, device=dev)
    mu_host = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    U_host = torch.empty(1, dtype=torch.float64).pin_memory()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    if args.multipole_only:
        if rank == 0:
            print(json.dumps({"config": {"workload": w.name, "n_atoms": n},
                              "multipole_energy": run_multipole(solver, dev_in, stream, flush)}), flush=True)
        return

    p = solver("fp64")
    n_pairs = None

    # The energy stays on the device (read back after the loop, and by the
    # end-to-end loop inside its timed region with mu): a host read of U
    # would add a synchronisation to every step.
    def step(inputs, marks=None):
        p.set_system(*inputs)
        p.permanent_field(out=E0)
        if marks:
            marks[0].record(stream)
        mu, it, rms = p.solve(E0)
        if marks:
            marks[1].record(stream)
        p.energy_on_device(mu, E0, U_dev)
        return mu, it, rms

    for _ in range(args.warmup):
        mu, it, rms = step(dev_in)
    n_pairs = p.pair_count()

    # ---- device-resident timed region
    clocks = ClockSampler(local) if rank == 0 else None
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = p.launch_count()
    step_ms, solve_ms, applications = [], [], []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        marks = [torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
        e0.record(stream)
        mu, it, rms = step(dev_in, marks)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        solve_ms.append(marks[0].elapsed_time(marks[1]))
        applications.append(1 + it)
    torch.cuda.synchronize()
    U = float(U_dev.item())
    # the context counts its own launches; the energy's two kernels per step
    # (amp_polarization_energy_noalloc, no context) are added here
    launches = p.launch_count() - launches0 + NOALLOC_ENERGY_LAUNCHES * args.steps
    clk = clocks.stop() if clocks else None
    t_total = max_over_ranks(sum(step_ms), world, dev)
    apps = sum(applications)
    value = whole_job_rate(n_pairs * apps, world, t_total)

    # ---- end to end through the public API with host buffers
    e2e_ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mu, it, rms = step(staging.upload())
        mu_host.copy_(mu, non_blocking=True)
        U_host.copy_(U_dev, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_total = max_over_ranks(sum(e2e_ms), world, dev)
    e2e_value = whole_job_rate(n_pairs * apps, world, e2e_total)
    d2h_bytes = mu_host.numel() * 8 + U_host.numel() * 8

    if rank != 0:
        if world > 1:
            torch.distributed.barrier()
        return

    # ---- phase timers (library events around each phase) on separate steps:
    # the event records cost ~0.1 ms per step, so the timed steps above run
    # without them
    prof_steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    p.profile(True)
    for _ in range(prof_steps):
        flush.zero_()
        step(dev_in)
    torch.cuda.synchronize()
    phases = p.profile_read()
    p.profile(False)

    # ---- rooflines of our two largest kernels; the dominant one is "roofline"
    rooflines = kernel_rooflines(phases, n_pairs, n, w.name, w.grid)
    roofline = max(rooflines, key=lambda r: r["ms_per_step"])
    phase_ms = {k: round(v[0] / prof_steps, 4) for k, v in phases.items()}

    # ---- mixed precision on the same workload, against the float64 result
    # and against the oracle's solutions of this box
    mixed = None
    gold = load_oracle_solution(w.name)
    if gold is not None:
        fp64_err = oracle_errors(mu, U, gold)
    else:
        fp64_err = None
    if not args.no_mixed:
        mixed, _, _ = precision_run(ap, w, "mixed", dev_in, stream, flush, args.warmup, 3, mu_ref=mu, U_ref=U,
                                    gold=gold)

    # ---- the 96,000-atom box (Puddle-sized), float64 and mixed
    large = None
    if not args.no_large and w.name != "water-96000":
        large = run_large_box(ap, dev, stream, flush)
    serving = None
    if not args.no_serving:
        serving = run_serving(args.requests, args.workers, [float(x) for x in args.rates.split(",")],
                              [float(x) for x in args.rates_capacity.split(",")])

    # ---- list reuse along a trajectory (not the headline step: every frame is
    # new positions, so each step does its full work except the cell search,
    # which the reuse path replaces by filtering the stored candidates)
    md = None
    if not args.no_md:
        md = run_md_reuse(solver, sysm, dev, dev_in, stream, flush)

    mpole = None
    if not args.no_multipole:
        mpole = run_multipole(solver, dev_in, stream, flush)
        if not args.no_cpu_baseline and rank == 0:
            mpole["cpu_baseline"] = oracle_multipole_sample(w)

    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baselines(w)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE, "dtype_note": DTYPE_NOTE, "data": "synthetic",
        "config": {"workload": w.name, "n_atoms": n, "box": w.L, "cutoff": w.cutoff, "beta": w.beta,
                   "pme_grid": w.grid, "tol_debye": w.tol_debye, "unique_pairs": n_pairs,
                   "tmu_applications_per_step": apps / args.steps,
                   "l2": "256 MB buffer written between timed steps",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "step_ms": t_total / args.steps,
        "solve_ms": statistics.mean(solve_ms),
        "iters": it,
        "fp64_vs_oracle": fp64_err,
        "tmu_pairs_per_s_operator": n_pairs / ((phases["t_real"][0] + phases["t_recip"][0])
                                               / max(phases["t_real"][1], 1) / 1e3),
        "phase_ms_per_step": phase_ms,
        "mixed": mixed,
        "mixed_solve_speedup_vs_fp64": (statistics.mean(solve_ms) / mixed["solve_ms"]) if mixed else None,
        "water_96000": large,
        "serving": serving,
        "md_list_reuse": md,
        "multipole_energy": mpole,
        "roofline": roofline,
        "roofline_other": [r for r in rooflines if r is not roofline],
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d_bytes,
                "d2h_bytes_per_step": d2h_bytes, "ms_per_step": e2e_total / args.steps},
        "gpu_launches": launches,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()


if __name__ == "__main__":
    main()
