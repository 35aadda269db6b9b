"""Python binding of libamoebapol (the C ABI in include/amoebapol.h).

Argument marshalling only: every step of the computation runs in the CUDA
library. The low-level functions carry the C names; ``Polarization`` wraps
them for torch CUDA tensors (PyTorch supplies device memory and the stream).

Importing this module loads ``libamoebapol.so`` and raises if it is missing:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libamoebapol.so")
HEADER_PATH = os.path.join(os.path.dirname(_HERE), "include", "amoebapol.h")

AMP_OK = 0
AMP_ERR_ARG = -1
AMP_ERR_CUDA = -2
AMP_ERR_OOM = -3
AMP_ERR_NOT_CONVERGED = -4
AMP_ERR_GEOMETRY = -5
AMP_ERR_STATE = -6
AMP_ERR_STALE = -8
AMP_FP64 = 0
AMP_MIXED = 1
PHASES = ("list", "pair", "e0_real", "e0_recip", "t_real", "t_recip", "pcg", "fp64_check", "energy", "forces",
          "t_spread", "t_fft", "t_gather", "list_search")


class amp_config(ctypes.Structure):
    _fields_ = [
        ("box", ctypes.c_double),
        ("cutoff", ctypes.c_double),
        ("ewald_beta", ctypes.c_double),
        ("pme_grid", ctypes.c_int),
        ("pme_order", ctypes.c_int),
        ("tol_debye", ctypes.c_double),
        ("max_iter", ctypes.c_int),
        ("precision", ctypes.c_int),
    ]


class amp_server_config(ctypes.Structure):
    _fields_ = [
        ("n_workers", ctypes.c_int),
        ("mem_budget_bytes", ctypes.c_longlong),
        ("precision", ctypes.c_int),
        ("tol_debye", ctypes.c_double),
        ("max_iter", ctypes.c_int),
        ("batch_max_atoms", ctypes.c_int),
        ("batch_arena_atoms", ctypes.c_int),
        ("batch_max_requests", ctypes.c_int),
        ("resident_bytes", ctypes.c_longlong),
    ]


class amp_server_result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("iters", ctypes.c_int),
        ("rms_debye", ctypes.c_double),
        ("energy", ctypes.c_double),
        ("t_submit", ctypes.c_double),
        ("t_start", ctypes.c_double),
        ("t_done", ctypes.c_double),
        ("path", ctypes.c_int),
        ("warm_start", ctypes.c_int),
        ("error", ctypes.c_char * 160),
    ]


class amp_server_counters(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_longlong),
        ("done", ctypes.c_longlong),
        ("failed", ctypes.c_longlong),
        ("queued", ctypes.c_int),
        ("running_batch", ctypes.c_int),
        ("running_workers", ctypes.c_int),
        ("contexts", ctypes.c_int),
        ("bytes_in_use", ctypes.c_longlong),
        ("budget", ctypes.c_longlong),
        ("batch_launches", ctypes.c_longlong),
    ]


class AmpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libamoebapol error {code}: {msg}")
        self.code = code


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} not found: build it with `python -m paper_1906_01211_gb300.build` "
            "(the CUDA library is required; there is no CPU path)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    I = ctypes.c_int
    D = ctypes.c_double
    sig = {
        "amp_create": (I, [ctypes.POINTER(P), ctypes.POINTER(amp_config), P]),
        "amp_destroy": (None, [P]),
        "amp_reconfigure": (I, [P, ctypes.POINTER(amp_config)]),
        "amp_last_error": (ctypes.c_char_p, [P]),
        "amp_set_system": (I, [P, I, P, P, P, P, P, P, P]),
        "amp_permanent_field": (I, [P, P]),
        "amp_apply_T": (I, [P, P, P]),
        "amp_solve_induced": (I, [P, P, P, I, ctypes.POINTER(I), ctypes.POINTER(D)]),
        "amp_polarization_energy": (I, [P, P, P, ctypes.POINTER(D)]),
        "amp_pair_count": (I, [P, ctypes.POINTER(ctypes.c_longlong)]),
        "amp_forces": (I, [P, P, P, P, P, P]),
        "amp_multipole_energy": (I, [P, ctypes.POINTER(D), P, P, P, P]),
        "amp_profile": (I, [P, I]),
        "amp_profile_read": (I, [P, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_longlong)]),
        "amp_last_solve_stats": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "amp_launch_count": (I, [P, ctypes.POINTER(ctypes.c_longlong)]),
        "amp_polarization_energy_noalloc": (I, [I, P, P, P, P]),
        "amp_set_list_skin": (I, [P, D]),
        "amp_update_positions": (I, [P, P, ctypes.POINTER(I)]),
        "amp_set_predictor": (I, [P, I]),
        "amp_predictor_coefficients": (I, [I, ctypes.POINTER(D)]),
        "amp_tcg1": (I, [P, P, P, ctypes.POINTER(D), P, P, P, P]),
        "amp_dcji": (I, [P, P, P, I, D, I, P, ctypes.POINTER(I), ctypes.POINTER(D)]),
        "amp_permanent_field_scaled": (I, [P, D, P]),
        "amp_two_rhs_forces": (I, [P, D, P, P, P, P, P, P]),
        "amp_frames_to_global": (I, [I, P, P, P, P, P, P, P, P, P]),
        "amp_frame_forces": (I, [I, P, P, P, P, P, P, P, P, P, P]),
        "amp_server_create": (I, [ctypes.POINTER(P), ctypes.POINTER(amp_server_config), I]),
        "amp_server_submit": (I, [P, I, D, D, D, I, P, P, P, P, P, P, P, ctypes.c_char_p,
                                  ctypes.POINTER(ctypes.c_longlong)]),
        "amp_server_poll": (I, [P, ctypes.c_longlong, P, ctypes.POINTER(amp_server_result)]),
        "amp_server_wait": (I, [P, ctypes.c_longlong, D, P, ctypes.POINTER(amp_server_result)]),
        "amp_server_stats": (I, [P, ctypes.POINTER(amp_server_counters)]),
        "amp_server_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def header_functions() -> list[str]:
    """Names of the functions declared in include/amoebapol.h."""
    text = open(HEADER_PATH).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+\**(amp_\w+)\s*\(", text, re.M)))


def _check(ctx, code: int):
    if code != AMP_OK:
        msg = _lib.amp_last_error(ctx)
        raise AmpError(code, msg.decode() if msg else "")


# ----------------------------------------------------------------- C names

def amp_create(cfg: amp_config, stream: int | None = None):
    h = ctypes.c_void_p()
    code = _lib.amp_create(ctypes.byref(h), ctypes.byref(cfg), ctypes.c_void_p(stream or 0))
    if code != AMP_OK:
        raise AmpError(code, "amp_create: invalid configuration or device error")
    return h


def amp_destroy(ctx):
    _lib.amp_destroy(ctx)


def amp_reconfigure(ctx, cfg: amp_config):
    _check(ctx, _lib.amp_reconfigure(ctx, ctypes.byref(cfg)))


def amp_last_error(ctx) -> str:
    m = _lib.amp_last_error(ctx)
    return m.decode() if m else ""


def amp_set_system(ctx, n, xyz, q, dip, quad, alpha, thole, mol):
    _check(ctx, _lib.amp_set_system(ctx, int(n), xyz, q, dip, quad, alpha, thole, mol))


def amp_set_list_skin(ctx, skin: float):
    _check(ctx, _lib.amp_set_list_skin(ctx, float(skin)))


def amp_update_positions(ctx, xyz) -> bool:
    """True if the lists were rebuilt from the stored candidates; False if an
    atom moved more than skin/2 (then nothing changed: set the system again)."""
    reused = ctypes.c_int(0)
    code = _lib.amp_update_positions(ctx, xyz, ctypes.byref(reused))
    if code == AMP_ERR_STALE:
        return False
    _check(ctx, code)
    return bool(reused.value)


def amp_permanent_field(ctx, E0):
    _check(ctx, _lib.amp_permanent_field(ctx, E0))


def amp_apply_T(ctx, mu, Tmu):
    _check(ctx, _lib.amp_apply_T(ctx, mu, Tmu))


def amp_solve_induced(ctx, E0, mu, use_guess: int):
    """use_guess: 0 start from alpha*E0, 1 from mu, 2 from the predictor."""
    it = ctypes.c_int(0)
    rms = ctypes.c_double(0.0)
    code = _lib.amp_solve_induced(ctx, E0, mu, int(use_guess), ctypes.byref(it), ctypes.byref(rms))
    return code, it.value, rms.value


def amp_set_predictor(ctx, order: int):
    _check(ctx, _lib.amp_set_predictor(ctx, int(order)))


def amp_predictor_coefficients(order: int) -> list[float]:
    b = (ctypes.c_double * 8)()
    code = _lib.amp_predictor_coefficients(int(order), b)
    if code != AMP_OK:
        raise AmpError(code, "order must be 0 .. 6")
    return [b[j] for j in range(order + 2)]


def amp_polarization_energy(ctx, mu, E0) -> float:
    u = ctypes.c_double(0.0)
    _check(ctx, _lib.amp_polarization_energy(ctx, mu, E0, ctypes.byref(u)))
    return u.value


def amp_forces(ctx, mu, F, gq=None, gdip=None, gquad=None):
    _check(ctx, _lib.amp_forces(ctx, mu, F, gq, gdip, gquad))


def amp_permanent_field_scaled(ctx, s_intra: float, E):
    _check(ctx, _lib.amp_permanent_field_scaled(ctx, float(s_intra), E))


def amp_two_rhs_forces(ctx, s_intra: float, mu_d, mu_p, F, gq=None, gdip=None, gquad=None):
    _check(ctx, _lib.amp_two_rhs_forces(ctx, float(s_intra), mu_d, mu_p, F, gq, gdip, gquad))


def amp_tcg1(ctx, E0, mu=None, F=None, gq=None, gdip=None, gquad=None) -> float:
    """TCG-1 energy (kcal/mol); mu_1 and the gradients into the non-null device pointers."""
    u = ctypes.c_double(0.0)
    _check(ctx, _lib.amp_tcg1(ctx, E0, mu, ctypes.byref(u), F, gq, gdip, gquad))
    return u.value


def amp_dcji(ctx, E0, block_of, n_blocks: int, tol_debye: float, max_iter: int, mu) -> tuple[int, float]:
    """DC-JI into mu (device pointers E0, mu; block_of a host int32 array):
    (iterations, final RMS in Debye)."""
    import numpy as np
    b = np.ascontiguousarray(block_of, dtype=np.int32)
    it = ctypes.c_int(0)
    rms = ctypes.c_double(0.0)
    _check(ctx, _lib.amp_dcji(ctx, E0, b.ctypes.data, int(n_blocks), float(tol_debye), int(max_iter), mu,
                              ctypes.byref(it), ctypes.byref(rms)))
    return it.value, rms.value


def cell_blocks(xyz, mol, box: float, cells_per_axis: int):
    """Blocks of whole molecules for DC-JI: (block_of [N], n_blocks). A
    regular grid of cells_per_axis^3 cells over the box (box > 0) or over the
    bounding cube of the sites (box = 0); each molecule goes to the cell of
    its first site; empty cells are dropped and the remaining blocks are
    numbered in cell order."""
    import numpy as np
    xyz = np.asarray(xyz, dtype=np.float64)
    mol = np.asarray(mol)
    n = xyz.shape[0]
    if box > 0.0:
        L, lo = float(box), np.zeros(3)
    else:
        L, lo = float(np.ptp(xyz, axis=0).max()) + 1e-9, xyz.min(axis=0)
    _, first = np.unique(mol, return_index=True)
    u = (xyz[first] - lo) / L
    if box > 0.0:
        u = u - np.floor(u)
    c = np.minimum((u * cells_per_axis).astype(np.int64), cells_per_axis - 1)
    key_of_mol = dict(zip(mol[first].tolist(), ((c[:, 0] * cells_per_axis + c[:, 1]) * cells_per_axis + c[:, 2]).tolist()))
    keys = np.array([key_of_mol[m] for m in mol.tolist()], dtype=np.int64)
    used, block_of = np.unique(keys, return_inverse=True)
    return block_of.astype(np.int32).reshape(n), int(used.size)


def amp_multipole_energy(ctx, F=None, gq=None, gdip=None, gquad=None) -> float:
    """Permanent-multipole energy (kcal/mol); gradients into the non-null device pointers."""
    u = ctypes.c_double(0.0)
    _check(ctx, _lib.amp_multipole_energy(ctx, ctypes.byref(u), F, gq, gdip, gquad))
    return u.value


def amp_pair_count(ctx) -> int:
    n = ctypes.c_longlong(0)
    _check(ctx, _lib.amp_pair_count(ctx, ctypes.byref(n)))
    return n.value


def amp_profile(ctx, enable: bool):
    _check(ctx, _lib.amp_profile(ctx, int(bool(enable))))


def amp_profile_read(ctx) -> dict:
    """{phase: (milliseconds, intervals)} since profiling was enabled."""
    n = len(PHASES)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_longlong * n)()
    _check(ctx, _lib.amp_profile_read(ctx, ms, cnt))
    return {name: (ms[k], cnt[k]) for k, name in enumerate(PHASES)}


AMP_PENDING = 1


def amp_frames_to_global(n, xyz, dip_local, quad_local, kind, zatom, xatom, dip, quad, stream=None):
    code = _lib.amp_frames_to_global(int(n), xyz, dip_local, quad_local, kind, zatom, xatom, dip, quad,
                                     ctypes.c_void_p(stream or 0))
    if code != AMP_OK:
        raise AmpError(code, "amp_frames_to_global")


def amp_frame_forces(n, xyz, dip_local, quad_local, kind, zatom, xatom, gdip, gquad, F, stream=None):
    code = _lib.amp_frame_forces(int(n), xyz, dip_local, quad_local, kind, zatom, xatom, gdip, gquad, F,
                                 ctypes.c_void_p(stream or 0))
    if code != AMP_OK:
        raise AmpError(code, "amp_frame_forces")


def frames_to_global(xyz, dip_local, quad_local, kind, zatom, xatom):
    """Global (dip, quad) torch tensors from local-frame moments (torch CUDA
    tensors: float64 positions and moments, int32 frame topology)."""
    import torch
    n = xyz.shape[0]
    dip = torch.empty((n, 3), dtype=torch.float64, device=xyz.device)
    quad = torch.empty((n, 6), dtype=torch.float64, device=xyz.device)
    amp_frames_to_global(n, xyz.data_ptr(), dip_local.data_ptr(), quad_local.data_ptr(), kind.data_ptr(),
                         zatom.data_ptr(), xatom.data_ptr(), dip.data_ptr(), quad.data_ptr(),
                         torch.cuda.current_stream().cuda_stream)
    return dip, quad


def add_frame_forces(F, xyz, dip_local, quad_local, kind, zatom, xatom, gdip, gquad):
    """F += the frame terms of the forces from the moment gradients (in place)."""
    import torch
    amp_frame_forces(xyz.shape[0], xyz.data_ptr(), dip_local.data_ptr(), quad_local.data_ptr(), kind.data_ptr(),
                     zatom.data_ptr(), xatom.data_ptr(), gdip.data_ptr(), gquad.data_ptr(), F.data_ptr(),
                     torch.cuda.current_stream().cuda_stream)
    return F


def amp_server_create(cfg: amp_server_config, device: int = 0):
    h = ctypes.c_void_p()
    code = _lib.amp_server_create(ctypes.byref(h), ctypes.byref(cfg), int(device))
    if code != AMP_OK:
        raise AmpError(code, "amp_server_create: invalid configuration or device error")
    return h


def amp_server_submit(srv, n, box, cutoff, beta, grid, xyz, q, dip, quad, alpha, thole, mol, key=None) -> int:
    """Host arrays (numpy, contiguous float64 / int32) in; the ticket out."""
    t = ctypes.c_longlong(-1)
    code = _lib.amp_server_submit(srv, int(n), float(box), float(cutoff), float(beta), int(grid),
                                  xyz.ctypes.data, q.ctypes.data, dip.ctypes.data, quad.ctypes.data,
                                  alpha.ctypes.data, thole.ctypes.data, mol.ctypes.data,
                                  key.encode() if key is not None else None, ctypes.byref(t))
    if code != AMP_OK:
        raise AmpError(code, "amp_server_submit")
    return t.value


def amp_server_poll(srv, ticket: int, mu_ptr, res: amp_server_result) -> int:
    return _lib.amp_server_poll(srv, ctypes.c_longlong(ticket), mu_ptr, ctypes.byref(res))


def amp_server_wait(srv, ticket: int, timeout_s: float, mu_ptr, res: amp_server_result) -> int:
    return _lib.amp_server_wait(srv, ctypes.c_longlong(ticket), float(timeout_s), mu_ptr, ctypes.byref(res))


def amp_server_stats(srv) -> amp_server_counters:
    c = amp_server_counters()
    code = _lib.amp_server_stats(srv, ctypes.byref(c))
    if code != AMP_OK:
        raise AmpError(code, "amp_server_stats")
    return c


def amp_server_destroy(srv):
    _lib.amp_server_destroy(srv)


AMP_ERR_TOO_LARGE = -7
AMP_NOALLOC_MAX_ATOMS = 1048576


def amp_polarization_energy_noalloc(n_atoms: int, mu_ptr: int, e0_ptr: int, u_dev_ptr: int,
                                    stream: int | None = None) -> int:
    """Energy into a device double, no allocation and no context (returns the status code).

    For callers that cannot allocate device memory when they need the energy;
    see include/amoebapol.h for the limits and the sharing rules of its scratch.
    """
    return _lib.amp_polarization_energy_noalloc(int(n_atoms), mu_ptr, e0_ptr, u_dev_ptr,
                                                ctypes.c_void_p(stream or 0))


def amp_launch_count(ctx) -> int:
    n = ctypes.c_longlong(0)
    _check(ctx, _lib.amp_launch_count(ctx, ctypes.byref(n)))
    return n.value


def amp_last_solve_stats(ctx):
    it = ctypes.c_int(0)
    chk = ctypes.c_int(0)
    _check(ctx, _lib.amp_last_solve_stats(ctx, ctypes.byref(it), ctypes.byref(chk)))
    return it.value, chk.value


# ----------------------------------------------------------------- torch wrapper

@dataclass
class Config:
    box: float
    cutoff: float = 7.0
    ewald_beta: float = 0.5446
    pme_grid: int = 24
    pme_order: int = 5
    tol_debye: float = 1e-8
    max_iter: int = 100
    precision: str = "fp64"

    def to_c(self) -> amp_config:
        prec = {"fp64": AMP_FP64, "mixed": AMP_MIXED}[self.precision]
        return amp_config(self.box, self.cutoff, self.ewald_beta, self.pme_grid, self.pme_order,
                          self.tol_debye, self.max_iter, prec)


class Polarization:
    """One solver context on the current CUDA device and stream.

    Tensors are torch CUDA float64 (mol: int32), contiguous, in the caller's
    atom order: xyz/dip/E0/mu (N, 3), quad (N, 6), q/alpha/thole/mol (N,).
    """

    def __init__(self, cfg: Config, stream=None):
        import torch
        self.torch = torch
        self.cfg = cfg
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.ctx = amp_create(cfg.to_c(), self.stream.cuda_stream)
        self.n = 0
        self._keep = ()
        self.generation = 0  # bumped by every set_system

    def close(self):
        if self.ctx is not None:
            amp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, t, dtype):
        torch = self.torch
        t = torch.as_tensor(t)
        if t.device.type != "cuda" or t.dtype != dtype or not t.is_contiguous():
            t = t.to(device="cuda", dtype=dtype).contiguous()
        return t

    def set_system(self, xyz, q, dip, quad, alpha, thole, mol):
        torch = self.torch
        f64 = torch.float64
        arrs = (self._dev(xyz, f64), self._dev(q, f64), self._dev(dip, f64), self._dev(quad, f64),
                self._dev(alpha, f64), self._dev(thole, f64), self._dev(mol, torch.int32))
        self.n = int(arrs[0].shape[0])
        amp_set_system(self.ctx, self.n, *[a.data_ptr() for a in arrs])
        self._keep = arrs  # inputs stay alive while the stream may read them
        self.generation += 1

    def set_predictor(self, order: int):
        """ASPC warm start of order k (-1: off) for solve(..., predict=True)."""
        amp_set_predictor(self.ctx, order)

    def set_list_skin(self, skin: float):
        """Neighbour-list skin (Angstrom) used from the next set_system on."""
        amp_set_list_skin(self.ctx, skin)

    def update_positions(self, xyz) -> bool:
        """New positions for the current atoms; True if the lists were reused
        (rebuilt from the candidates of the last set_system), False if an atom
        moved more than skin/2 (nothing changed: call set_system)."""
        x = self._dev(xyz, self.torch.float64)
        ok = amp_update_positions(self.ctx, x.data_ptr())
        if ok:
            self._keep = (x,) + tuple(self._keep[1:])
            self.generation += 1
        return ok

    def set_synthetic(self, system):
        """Upload a ``synth.System`` (numpy arrays)."""
        self.set_system(system.xyz, system.q, system.dip, system.quad, system.alpha, system.thole, system.mol)

    def permanent_field(self, out=None):
        torch = self.torch
        out = out if out is not None else torch.empty((self.n, 3), dtype=torch.float64, device="cuda")
        amp_permanent_field(self.ctx, out.data_ptr())
        return out

    def apply_T(self, mu, out=None):
        torch = self.torch
        mu = self._dev(mu, torch.float64)
        out = out if out is not None else torch.empty_like(mu)
        amp_apply_T(self.ctx, mu.data_ptr(), out.data_ptr())
        return out

    def solve(self, E0, mu=None, check=True, predict=False):
        """Returns (mu, iterations, final RMS in Debye). mu: initial guess;
        predict: start from the predictor of set_predictor instead."""
        torch = self.torch
        E0 = self._dev(E0, torch.float64)
        guess = 2 if predict else (1 if mu is not None else 0)
        mu = self._dev(mu, torch.float64).clone() if guess == 1 else torch.empty_like(E0)
        code, it, rms = amp_solve_induced(self.ctx, E0.data_ptr(), mu.data_ptr(), guess)
        if check:
            _check(self.ctx, code)
        return mu, it, rms

    def energy(self, mu, E0) -> float:
        torch = self.torch
        mu = self._dev(mu, torch.float64)
        E0 = self._dev(E0, torch.float64)
        return amp_polarization_energy(self.ctx, mu.data_ptr(), E0.data_ptr())

    def energy_on_device(self, mu, E0, out):
        """U into out (a one-element float64 CUDA tensor) on the context's
        stream, without waiting for it (amp_polarization_energy_noalloc): a
        loop of steps reads it back when it needs it, not every step. At most
        AMP_NOALLOC_MAX_ATOMS atoms; its scratch is shared by every call of
        the process, so calls whose kernels could overlap (other streams)
        must not be issued concurrently."""
        torch = self.torch
        mu = self._dev(mu, torch.float64)
        E0 = self._dev(E0, torch.float64)
        if out.device.type != "cuda" or out.dtype != torch.float64 or out.numel() < 1:
            raise ValueError("out must be a float64 CUDA tensor with at least one element")
        code = amp_polarization_energy_noalloc(int(mu.shape[0]), mu.data_ptr(), E0.data_ptr(), out.data_ptr(),
                                               self.stream.cuda_stream)
        if code != AMP_OK:
            raise AmpError(code, "amp_polarization_energy_noalloc failed")
        return out

    def forces(self, mu):
        """(F, dU/dq, dU/dd, dU/dTheta6) at the converged dipoles mu."""
        torch = self.torch
        mu = self._dev(mu, torch.float64)
        n = mu.shape[0]
        F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        gq = torch.empty((n,), dtype=torch.float64, device="cuda")
        gd = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        gt = torch.empty((n, 6), dtype=torch.float64, device="cuda")
        amp_forces(self.ctx, mu.data_ptr(), F.data_ptr(), gq.data_ptr(), gd.data_ptr(), gt.data_ptr())
        return F, gq, gd, gt

    def permanent_field_scaled(self, s_intra: float, out=None):
        """The permanent field with scale s_intra for two sites of one molecule (E_p)."""
        torch = self.torch
        out = out if out is not None else torch.empty((self.n, 3), dtype=torch.float64, device="cuda")
        amp_permanent_field_scaled(self.ctx, s_intra, out.data_ptr())
        return out

    def two_rhs_forces(self, s_intra: float, mu_d, mu_p):
        """(F, dU/dq, dU/dd, dU/dTheta6) of U = -1/2 C mu_d . E_p at the two solutions."""
        torch = self.torch
        mu_d = self._dev(mu_d, torch.float64)
        mu_p = self._dev(mu_p, torch.float64)
        n = mu_d.shape[0]
        F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        gq = torch.empty((n,), dtype=torch.float64, device="cuda")
        gd = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        gt = torch.empty((n, 6), dtype=torch.float64, device="cuda")
        amp_two_rhs_forces(self.ctx, s_intra, mu_d.data_ptr(), mu_p.data_ptr(), F.data_ptr(), gq.data_ptr(),
                           gd.data_ptr(), gt.data_ptr())
        return F, gq, gd, gt

    def tcg1(self, E0, gradients: bool = True):
        """TCG-1: (mu_1, U_1, F, dU_1/dq, dU_1/dd, dU_1/dTheta6); the four
        gradients are None when gradients is False."""
        torch = self.torch
        E0 = self._dev(E0, torch.float64)
        n = E0.shape[0]
        mu = torch.empty_like(E0)
        if not gradients:
            return (mu, amp_tcg1(self.ctx, E0.data_ptr(), mu.data_ptr()), None, None, None, None)
        F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        gq = torch.empty((n,), dtype=torch.float64, device="cuda")
        gd = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        gt = torch.empty((n, 6), dtype=torch.float64, device="cuda")
        U = amp_tcg1(self.ctx, E0.data_ptr(), mu.data_ptr(), F.data_ptr(), gq.data_ptr(), gd.data_ptr(),
                     gt.data_ptr())
        return mu, U, F, gq, gd, gt

    def dcji(self, E0, block_of, n_blocks: int, tol_debye: float = 1e-8, max_iter: int = 200):
        """DC-JI (block Jacobi over blocks of whole molecules, block_of from
        cell_blocks): (mu, iterations, final RMS in Debye)."""
        torch = self.torch
        E0 = self._dev(E0, torch.float64)
        mu = torch.empty_like(E0)
        it, rms = amp_dcji(self.ctx, E0.data_ptr(), block_of, n_blocks, tol_debye, max_iter, mu.data_ptr())
        return mu, it, rms

    def multipole_energy(self, gradients: bool = True):
        """Permanent-multipole energy U (kcal/mol) and, if asked, (F, dU/dq, dU/dd,
        dU/dTheta6) of the current system; quadrupole gradients projected onto
        traceless changes."""
        if not gradients:
            return amp_multipole_energy(self.ctx)
        torch = self.torch
        n = self.n
        F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        gq = torch.empty((n,), dtype=torch.float64, device="cuda")
        gd = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        gt = torch.empty((n, 6), dtype=torch.float64, device="cuda")
        U = amp_multipole_energy(self.ctx, F.data_ptr(), gq.data_ptr(), gd.data_ptr(), gt.data_ptr())
        return U, F, gq, gd, gt

    def pair_count(self) -> int:
        return amp_pair_count(self.ctx)

    def reconfigure(self, cfg: Config):
        """New box/cutoff/beta/tolerance with the same grid, precision and mode."""
        amp_reconfigure(self.ctx, cfg.to_c())
        self.cfg = cfg
        self.n = 0

    def profile(self, enable: bool):
        amp_profile(self.ctx, enable)

    def profile_read(self) -> dict:
        return amp_profile_read(self.ctx)

    def launch_count(self) -> int:
        return amp_launch_count(self.ctx)

    def last_solve_stats(self):
        return amp_last_solve_stats(self.ctx)
