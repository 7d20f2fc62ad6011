"""Python binding of the GB300 voxel electrophysiology library (libep.so).

Argument marshalling only: every step of the time step runs in the CUDA
kernels behind the C ABI declared in ``include/ep.h``.  There is no CPU
fallback; importing fails if the library has not been built (run
``python -m paper_2302_12519_gb300.build``).  PyTorch, when present, is used
only to supply device memory (its caching allocator) and the CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libep.so")

(EP_OK, EP_EINVAL, EP_ENOMEM, EP_ECUDA, EP_ENOCONV, EP_ENONFINITE, EP_ESTATE, EP_EBUSY, EP_EREJECTED,
 EP_ECANCELLED) = range(10)
STATUS_NAMES = ["EP_OK", "EP_EINVAL", "EP_ENOMEM", "EP_ECUDA", "EP_ENOCONV", "EP_ENONFINITE", "EP_ESTATE",
                "EP_EBUSY", "EP_EREJECTED", "EP_ECANCELLED"]
EP_MONO, EP_BI = 0, 1
EP_EXPLICIT, EP_IMPLICIT = 0, 1
EP_SOLVER_JACOBI, EP_SOLVER_CHEBYSHEV, EP_SOLVER_GAUSS_SEIDEL = 0, 1, 2
EP_FP32, EP_FP64 = 0, 1
EP_VM_MV, EP_W, EP_VE_MV, EP_TACT, EP_V, EP_VE = range(6)

# every symbol include/ep.h declares
EXPORTS = ["ep_create", "ep_set_mask", "ep_set_fibres", "ep_set_params", "ep_add_stimulus", "ep_set_state",
           "ep_step", "ep_read", "ep_state_bytes", "ep_read_state", "ep_write_state", "ep_apply_operator",
           "ep_get_info", "ep_step_noalloc", "ep_profile_enable", "ep_get_profile", "ep_last_error",
           "ep_destroy", "ep_batch_create", "ep_batch_add", "ep_batch_remove", "ep_batch_step",
           "ep_batch_slot_stats", "ep_batch_autotune", "ep_batch_get_info", "ep_batch_last_error",
           "ep_batch_destroy", "ep_footprint", "ep_batch_set_schedule", "ep_server_create", "ep_server_submit",
           "ep_server_cancel", "ep_server_collect", "ep_server_drain", "ep_server_get_stats", "ep_server_now",
           "ep_server_last_error", "ep_server_destroy", "ep_set_torso", "ep_set_ecg", "ep_read_ecg",
           "ep_apply_elliptic", "ep_sdf_encode", "ep_sdf_encode_device", "ep_sdf_last_error"]

_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class GridDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("dx_mm", ctypes.c_double),
                ("model", ctypes.c_int), ("precision", ctypes.c_int), ("cuda_stream", ctypes.c_void_p),
                ("dev_alloc", _ALLOC_T), ("dev_free", _FREE_T), ("alloc_ctx", ctypes.c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("tau_in", "tau_out", "tau_open", "tau_close", "v_gate", "sig_iL", "sig_iT", "sig_eL", "sig_eT",
                 "lambda_", "K", "dt_ms", "jacobi_omega", "rel_tol")] + \
               [("check_every", ctypes.c_int), ("max_iter", ctypes.c_int), ("diffusion", ctypes.c_int),
                ("solver", ctypes.c_int), ("cheb_lmin", ctypes.c_double), ("cheb_lmax", ctypes.c_double)]


class StepStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("rel_res", ctypes.c_double), ("converged", ctypes.c_int),
                ("total_iters", ctypes.c_longlong), ("step", ctypes.c_longlong),
                ("ie_total_iters", ctypes.c_longlong)]


class Info(ctypes.Structure):
    _fields_ = [("n_voxels", ctypes.c_longlong), ("n_tissue", ctypes.c_longlong), ("n_components", ctypes.c_int),
                ("n_segments", ctypes.c_int), ("omega", ctypes.c_double), ("device_bytes", ctypes.c_size_t),
                ("cheb_lmin", ctypes.c_double), ("cheb_lmax", ctypes.c_double),
                ("n_domain", ctypes.c_longlong), ("n_segments_elliptic", ctypes.c_int),
                ("n_segments_far", ctypes.c_int)]


class SdfNode(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("a", ctypes.c_float), ("b", ctypes.c_float), ("c", ctypes.c_float),
                ("centre", ctypes.c_float * 3), ("rot", ctypes.c_float * 9)]


class SdfRegion(ctypes.Structure):
    _fields_ = [("first", ctypes.c_int), ("count", ctypes.c_int), ("kind", ctypes.c_int),
                ("axis", ctypes.c_float * 3), ("scale", ctypes.c_float)]


class EcgSample(ctypes.Structure):
    _fields_ = [("t_ms", ctypes.c_double), ("phi_mV", ctypes.c_double * 3), ("lead_mV", ctypes.c_double * 6)]


class Profile(ctypes.Structure):
    _fields_ = [("sweep_ms", ctypes.c_double), ("other_ms", ctypes.c_double),
                ("sweep_launches", ctypes.c_longlong), ("sweeps", ctypes.c_longlong),
                ("other_launches", ctypes.c_longlong), ("steps", ctypes.c_longlong),
                ("ie_sweep_ms", ctypes.c_double), ("ie_sweeps", ctypes.c_longlong)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("instances", ctypes.c_int), ("stencil_items", ctypes.c_longlong),
                ("chunk_items", ctypes.c_longlong), ("device_bytes", ctypes.c_size_t),
                ("budget_bytes", ctypes.c_size_t),
                ("sweeps_per_check", ctypes.c_int), ("zseg", ctypes.c_int),
                ("group_bytes", ctypes.c_size_t), ("groups", ctypes.c_int), ("solo_members", ctypes.c_int)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int), ("chunk_steps", ctypes.c_int), ("sweeps_per_check", ctypes.c_int),
                ("hbm_budget_bytes", ctypes.c_size_t), ("cuda_stream", ctypes.c_void_p),
                ("max_active_items", ctypes.c_longlong)]


class RequestResult(ctypes.Structure):
    _fields_ = [("id", ctypes.c_longlong), ("status", ctypes.c_int), ("steps_done", ctypes.c_int),
                ("n_tissue", ctypes.c_longlong), ("total_iters", ctypes.c_longlong),
                ("t_release_s", ctypes.c_double), ("t_admit_s", ctypes.c_double), ("t_done_s", ctypes.c_double),
                ("device_bytes", ctypes.c_size_t), ("sim", ctypes.c_void_p)]


class ServerStats(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int), ("active", ctypes.c_int), ("finished", ctypes.c_int)] + \
               [(n, ctypes.c_longlong) for n in ("submitted", "admitted", "completed", "cancelled", "rejected",
                                                  "chunks", "voxel_steps")] + \
               [("hbm_in_use", ctypes.c_size_t), ("hbm_peak", ctypes.c_size_t), ("busy_s", ctypes.c_double),
                ("now_s", ctypes.c_double)]


class EPError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load libep.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing; build it with `python -m paper_2302_12519_gb300.build`")
    L = ctypes.CDLL(path)
    vp, ip, dp, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    sigs = {
        "ep_create": ([ctypes.POINTER(GridDesc), ctypes.POINTER(vp)], ip),
        "ep_set_mask": ([vp, vp, sz], ip),
        "ep_set_fibres": ([vp, vp, sz], ip),
        "ep_set_params": ([vp, ctypes.POINTER(Params)], ip),
        "ep_add_stimulus": ([vp, ctypes.POINTER(ctypes.c_int * 3), ctypes.POINTER(ctypes.c_int * 3), dp, dp, dp], ip),
        "ep_set_state": ([vp, vp, vp, vp, sz, ctypes.c_longlong], ip),
        "ep_step": ([vp, ip, ctypes.POINTER(StepStats)], ip),
        "ep_step_noalloc": ([vp, ip, ctypes.POINTER(StepStats)], ip),
        "ep_read": ([vp, ip, vp, sz], ip),
        "ep_state_bytes": ([vp, ctypes.POINTER(sz)], ip),
        "ep_read_state": ([vp, vp, sz], ip),
        "ep_write_state": ([vp, vp, sz], ip),
        "ep_apply_operator": ([vp, dp, dp, vp, vp, sz], ip),
        "ep_get_info": ([vp, ctypes.POINTER(Info)], ip),
        "ep_set_torso": ([vp, vp, sz, dp], ip),
        "ep_set_ecg": ([vp, ctypes.POINTER(ctypes.c_int * 9), ip], ip),
        "ep_read_ecg": ([vp, vp, ip, ctypes.POINTER(ip)], ip),
        "ep_apply_elliptic": ([vp, vp, vp, sz], ip),
        "ep_sdf_encode": ([ctypes.POINTER(SdfNode), ip, ctypes.POINTER(SdfRegion), ip, ip, ip, ip, ctypes.c_float,
                           ctypes.POINTER(ctypes.c_float * 3), dp, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_longlong),
                           vp], ip),
        "ep_sdf_encode_device": ([ctypes.POINTER(SdfNode), ip, ctypes.POINTER(SdfRegion), ip, ip, ip, ip,
                                  ctypes.c_float, ctypes.POINTER(ctypes.c_float * 3), dp, vp, vp, vp, vp, vp, vp,
                                  vp, vp], ip),
        "ep_sdf_last_error": ([], ctypes.c_char_p),
        "ep_profile_enable": ([vp, ip], ip),
        "ep_get_profile": ([vp, ctypes.POINTER(Profile)], ip),
        "ep_last_error": ([vp], ctypes.c_char_p),
        "ep_batch_create": ([ip, sz, vp, ctypes.POINTER(vp)], ip),
        "ep_batch_add": ([vp, vp, ctypes.POINTER(ip)], ip),
        "ep_batch_remove": ([vp, ip], ip),
        "ep_batch_step": ([vp, ip], ip),
        "ep_batch_slot_stats": ([vp, ip, ctypes.POINTER(StepStats)], ip),
        "ep_batch_autotune": ([vp, ip], ip),
        "ep_batch_get_info": ([vp, ctypes.POINTER(BatchInfo)], ip),
        "ep_batch_last_error": ([vp], ctypes.c_char_p),
        "ep_batch_destroy": ([vp], None),
        "ep_footprint": ([vp, ctypes.POINTER(sz), ctypes.POINTER(sz)], ip),
        "ep_batch_set_schedule": ([vp, ip, ip, ctypes.c_longlong], ip),
        "ep_server_create": ([ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)], ip),
        "ep_server_submit": ([vp, vp, ip, dp, ctypes.POINTER(ctypes.c_longlong)], ip),
        "ep_server_cancel": ([vp, ctypes.c_longlong], ip),
        "ep_server_collect": ([vp, ctypes.POINTER(RequestResult), ip, ctypes.POINTER(ip), dp], ip),
        "ep_server_drain": ([vp, dp], ip),
        "ep_server_get_stats": ([vp, ctypes.POINTER(ServerStats)], ip),
        "ep_server_now": ([vp], dp),
        "ep_server_last_error": ([vp], ctypes.c_char_p),
        "ep_server_destroy": ([vp], None),
        "ep_destroy": ([vp], None),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def torch_allocator():
    """(alloc(nbytes) -> pointer, free(pointer)) backed by torch's caching
    allocator on the current device and stream, or None without a GPU."""
    try:
        import torch
    except Exception:
        return None
    if not torch.cuda.is_available():
        return None
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream(dev)

    def alloc(nbytes):
        return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream))

    def free(ptr):
        torch.cuda.caching_allocator_delete(int(ptr))

    return alloc, free


def _torch_hooks(allocator=None):
    """Device allocator callbacks for ep_grid_desc (from `allocator`, a pair of
    Python callables alloc(nbytes) -> pointer (0 = failure) and free(pointer),
    else torch's caching allocator) and the current torch stream.  Returns
    (alloc, free, stream) or None."""
    try:
        import torch
    except Exception:
        return None
    if not torch.cuda.is_available():
        return None
    alloc, free = allocator if allocator is not None else torch_allocator()
    stream = torch.cuda.current_stream(torch.cuda.current_device())

    def _alloc(nbytes, ctx):
        return int(alloc(int(nbytes)) or 0)

    def _free(ptr, ctx):
        free(int(ptr))

    return _ALLOC_T(_alloc), _FREE_T(_free), int(stream.cuda_stream)


def _f64(a, n: int) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
    if a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


class Sim:
    """One simulation handle (ep_sim).  Mirrors the C ABI one call per method."""

    def __init__(self, nx: int, ny: int, nz: int, dx_mm: float, model: int = EP_BI, precision: int = EP_FP32,
                 use_torch: bool = True, stream: Optional[int] = None, allocator=None):
        """allocator: optional (alloc(nbytes) -> pointer, free(pointer)) used for
        the handle's device memory instead of torch's caching allocator."""
        L = load()
        self._L = L
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.n = self.nx * self.ny * self.nz
        d = GridDesc()
        d.nx, d.ny, d.nz, d.dx_mm, d.model, d.precision = self.nx, self.ny, self.nz, float(dx_mm), int(model), int(precision)
        self._hooks = _torch_hooks(allocator) if use_torch else None
        if self._hooks is not None:
            d.dev_alloc, d.dev_free = self._hooks[0], self._hooks[1]
            d.cuda_stream = self._hooks[2] if stream is None else stream
        elif stream is not None:
            d.cuda_stream = stream
        self._desc = d
        h = ctypes.c_void_p()
        st = L.ep_create(ctypes.byref(d), ctypes.byref(h))
        if st != EP_OK:
            raise EPError(st, "ep_create")
        self._h = h

    # -- helpers -------------------------------------------------------------
    def _check(self, st: int, what: str):
        if st != EP_OK:
            raise EPError(st, f"{what}: {self._L.ep_last_error(self._h).decode()}")

    def close(self):
        if getattr(self, "_h", None):
            self._L.ep_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- set-up --------------------------------------------------------------
    def set_mask(self, mask):
        m = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8).reshape(-1))
        self._check(self._L.ep_set_mask(self._h, m.ctypes.data, m.size), "ep_set_mask")

    def set_fibres(self, fib):
        f = np.ascontiguousarray(np.asarray(fib, dtype=np.float32).reshape(-1))
        self._check(self._L.ep_set_fibres(self._h, f.ctypes.data, f.size), "ep_set_fibres")

    def set_params(self, p):
        P = Params(p.tau_in, p.tau_out, p.tau_open, p.tau_close, p.v_gate, p.sig_iL, p.sig_iT, p.sig_eL, p.sig_eT,
                   p.lam, p.K, p.dt, p.omega, p.rel_tol, int(p.check_every), int(p.max_iter),
                   int(getattr(p, "diffusion", 0)), int(getattr(p, "solver", 0)),
                   float(getattr(p, "cheb_lmin", 0.0)), float(getattr(p, "cheb_lmax", 0.0)))
        self._check(self._L.ep_set_params(self._h, ctypes.byref(P)), "ep_set_params")

    def add_stimulus(self, lo: Sequence[int], hi: Sequence[int], t_start: float, dur: float, amp: float):
        a, b = (ctypes.c_int * 3)(*lo), (ctypes.c_int * 3)(*hi)
        self._check(self._L.ep_add_stimulus(self._h, ctypes.byref(a), ctypes.byref(b), float(t_start), float(dur),
                                            float(amp)), "ep_add_stimulus")

    def set_state(self, v=None, w=None, ve=None, step: int = 0):
        arrs = [None if a is None else _f64(a, self.n) for a in (v, w, ve)]
        ptrs = [None if a is None else a.ctypes.data for a in arrs]
        self._check(self._L.ep_set_state(self._h, *ptrs, self.n, int(step)), "ep_set_state")

    # -- stepping and reads --------------------------------------------------
    def step(self, n_steps: int = 1, allow_noconv: bool = False) -> StepStats:
        s = StepStats()
        st = self._L.ep_step(self._h, int(n_steps), ctypes.byref(s))
        if not (allow_noconv and st == EP_ENOCONV):
            self._check(st, "ep_step")
        self.last_status = st
        return s

    def step_noalloc(self, n_steps: int = 1, allow_noconv: bool = False) -> StepStats:
        """ep_step_noalloc: same as step() with no device allocation in the call."""
        s = StepStats()
        st = self._L.ep_step_noalloc(self._h, int(n_steps), ctypes.byref(s))
        if not (allow_noconv and st == EP_ENOCONV):
            self._check(st, "ep_step_noalloc")
        self.last_status = st
        return s

    def read(self, field: int) -> np.ndarray:
        out = np.empty(self.n, np.float64)
        self._check(self._L.ep_read(self._h, int(field), out.ctypes.data, out.nbytes), "ep_read")
        return out

    def state_bytes(self) -> int:
        b = ctypes.c_size_t(0)
        self._check(self._L.ep_state_bytes(self._h, ctypes.byref(b)), "ep_state_bytes")
        return b.value

    def read_state(self, out: Optional[np.ndarray] = None) -> np.ndarray:
        nb = self.state_bytes()
        if out is None:
            out = np.empty(nb, np.uint8)
        self._check(self._L.ep_read_state(self._h, out.ctypes.data, nb), "ep_read_state")
        return out

    def write_state(self, blob: np.ndarray):
        blob = np.ascontiguousarray(blob, dtype=np.uint8)
        self._check(self._L.ep_write_state(self._h, blob.ctypes.data, blob.nbytes), "ep_write_state")

    def apply_operator(self, sig_L: float, sig_T: float, u) -> np.ndarray:
        u = _f64(u, self.n)
        out = np.empty(self.n, np.float64)
        self._check(self._L.ep_apply_operator(self._h, float(sig_L), float(sig_T), u.ctypes.data, out.ctypes.data,
                                              self.n), "ep_apply_operator")
        return out

    def apply_elliptic(self, u) -> np.ndarray:
        """ep_apply_elliptic: the elliptic operator (with the torso, if set) applied to u."""
        u = _f64(u, self.n)
        out = np.empty(self.n, np.float64)
        self._check(self._L.ep_apply_elliptic(self._h, u.ctypes.data, out.ctypes.data, self.n), "ep_apply_elliptic")
        return out

    def set_torso(self, torso, sig_o: float):
        t = np.ascontiguousarray(np.asarray(torso, dtype=np.uint8).reshape(-1))
        self._check(self._L.ep_set_torso(self._h, t.ctypes.data, t.size, float(sig_o)), "ep_set_torso")

    def set_ecg(self, electrodes, capacity: int):
        """electrodes: (i, j, k) of RA, LA, LL (None with capacity 0 switches the ECG off)."""
        if electrodes is None:
            self._check(self._L.ep_set_ecg(self._h, None, int(capacity)), "ep_set_ecg")
            return
        e = (ctypes.c_int * 9)(*[int(a) for ijk in electrodes for a in ijk])
        self._check(self._L.ep_set_ecg(self._h, ctypes.byref(e), int(capacity)), "ep_set_ecg")

    def read_ecg(self, max_samples: int = 1 << 16):
        """Samples since the last read: (t_ms (m,), phi_mV (m, 3), lead_mV (m, 6))."""
        buf = (EcgSample * max(1, int(max_samples)))()
        n = ctypes.c_int(0)
        self._check(self._L.ep_read_ecg(self._h, buf, int(max_samples), ctypes.byref(n)), "ep_read_ecg")
        m = n.value
        t = np.array([buf[i].t_ms for i in range(m)])
        phi = np.array([list(buf[i].phi_mV) for i in range(m)]).reshape(m, 3)
        lead = np.array([list(buf[i].lead_mV) for i in range(m)]).reshape(m, 6)
        return t, phi, lead

    def footprint(self):
        """(resident, peak) device bytes, planned on the host (ep_footprint)."""
        r, p = ctypes.c_size_t(), ctypes.c_size_t()
        self._check(self._L.ep_footprint(self._h, ctypes.byref(r), ctypes.byref(p)), "ep_footprint")
        return r.value, p.value

    def profile_enable(self, on: bool = True):
        self._check(self._L.ep_profile_enable(self._h, int(bool(on))), "ep_profile_enable")

    def profile(self) -> Profile:
        p = Profile()
        self._check(self._L.ep_get_profile(self._h, ctypes.byref(p)), "ep_get_profile")
        return p

    def info(self) -> Info:
        i = Info()
        self._check(self._L.ep_get_info(self._h, ctypes.byref(i)), "ep_get_info")
        return i


class Batch:
    """A batch of handles advanced together (ep_batch).  Members stay owned by
    the caller and must outlive their membership."""

    def __init__(self, max_instances: int, hbm_budget_bytes: int = 0, stream: Optional[int] = None):
        L = load()
        self._L = L
        h = ctypes.c_void_p()
        st = L.ep_batch_create(int(max_instances), int(hbm_budget_bytes), stream, ctypes.byref(h))
        if st != EP_OK:
            raise EPError(st, "ep_batch_create")
        self._h = h
        self._members = {}

    def _check(self, st: int, what: str):
        if st != EP_OK:
            raise EPError(st, f"{what}: {self._L.ep_batch_last_error(self._h).decode()}")

    def add(self, sim: "Sim") -> int:
        slot = ctypes.c_int(-1)
        self._check(self._L.ep_batch_add(self._h, sim._h, ctypes.byref(slot)), "ep_batch_add")
        self._members[slot.value] = sim
        return slot.value

    def remove(self, slot: int):
        self._check(self._L.ep_batch_remove(self._h, int(slot)), "ep_batch_remove")
        self._members.pop(slot, None)

    def step(self, n_steps: int, allow_noconv: bool = False) -> int:
        st = self._L.ep_batch_step(self._h, int(n_steps))
        if not (allow_noconv and st == EP_ENOCONV):
            self._check(st, "ep_batch_step")
        return st

    def slot_stats(self, slot: int) -> StepStats:
        s = StepStats()
        self._check(self._L.ep_batch_slot_stats(self._h, int(slot), ctypes.byref(s)), "ep_batch_slot_stats")
        return s

    def autotune(self, trial_sweeps: int = 20):
        self._check(self._L.ep_batch_autotune(self._h, int(trial_sweeps)), "ep_batch_autotune")

    def set_schedule(self, sweeps_per_check: int = 0, zseg: int = 0, group_bytes: int = -1):
        self._check(self._L.ep_batch_set_schedule(self._h, int(sweeps_per_check), int(zseg), int(group_bytes)),
                    "ep_batch_set_schedule")

    def info(self) -> BatchInfo:
        i = BatchInfo()
        self._check(self._L.ep_batch_get_info(self._h, ctypes.byref(i)), "ep_batch_get_info")
        return i

    def close(self):
        if getattr(self, "_h", None):
            self._L.ep_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Request loop with continuous batching (ep_server).  A submitted Sim is
    handed to the server (its Python object stops owning the handle) and
    comes back, attached again, in the result of ``collect``.  Handles must
    use the library's own device allocations (``use_torch=False``): the
    serving thread allocates them."""

    def __init__(self, max_slots: int, chunk_steps: int = 10, hbm_budget_bytes: int = 0, sweeps_per_check: int = 0,
                 stream: Optional[int] = None, max_active_items: int = 0):
        L = load()
        self._L = L
        c = ServerConfig()
        c.max_slots, c.chunk_steps, c.sweeps_per_check = int(max_slots), int(chunk_steps), int(sweeps_per_check)
        c.hbm_budget_bytes, c.cuda_stream = int(hbm_budget_bytes), stream
        c.max_active_items = int(max_active_items)
        h = ctypes.c_void_p()
        st = L.ep_server_create(ctypes.byref(c), ctypes.byref(h))
        if st != EP_OK:
            raise EPError(st, "ep_server_create")
        self._h = h
        self._held = {}

    def _check(self, st: int, what: str):
        if st != EP_OK:
            raise EPError(st, f"{what}: {self._L.ep_server_last_error(self._h).decode()}")

    def submit(self, sim: "Sim", n_steps: int, release_s: float = 0.0) -> int:
        if sim._hooks is not None:
            raise ValueError("served handles must be created with use_torch=False")
        rid = ctypes.c_longlong()
        self._check(self._L.ep_server_submit(self._h, sim._h, int(n_steps), float(release_s), ctypes.byref(rid)),
                    "ep_server_submit")
        self._held[rid.value] = (sim, sim._h)
        sim._h = None   # the server owns the handle until collected
        return rid.value

    def cancel(self, rid: int):
        self._check(self._L.ep_server_cancel(self._h, int(rid)), "ep_server_cancel")

    def collect(self, max_results: int = 64, wait_s: float = 0.0):
        """Finished requests: list of (RequestResult, Sim) with the Sim attached again."""
        buf = (RequestResult * int(max_results))()
        n = ctypes.c_int()
        self._check(self._L.ep_server_collect(self._h, buf, int(max_results), ctypes.byref(n), float(wait_s)),
                    "ep_server_collect")
        out = []
        for i in range(n.value):
            r = buf[i]
            sim, h = self._held.pop(r.id)
            sim._h = h
            out.append((r, sim))
        return out

    def collect_n(self, n: int, timeout_s: float = 600.0):
        """Collect until n results arrived (collecting as they finish keeps
        admission from waiting on memory held by results)."""
        import time
        out, t_end = [], time.monotonic() + timeout_s
        while len(out) < n:
            left = t_end - time.monotonic()
            if left <= 0:
                raise EPError(EP_EBUSY, f"collect_n: {len(out)} of {n} results after {timeout_s} s")
            out += self.collect(max_results=max(1, n - len(out)), wait_s=min(left, 1.0))
        return out

    def drain(self, timeout_s: float = -1.0):
        self._check(self._L.ep_server_drain(self._h, float(timeout_s)), "ep_server_drain")

    def stats(self) -> ServerStats:
        s = ServerStats()
        self._check(self._L.ep_server_get_stats(self._h, ctypes.byref(s)), "ep_server_get_stats")
        return s

    def now(self) -> float:
        return self._L.ep_server_now(self._h)

    def close(self):
        if getattr(self, "_h", None):
            self._L.ep_server_destroy(self._h)   # destroys the handles it still holds
            self._h = None
            self._held.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sdf_tables(nodes, regions):
    """ctypes arrays of ep_sdf_node / ep_sdf_region from node and region
    objects (op, a, b, c, centre, rot / first, count, kind, axis, scale)."""
    N = (SdfNode * len(nodes))()
    for i, nd in enumerate(nodes):
        N[i].op, N[i].a, N[i].b, N[i].c = int(nd.op), float(nd.a), float(nd.b), float(nd.c)
        N[i].centre[:] = [float(v) for v in nd.centre]
        N[i].rot[:] = [float(v) for v in nd.rot]
    R = (SdfRegion * len(regions))()
    for i, rg in enumerate(regions):
        R[i].first, R[i].count, R[i].kind = int(rg.first), int(rg.count), int(rg.kind)
        R[i].axis[:] = [float(v) for v in rg.axis]
        R[i].scale = float(rg.scale)
    return N, R


def sdf_encode(nodes, regions, nx: int, ny: int, nz: int, dx_mm: float, origin_mm, helix_rad: float,
               want_vertices: bool = True, stream: Optional[int] = None):
    """ep_sdf_encode.  nodes: sequence of objects with op, a, b, c, centre (3),
    rot (9); regions: objects with first, count, kind, axis (3), scale.
    Returns a dict of label, mask (uint8, n), fibres (float32, 3n), vertices
    (uint8, (nx+1)(ny+1)(nz+1)) and n_tissue."""
    L = load()
    N, R = sdf_tables(nodes, regions)
    n = nx * ny * nz
    label = np.empty(n, np.uint8)
    mask = np.empty(n, np.uint8)
    fib = np.empty(3 * n, np.float32)
    vert = np.empty((nx + 1) * (ny + 1) * (nz + 1), np.uint8) if want_vertices else None
    cnt = ctypes.c_longlong(0)
    org = (ctypes.c_float * 3)(*[float(v) for v in origin_mm])
    st = L.ep_sdf_encode(N, len(nodes), R, len(regions), nx, ny, nz, float(dx_mm), ctypes.byref(org),
                         float(helix_rad), label.ctypes.data, mask.ctypes.data, fib.ctypes.data,
                         None if vert is None else vert.ctypes.data, ctypes.byref(cnt), stream)
    if st != EP_OK:
        raise EPError(st, f"ep_sdf_encode: {L.ep_sdf_last_error().decode()}")
    return {"label": label, "mask": mask, "fibres": fib, "vertices": vert, "n_tissue": cnt.value}


def _is_bi(case, model: Optional[int]) -> bool:
    return (case.model if model is None else model) == EP_BI


def sim_from_case(case, use_torch: bool = True, model: Optional[int] = None, precision: Optional[int] = None,
                  ecg_capacity: int = 4096, allocator=None) -> Sim:
    """Create a handle from a ``workloads.Case`` (mask, fibres, parameters,
    stimuli; the torso and the ECG electrodes if the case has them)."""
    s = Sim(case.nx, case.ny, case.nz, case.dx, case.model if model is None else model,
            case.precision if precision is None else precision, use_torch=use_torch, allocator=allocator)
    s.set_mask(case.mask_flat())
    s.set_fibres(case.fib_flat())
    s.set_params(case.params)
    for st in case.stimuli:
        s.add_stimulus(st.lo, st.hi, st.t_start, st.dur, st.amp)
    if getattr(case, "torso", None) is not None:
        s.set_torso(case.torso, case.params.sig_o)
    if getattr(case, "electrodes", None) is not None and _is_bi(case, model):
        s.set_ecg(case.electrodes, ecg_capacity)
    return s
