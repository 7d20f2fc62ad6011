"""Plain FP64 CPU oracle for the voxel bidomain/monodomain time step.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke``
and by the CPU-baseline leg of ``bench.py``.  The product (the CUDA library and
its binding) never imports, links or runs anything from this package.

The arithmetic lives in ``ep_oracle.c`` (plain C, FP64, written from the
thesis' definitions; see its header for every equation it follows).  This
module only builds it with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ep_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libep_oracle.so")
_lib = None

OG_MONO = 0
OG_BI = 1


def build(force: bool = False) -> str:
    """Compile ep_oracle.c into libep_oracle.so (gcc, OpenMP, no FP contraction)."""
    if not force and os.path.exists(_LIB_PATH) and \
            os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                               os.path.getmtime(os.path.join(_HERE, "ep_oracle.h"))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("mask", ctypes.c_void_p), ("fib", ctypes.c_void_p),
                ("torso", ctypes.c_void_p), ("sig_o", ctypes.c_double)]


class _Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("tau_in", "tau_out", "tau_open", "tau_close", "v_gate",
                 "sig_iL", "sig_iT", "sig_eL", "sig_eT", "lam", "K", "dt", "omega", "rel_tol")] + \
               [("check_every", ctypes.c_int), ("max_iter", ctypes.c_int), ("model", ctypes.c_int),
                ("diffusion", ctypes.c_int), ("solver", ctypes.c_int),
                ("cheb_lmin", ctypes.c_double), ("cheb_lmax", ctypes.c_double), ("sig_o", ctypes.c_double)]


class _SdfNode(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("a", ctypes.c_float), ("b", ctypes.c_float), ("c", ctypes.c_float),
                ("centre", ctypes.c_float * 3), ("rot", ctypes.c_float * 9)]


class _SdfRegion(ctypes.Structure):
    _fields_ = [("first", ctypes.c_int), ("count", ctypes.c_int), ("kind", ctypes.c_int),
                ("axis", ctypes.c_float * 3), ("scale", ctypes.c_float)]


class _Stim(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_int * 3), ("hi", ctypes.c_int * 3),
                ("t_start", ctypes.c_double), ("dur", ctypes.c_double), ("amp", ctypes.c_double)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        vp, dp, ip = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
        L.og_apply_L.argtypes = [ctypes.POINTER(_Grid), dp, dp, vp, vp]
        L.og_diag_L.argtypes = [ctypes.POINTER(_Grid), dp, dp, vp]
        L.og_components.argtypes = [ctypes.POINTER(_Grid), vp]
        L.og_components.restype = ip
        L.og_jacobi.argtypes = [ctypes.POINTER(_Grid), dp, dp, vp, vp, dp, dp, ip, ip,
                                ctypes.POINTER(ip), ctypes.POINTER(dp)]
        L.og_jacobi.restype = ip
        L.og_ie_jacobi.argtypes = [ctypes.POINTER(_Grid), dp, dp, dp, vp, vp, dp, ip, ip,
                                   ctypes.POINTER(ip), ctypes.POINTER(dp)]
        L.og_ie_jacobi.restype = ip
        L.og_chebyshev.argtypes = [ctypes.POINTER(_Grid), dp, dp, vp, vp, dp, dp, dp, ip, ip,
                                   ctypes.POINTER(ip), ctypes.POINTER(dp)]
        L.og_chebyshev.restype = ip
        L.og_gauss_seidel.argtypes = [ctypes.POINTER(_Grid), dp, dp, vp, vp, dp, dp, ip, ip,
                                      ctypes.POINTER(ip), ctypes.POINTER(dp)]
        L.og_gauss_seidel.restype = ip
        L.og_default_omega.argtypes = [dp, dp]
        L.og_default_omega.restype = dp
        L.og_create.argtypes = [ip, ip, ip, dp, vp, vp, ctypes.POINTER(_Params),
                                ctypes.POINTER(_Stim), ip]
        L.og_create.restype = vp
        L.og_destroy.argtypes = [vp]
        L.og_set_torso.argtypes = [vp, vp]
        L.og_set_torso.restype = ip
        L.og_set_state.argtypes = [vp, vp, vp, vp, ctypes.c_long]
        L.og_get_state.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_long)]
        L.og_step.argtypes = [vp, ctypes.POINTER(ip), ctypes.POINTER(dp)]
        L.og_step.restype = ip
        L.og_run.argtypes = [vp, ip, ctypes.POINTER(ip), ctypes.POINTER(dp)]
        L.og_run.restype = ip
        L.og_ncomp.argtypes = [vp]
        L.og_ncomp.restype = ip
        L.og_total_iters.argtypes = [vp]
        L.og_total_iters.restype = ctypes.c_long
        L.og_ie_total_iters.argtypes = [vp]
        L.og_ie_total_iters.restype = ctypes.c_long
        L.og_num_threads.restype = ip
        L.og_sdf_eval.argtypes = [ctypes.POINTER(_SdfNode), ip, ctypes.POINTER(ctypes.c_float * 3)]
        L.og_sdf_eval.restype = ctypes.c_float
        L.og_sdf_encode.argtypes = [ctypes.POINTER(_SdfNode), ctypes.POINTER(_SdfRegion), ip, ip, ip, ip,
                                    ctypes.c_float, ctypes.POINTER(ctypes.c_float * 3), dp, vp, vp, vp, vp]
        L.og_sdf_encode.restype = ip
        _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class Grid:
    """Holds contiguous FP64 copies of a mask and fibre field, and optionally a
    conducting torso (voxels outside the tissue, conductivity sig_o I) that
    joins the domain of the operator."""

    def __init__(self, nx: int, ny: int, nz: int, dx: float, mask, fib, torso=None, sig_o: float = 0.0):
        self.nx, self.ny, self.nz, self.dx = nx, ny, nz, float(dx)
        self.mask = np.ascontiguousarray(np.asarray(mask).reshape(-1), dtype=np.uint8)
        self.fib = np.ascontiguousarray(np.asarray(fib, dtype=np.float64).reshape(-1))
        assert self.mask.size == nx * ny * nz and self.fib.size == 3 * nx * ny * nz
        self.torso = None
        tp = None
        if torso is not None:
            self.torso = np.ascontiguousarray((np.asarray(torso).reshape(-1) != 0) & (self.mask == 0), dtype=np.uint8)
            tp = _ptr(self.torso)
        self._g = _Grid(nx, ny, nz, self.dx, _ptr(self.mask), _ptr(self.fib), tp, float(sig_o))

    @classmethod
    def from_case(cls, case) -> "Grid":
        """The tissue grid of a case (torso left out: the intracellular operator)."""
        return cls(case.nx, case.ny, case.nz, case.dx, case.mask, case.fib)

    @classmethod
    def elliptic_from_case(cls, case) -> "Grid":
        """The domain of the case's elliptic equation: tissue plus its torso, if any."""
        return cls(case.nx, case.ny, case.nz, case.dx, case.mask, case.fib, case.torso, case.params.sig_o)

    def domain(self) -> np.ndarray:
        """Boolean membership of every voxel in the operator's domain."""
        d = self.mask != 0
        return d | (self.torso != 0) if self.torso is not None else d

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    def apply_L(self, sL: float, sT: float, u) -> np.ndarray:
        u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1))
        out = np.zeros(self.n)
        lib().og_apply_L(ctypes.byref(self._g), sL, sT, _ptr(u), _ptr(out))
        return out

    def diag_L(self, sL: float, sT: float) -> np.ndarray:
        out = np.zeros(self.n)
        lib().og_diag_L(ctypes.byref(self._g), sL, sT, _ptr(out))
        return out

    def components(self) -> Tuple[int, np.ndarray]:
        comp = np.zeros(self.n, np.int32)
        nc = lib().og_components(ctypes.byref(self._g), _ptr(comp))
        return nc, comp

    def jacobi(self, sL, sT, b, x0, omega=0.0, tol=1e-6, m=10, max_iter=100000):
        b = np.ascontiguousarray(np.asarray(b, dtype=np.float64).reshape(-1))
        x = np.ascontiguousarray(np.array(x0, dtype=np.float64).reshape(-1))
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        st = lib().og_jacobi(ctypes.byref(self._g), sL, sT, _ptr(b), _ptr(x), omega, tol, m,
                             max_iter, ctypes.byref(it), ctypes.byref(rr))
        return x, it.value, rr.value, st

    def chebyshev(self, sL, sT, b, x0, lmin, lmax, tol=1e-6, m=10, max_iter=100000):
        """Chebyshev-accelerated Jacobi for L x = b with D^-1 L's interval [lmin, lmax]."""
        b = np.ascontiguousarray(np.asarray(b, dtype=np.float64).reshape(-1))
        x = np.ascontiguousarray(np.array(x0, dtype=np.float64).reshape(-1))
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        st = lib().og_chebyshev(ctypes.byref(self._g), sL, sT, _ptr(b), _ptr(x), lmin, lmax, tol, m, max_iter,
                                ctypes.byref(it), ctypes.byref(rr))
        return x, it.value, rr.value, st

    def gauss_seidel(self, sL, sT, b, x0, omega=1.0, tol=1e-6, m=10, max_iter=100000):
        """Eight-colour Gauss-Seidel (omega = 1) or SOR for L x = b."""
        b = np.ascontiguousarray(np.asarray(b, dtype=np.float64).reshape(-1))
        x = np.ascontiguousarray(np.array(x0, dtype=np.float64).reshape(-1))
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        st = lib().og_gauss_seidel(ctypes.byref(self._g), sL, sT, _ptr(b), _ptr(x), omega, tol, m, max_iter,
                                   ctypes.byref(it), ctypes.byref(rr))
        return x, it.value, rr.value, st

    def ie_jacobi(self, sL, sT, alpha, f, x0, tol=1e-6, m=10, max_iter=100000):
        """Implicit-Euler Jacobi (Eq. iejac1) for (I + alpha L) x = f."""
        f = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(-1))
        x = np.ascontiguousarray(np.array(x0, dtype=np.float64).reshape(-1))
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        st = lib().og_ie_jacobi(ctypes.byref(self._g), sL, sT, alpha, _ptr(f), _ptr(x), tol, m, max_iter,
                                ctypes.byref(it), ctypes.byref(rr))
        return x, it.value, rr.value, st


def _params_struct(p, model: int) -> _Params:
    return _Params(p.tau_in, p.tau_out, p.tau_open, p.tau_close, p.v_gate,
                   p.sig_iL, p.sig_iT, p.sig_eL, p.sig_eT, p.lam, p.K, p.dt, p.omega,
                   p.rel_tol, int(p.check_every), int(p.max_iter), int(model),
                   int(getattr(p, "diffusion", 0)), int(getattr(p, "solver", 0)),
                   float(getattr(p, "cheb_lmin", 0.0)), float(getattr(p, "cheb_lmax", 0.0)),
                   float(getattr(p, "sig_o", 0.0)))


class Sim:
    """FP64 oracle simulation of one case (see workloads.Case)."""

    def __init__(self, case, params=None, model: Optional[int] = None):
        self.case = case
        self.grid = Grid.from_case(case)
        p = params if params is not None else case.params
        self.model = case.model if model is None else model
        self._p = _params_struct(p, self.model)
        st = (_Stim * max(1, len(case.stimuli)))()
        for i, s in enumerate(case.stimuli):
            st[i].lo[:] = list(s.lo)
            st[i].hi[:] = list(s.hi)
            st[i].t_start, st[i].dur, st[i].amp = s.t_start, s.dur, s.amp
        self._st = st
        self._h = lib().og_create(case.nx, case.ny, case.nz, float(case.dx),
                                  _ptr(self.grid.mask), _ptr(self.grid.fib),
                                  ctypes.byref(self._p), st, len(case.stimuli))
        self._torso = None
        if getattr(case, "torso", None) is not None:
            self._torso = np.ascontiguousarray(np.asarray(case.torso).reshape(-1), dtype=np.uint8)
            lib().og_set_torso(self._h, _ptr(self._torso))
        self.last_iters = 0
        self.last_relres = 0.0

    def close(self):
        if self._h:
            lib().og_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def ncomp(self) -> int:
        return lib().og_ncomp(self._h)

    @property
    def total_iters(self) -> int:
        return lib().og_total_iters(self._h)

    @property
    def ie_total_iters(self) -> int:
        return lib().og_ie_total_iters(self._h)

    def set_state(self, v=None, w=None, ve=None, step: int = 0):
        arrs = [None if a is None else np.ascontiguousarray(np.asarray(a, np.float64).reshape(-1))
                for a in (v, w, ve)]
        lib().og_set_state(self._h, *[None if a is None else _ptr(a) for a in arrs], int(step))

    def state(self):
        n = self.grid.n
        v, w, ve, ta = (np.zeros(n) for _ in range(4))
        step = ctypes.c_long(0)
        lib().og_get_state(self._h, _ptr(v), _ptr(w), _ptr(ve), _ptr(ta), ctypes.byref(step))
        return {"v": v, "w": w, "ve": ve, "tact": ta, "step": step.value}

    def step(self) -> int:
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        st = lib().og_step(self._h, ctypes.byref(it), ctypes.byref(rr))
        self.last_iters, self.last_relres = it.value, rr.value
        return st

    def run(self, nsteps: int) -> int:
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        st = lib().og_run(self._h, int(nsteps), ctypes.byref(it), ctypes.byref(rr))
        self.last_iters, self.last_relres = it.value, rr.value
        return st


def num_threads() -> int:
    return lib().og_num_threads()


def vm_mV(v):
    """Transmembrane potential in mV from dimensionless v (V_m = 100 v - 80)."""
    return 100.0 * np.asarray(v) - 80.0


def electrode_potentials(case, ve) -> np.ndarray:
    """Potentials (mV, V_e = 100 v_e) at the case's three electrodes RA, LA, LL."""
    ve = np.asarray(ve).reshape(-1)
    return np.array([100.0 * ve[i + case.nx * (j + case.ny * k)] for (i, j, k) in case.electrodes])


def ecg_leads(phi) -> np.ndarray:
    """The six limb leads from the electrode potentials (RA, LA, LL) (Sec.
    "Electrocardiogram"): I = LA - RA, II = LL - RA, III = LL - LA, and the
    augmented leads aVR, aVL, aVF, each one electrode minus the mean of the
    other two.  phi: (..., 3); returns (..., 6) in the order I, II, III, aVR,
    aVL, aVF."""
    phi = np.asarray(phi, dtype=np.float64)
    ra, la, ll = phi[..., 0], phi[..., 1], phi[..., 2]
    return np.stack([la - ra, ll - ra, ll - la,
                     ra - 0.5 * (la + ll), la - 0.5 * (ra + ll), ll - 0.5 * (ra + la)], axis=-1)


def _sdf_nodes(nodes):
    N = (_SdfNode * len(nodes))()
    for i, nd in enumerate(nodes):
        N[i].op, N[i].a, N[i].b, N[i].c = int(nd.op), float(nd.a), float(nd.b), float(nd.c)
        N[i].centre[:] = [float(v) for v in nd.centre]
        N[i].rot[:] = [float(v) for v in nd.rot]
    return N


def sdf_eval(nodes, x) -> float:
    """Value (FP32) of a postfix SDF program at the point x (mm)."""
    N = _sdf_nodes(nodes)
    p = (ctypes.c_float * 3)(*[float(v) for v in x])
    return float(lib().og_sdf_eval(N, len(nodes), ctypes.byref(p)))


def sdf_encode(nodes, regions, nx, ny, nz, dx, origin, helix_rad):
    """Two-pass encoding of a scene (Sec. "Geometry", "Encoding"): per voxel
    label, tissue mask and fibre (FP64), per vertex class; tissue count."""
    N = _sdf_nodes(nodes)
    R = (_SdfRegion * len(regions))()
    for i, rg in enumerate(regions):
        R[i].first, R[i].count, R[i].kind = int(rg.first), int(rg.count), int(rg.kind)
        R[i].axis[:] = [float(v) for v in rg.axis]
        R[i].scale = float(rg.scale)
    n = nx * ny * nz
    label = np.zeros(n, np.uint8)
    mask = np.zeros(n, np.uint8)
    fib = np.zeros(3 * n)
    vert = np.zeros((nx + 1) * (ny + 1) * (nz + 1), np.uint8)
    org = (ctypes.c_float * 3)(*[float(v) for v in origin])
    cnt = lib().og_sdf_encode(N, R, len(regions), nx, ny, nz, float(dx), ctypes.byref(org), float(helix_rad),
                              _ptr(label), _ptr(mask), _ptr(fib), _ptr(vert))
    return {"label": label, "mask": mask, "fibres": fib, "vertices": vert, "n_tissue": cnt}
