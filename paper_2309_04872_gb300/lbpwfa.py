"""Thin ctypes binding of liblbpwfa.so (include/lbpwfa.h).

Argument marshalling only: every step of the solver runs in the CUDA
library.  If the library has not been built the import of a run fails
loudly; there is no CPU fallback.  Device buffers may be passed as torch
CUDA tensors (their data pointer is handed to the library); host buffers are
numpy float64 arrays.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LEC, WARMC = 0, 1
FP64, FP32, FP16S, FP32C = 0, 1, 2, 3
OPEN, PERIODIC = 0, 1
CARTESIAN, AXISYMMETRIC = 0, 1
_PREC = {"fp64": FP64, "fp32": FP32, "fp16s": FP16S, "fp32c": FP32C}

M_N, M_UZ, M_UX, M_UY, M_GAMMA, M_PZ, M_PX, M_PY = (1 << b for b in range(8))
M_P0, M_LAMBDA = 1 << 8, 1 << 9
M_TH_ZZ, M_TH_XX, M_TH_YY, M_TH_ZX, M_TH_ZY, M_TH_XY = (1 << b for b in range(10, 16))
M_P_PAR, M_P_PERP = 1 << 16, 1 << 17
F_EX, F_EY, F_EZ, F_BX, F_BY, F_BZ = (1 << b for b in range(6))

STATUS = {0: "ok", -1: "invalid argument", -2: "out of memory", -3: "CUDA error",
          -4: "non-finite populations", -5: "device wait timed out", -6: "invalid state",
          -7: "checkpoint I/O error"}


class LbpwfaError(RuntimeError):
    def __init__(self, status: int, detail: str = ""):
        self.status = status
        super().__init__(f"lbpwfa status {status} ({STATUS.get(status, '?')}) {detail}".strip())


class Params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("dx", ctypes.c_double),
        ("courant", ctypes.c_double), ("tau", ctypes.c_double), ("closure", ctypes.c_int),
        ("dv", ctypes.c_int), ("mu", ctypes.c_double), ("alpha", ctypes.c_double),
        ("sigma_z", ctypes.c_double), ("sigma_r", ctypes.c_double), ("z0", ctypes.c_double),
        ("profile", ctypes.POINTER(ctypes.c_double)), ("profile_len", ctypes.c_int),
        ("profile_dz", ctypes.c_double), ("precision", ctypes.c_int), ("boundary", ctypes.c_int),
        ("init_fields", ctypes.c_int), ("stream", ctypes.c_void_p), ("kernel_variant", ctypes.c_int),
        ("geometry", ctypes.c_int), ("device_bytes_cap", ctypes.c_size_t),
        ("record_tape", ctypes.c_int64), ("checkpoint_every", ctypes.c_int64),
    ]


class FitParams(ctypes.Structure):
    _fields_ = [("quantity", ctypes.c_int), ("line", ctypes.c_int * 2), ("xi_lo", ctypes.c_double),
                ("xi_hi", ctypes.c_double), ("k_lo", ctypes.c_double), ("k_hi", ctypes.c_double),
                ("nk", ctypes.c_int)]


FIT_EZ, FIT_N = 0, 1


class Info(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int), ("Q", ctypes.c_int), ("ncell", ctypes.c_int64),
                ("step", ctypes.c_int64), ("dt", ctypes.c_double), ("time", ctypes.c_double),
                ("device_bytes", ctypes.c_size_t), ("bytes_per_update", ctypes.c_double),
                ("kernel_variant", ctypes.c_int), ("algorithmic_bytes_per_update", ctypes.c_double)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("nruns", ctypes.c_int), ("ncell", ctypes.c_int64), ("nitems", ctypes.c_int64),
                ("tile", (ctypes.c_int * 2) * 2), ("grid", ctypes.c_int * 2), ("graph_steps", ctypes.c_int),
                ("step", ctypes.c_int64), ("device_bytes", ctypes.c_size_t), ("bytes_per_step", ctypes.c_double),
                ("tuned_ms", (ctypes.c_double * 4) * 2), ("algorithmic_bytes_per_step", ctypes.c_double)]


class RecordParams(ctypes.Structure):
    _fields_ = [("max_steps", ctypes.c_int64), ("checkpoint_every", ctypes.c_int64)]


class AdjointIO(ctypes.Structure):
    _fields_ = [("witness", ctypes.c_int * 3), ("seed", ctypes.c_double), ("J", ctypes.c_double),
                ("grad_driver", ctypes.c_double * 3), ("grad_profile", ctypes.POINTER(ctypes.c_double))]


_lib = None
_DP = ctypes.POINTER(ctypes.c_double)
EXPORTED = ["lbpwfa_create", "lbpwfa_step", "lbpwfa_moments", "lbpwfa_fields", "lbpwfa_advected",
            "lbpwfa_set_state", "lbpwfa_get_state", "lbpwfa_reduce", "lbpwfa_info", "lbpwfa_save",
            "lbpwfa_load", "lbpwfa_set_stream", "lbpwfa_synchronize", "lbpwfa_destroy",
            "lbpwfa_status_string", "lbpwfa_last_error", "lbpwfa_reduce_noalloc",
            "lbpwfa_batch_create", "lbpwfa_batch_step", "lbpwfa_batch_member", "lbpwfa_batch_info",
            "lbpwfa_batch_destroy", "lbpwfa_record", "lbpwfa_adjoint_step", "lbpwfa_line_fit",
            "lbpwfa_gauss_residual", "lbpwfa_set_wait_limit", "lbpwfa_measure_fp64_rate",
            "lbpwfa_create_batch", "lbpwfa_autotune"]


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = False) -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"liblbpwfa.so is not built ({path}); call "
                               "paper_2309_04872_gb300.build.build() first")
        _build.build()
    L = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    L.lbpwfa_create.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(vp)]
    L.lbpwfa_step.argtypes = [vp, ctypes.c_int64]
    L.lbpwfa_moments.argtypes = [vp, ctypes.c_uint32, vp, ctypes.c_size_t, ctypes.c_int]
    L.lbpwfa_fields.argtypes = [vp, ctypes.c_uint32, vp, ctypes.c_size_t, ctypes.c_int]
    L.lbpwfa_line_fit.argtypes = [vp, ctypes.POINTER(FitParams), _DP]
    L.lbpwfa_gauss_residual.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _DP]
    L.lbpwfa_advected.argtypes = [vp, vp, ctypes.c_size_t, ctypes.c_int]
    L.lbpwfa_set_state.argtypes = [vp, vp, vp, vp, ctypes.c_int]
    L.lbpwfa_get_state.argtypes = [vp, vp, vp, vp, ctypes.c_int]
    L.lbpwfa_reduce.argtypes = [vp, _DP]
    L.lbpwfa_reduce_noalloc.argtypes = [vp, vp, ctypes.c_int]
    L.lbpwfa_info.argtypes = [vp, ctypes.POINTER(Info)]
    L.lbpwfa_save.argtypes = [vp, ctypes.c_char_p]
    L.lbpwfa_load.argtypes = [vp, ctypes.c_char_p]
    L.lbpwfa_set_stream.argtypes = [vp, vp]
    L.lbpwfa_synchronize.argtypes = [vp]
    L.lbpwfa_set_wait_limit.argtypes = [vp, ctypes.c_uint32]
    L.lbpwfa_autotune.argtypes = [vp, _DP]
    L.lbpwfa_measure_fp64_rate.argtypes = [_DP]
    L.lbpwfa_destroy.argtypes = [vp]
    L.lbpwfa_destroy.restype = None
    L.lbpwfa_status_string.argtypes = [ctypes.c_int]
    L.lbpwfa_status_string.restype = ctypes.c_char_p
    L.lbpwfa_last_error.argtypes = [vp]
    L.lbpwfa_last_error.restype = ctypes.c_char_p
    L.lbpwfa_batch_create.argtypes = [ctypes.POINTER(Params), ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)]
    L.lbpwfa_batch_step.argtypes = [vp, ctypes.c_int64]
    L.lbpwfa_create_batch.argtypes = [ctypes.POINTER(Params), ctypes.c_int, ctypes.POINTER(vp)]
    L.lbpwfa_batch_member.argtypes = [vp, ctypes.c_int, ctypes.POINTER(vp)]
    L.lbpwfa_batch_info.argtypes = [vp, ctypes.POINTER(BatchInfo)]
    L.lbpwfa_batch_destroy.argtypes = [vp]
    L.lbpwfa_batch_destroy.restype = None
    L.lbpwfa_record.argtypes = [vp, ctypes.POINTER(RecordParams)]
    L.lbpwfa_adjoint_step.argtypes = [vp, ctypes.POINTER(AdjointIO)]
    _lib = L
    return L


def measure_fp64_rate() -> float:
    """FP64 FMA rate of the current GPU in FLOP/s (lbpwfa_measure_fp64_rate)."""
    out = ctypes.c_double()
    st = load_library().lbpwfa_measure_fp64_rate(ctypes.byref(out))
    if st != 0:
        raise LbpwfaError(st, "lbpwfa_measure_fp64_rate")
    return out.value


def _code(v, table):
    return table[v.lower()] if isinstance(v, str) else int(v)


def make_params(cfg: dict, precision="fp64", stream=None, variant=0):
    """Parameter struct from a configuration dict (same keys as the oracle's:
    dim, n, dx, courant, tau, closure, dv, mu, alpha, sigma_z, sigma_r, z0,
    profile, profile_dz, boundary, init_fields, geometry ('cartesian' |
    'axisymmetric'))."""
    n = list(cfg["n"]) + [1, 1]
    prof = cfg.get("profile")
    keep = None
    p = Params()
    p.dim = int(cfg["dim"])
    for a in range(3):
        p.n[a] = int(n[a]) if a < p.dim else 1
    p.dx = float(cfg["dx"])
    p.courant = float(cfg["courant"])
    p.tau = float(cfg["tau"])
    p.closure = _code(cfg.get("closure", "lec"), {"lec": LEC, "warmc": WARMC})
    p.dv = int(cfg.get("dv", 3))
    p.mu = float(cfg.get("mu", 0.0))
    p.alpha = float(cfg.get("alpha", 0.0))
    p.sigma_z = float(cfg.get("sigma_z", 1.0))
    p.sigma_r = float(cfg.get("sigma_r", 1.0))
    p.z0 = float(cfg.get("z0", 0.0))
    if prof is not None:
        keep = np.ascontiguousarray(np.asarray(prof, dtype=np.float64))
        p.profile = keep.ctypes.data_as(_DP)
        p.profile_len = int(keep.size)
        p.profile_dz = float(cfg["profile_dz"])
    p.precision = _code(precision, _PREC)
    p.boundary = _code(cfg.get("boundary", "open"), {"open": OPEN, "periodic": PERIODIC})
    p.init_fields = int(bool(cfg.get("init_fields", p.dim >= 2)))
    p.stream = stream
    p.kernel_variant = int(variant)
    p.geometry = _code(cfg.get("geometry", "cartesian"), {"cartesian": CARTESIAN, "axisymmetric": AXISYMMETRIC})
    p.device_bytes_cap = int(cfg.get("device_bytes_cap", 0))
    p.record_tape = int(cfg.get("record_tape", 0))
    p.checkpoint_every = int(cfg.get("checkpoint_every", 0))
    return p, keep


def _buf(x, count=None):
    """(pointer, is_device, keepalive) of a numpy array or torch tensor."""
    if x is None:
        return None, 0, None
    if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
        if x.dtype.__str__() != "torch.float64" or not x.is_contiguous():
            raise ValueError("device buffers must be contiguous float64 torch tensors")
        return ctypes.c_void_p(x.data_ptr()), int(x.is_cuda), x
    a = np.asarray(x)
    if a.dtype != np.float64 or not a.flags.c_contiguous:
        raise ValueError("host buffers must be C-contiguous float64 numpy arrays")
    return ctypes.c_void_p(a.ctypes.data), 0, a


class Run:
    """One simulation on the GPU behind the C ABI."""

    def __init__(self, cfg: dict, precision="fp64", stream=None, variant=0):
        L = load_library()
        self.cfg = dict(cfg)
        self.precision = precision
        self._p, self._keep = make_params(cfg, precision, stream, variant)
        h = ctypes.c_void_p()
        st = L.lbpwfa_create(ctypes.byref(self._p), ctypes.byref(h))
        if st != 0:
            raise LbpwfaError(st, "lbpwfa_create")
        self._h = h
        inf = self.info()
        self.K, self.Q, self.ncell = inf.K, inf.Q, inf.ncell

    def _check(self, st, what):
        if st != 0:
            detail = load_library().lbpwfa_last_error(self._h) or b""
            raise LbpwfaError(st, f"{what}: {detail.decode(errors='replace')}")

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            load_library().lbpwfa_destroy(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def info(self) -> Info:
        inf = Info()
        self._check(load_library().lbpwfa_info(self._h, ctypes.byref(inf)), "lbpwfa_info")
        return inf

    def step(self, nsteps: int = 1):
        self._check(load_library().lbpwfa_step(self._h, int(nsteps)), "lbpwfa_step")

    def synchronize(self):
        self._check(load_library().lbpwfa_synchronize(self._h), "lbpwfa_synchronize")

    def autotune(self):
        """Time every step kernel this run can take and keep the fastest
        (lbpwfa_autotune): returns the step time in ms per variant 1..4
        (None where not timed, every entry when the choice came from the
        LBPWFA_TUNE_CACHE file) and the variant in use."""
        ms = np.full(5, -1.0)
        self._check(load_library().lbpwfa_autotune(self._h, ms.ctypes.data_as(_DP)), "lbpwfa_autotune")
        return {v: (float(ms[v]) if ms[v] >= 0 else None) for v in range(1, 5)}, self.info().kernel_variant

    def set_wait_limit(self, polls: int):
        """Polls of each tile's first barrier wait before it gives up
        (lbpwfa_set_wait_limit; a failure-detection test hook)."""
        self._check(load_library().lbpwfa_set_wait_limit(self._h, int(polls)), "lbpwfa_set_wait_limit")

    def moments(self, mask: int, out=None):
        nb = bin(mask & 0x3FFFF).count("1")
        if out is None:
            out = np.zeros((nb, self.ncell))
        ptr, dev, keep = _buf(out)
        self._check(load_library().lbpwfa_moments(self._h, mask, ptr, nb * self.ncell, dev), "lbpwfa_moments")
        return out

    def line_fit(self, quantity="ez", line=(0, 0), xi=(-25.0, -5.0), k=(0.5, 1.5, 201)):
        """Least-squares sinusoid fit along one grid line in z (lbpwfa_line_fit):
        returns dict(k, amplitude, phase, rms, points)."""
        fp = FitParams()
        fp.quantity = {"ez": FIT_EZ, "n": FIT_N}[quantity]
        fp.line[0], fp.line[1] = int(line[0]), int(line[1])
        fp.xi_lo, fp.xi_hi = float(xi[0]), float(xi[1])
        fp.k_lo, fp.k_hi, fp.nk = float(k[0]), float(k[1]), int(k[2])
        out = (ctypes.c_double * 5)()
        self._check(load_library().lbpwfa_line_fit(self._h, ctypes.byref(fp), out), "lbpwfa_line_fit")
        return dict(k=out[0], amplitude=out[1], phase=out[2], rms=out[3], points=int(out[4]))

    def gauss_residual(self, lo, hi):
        """Gauss's law residual over the dual cells lo <= index < hi
        (lbpwfa_gauss_residual): dict(res2, rho2, cells)."""
        a = (ctypes.c_int * 3)(*(list(lo) + [0, 0, 0])[:3])
        b = (ctypes.c_int * 3)(*(list(hi) + [1, 1, 1])[:3])
        out = (ctypes.c_double * 3)()
        self._check(load_library().lbpwfa_gauss_residual(self._h, a, b, out), "lbpwfa_gauss_residual")
        return dict(res2=out[0], rho2=out[1], cells=int(out[2]))

    def fields(self, mask: int = 0x3F, out=None):
        nb = bin(mask & 0x3F).count("1")
        if out is None:
            out = np.zeros((nb, self.ncell))
        ptr, dev, keep = _buf(out)
        self._check(load_library().lbpwfa_fields(self._h, mask, ptr, nb * self.ncell, dev), "lbpwfa_fields")
        return out

    def advected(self, out=None):
        if out is None:
            out = np.zeros((self.K, self.ncell))
        ptr, dev, keep = _buf(out)
        self._check(load_library().lbpwfa_advected(self._h, ptr, self.K * self.ncell, dev), "lbpwfa_advected")
        return out

    def set_state(self, f=None, E=None, B=None):
        arrs = [x if (x is None or hasattr(x, "data_ptr")) else np.ascontiguousarray(x, dtype=np.float64)
                for x in (f, E, B)]
        bufs = [_buf(a) for a in arrs]
        devs = {b[1] for b in bufs if b[2] is not None}
        if len(devs) > 1:
            raise ValueError("mix of host and device buffers")
        dev = devs.pop() if devs else 0
        self._check(load_library().lbpwfa_set_state(self._h, bufs[0][0], bufs[1][0], bufs[2][0], dev),
                    "lbpwfa_set_state")

    def get_state(self):
        f = np.zeros((self.K, self.Q, self.ncell))
        E = np.zeros((3, self.ncell))
        B = np.zeros((3, self.ncell))
        self._check(load_library().lbpwfa_get_state(self._h, ctypes.c_void_p(f.ctypes.data),
                                                    ctypes.c_void_p(E.ctypes.data),
                                                    ctypes.c_void_p(B.ctypes.data), 0), "lbpwfa_get_state")
        return f, E, B

    def reduce(self, status: bool = False):
        """FP64 sums (sum n, sum n_b, non-finite populations); with status
        also the call's status code (0, or -4 when out[2] > 0)."""
        out = np.zeros(3)
        st = load_library().lbpwfa_reduce(self._h, out.ctypes.data_as(_DP))
        if st not in (0, -4):
            self._check(st, "lbpwfa_reduce")
        return (out, st) if status else out

    def save(self, path: str):
        self._check(load_library().lbpwfa_save(self._h, path.encode()), "lbpwfa_save")

    def load(self, path: str):
        self._check(load_library().lbpwfa_load(self._h, path.encode()), "lbpwfa_load")

    def record(self, max_steps: int, checkpoint_every: int = 0):
        """Start an adjoint recording window of up to max_steps steps
        (checkpoint_every = 0 keeps every step's tape)."""
        rp = RecordParams(int(max_steps), int(checkpoint_every))
        self._check(load_library().lbpwfa_record(self._h, ctypes.byref(rp)), "lbpwfa_record")

    def adjoint(self, witness, seed: float = 1.0):
        """Reverse sweep over the recorded window: returns (J, dL/d(alpha,
        sigma_z, sigma_r), dL/d(profile samples) or None) for J = E_z at the
        witness node's slot and L = seed J."""
        io = AdjointIO()
        w = list(witness) + [0, 0]
        for a in range(3):
            io.witness[a] = int(w[a])
        io.seed = float(seed)
        gp = None
        if self._keep is not None:
            gp = np.zeros(self._keep.size)
            io.grad_profile = gp.ctypes.data_as(_DP)
        self._check(load_library().lbpwfa_adjoint_step(self._h, ctypes.byref(io)), "lbpwfa_adjoint_step")
        return float(io.J), np.array([io.grad_driver[q] for q in range(3)]), gp


class _Member(Run):
    """View of one run of a batch (outputs and state; stepping goes through
    the batch)."""

    def __init__(self, batch, handle, cfg, precision):
        self.cfg = dict(cfg)
        self.precision = precision
        self._batch = batch  # keeps the batch alive
        self._h = handle
        inf = self.info()
        self.K, self.Q, self.ncell = inf.K, inf.Q, inf.ncell

    def close(self):
        self._h = None  # owned by the batch


class Batch:
    """Many 2D runs advanced together by one persistent launch per step."""

    def __init__(self, cfgs, precision="fp32", stream=None, tune=True):
        L = load_library()
        self.cfgs = [dict(c) for c in cfgs]
        arr = (Params * len(cfgs))()
        self._keep = []
        for i, c in enumerate(cfgs):
            p, keep = make_params(c, precision, stream if i == 0 else None)
            arr[i] = p
            self._keep.append(keep)
        h = ctypes.c_void_p()
        st = L.lbpwfa_batch_create(arr, len(cfgs), 0 if tune else 1, ctypes.byref(h))
        if st != 0:
            raise LbpwfaError(st, "lbpwfa_batch_create")
        self._h = h
        self.members = []
        for i, c in enumerate(cfgs):
            m = ctypes.c_void_p()
            st = L.lbpwfa_batch_member(self._h, i, ctypes.byref(m))
            if st != 0:
                raise LbpwfaError(st, "lbpwfa_batch_member")
            self.members.append(_Member(self, m, c, precision))

    def step(self, nsteps: int = 1):
        st = load_library().lbpwfa_batch_step(self._h, int(nsteps))
        if st != 0:
            raise LbpwfaError(st, "lbpwfa_batch_step")

    def info(self) -> BatchInfo:
        inf = BatchInfo()
        st = load_library().lbpwfa_batch_info(self._h, ctypes.byref(inf))
        if st != 0:
            raise LbpwfaError(st, "lbpwfa_batch_info")
        return inf

    def synchronize(self):
        self.members[0].synchronize()

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            for m in self.members:
                m._h = None
            load_library().lbpwfa_batch_destroy(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
