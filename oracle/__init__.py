"""FP64 CPU oracle for the moment-matching lattice Boltzmann warm-plasma
wakefield scheme of arXiv 2309.04872.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this package.
The CUDA library never imports, links or calls it, and the two share no
source: the C file next to this module restates the scheme on its own.

The shared library is built with plain gcc (``build()``) into ``_build/``.
Every array crossing this wrapper is float64 with the layouts documented in
``lbpwfa_oracle.h``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbpwfa_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
# ORC_PLANT=n builds and loads a copy of the oracle with planted mistake n
# (the PLANTED sites of the C file), for the test that the pins catch it
_PLANT = os.environ.get("ORC_PLANT", "").strip()
if _PLANT and not _PLANT.isdigit():
    raise ValueError(f"ORC_PLANT must be a mistake number, not {_PLANT!r}")
_LIB_PATH = os.path.join(_BUILD, f"liblbpwfa_oracle_plant{_PLANT}.so" if _PLANT else "liblbpwfa_oracle.so")
_lib = None

LEC, WARMC = 0, 1
OPEN, PERIODIC = 0, 1
CARTESIAN, AXISYMMETRIC = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, OpenMP on)."""
    os.makedirs(_BUILD, exist_ok=True)
    hdr = os.path.join(_HERE, "lbpwfa_oracle.h")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC), os.path.getmtime(hdr))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"] + ([f"-DORC_PLANT={_PLANT}"] if _PLANT else [])
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nz", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("dx", ctypes.c_double), ("courant", ctypes.c_double), ("tau", ctypes.c_double),
        ("closure", ctypes.c_int), ("dv", ctypes.c_int), ("mu", ctypes.c_double),
        ("alpha", ctypes.c_double), ("sigma_z", ctypes.c_double), ("sigma_r", ctypes.c_double),
        ("z0", ctypes.c_double), ("profile", ctypes.POINTER(ctypes.c_double)),
        ("profile_len", ctypes.c_int), ("profile_dz", ctypes.c_double),
        ("boundary", ctypes.c_int), ("init_fields", ctypes.c_int),
        ("geometry", ctypes.c_int),
    ]


_DP = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.POINTER(_Params), ctypes.POINTER(ctypes.c_int)]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_sizes.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_long)]
        L.orc_get_step.restype = ctypes.c_long
        L.orc_get_step.argtypes = [ctypes.c_void_p]
        L.orc_get_dt.restype = ctypes.c_double
        L.orc_get_dt.argtypes = [ctypes.c_void_p]
        L.orc_rest_advected.argtypes = [ctypes.c_void_p, _DP]
        L.orc_set_state.argtypes = [ctypes.c_void_p, _DP, _DP, _DP]
        L.orc_get_state.argtypes = [ctypes.c_void_p, _DP, _DP, _DP]
        L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
        L.orc_advected.argtypes = [ctypes.c_void_p, _DP]
        L.orc_moments.restype = ctypes.c_int
        L.orc_moments.argtypes = [ctypes.c_void_p, ctypes.c_uint, _DP]
        L.orc_rest_pressures.restype = None
        L.orc_rest_pressures.argtypes = [_DP, _DP, _DP]
        L.orc_reduce.argtypes = [ctypes.c_void_p, _DP]
        L.orc_stencil.restype = ctypes.c_int
        L.orc_stencil.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), _DP]
        L.orc_equilibrium.argtypes = [ctypes.c_int, ctypes.c_double, _DP, ctypes.c_double, _DP]
        L.orc_decode_lec.restype = ctypes.c_int
        L.orc_decode_lec.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _DP,
                                     _DP, _DP, _DP, _DP]
        L.orc_decode_warmc.argtypes = [ctypes.c_int, _DP, _DP]
        L.orc_lec_source.argtypes = [ctypes.c_double, ctypes.c_double, _DP, _DP, _DP, _DP, _DP]
        L.orc_warmc_source.argtypes = [ctypes.c_double, _DP, _DP, _DP, ctypes.c_double, _DP, _DP,
                                       _DP, _DP, _DP, _DP, _DP, _DP, _DP, _DP]
        L.orc_driver_density.restype = ctypes.c_double
        L.orc_driver_density.argtypes = [ctypes.POINTER(_Params), ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double]
        L.orc_adjoint_run.restype = ctypes.c_double
        L.orc_adjoint_run.argtypes = [ctypes.c_void_p, ctypes.c_long, ctypes.c_long, _DP, _DP,
                                      _DP, _DP, _DP]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


def _arr(x, n=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None:
        a = np.ascontiguousarray(np.resize(a, n)) if a.size != n else a
    return a


def _closure_code(c):
    if isinstance(c, str):
        return {"lec": LEC, "warmc": WARMC}[c.lower()]
    return int(c)


def _boundary_code(b):
    if isinstance(b, str):
        return {"open": OPEN, "periodic": PERIODIC}[b.lower()]
    return int(b)


def _geometry_code(g):
    if isinstance(g, str):
        return {"cartesian": CARTESIAN, "axisymmetric": AXISYMMETRIC}[g.lower()]
    return int(g)


def make_params(cfg: dict):
    """Build the C parameter struct from a plain configuration dict.

    Keys: dim, n (z, x, y), dx, courant, tau, closure ('lec'|'warmc'), dv,
    mu, alpha, sigma_z, sigma_r, z0, profile (array or None), profile_dz,
    boundary ('open'|'periodic'), init_fields (bool), geometry
    ('cartesian'|'axisymmetric'; axisymmetric: dim 2, open, x is r = j dx).
    The returned tuple keeps the profile buffer alive."""
    n = list(cfg["n"]) + [1, 1]
    prof = cfg.get("profile")
    prof_arr = None
    if prof is not None:
        prof_arr = _arr(prof)
    p = _Params(
        dim=int(cfg["dim"]), nz=int(n[0]), nx=int(n[1]), ny=int(n[2]),
        dx=float(cfg["dx"]), courant=float(cfg["courant"]), tau=float(cfg["tau"]),
        closure=_closure_code(cfg.get("closure", "lec")), dv=int(cfg.get("dv", 3)),
        mu=float(cfg.get("mu", 0.0)), alpha=float(cfg.get("alpha", 0.0)),
        sigma_z=float(cfg.get("sigma_z", 1.0)), sigma_r=float(cfg.get("sigma_r", 1.0)),
        z0=float(cfg.get("z0", 0.0)),
        profile=_ptr(prof_arr) if prof_arr is not None else None,
        profile_len=int(prof_arr.size) if prof_arr is not None else 0,
        profile_dz=float(cfg.get("profile_dz", 0.0)),
        boundary=_boundary_code(cfg.get("boundary", "open")),
        init_fields=int(bool(cfg.get("init_fields", cfg["dim"] >= 2))),
        geometry=_geometry_code(cfg.get("geometry", "cartesian")),
    )
    return p, prof_arr


class Oracle:
    """One oracle run.  State: populations f^n (after streaming), E at
    t_{n-1/2}, B at t_n."""

    def __init__(self, cfg: dict):
        self.cfg = dict(cfg)
        self._p, self._prof = make_params(cfg)
        st = ctypes.c_int(0)
        h = lib().orc_create(ctypes.byref(self._p), ctypes.byref(st))
        if not h or st.value != 0:
            raise ValueError(f"oracle rejected the configuration (status {st.value})")
        self._h = ctypes.c_void_p(h)
        K, Q, nc = ctypes.c_int(), ctypes.c_int(), ctypes.c_long()
        lib().orc_sizes(self._h, ctypes.byref(K), ctypes.byref(Q), ctypes.byref(nc))
        self.K, self.Q, self.ncell = K.value, Q.value, nc.value
        d = int(cfg["dim"])
        n = list(cfg["n"]) + [1, 1]
        self.shape = tuple(int(v) for v in n[:d])  # (nz, nx, ny) for present axes

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and lib is not None:
            try:
                lib().orc_destroy(h)
            except Exception:
                pass
            self._h = None

    @property
    def step_count(self) -> int:
        return int(lib().orc_get_step(self._h))

    @property
    def dt(self) -> float:
        return float(lib().orc_get_dt(self._h))

    def rest_advected(self) -> np.ndarray:
        a = np.zeros(self.K)
        lib().orc_rest_advected(self._h, _ptr(a))
        return a

    def step(self, nsteps: int = 1):
        lib().orc_step(self._h, int(nsteps))

    def set_state(self, f=None, E=None, B=None):
        fa = _arr(f).reshape(-1) if f is not None else None
        Ea = _arr(E).reshape(-1) if E is not None else None
        Ba = _arr(B).reshape(-1) if B is not None else None
        if fa is not None:
            assert fa.size == self.K * self.Q * self.ncell
        for a in (Ea, Ba):
            if a is not None:
                assert a.size == 3 * self.ncell
        lib().orc_set_state(self._h, _ptr(fa) if fa is not None else None,
                            _ptr(Ea) if Ea is not None else None,
                            _ptr(Ba) if Ba is not None else None)

    def get_state(self):
        f = np.zeros(self.K * self.Q * self.ncell)
        E = np.zeros(3 * self.ncell)
        B = np.zeros(3 * self.ncell)
        lib().orc_get_state(self._h, _ptr(f), _ptr(E), _ptr(B))
        return (f.reshape(self.K, self.Q, self.ncell), E.reshape(3, self.ncell),
                B.reshape(3, self.ncell))

    def advected(self) -> np.ndarray:
        A = np.zeros(self.K * self.ncell)
        lib().orc_advected(self._h, _ptr(A))
        return A.reshape(self.K, self.ncell)

    def moments(self, mask: int) -> np.ndarray:
        nb = bin(mask & 0x3FFFF).count("1")
        out = np.zeros(nb * self.ncell)
        lib().orc_moments(self._h, ctypes.c_uint(mask), _ptr(out))
        return out.reshape(nb, self.ncell)

    def fields(self):
        _, E, B = self.get_state()
        return E, B

    def reduce(self) -> np.ndarray:
        out = np.zeros(3)
        lib().orc_reduce(self._h, _ptr(out))
        return out

    def adjoint(self, nsteps: int, witness: int, state_grad: bool = False):
        """Run ``nsteps`` steps and return (J, dJ/d(alpha, sigma_z, sigma_r),
        dJ/d(profile samples)) with J = E.flat[witness] at the end (the
        discrete adjoint of the whole run; 1D and 2D).  With ``state_grad``
        a fourth item (dJ/df, dJ/dE, dJ/dB) of the starting state follows."""
        g3 = np.zeros(3)
        npr = self._prof.size if self._prof is not None else 0
        gp = np.zeros(max(1, npr))
        lf = np.zeros(self.K * self.Q * self.ncell) if state_grad else None
        lE = np.zeros(3 * self.ncell) if state_grad else None
        lB = np.zeros(3 * self.ncell) if state_grad else None
        J = lib().orc_adjoint_run(self._h, int(nsteps), int(witness), _ptr(g3), _ptr(gp),
                                  _ptr(lf) if state_grad else None,
                                  _ptr(lE) if state_grad else None,
                                  _ptr(lB) if state_grad else None)
        out = (float(J), g3, gp[:npr])
        if state_grad:
            out = out + ((lf, lE.reshape(3, self.ncell), lB.reshape(3, self.ncell)),)
        return out


# ---------------------------------------------------------------------------
# pieces for the pins
# ---------------------------------------------------------------------------
def stencil(dim: int):
    xi = (ctypes.c_int * (19 * 3))()
    w = np.zeros(19)
    Q = lib().orc_stencil(int(dim), xi, _ptr(w))
    return np.array(xi[: 3 * Q], dtype=np.int64).reshape(Q, 3), w[:Q].copy()


def equilibrium(dim: int, A: float, u_phys, courant: float) -> np.ndarray:
    u = _arr(u_phys, 3)
    out = np.zeros(19)
    lib().orc_equilibrium(int(dim), float(A), _ptr(u), float(courant), _ptr(out))
    Q = {1: 3, 2: 9, 3: 19}[int(dim)]
    return out[:Q].copy()


def decode_lec(Ds: int, D: int, mu: float, A):
    a = _arr(A, 1 + Ds)
    a = np.concatenate([a, np.zeros(4)])
    n, g, Pi = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    u = np.zeros(3)
    its = lib().orc_decode_lec(int(Ds), int(D), float(mu), _ptr(a), ctypes.byref(n), _ptr(u),
                               ctypes.byref(g), ctypes.byref(Pi))
    return dict(n=n.value, u=u, gamma=g.value, Pi=Pi.value, iterations=its)


def decode_warmc(dim: int, A):
    a = np.concatenate([_arr(A), np.zeros(4)])
    o = np.zeros(22)
    lib().orc_decode_warmc(int(dim), _ptr(a), _ptr(o))
    return dict(n=o[0], lam=o[1], u=o[2:5].copy(), gamma=o[5], th=o[6:15].reshape(3, 3).copy(),
                th0=o[15:18].copy(), th00=o[18], w=o[19:22].copy())


def rest_pressures(th, u):
    """(P_par, P_perp) of a WARMC tensor theta^{ij} ([3][3], order z, x, y)
    at 3-velocity u = (u_z, u_x, u_y): App. A's inversion, r -> x, phi -> y."""
    th = np.ascontiguousarray(np.asarray(th, dtype=np.float64).reshape(9))
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(3))
    out = np.zeros(2)
    lib().orc_rest_pressures(_ptr(th), _ptr(u), _ptr(out))
    return float(out[0]), float(out[1])


def lec_source(mu, n, u, gradPi, E, B):
    F = np.zeros(3)
    lib().orc_lec_source(float(mu), float(n), _ptr(_arr(u, 3)), _ptr(_arr(gradPi, 3)),
                         _ptr(_arr(E, 3)), _ptr(_arr(B, 3)), _ptr(F))
    return F


def warmc_source(n, u, th, th0, dth00_dt, dth0_dt, dw_dt, dth, dth0, dw, E, B):
    """Sources of Eq. (lb-ade-warmc-comps-F).  dth[a, b, k] = d_k theta^{ab},
    dth0[a, k] = d_k theta^{0a}, dw[a, k] = d_k w^a."""
    Fnl = ctypes.c_double()
    Fnlu = np.zeros(3)
    Fth = np.zeros(9)
    lib().orc_warmc_source(float(n), _ptr(_arr(u, 3)), _ptr(_arr(th, 9)), _ptr(_arr(th0, 3)),
                           float(dth00_dt), _ptr(_arr(dth0_dt, 3)), _ptr(_arr(dw_dt, 3)),
                           _ptr(_arr(dth, 27)), _ptr(_arr(dth0, 9)), _ptr(_arr(dw, 9)),
                           _ptr(_arr(E, 3)), _ptr(_arr(B, 3)), ctypes.byref(Fnl), _ptr(Fnlu),
                           _ptr(Fth))
    return Fnl.value, Fnlu, Fth.reshape(3, 3)


def driver_density(cfg: dict, z, x=0.0, y=0.0, t=0.0) -> float:
    p, keep = make_params(cfg)
    return float(lib().orc_driver_density(ctypes.byref(p), float(z), float(x), float(y), float(t)))
