"""TEST INFRASTRUCTURE ONLY: ctypes front end of the FP64 CPU oracle.

The oracle (``fs_oracle.c``) is a plain single-threaded hybrid PIC
implementation of the faux-shock box of Simon et al. (Sec. 2, Eq. 1). Only the
tests, the smoke check and the benchmark's CPU-baseline leg may use it; the
product path never imports this module.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fs_oracle.c")
_HDR = os.path.join(_HERE, "fs_oracle.h")
_LIB = os.path.join(_HERE, "libfsoracle.so")
_lock = threading.Lock()
_lib = None

BC_FAUXSHOCK, BC_PERIODIC = 0, 1
FS_OPEN, FS_SHOCK = 0, 1
FRAME_SHOCK, FRAME_DOWNSTREAM = 0, 1
ID_MASK, ID_CR, ID_RETURNED = 0x3FFFFFFF, 0x40000000, 0x80000000

GRID_B, GRID_E, GRID_BBAR, GRID_N, GRID_J, GRID_U = 0, 1, 2, 3, 4, 5
GRID_PROFILE_N, GRID_PROFILE_DB2 = 6, 7


class OrParams(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
        ("dx", C.c_double), ("dy", C.c_double), ("dt", C.c_double),
        ("mach_a", C.c_double), ("theta_bn_deg", C.c_double),
        ("beta_i", C.c_double), ("beta_e", C.c_double),
        ("ppc", C.c_int), ("bc_x", C.c_int), ("fs_mode_thermal", C.c_int),
        ("fs_speed_frame", C.c_int),
        ("r_comp", C.c_double), ("u2", C.c_double),
        ("inject_thermal", C.c_int), ("cr_enable", C.c_int),
        ("n_cr_ratio", C.c_double), ("p_iso", C.c_double), ("u_cr", C.c_double),
        ("n_sub", C.c_int),
        ("n_floor", C.c_double), ("eta", C.c_double), ("j_cr_ext", C.c_double),
        ("init_plasma", C.c_int),
        ("seed", C.c_uint64),
        ("hist_nx", C.c_int), ("hist_np", C.c_int),
        ("hist_pmin", C.c_double), ("hist_pmax", C.c_double),
        ("c_light", C.c_double),
        ("spec_np", C.c_int), ("spec_pmin", C.c_double), ("spec_pmax", C.c_double),
    ]


class OrDiag(C.Structure):
    _fields_ = [
        ("step", C.c_longlong), ("n_particles", C.c_longlong),
        ("next_id", C.c_longlong),
        ("incident", C.c_longlong), ("transmitted", C.c_longlong),
        ("reflected", C.c_longlong), ("escaped", C.c_longlong),
        ("injected", C.c_longlong),
        ("kinetic", C.c_double), ("magnetic", C.c_double),
        ("px", C.c_double), ("py", C.c_double), ("pz", C.c_double),
        ("fs_energy", C.c_double),
        ("injected_energy", C.c_double), ("removed_energy", C.c_double),
        ("push_work", C.c_double),
    ]


DEFAULTS = dict(
    dim=1, nx=64, ny=1, dx=0.5, dy=0.5, dt=0.005, mach_a=10.0,
    theta_bn_deg=0.0, beta_i=1.0, beta_e=1.0, ppc=8, bc_x=BC_FAUXSHOCK,
    fs_mode_thermal=FS_SHOCK, fs_speed_frame=FRAME_SHOCK, r_comp=4.0, u2=0.0,
    inject_thermal=1, cr_enable=0, n_cr_ratio=0.01, p_iso=100.0, u_cr=0.0,
    n_sub=2, n_floor=0.05, eta=0.0, j_cr_ext=0.0, init_plasma=1, seed=1,
    hist_nx=64, hist_np=64, hist_pmin=-40.0, hist_pmax=40.0,
    c_light=0.0, spec_np=64, spec_pmin=1.0, spec_pmax=1.0e4,
)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction) if it is stale."""
    with _lock:
        stale = (not os.path.exists(_LIB) or
                 os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC),
                                              os.path.getmtime(_HDR)))
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off",
                   "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.POINTER
        L.or_create.restype = C.c_void_p
        L.or_create.argtypes = [P(OrParams)]
        L.or_destroy.argtypes = [C.c_void_p]
        L.or_nxn.argtypes = [C.c_void_p]
        L.or_step.argtypes = [C.c_void_p, C.c_int]
        L.or_num_particles.restype = C.c_longlong
        L.or_num_particles.argtypes = [C.c_void_p]
        L.or_get_particles.argtypes = [C.c_void_p] + [C.c_void_p] * 8
        L.or_get_grid.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
        L.or_set_B.argtypes = [C.c_void_p, C.c_void_p]
        L.or_set_node_fields.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_inject.argtypes = [C.c_void_p, C.c_longlong] + [C.c_void_p] * 8
        L.or_diag.argtypes = [C.c_void_p, P(OrDiag)]
        L.or_histogram.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
        L.or_spectrum_p.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
        L.or_boris_rel.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                   C.c_double]
        L.or_gather.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_double,
                                C.c_double, C.c_void_p]
        L.or_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_u01.restype = C.c_double
        L.or_u01.argtypes = [C.c_uint32]
        L.or_log.restype = C.c_double
        L.or_log.argtypes = [C.c_double]
        L.or_sincos2pi.argtypes = [C.c_double, P(C.c_double), P(C.c_double)]
        L.or_boris.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double]
        L.or_fs_rule.argtypes = [P(OrParams), C.c_void_p, C.c_uint32,
                                 C.c_longlong, P(C.c_double)]
        _lib = L
    return _lib


def make_params(**kw) -> OrParams:
    d = dict(DEFAULTS)
    unknown = set(kw) - set(d)
    if unknown:
        raise KeyError(f"unknown oracle parameters {sorted(unknown)}")
    d.update(kw)
    p = OrParams()
    for name, _ in OrParams._fields_:
        setattr(p, name, d[name])
    return p


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------- primitives
def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def u01(k: int) -> float:
    return lib().or_u01(k)


def log(x: float) -> float:
    return lib().or_log(x)


def sincos2pi(u: float):
    c, s = C.c_double(), C.c_double()
    lib().or_sincos2pi(u, C.byref(c), C.byref(s))
    return c.value, s.value


def profile_B(B: np.ndarray) -> np.ndarray:
    """Transversely averaged lineouts of Bx, By, Bz (Sec. 3.1, Fig. 2(b)):
    B given as [ny][nx][3] at cell centres; returns [nx][3]."""
    return np.asarray(B, dtype=np.float64).mean(axis=0)


def bperp_spectrum(B: np.ndarray) -> np.ndarray:
    """Perpendicular magnetic power spectrum averaged over the transverse
    direction (Sec. 3.1, Fig. 3 caption): |F[By](k, y)|^2 + |F[Bz](k, y)|^2
    averaged over y, F the discrete Fourier transform along x divided by nx,
    for k = 0 .. nx/2 (wavenumber 2 pi k / (nx dx)). B as [ny][nx][3]. The
    transforms are numpy's FFT of each component separately."""
    B = np.asarray(B, dtype=np.float64)
    nx = B.shape[1]
    Fy = np.fft.fft(B[:, :, 1], axis=1) / nx
    Fz = np.fft.fft(B[:, :, 2], axis=1) / nx
    P = (np.abs(Fy) ** 2 + np.abs(Fz) ** 2).mean(axis=0)
    return P[: nx // 2 + 1]


def boris_rel(u, E, B, dt, c_light) -> np.ndarray:
    """One relativistic Boris step of u = gamma v (c_light = c / v_A)."""
    uu = np.ascontiguousarray(u, dtype=np.float64).copy()
    lib().or_boris_rel(_ptr(uu), _ptr(np.ascontiguousarray(E, np.float64)),
                       _ptr(np.ascontiguousarray(B, np.float64)), dt, c_light)
    return uu


def boris(v, E, B, dt) -> np.ndarray:
    vv = np.array(v, dtype=np.float64)
    e = np.ascontiguousarray(E, dtype=np.float64)
    b = np.ascontiguousarray(B, dtype=np.float64)
    lib().or_boris(_ptr(vv), _ptr(e), _ptr(b), dt)
    return vv


def fs_rule(v, pid: int, step: int, **params):
    """Returns (returned?, new velocity, mu') for one faux-shock crossing."""
    p = make_params(**params)
    vv = np.array(v, dtype=np.float64)
    mu = C.c_double(np.nan)
    r = lib().or_fs_rule(C.byref(p), _ptr(vv), pid, step, C.byref(mu))
    return bool(r), vv, mu.value


# ---------------------------------------------------------------- simulation
class Oracle:
    def __init__(self, **params):
        self.params = dict(DEFAULTS)
        self.params.update(params)
        self._p = make_params(**params)
        self._h = lib().or_create(C.byref(self._p))
        if not self._h:
            raise ValueError("oracle rejected the parameters")
        self.nx, self.ny = self._p.nx, self._p.ny
        self.nxn = lib().or_nxn(self._h)

    def close(self):
        if self._h:
            lib().or_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        if lib().or_step(self._h, n) != 0:
            raise RuntimeError("oracle step failed (non-finite motion)")

    @property
    def num_particles(self) -> int:
        return lib().or_num_particles(self._h)

    def particles(self) -> dict:
        n = self.num_particles
        out = dict(ci=np.zeros(n, np.int32), cj=np.zeros(n, np.int32),
                   fx=np.zeros(n), fy=np.zeros(n), vx=np.zeros(n),
                   vy=np.zeros(n), vz=np.zeros(n), id=np.zeros(n, np.uint32))
        lib().or_get_particles(self._h, *[_ptr(out[k]) for k in
                                          ("ci", "cj", "fx", "fy", "vx", "vy",
                                           "vz", "id")])
        return out

    def grid(self, what: int) -> np.ndarray:
        nx, ny, nxn = self.nx, self.ny, self.nxn
        shape = {GRID_B: (ny, nx, 3), GRID_E: (ny, nxn, 3),
                 GRID_BBAR: (ny, nxn, 3), GRID_N: (ny, nxn),
                 GRID_J: (ny, nxn, 3), GRID_U: (ny, nxn, 3),
                 GRID_PROFILE_N: (nxn,), GRID_PROFILE_DB2: (nx,)}[what]
        out = np.zeros(shape)
        if lib().or_get_grid(self._h, what, _ptr(out)) != 0:
            raise ValueError(what)
        return out

    def set_B(self, B: np.ndarray):
        b = np.ascontiguousarray(B, dtype=np.float64).reshape(self.ny, self.nx, 3)
        lib().or_set_B(self._h, _ptr(b))

    def set_node_fields(self, E: np.ndarray, Bbar: np.ndarray):
        e = np.ascontiguousarray(E, dtype=np.float64)
        b = np.ascontiguousarray(Bbar, dtype=np.float64)
        assert e.size == 3 * self.ny * self.nxn and b.size == e.size
        lib().or_set_node_fields(self._h, _ptr(e), _ptr(b))

    def inject(self, ci, cj, fx, fy, vx, vy, vz, ids=None):
        n = len(ci)
        arr = [np.ascontiguousarray(ci, np.int32), np.ascontiguousarray(cj, np.int32),
               np.ascontiguousarray(fx, np.float64), np.ascontiguousarray(fy, np.float64),
               np.ascontiguousarray(vx, np.float64), np.ascontiguousarray(vy, np.float64),
               np.ascontiguousarray(vz, np.float64)]
        idp = None
        if ids is not None:
            ida = np.ascontiguousarray(ids, np.uint32)
            arr.append(ida)
            idp = _ptr(ida)
        r = lib().or_inject(self._h, n, *[_ptr(a) for a in arr[:7]], idp)
        if r != 0:
            raise ValueError("oracle rejected the injected particles")

    def diag(self) -> dict:
        d = OrDiag()
        lib().or_diag(self._h, C.byref(d))
        return {name: getattr(d, name) for name, _ in OrDiag._fields_}

    def spectrum_p(self, species: int = 1) -> np.ndarray:
        """Counts of |u| in the log-spaced momentum bins (species -1 all,
        0 thermal, 1 cosmic rays)."""
        out = np.zeros(self._p.spec_np, dtype=np.int64)
        if lib().or_spectrum_p(self._h, species, _ptr(out)) != 0:
            raise ValueError("momentum spectrum needs spec_np >= 1 and 0 < pmin < pmax")
        return out

    def histogram(self, species: int = -1) -> np.ndarray:
        out = np.zeros((self._p.hist_nx, self._p.hist_np), dtype=np.int64)
        lib().or_histogram(self._h, species, _ptr(out))
        return out

    def gather(self, i, j, fx, fy) -> np.ndarray:
        out = np.zeros(6)
        lib().or_gather(self._h, i, j, fx, fy, _ptr(out))
        return out
