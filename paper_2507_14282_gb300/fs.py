"""Thin ctypes binding of the C ABI in include/fs.h.

Argument marshalling only: every step of the simulation runs in libfs.so's
CUDA kernels. PyTorch provides the device buffer (one uint8 tensor sized by
fs_query) and the CUDA stream. There is no CPU fallback: constructing a
simulation without the built library or without a CUDA device raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfs.so")

FS_FP64, FS_FP32 = 0, 1
FS_BC_FAUXSHOCK, FS_BC_PERIODIC = 0, 1
FS_OPEN, FS_SHOCK = 0, 1
FS_FRAME_SHOCK, FS_FRAME_DOWNSTREAM = 0, 1
FS_B, FS_E, FS_BBAR, FS_N, FS_J, FS_U = 0, 1, 2, 3, 4, 5
FS_PROFILE_N, FS_PROFILE_DB2, FS_HIST_XPX, FS_HIST_XPX_CR = 6, 7, 8, 9
FS_PROFILE_B, FS_SPECTRUM_BPERP = 10, 11
FS_SPECTRUM_P_CR, FS_SPECTRUM_P_ALL = 12, 13
FS_STATE = 14
ID_MASK, ID_CR, ID_RETURNED = 0x3FFFFFFF, 0x40000000, 0x80000000
FS_EUNSTABLE = -7
FS_ENOMEM = -8
FS_ETIMEOUT, FS_ENAN, FS_ECAPACITY, FS_EBADCELL = -6, -3, -2, -9
FS_RK4_Z_MAX = 2.8284271247461903  # 2 sqrt 2: RK4 on the imaginary axis


class FsParams(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
        ("dx", C.c_double), ("dy", C.c_double), ("dt", C.c_double),
        ("precision", C.c_int),
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
        ("seed", C.c_ulonglong),
        ("capacity_factor", C.c_double), ("mover_fraction", C.c_double),
        ("tile_x", C.c_int), ("tile_y", C.c_int),
        ("hist_nx", C.c_int), ("hist_np", C.c_int),
        ("hist_pmin", C.c_double), ("hist_pmax", C.c_double),
        ("use_graph", C.c_int),
        ("c_light", C.c_double),
        ("spec_np", C.c_int), ("spec_pmin", C.c_double), ("spec_pmax", C.c_double),
        ("push_chunk", C.c_int), ("push_ctas_per_sm", C.c_int),
    ]


class FsSizes(C.Structure):
    _fields_ = [
        ("device_bytes", C.c_size_t), ("device_alignment", C.c_size_t),
        ("particle_capacity", C.c_longlong), ("tiles", C.c_longlong),
        ("tile_x", C.c_int), ("tile_y", C.c_int), ("nxn", C.c_int),
    ]


class FsDiag(C.Structure):
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
        ("status", C.c_int), ("launches", C.c_longlong),
        ("max_z", C.c_double),
    ]


class FsRunState(C.Structure):
    _fields_ = [
        ("step", C.c_longlong), ("next_id", C.c_longlong),
        ("incident", C.c_longlong), ("transmitted", C.c_longlong),
        ("reflected", C.c_longlong), ("escaped", C.c_longlong),
        ("injected", C.c_longlong),
        ("fs_energy", C.c_double), ("injected_energy", C.c_double),
        ("removed_energy", C.c_double),
        ("ny", C.c_int), ("reserved", C.c_int),
    ]


class FsError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


_lib = None


def lib():
    """Loads libfs.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise FileNotFoundError(
                f"{LIB_PATH} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        P, V = C.POINTER, C.c_void_p
        L.fs_params_default.argtypes = [C.c_int, P(FsParams)]
        L.fs_query.argtypes = [P(FsParams), P(FsSizes)]
        L.fs_init.argtypes = [P(FsParams), V, C.c_size_t, V, P(V)]
        L.fs_inject.argtypes = [V, C.c_longlong] + [V] * 8
        L.fs_load_fields.argtypes = [V, V]
        L.fs_step.argtypes = [V, C.c_int]
        L.fs_moments.argtypes = [V, C.c_int, V, C.c_size_t, C.c_int]
        L.fs_num_particles.argtypes = [V, P(C.c_longlong)]
        L.fs_restore_state.argtypes = [V, V, C.c_size_t]
        L.fs_get_particles.argtypes = [V, C.c_longlong] + [V] * 8 + [P(C.c_longlong)]
        L.fs_diag.argtypes = [V, P(FsDiag)]
        L.fs_destroy.argtypes = [V]
        L.fs_profile.argtypes = [V, C.c_int]
        L.fs_profile_read.argtypes = [V, V, V, C.c_int]
        L.fs_strerror.argtypes = [C.c_int]
        L.fs_strerror.restype = C.c_char_p
        L.fs_batch_plan.argtypes = [C.c_int, V, V, C.c_int, V]
        L.fs_batch_query.argtypes = [C.c_int, C.c_int, P(C.c_size_t)]
        L.fs_batch_init.argtypes = [V, C.c_int, V, C.c_size_t, P(V)]
        L.fs_batch_step.argtypes = [V, C.c_int]
        L.fs_batch_destroy.argtypes = [V]
        L.fs_window_query.argtypes = [P(FsParams), C.c_int, C.c_int, C.c_longlong, C.c_int,
                                      P(C.c_size_t)]
        L.fs_window_init.argtypes = [P(FsParams), C.c_int, C.c_int, C.c_longlong, V, V,
                                     C.c_int, V, C.c_int, V, C.c_size_t, V, P(V)]
        L.fs_window_forward.argtypes = [V, V, P(C.c_double)]
        L.fs_window_backward.argtypes = [V, C.c_double, V]
        L.fs_window_counts.argtypes = [V, V]
        L.fs_window_destroy.argtypes = [V]
        L.fs_fp64_fma_rate.argtypes = [C.c_int, V, P(C.c_double)]
        L.fs_selftest_wait.argtypes = [C.c_int, V, V]
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().fs_strerror(code).decode()


def fp64_fma_rate(iters: int = 1 << 14, stream=None) -> float:
    """This GPU's FP64 fused multiply-add rate in FMA lane operations per
    second (fs_fp64_fma_rate; the FP64 push's roofline denominator)."""
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("fp64_fma_rate needs a CUDA device")
    st = stream if stream is not None else torch.cuda.current_stream()
    out = C.c_double()
    _check(lib().fs_fp64_fma_rate(int(iters), C.c_void_p(st.cuda_stream), C.byref(out)),
           "fs_fp64_fma_rate")
    return out.value


def selftest_wait(limit: int = 4096, stream=None) -> int:
    """fs_selftest_wait: one CTA waits with the push's bounded mbarrier wait on
    a barrier nothing arrives on; returns the status code (FS_ETIMEOUT when
    the wait ran out, as it should)."""
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("selftest_wait needs a CUDA device")
    st = stream if stream is not None else torch.cuda.current_stream()
    word = torch.zeros(1, dtype=torch.int32, device=st.device)
    return int(lib().fs_selftest_wait(int(limit), C.c_void_p(word.data_ptr()),
                                      C.c_void_p(st.cuda_stream)))


def _check(code: int, what: str):
    if code != 0:
        raise FsError(code, what)


def params_default(dim: int) -> dict:
    p = FsParams()
    _check(lib().fs_params_default(dim, C.byref(p)), "fs_params_default")
    return {name: getattr(p, name) for name, _ in FsParams._fields_}


def make_params(**kw) -> FsParams:
    d = params_default(kw.get("dim", 1))
    unknown = set(kw) - set(d)
    if unknown:
        raise KeyError(f"unknown parameters {sorted(unknown)}")
    d.update(kw)
    p = FsParams()
    for name, _ in FsParams._fields_:
        setattr(p, name, d[name])
    return p


def query(**kw) -> FsSizes:
    p = make_params(**kw)
    s = FsSizes()
    _check(lib().fs_query(C.byref(p), C.byref(s)), "fs_query")
    return s


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class FauxShock:
    """One simulation: a device buffer from torch plus a library handle."""

    def __init__(self, device: str = "cuda:0", stream=None, **params):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("FauxShock needs a CUDA device; there is no CPU path")
        self.torch = torch
        self.device = torch.device(device)
        self._p = make_params(**params)
        self.params = {name: getattr(self._p, name) for name, _ in FsParams._fields_}
        sz = FsSizes()
        _check(lib().fs_query(C.byref(self._p), C.byref(sz)), "fs_query")
        self.sizes = sz
        self.nx, self.ny, self.nxn = self._p.nx, self._p.ny, sz.nxn
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream()
            align = int(sz.device_alignment)
            self._mem = torch.empty(int(sz.device_bytes) + align, dtype=torch.uint8,
                                    device=self.device)
            base = self._mem.data_ptr()
            off = (-base) % align
            self._base = base + off
            h = C.c_void_p()
            _check(lib().fs_init(C.byref(self._p), C.c_void_p(self._base),
                                 C.c_size_t(int(sz.device_bytes)),
                                 C.c_void_p(self.stream.cuda_stream), C.byref(h)),
                   "fs_init")
        self._h = h

    # ----------------------------------------------------------- lifecycle
    def close(self):
        """Releases the handle, then the device buffer (back to torch's cache)."""
        if getattr(self, "_h", None):
            lib().fs_destroy(self._h)
            self._h = None
        self._mem = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ----------------------------------------------------------- stepping
    def step(self, n: int = 1):
        _check(lib().fs_step(self._h, n), "fs_step")

    # ----------------------------------------------------------- tracing
    PHASES = ("push", "movers", "inject", "moments", "fields")

    def profile(self, enable: bool = True):
        _check(lib().fs_profile(self._h, 1 if enable else 0), "fs_profile")

    def profile_read(self) -> dict:
        """Summed ms and step counts per phase since the last read."""
        ms = np.zeros(5)
        cnt = np.zeros(5, dtype=np.int64)
        _check(lib().fs_profile_read(self._h, _ptr(ms), _ptr(cnt), 5), "fs_profile_read")
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(self.PHASES)}

    # ----------------------------------------------------------- outputs
    def num_particles(self) -> int:
        n = C.c_longlong()
        _check(lib().fs_num_particles(self._h, C.byref(n)), "fs_num_particles")
        return n.value

    def diag(self) -> dict:
        """fs_diag as a dict; 'unstable' is True when the field integrator's
        stability number max_z exceeds the RK4 bound (FS_EUNSTABLE)."""
        d = FsDiag()
        rc = lib().fs_diag(self._h, C.byref(d))
        if rc != FS_EUNSTABLE:
            _check(rc, "fs_diag")
        out = {name: getattr(d, name) for name, _ in FsDiag._fields_}
        out["unstable"] = rc == FS_EUNSTABLE
        return out

    def grid(self, what: int) -> np.ndarray:
        nx, ny, nxn = self.nx, self.ny, self.nxn
        shape = {FS_B: (ny, nx, 3), FS_E: (ny, nxn, 3), FS_BBAR: (ny, nxn, 3),
                 FS_N: (ny, nxn), FS_J: (ny, nxn, 3), FS_U: (ny, nxn, 3),
                 FS_PROFILE_N: (nxn,), FS_PROFILE_DB2: (nx,), FS_PROFILE_B: (nx, 3),
                 FS_SPECTRUM_BPERP: (nx // 2 + 1,)}[what]
        out = np.zeros(shape)
        _check(lib().fs_moments(self._h, what, _ptr(out), out.nbytes, 0), "fs_moments")
        return out

    def grid_device(self, what: int, out) -> None:
        """Writes a grid quantity as FP64 into a CUDA tensor (no host copy)."""
        _check(lib().fs_moments(self._h, what, C.c_void_p(out.data_ptr()),
                                out.numel() * out.element_size(), 1), "fs_moments")

    def spectrum_p(self, cr_only: bool = True) -> np.ndarray:
        """Momentum spectrum n(p): counts of |u| in spec_np log-spaced bins."""
        out = np.zeros(self._p.spec_np, dtype=np.int64)
        what = FS_SPECTRUM_P_CR if cr_only else FS_SPECTRUM_P_ALL
        _check(lib().fs_moments(self._h, what, _ptr(out), out.nbytes, 0), "fs_moments")
        return out

    def histogram(self, cr_only: bool = False) -> np.ndarray:
        out = np.zeros((self._p.hist_nx, self._p.hist_np), dtype=np.int64)
        what = FS_HIST_XPX_CR if cr_only else FS_HIST_XPX
        _check(lib().fs_moments(self._h, what, _ptr(out), out.nbytes, 0), "fs_moments")
        return out

    def particles(self) -> dict:
        n = self.num_particles()
        out = dict(ci=np.zeros(n, np.int32), cj=np.zeros(n, np.int32),
                   fx=np.zeros(n), fy=np.zeros(n), vx=np.zeros(n), vy=np.zeros(n),
                   vz=np.zeros(n), id=np.zeros(n, np.uint32))
        got = C.c_longlong()
        _check(lib().fs_get_particles(self._h, n, *[_ptr(out[k]) for k in
                                                     ("ci", "cj", "fx", "fy", "vx", "vy",
                                                      "vz", "id")], C.byref(got)),
               "fs_get_particles")
        assert got.value == n
        return out

    # ----------------------------------------------------------- inputs
    def inject(self, ci, cj, fx, fy, vx, vy, vz, ids=None):
        arrs = [np.ascontiguousarray(ci, np.int32), np.ascontiguousarray(cj, np.int32),
                np.ascontiguousarray(fx, np.float64), np.ascontiguousarray(fy, np.float64),
                np.ascontiguousarray(vx, np.float64), np.ascontiguousarray(vy, np.float64),
                np.ascontiguousarray(vz, np.float64)]
        idp = None
        if ids is not None:
            ida = np.ascontiguousarray(ids, np.uint32)
            arrs.append(ida)
            idp = _ptr(ida)
        _check(lib().fs_inject(self._h, len(arrs[0]), *[_ptr(a) for a in arrs[:7]], idp),
               "fs_inject")

    def load_fields(self, B: np.ndarray):
        b = np.ascontiguousarray(B, dtype=np.float64).reshape(self.ny, self.nx, 3)
        _check(lib().fs_load_fields(self._h, _ptr(b)), "fs_load_fields")

    # ----------------------------------------------------------- checkpoint
    def run_state(self) -> np.ndarray:
        """fs_moments(FS_STATE): the run state beyond particles and field
        (step, next id, flux counters, energy sums, inflow accumulators) as
        raw bytes; fields(blob) decodes them."""
        blob = np.zeros(C.sizeof(FsRunState) + 8 * self.ny, dtype=np.uint8)
        _check(lib().fs_moments(self._h, FS_STATE, _ptr(blob), blob.nbytes, 0), "fs_moments")
        return blob

    @staticmethod
    def run_state_fields(blob: np.ndarray) -> dict:
        st = FsRunState.from_buffer_copy(blob[:C.sizeof(FsRunState)].tobytes())
        out = {name: getattr(st, name) for name, _ in FsRunState._fields_}
        out["row_acc"] = blob[C.sizeof(FsRunState):].view(np.float64).copy()
        return out

    def restore_state(self, blob: np.ndarray):
        b = np.ascontiguousarray(blob, dtype=np.uint8)
        _check(lib().fs_restore_state(self._h, _ptr(b), b.nbytes), "fs_restore_state")

    def checkpoint(self) -> dict:
        """Everything a restart needs: the particles (with ids), B at the
        cell centres and the run state."""
        return {"particles": self.particles(), "B": self.grid(FS_B),
                "state": self.run_state()}

    @classmethod
    def restart(cls, ckpt: dict, device: str = "cuda:0", stream=None, **params):
        """A fresh handle with the same parameters holding a checkpoint: no
        initial plasma, then the field, the particles with their ids and the
        run state (fs_load_fields, fs_inject, fs_restore_state)."""
        params = dict(params)
        params["init_plasma"] = 0
        sim = cls(device=device, stream=stream, **params)
        sim.load_fields(ckpt["B"])
        p = ckpt["particles"]
        if len(p["id"]):
            sim.inject(p["ci"], p["cj"], p["fx"], p["fy"], p["vx"], p["vy"], p["vz"],
                       ids=p["id"])
        sim.restore_state(ckpt["state"])
        return sim


def batch_plan(n_particles, ntiles, ncta_max: int) -> list:
    """CTA groups of a batch (fs_batch_plan; host-only, no GPU needed)."""
    n = np.ascontiguousarray(n_particles, dtype=np.int64)
    t = np.ascontiguousarray(ntiles, dtype=np.int32)
    out = np.zeros(len(n), dtype=np.int32)
    _check(lib().fs_batch_plan(len(n), _ptr(n), _ptr(t), int(ncta_max), _ptr(out)),
           "fs_batch_plan")
    return out.tolist()


class FsBatch:
    """Independent FauxShock runs stepped together (fs_batch_*): one push
    launch per class of runs over every run's CTA group per step (1D FP32 runs
    of a tile width in COMPILED_WIDTHS form a class with that width compiled
    in), the rest of the step batched too (1D runs with x walls) or in
    parallel branches of one CUDA graph. The runs must share precision,
    dimension and stream; they are not stepped on their own while the batch
    lives."""

    COMPILED_WIDTHS = (4, 8, 16)

    def __init__(self, sims):
        import torch
        if not sims:
            raise ValueError("a batch needs at least one run")
        self.sims = list(sims)
        prec = self.sims[0].params["precision"]
        nb = C.c_size_t()
        _check(lib().fs_batch_query(len(self.sims), prec, C.byref(nb)), "fs_batch_query")
        align = 256
        dev = self.sims[0].device
        self._mem = torch.empty(int(nb.value) + align, dtype=torch.uint8, device=dev)
        base = self._mem.data_ptr()
        base += (-base) % align
        hs = (C.c_void_p * len(self.sims))(*[s._h.value for s in self.sims])
        h = C.c_void_p()
        _check(lib().fs_batch_init(hs, len(self.sims), C.c_void_p(base), nb, C.byref(h)),
               "fs_batch_init")
        self._h = h

    def step(self, n: int = 1):
        _check(lib().fs_batch_step(self._h, n), "fs_batch_step")

    def close(self):
        if getattr(self, "_h", None):
            lib().fs_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
