"""ctypes binding of libhotrg's C ABI (``include/hotrg.h``).

Argument marshalling only: every step of the coarse-graining runs in the
library's CUDA kernels.  The shared object is built in-tree by
``paper_2602_05900_gb300.build`` (``__graft_entry__.build()``); if it is
missing, loading fails loudly -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# HOTRG_LIB selects another build of the library (the bounds-checked one)
LIB_PATH = os.environ.get("HOTRG_LIB") or os.path.join(HERE, "libhotrg.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "hotrg.h")

HOTRG_OK, HOTRG_EINVAL, HOTRG_ENOMEM, HOTRG_ECUDA, HOTRG_EEIG, HOTRG_ENONFINITE, \
    HOTRG_ETIMEOUT, HOTRG_ESTATE, HOTRG_EBOUNDS = range(9)
DIR_X, DIR_Y = 0, 1
PRECISIONS = {"fp64": 0, "tf32": 1, "bf16x3": 2, "bf16x6": 3, "bf16xs": 4}


OPT_EIG_TC_PRODUCTS = 0
OPT_XS_DIGITS = 1
OPT_GEMM_AUTOTUNE = 2
OPT_GRAPHS = 3
OPT_EIG_MAX_ITERS = 4
OPT_WAIT_CYCLES = 5
OPT_TEST_STALL = 6
OPT_FUSED_CHAIN = 7
WAIT_CYCLES_DEFAULT = 2_000_000_000


class StepInfo(ctypes.Structure):
    """Mirror of ``hotrg_step_info_t``."""
    _fields_ = [("dir", ctypes.c_int), ("Dx", ctypes.c_int), ("Dy", ctypes.c_int),
                ("Dn", ctypes.c_int), ("side", ctypes.c_int), ("ln_c", ctypes.c_double),
                ("eps_L", ctypes.c_double), ("eps_R", ctypes.c_double),
                ("cut_gap", ctypes.c_double), ("trace_G", ctypes.c_double),
                ("eig_path", ctypes.c_int), ("eig_iters", ctypes.c_int),
                ("eig_residual", ctypes.c_double), ("eig_rr", ctypes.c_int),
                ("eig_sweeps", ctypes.c_int), ("eig_sweeps32", ctypes.c_int)]


STAGES = ["prep", "env", "gram", "eig", "proj_p", "proj_q", "proj_t", "rescale"]


class Profile(ctypes.Structure):
    """Mirror of ``hotrg_profile_t``."""
    _fields_ = [("steps", ctypes.c_int), ("launches", ctypes.c_longlong),
                ("stage_launches", ctypes.c_longlong * 8), ("ms", ctypes.c_double * 8),
                ("flops", ctypes.c_double * 8)]


class HotrgError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_SIGS = {
    "hotrg_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "hotrg_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "hotrg_ising_tensor": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, _dp]),
    "hotrg_potts_tensor": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, _dp]),
    "hotrg_xxz_tensor": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp]),
    "hotrg_trace_y": (ctypes.c_int, [ctypes.c_void_p]),
    "hotrg_itebd_create": (ctypes.c_int, [ctypes.c_int, _dp, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "hotrg_itebd_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "hotrg_itebd_energy": (ctypes.c_int, [ctypes.c_void_p, _dp]),
    "hotrg_itebd_lambda": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _dp, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int)]),
    "hotrg_itebd_discarded": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _dp]),
    "hotrg_itebd_dims": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong)]),
    "hotrg_itebd_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "hotrg_itebd_destroy": (None, [ctypes.c_void_p]),
    "hotrg_create": (ctypes.c_int, [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "hotrg_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "hotrg_log_z_per_site": (ctypes.c_int, [ctypes.c_void_p, _dp]),
    "hotrg_free_energy": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, _dp]),
    "hotrg_step_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(StepInfo)]),
    "hotrg_spectrum": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _dp, ctypes.c_int, _ip]),
    "hotrg_get_tensor": (ctypes.c_int, [ctypes.c_void_p, _dp, ctypes.c_longlong, _ip]),
    "hotrg_get_isometry": (ctypes.c_int, [ctypes.c_void_p, _dp, ctypes.c_longlong, _ip, _ip]),
    "hotrg_dims": (ctypes.c_int, [ctypes.c_void_p, _ip, _ip, _ip]),
    "hotrg_profile_enable": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "hotrg_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Profile)]),
    "hotrg_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_dp), _ip, _ip, ctypes.c_int,
                                          ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "hotrg_batch_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "hotrg_batch_size": (ctypes.c_int, [ctypes.c_void_p, _ip]),
    "hotrg_batch_log_z": (ctypes.c_int, [ctypes.c_void_p, _dp]),
    "hotrg_batch_step_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                             ctypes.POINTER(StepInfo)]),
    "hotrg_batch_get_tensor": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _dp, ctypes.c_longlong,
                                              _ip]),
    "hotrg_dgemm_emu": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_longlong, ctypes.c_void_p, ctypes.c_longlong,
                                       ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int, ctypes.c_void_p]),
    "hotrg_set_option": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "hotrg_destroy": (None, [ctypes.c_void_p]),
    "hotrg_rescale_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_double,
                                             ctypes.c_void_p, ctypes.c_void_p]),
}


def header_symbols(path: str = HEADER):
    """Names of the functions declared in ``include/hotrg.h``."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hotrg_[a-z_0-9]+)\s*\(", text)))


def load(path: str = LIB_PATH):
    """Load libhotrg.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise OSError(f"libhotrg.so not found at {path}; run __graft_entry__.build() first")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def status_string(s: int) -> str:
    return load().hotrg_status_string(s).decode()


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _stream_handle(stream):
    return ctypes.c_void_p(stream if isinstance(stream, int) else
                           (stream.cuda_stream if stream is not None else 0))


def ising_tensor(beta: float, h: float = 0.0) -> np.ndarray:
    out = np.zeros((2, 2, 2, 2))
    s = load().hotrg_ising_tensor(beta, h, _ptr(out))
    if s:
        raise HotrgError(s, "hotrg_ising_tensor rejected its arguments")
    return out


def potts_tensor(q: int, beta: float) -> np.ndarray:
    out = np.zeros((q, q, q, q))
    s = load().hotrg_potts_tensor(q, beta, _ptr(out))
    if s:
        raise HotrgError(s, "hotrg_potts_tensor rejected its arguments")
    return out


def xxz_tensor(Jxy: float, Jz: float, tau: float) -> np.ndarray:
    """Cell tensor (4, 4, 4, 4) of the Trotterised XXZ chain (two sites, one period)."""
    out = np.zeros((4, 4, 4, 4))
    s = load().hotrg_xxz_tensor(Jxy, Jz, tau, _ptr(out))
    if s:
        raise HotrgError(s, "hotrg_xxz_tensor rejected its arguments")
    return out


class Hotrg:
    """One HOTRG instance on the GPU (owns a ``hotrg_ctx``)."""

    def __init__(self, T0: np.ndarray, D_cut: int, precision: str = "fp64", stream=None):
        lib = load()
        T0 = np.ascontiguousarray(T0, dtype=np.float64)
        D0 = T0.shape[0]
        if T0.shape != (D0, D0, D0, D0):
            raise ValueError("T0 must have shape (D0, D0, D0, D0)")
        handle = ctypes.c_void_p()
        s = lib.hotrg_create(_ptr(T0), D0, int(D_cut), PRECISIONS[precision],
                             _stream_handle(stream), ctypes.byref(handle))
        if s:
            raise HotrgError(s, f"hotrg_create failed: {status_string(s)}")
        self._h = handle
        self.D_cut = int(D_cut)
        self.precision = precision

    def _check(self, s: int, what: str):
        if s:
            msg = load().hotrg_last_error(self._h)
            raise HotrgError(s, f"{what}: {status_string(s)}: {msg.decode() if msg else ''}")

    def step(self, direction: str):
        self._check(load().hotrg_step(self._h, DIR_X if direction == "x" else DIR_Y), "hotrg_step")

    def run(self, nsteps: int, first: str = "x"):
        for i in range(nsteps):
            self.step(first if i % 2 == 0 else ("y" if first == "x" else "x"))
        return self

    def trace_y(self):
        """Close the y legs (T[x,x'] = sum_y T[x,x',y,y]) of every instance."""
        self._check(load().hotrg_trace_y(self._h), "hotrg_trace_y")
        return self

    def run_quantum(self, n_time: int, n_space: int):
        """n_time Y steps (beta = 2^n_time tau), the time trace, n_space X steps."""
        for _ in range(n_time):
            self.step("y")
        self.trace_y()
        for _ in range(n_space):
            self.step("x")
        return self

    def ln_z_per_site(self) -> float:
        out = ctypes.c_double()
        self._check(load().hotrg_log_z_per_site(self._h, ctypes.byref(out)), "hotrg_log_z_per_site")
        return out.value

    def free_energy(self, beta: float) -> float:
        out = ctypes.c_double()
        self._check(load().hotrg_free_energy(self._h, beta, ctypes.byref(out)), "hotrg_free_energy")
        return out.value

    def step_info(self, step: int) -> StepInfo:
        out = StepInfo()
        self._check(load().hotrg_step_info(self._h, step, ctypes.byref(out)), "hotrg_step_info")
        return out

    def spectrum(self, step: int) -> np.ndarray:
        n = ctypes.c_int()
        buf = np.zeros(self.D_cut + 2)
        self._check(load().hotrg_spectrum(self._h, step, _ptr(buf), buf.size, ctypes.byref(n)),
                    "hotrg_spectrum")
        return buf[: n.value].copy()

    def dims(self):
        dx, dy, ns = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(load().hotrg_dims(self._h, ctypes.byref(dx), ctypes.byref(dy), ctypes.byref(ns)),
                    "hotrg_dims")
        return dx.value, dy.value, ns.value

    def tensor(self) -> np.ndarray:
        dx, dy, _ = self.dims()
        out = np.zeros((dx, dx, dy, dy))
        dims = (ctypes.c_int * 4)()
        self._check(load().hotrg_get_tensor(self._h, _ptr(out), out.size, dims), "hotrg_get_tensor")
        return out

    def isometry(self) -> np.ndarray:
        rows, cols = ctypes.c_int(), ctypes.c_int()
        load().hotrg_get_isometry(self._h, None, 0, ctypes.byref(rows), ctypes.byref(cols))
        out = np.zeros(rows.value * cols.value)
        self._check(load().hotrg_get_isometry(self._h, _ptr(out), out.size, ctypes.byref(rows),
                                              ctypes.byref(cols)), "hotrg_get_isometry")
        return out.reshape(cols.value, rows.value).T.copy()   # column-major -> [row, col]

    def set_option(self, option: int, value: int):
        self._check(load().hotrg_set_option(self._h, option, value), "hotrg_set_option")

    def profile_enable(self, on: bool = True):
        self._check(load().hotrg_profile_enable(self._h, 1 if on else 0), "hotrg_profile_enable")

    def profile_read(self) -> dict:
        p = Profile()
        self._check(load().hotrg_profile_read(self._h, ctypes.byref(p)), "hotrg_profile_read")
        return {"steps": p.steps, "launches": p.launches,
                "stage_launches": {k: int(p.stage_launches[i]) for i, k in enumerate(STAGES)},
                "ms": {k: float(p.ms[i]) for i, k in enumerate(STAGES)},
                "flops": {k: float(p.flops[i]) for i, k in enumerate(STAGES)}}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().hotrg_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class HotrgBatch:
    """Many independent HOTRG instances in one context (``hotrg_batch_*``).

    ``T0s`` is a sequence of initial tensors (each (D0, D0, D0, D0)) and
    ``D_cuts`` the matching cuts; all instances take the same step directions.
    """

    def __init__(self, T0s, D_cuts, precision: str = "tf32", stream=None):
        lib = load()
        self._T0s = [np.ascontiguousarray(t, dtype=np.float64) for t in T0s]
        n = len(self._T0s)
        if n == 0 or len(D_cuts) != n:
            raise ValueError("need one D_cut per initial tensor")
        for t in self._T0s:
            if t.ndim != 4 or len(set(t.shape)) != 1:
                raise ValueError("every T0 must have shape (D0, D0, D0, D0)")
        ptrs = (_dp * n)(*[_ptr(t) for t in self._T0s])
        d0 = (ctypes.c_int * n)(*[t.shape[0] for t in self._T0s])
        dc = (ctypes.c_int * n)(*[int(d) for d in D_cuts])
        handle = ctypes.c_void_p()
        s = lib.hotrg_batch_create(n, ptrs, d0, dc, PRECISIONS[precision], _stream_handle(stream),
                                   ctypes.byref(handle))
        if s:
            raise HotrgError(s, f"hotrg_batch_create failed: {status_string(s)}")
        self._h = handle
        self.n = n
        self.D_cuts = [int(d) for d in D_cuts]
        self.precision = precision

    _check = Hotrg._check
    close = Hotrg.close
    __del__ = Hotrg.__del__
    __enter__ = Hotrg.__enter__
    __exit__ = Hotrg.__exit__
    profile_enable = Hotrg.profile_enable
    set_option = Hotrg.set_option
    profile_read = Hotrg.profile_read

    def step(self, direction: str):
        self._check(load().hotrg_batch_step(self._h, DIR_X if direction == "x" else DIR_Y),
                    "hotrg_batch_step")

    run = Hotrg.run
    trace_y = Hotrg.trace_y
    run_quantum = Hotrg.run_quantum

    def size(self) -> int:
        n = ctypes.c_int()
        self._check(load().hotrg_batch_size(self._h, ctypes.byref(n)), "hotrg_batch_size")
        return n.value

    def ln_z_per_site(self) -> np.ndarray:
        out = np.zeros(self.n)
        self._check(load().hotrg_batch_log_z(self._h, _ptr(out)), "hotrg_batch_log_z")
        return out

    def step_info(self, inst: int, step: int) -> StepInfo:
        out = StepInfo()
        self._check(load().hotrg_batch_step_info(self._h, inst, step, ctypes.byref(out)),
                    "hotrg_batch_step_info")
        return out

    def tensor(self, inst: int) -> np.ndarray:
        dims = (ctypes.c_int * 4)()
        load().hotrg_batch_get_tensor(self._h, inst, None, 0, dims)
        out = np.zeros((dims[0], dims[1], dims[2], dims[3]))
        self._check(load().hotrg_batch_get_tensor(self._h, inst, _ptr(out), out.size, dims),
                    "hotrg_batch_get_tensor")
        return out


class Itebd:
    """A batch of iTEBD chains on the GPU (``hotrg_itebd_*``).

    ``couplings`` is a sequence of (Jxy, Jz, tau), one per chain; ``init`` is
    None (the Neel state) or one (P, Q, lam) per chain, all with the same D0.
    """

    def __init__(self, couplings, D_b: int, init=None, stream=None):
        lib = load()
        cp = np.ascontiguousarray(np.asarray(couplings, dtype=np.float64).reshape(-1, 3))
        n = cp.shape[0]
        self._keep = [cp]
        arrays = [None, None, None]
        D0 = 1
        if init is not None:
            if len(init) != n:
                raise ValueError("need one initial state per chain")
            D0 = int(np.asarray(init[0][2]).size)
            for k in range(3):
                parts = [np.ascontiguousarray(st[k], dtype=np.float64) for st in init]
                self._keep += parts
                arrays[k] = ctypes.cast((_dp * n)(*[_ptr(a) for a in parts]), ctypes.c_void_p)
        handle = ctypes.c_void_p()
        s = lib.hotrg_itebd_create(n, _ptr(cp), int(D_b), D0, arrays[0], arrays[1], arrays[2],
                                   _stream_handle(stream), ctypes.byref(handle))
        if s:
            raise HotrgError(s, f"hotrg_itebd_create failed: {status_string(s)}")
        self._h = handle
        self.n = n
        self.D_b = int(D_b)

    def _check(self, s: int, what: str):
        if s:
            msg = load().hotrg_itebd_last_error(self._h)
            raise HotrgError(s, f"{what}: {status_string(s)}: {msg.decode() if msg else ''}")

    def step(self, nsteps: int = 1):
        self._check(load().hotrg_itebd_step(self._h, int(nsteps)), "hotrg_itebd_step")
        return self

    def energy(self) -> np.ndarray:
        out = np.zeros(self.n)
        self._check(load().hotrg_itebd_energy(self._h, _ptr(out)), "hotrg_itebd_energy")
        return out

    def lam(self, inst: int = 0) -> np.ndarray:
        buf = np.zeros(self.D_b)
        k = ctypes.c_int()
        self._check(load().hotrg_itebd_lambda(self._h, inst, _ptr(buf), buf.size, ctypes.byref(k)),
                    "hotrg_itebd_lambda")
        return buf[:k.value].copy()

    def discarded(self, inst: int = 0) -> float:
        out = ctypes.c_double()
        self._check(load().hotrg_itebd_discarded(self._h, inst, ctypes.byref(out)), "hotrg_itebd_discarded")
        return out.value

    def dims(self):
        o, m, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
        self._check(load().hotrg_itebd_dims(self._h, ctypes.byref(o), ctypes.byref(m), ctypes.byref(k)),
                    "hotrg_itebd_dims")
        return o.value, m.value, k.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().hotrg_itebd_destroy(self._h)
            self._h = ctypes.c_void_p()

    __del__ = Hotrg.__del__
    __enter__ = Hotrg.__enter__
    __exit__ = Hotrg.__exit__


def dgemm_emu(A, B, C, slices: int = 7, stream=None):
    """C = A @ B.T through ``hotrg_dgemm_emu`` on torch CUDA float64 tensors
    (row-major, unit column stride); returns C."""
    for t in (A, B, C):
        if t.dtype.itemsize != 8 or not t.is_cuda or t.stride(1) != 1:
            raise ValueError("A, B, C must be float64 CUDA tensors with unit column stride")
    M, K = A.shape
    N = B.shape[0]
    s = load().hotrg_dgemm_emu(M, N, K, A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0),
                               C.data_ptr(), C.stride(0), slices, _stream_handle(stream))
    if s:
        raise HotrgError(s, f"hotrg_dgemm_emu failed: {status_string(s)}")
    return C
