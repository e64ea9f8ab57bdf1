"""ctypes binding of libitp (include/itp.h): the same entry points, argument
marshalling only.  Every step of the method runs in the CUDA library; there
is no Python or CPU fallback, and loading fails loudly if libitp.so is
missing."""
from __future__ import annotations

import ctypes
import os

import numpy as np

ITP_OK = 0
ITP_ERR_ARG = 1
ITP_ERR_CUDA = 2
ITP_ERR_NOT_PD = 3
ITP_ERR_TIMEOUT = 4
ITP_ERR_OOM = 5
ITP_ERR_STATE = 6
ITP_ERR_NOCONV = 7
ITP_FP64 = 0
ITP_MIXED = 1
ITP_RITZ = 1
ITP_RITZ_VALUES = 2
ITP_EVAL_FP64 = 8
ITP_STEP_FP64 = 4
ITP_TUNE_PENCIL_W, ITP_TUNE_SPLIT, ITP_TUNE_ROW_TB, ITP_TUNE_GRAM = 0, 1, 2, 3
ITP_TUNING_LEN = 4

_ERR_NAMES = {1: "ITP_ERR_ARG", 2: "ITP_ERR_CUDA", 3: "ITP_ERR_NOT_PD", 4: "ITP_ERR_TIMEOUT",
              5: "ITP_ERR_OOM", 6: "ITP_ERR_STATE", 7: "ITP_ERR_NOCONV"}

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libitp.so")

# (name, restype, argtypes) of every exported entry point
_H = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_PD = ctypes.c_void_p
SIGNATURES = [
    ("itp_create_grid", _I, [ctypes.POINTER(_H), _I, _I, _I, _D, _D, _D, _I, _I, _I, ctypes.c_void_p]),
    ("itp_destroy", None, [_H]),
    ("itp_set_potential", _I, [_H, _PD]),
    ("itp_set_states", _I, [_H, _PD]),
    ("itp_set_states_device", _I, [_H, ctypes.c_void_p]),
    ("itp_get_states", _I, [_H, _PD]),
    ("itp_get_phi", _I, [_H, _PD]),
    ("itp_propagate", _I, [_H, _I, _D]),
    ("itp_orthonormalize", _I, [_H]),
    ("itp_energies", _I, [_H, _PD, _I]),
    ("itp_step", _I, [_H, _I, _D, _I, _PD]),
    ("itp_step_host", _I, [_H, _I, _D, _I, _PD, _PD, _PD]),
    ("itp_polish", _I, [_H, _I, _D, _D, _I, ctypes.POINTER(_I), _PD]),
    ("itp_propagate_romberg6", _I, [_H, _D]),
    ("itp_solve_adaptive", _I, [_H, _I, _D, _D, _D, _I, _I, ctypes.POINTER(_I), _PD, _PD, _PD]),
    ("itp_synchronize", _I, [_H]),
    ("itp_test_expire_waits", _I, [_H, _I]),
    ("itp_last_error", ctypes.c_char_p, [_H]),
    ("itp_kernel_launches", ctypes.c_longlong, [_H]),
    ("itp_profile", _I, [_H, _I]),
    ("itp_profile_read", _I, [_H, _I, ctypes.POINTER(ctypes.c_longlong),
                              ctypes.POINTER(ctypes.c_double)]),
    ("itp_peak_probe", _I, [_I, ctypes.c_void_p, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    ("itp_orthonormalize_noalloc", _I, [ctypes.c_void_p, ctypes.c_void_p, _I, ctypes.c_longlong,
                                        _D, ctypes.c_void_p]),
    ("itp_get_tuning", _I, [_H, _PD]),
    ("itp_set_tuning", _I, [_H, _PD]),
    ("itp_autotune", _I, [_H, _I, _D, _PD, ctypes.c_char_p, _I]),
    ("itp_create_batch", _I, [ctypes.POINTER(_H), _I, _PD, _PD, _PD, _PD, _I, ctypes.c_void_p]),
    ("itp_batch_problem", _H, [_H, _I]),
    ("itp_batch_count", _I, [_H]),
    ("itp_batch_step", _I, [_H, _I, _D, _I, _PD]),
    ("itp_batch_kernel_launches", ctypes.c_longlong, [_H]),
    ("itp_batch_set_grouping", _I, [_H, _I]),
    ("itp_batch_groups", _I, [_H]),
    ("itp_batch_last_error", ctypes.c_char_p, [_H]),
    ("itp_batch_destroy", None, [_H]),
]

KERNEL_KINDS = ["plane_fwd", "plane_merged", "plane_combine", "plane_hpsi", "pencil",
                "pencil_kinetic", "gram", "gram_reduce", "cholesky", "eigh", "apply", "other"]

_lib = None


class ItpError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{_ERR_NAMES.get(code, code)}: {message}")
        self.code = code


def load() -> ctypes.CDLL:
    """Load libitp.so (built by paper_0809_3739_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(h, code: int):
    if code != ITP_OK:
        msg = load().itp_last_error(h)
        raise ItpError(code, msg.decode() if msg else "")


def _f64(a, count=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if count is not None and a.size != count:
        raise ValueError(f"expected {count} values, got {a.size}")
    return a


# ---- the C entry points ------------------------------------------------------
def itp_create_grid(nx, ny, nz, lx, ly, lz, n_states, n_guard=0, precision=ITP_FP64,
                    cuda_stream=0):
    h = _H()
    code = load().itp_create_grid(ctypes.byref(h), nx, ny, nz, lx, ly, lz, n_states, n_guard,
                                  precision, ctypes.c_void_p(cuda_stream or None))
    _check(None, code)
    return h


def itp_destroy(h):
    load().itp_destroy(h)


def itp_set_potential(h, V):
    V = _f64(V)
    _check(h, load().itp_set_potential(h, V.ctypes.data))


def itp_set_states(h, psi):
    psi = _f64(psi)
    _check(h, load().itp_set_states(h, psi.ctypes.data))


def itp_set_states_device(h, device_ptr: int):
    _check(h, load().itp_set_states_device(h, ctypes.c_void_p(device_ptr)))


def itp_get_states(h, out: np.ndarray):
    if out.dtype != np.float64 or not out.flags.c_contiguous:
        raise ValueError("out must be a C-contiguous float64 array")
    _check(h, load().itp_get_states(h, out.ctypes.data))
    return out


def itp_get_phi(h, out: np.ndarray):
    if out.dtype != np.float64 or not out.flags.c_contiguous:
        raise ValueError("out must be a C-contiguous float64 array")
    _check(h, load().itp_get_phi(h, out.ctypes.data))
    return out


def itp_propagate(h, order: int, tau: float):
    _check(h, load().itp_propagate(h, int(order), float(tau)))


def itp_propagate_romberg6(h, tau: float):
    _check(h, load().itp_propagate_romberg6(h, float(tau)))


def itp_orthonormalize(h):
    _check(h, load().itp_orthonormalize(h))


def itp_energies(h, out: np.ndarray | None, flags: int = ITP_RITZ):
    ptr = None if out is None else out.ctypes.data
    _check(h, load().itp_energies(h, ptr, int(flags)))
    return out


def itp_step(h, order, tau, flags=ITP_RITZ_VALUES, out: np.ndarray | None = None):
    ptr = None if out is None else out.ctypes.data
    _check(h, load().itp_step(h, int(order), float(tau), int(flags), ptr))
    return out


def _host_buffer(a, count: int, writable: bool) -> int:
    """Address of a host buffer of `count` doubles: a C-contiguous float64
    numpy array (checked), or a raw address (int) the caller vouches for."""
    if isinstance(a, int):
        return a
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
        raise ValueError("host buffer must be a C-contiguous float64 array")
    if a.size != count:
        raise ValueError(f"expected {count} values, got {a.size}")
    if writable and not a.flags.writeable:
        raise ValueError("output buffer is read-only")
    return a.ctypes.data


def itp_step_host(h, m, n_points, order, tau, psi_in, psi_out, flags=ITP_RITZ_VALUES,
                  out: np.ndarray | None = None):
    """One step between host buffers (itp_step_host): psi_in and psi_out
    are float64 arrays of m * n_points values (or raw host addresses)."""
    pin = _host_buffer(psi_in, m * n_points, False)
    pout = _host_buffer(psi_out, m * n_points, True)
    ptr = None if out is None else out.ctypes.data
    _check(h, load().itp_step_host(h, int(order), float(tau), int(flags), pin, pout, ptr))
    return out


def itp_polish(h, order, tau, tol, max_steps, out: np.ndarray | None = None):
    steps = _I(0)
    ptr = None if out is None else out.ctypes.data
    _check(h, load().itp_polish(h, int(order), float(tau), float(tol), int(max_steps),
                                ctypes.byref(steps), ptr))
    return steps.value


def itp_solve_adaptive(h, m, order, tau0, reduce, gamma, max_steps=200, max_levels=12):
    """Returns dict(E, RH, levels=[(tau, steps, propagated state-steps)], converged)."""
    lv = _I(0)
    stats = np.zeros((max_levels, 3), dtype=np.float64)
    RH = np.empty(m, dtype=np.float64)
    E = np.empty(m, dtype=np.float64)
    code = load().itp_solve_adaptive(h, int(order), float(tau0), float(reduce), float(gamma),
                                     int(max_steps), int(max_levels), ctypes.byref(lv),
                                     stats.ctypes.data, RH.ctypes.data, E.ctypes.data)
    if code not in (ITP_OK, ITP_ERR_NOCONV):
        _check(h, code)
    levels = [(float(t), int(s), int(p)) for t, s, p in stats[:lv.value]]
    return {"E": E, "RH": RH, "levels": levels, "converged": code == ITP_OK}


def itp_synchronize(h):
    _check(h, load().itp_synchronize(h))


def itp_test_expire_waits(h, launches: int):
    _check(h, load().itp_test_expire_waits(h, int(launches)))


def itp_last_error(h) -> str:
    r = load().itp_last_error(h)
    return r.decode() if r else ""


def itp_kernel_launches(h) -> int:
    return int(load().itp_kernel_launches(h))


def itp_profile(h, enable: bool):
    _check(h, load().itp_profile(h, 1 if enable else 0))


def itp_profile_read(h, kind: int):
    n = ctypes.c_longlong(0)
    ms = ctypes.c_double(0.0)
    _check(h, load().itp_profile_read(h, int(kind), ctypes.byref(n), ctypes.byref(ms)))
    return int(n.value), float(ms.value)


def itp_orthonormalize_noalloc(phi_device_ptr: int, psi_device_ptr: int, m: int,
                               n_points: int, dV: float, cuda_stream: int = 0):
    """Allocation-free orthonormalisation of caller-owned device buffers
    (device pointers as integers, e.g. torch tensors' data_ptr())."""
    code = load().itp_orthonormalize_noalloc(ctypes.c_void_p(phi_device_ptr),
                                            ctypes.c_void_p(psi_device_ptr), int(m),
                                            int(n_points), float(dV),
                                            ctypes.c_void_p(cuda_stream or None))
    if code != ITP_OK:
        raise ItpError(code, "itp_orthonormalize_noalloc failed")


ITP_PROBE_FFMA, ITP_PROBE_FFMA2, ITP_PROBE_DFMA, ITP_PROBE_TF32_MMA = 0, 1, 2, 3
PROBE_KINDS = {"ffma": ITP_PROBE_FFMA, "ffma2": ITP_PROBE_FFMA2, "dfma": ITP_PROBE_DFMA,
               "tf32_mma": ITP_PROBE_TF32_MMA}


def itp_peak_probe(kind, cuda_stream: int = 0):
    """Measured rate of one kind of arithmetic on the current device:
    returns (TFLOP/s, ms per probe launch)."""
    t = ctypes.c_double()
    ms = ctypes.c_double()
    code = load().itp_peak_probe(PROBE_KINDS.get(kind, kind), ctypes.c_void_p(cuda_stream or None),
                                 ctypes.byref(t), ctypes.byref(ms))
    if code != ITP_OK:
        raise ItpError(code, f"itp_peak_probe({kind}) failed")
    return t.value, ms.value


def itp_get_tuning(h) -> dict:
    t = (ctypes.c_int * ITP_TUNING_LEN)()
    _check(h, load().itp_get_tuning(h, t))
    return {"pencil_w": t[0], "split": t[1], "row_tb": t[2], "gram_ctas": t[3]}


def itp_set_tuning(h, pencil_w, split, row_tb, gram_ctas):
    t = (ctypes.c_int * ITP_TUNING_LEN)(int(pencil_w), int(split), int(row_tb), int(gram_ctas))
    _check(h, load().itp_set_tuning(h, t))


def itp_autotune(h, order, tau):
    """Returns (chosen shapes as a dict, the candidates' timing report)."""
    t = (ctypes.c_int * ITP_TUNING_LEN)()
    rep = ctypes.create_string_buffer(1024)
    _check(h, load().itp_autotune(h, int(order), float(tau), t, rep, len(rep)))
    return ({"pencil_w": t[0], "split": t[1], "row_tb": t[2], "gram_ctas": t[3]},
            rep.value.decode())


def _check_batch(b, code: int):
    if code != ITP_OK:
        msg = load().itp_batch_last_error(b)
        raise ItpError(code, msg.decode() if msg else "")


def itp_create_batch(dims, boxes, n_states, n_guard=None, precision=ITP_MIXED, cuda_stream=0):
    """dims: (count, 3) ints (nx, ny, nz); boxes: (count, 3) box lengths."""
    dims = np.ascontiguousarray(dims, dtype=np.int32).reshape(-1, 3)
    boxes = np.ascontiguousarray(boxes, dtype=np.float64).reshape(-1, 3)
    ns = np.ascontiguousarray(n_states, dtype=np.int32)
    count = dims.shape[0]
    if boxes.shape[0] != count or ns.size != count:
        raise ValueError("dims, boxes and n_states need one entry per problem")
    ng = None if n_guard is None else np.ascontiguousarray(n_guard, dtype=np.int32)
    if ng is not None and ng.size != count:
        raise ValueError("n_guard needs one entry per problem")
    b = _H()
    code = load().itp_create_batch(ctypes.byref(b), count, dims.ctypes.data, boxes.ctypes.data,
                                   ns.ctypes.data, None if ng is None else ng.ctypes.data,
                                   precision, ctypes.c_void_p(cuda_stream or None))
    _check_batch(None, code)
    return b


def itp_batch_problem(b, p: int):
    h = load().itp_batch_problem(b, int(p))
    if not h:
        raise IndexError(f"no problem {p} in the batch")
    return _H(h)


def itp_batch_step(b, order, tau, flags=ITP_RITZ_VALUES, out: np.ndarray | None = None):
    ptr = None if out is None else out.ctypes.data
    _check_batch(b, load().itp_batch_step(b, int(order), float(tau), int(flags), ptr))
    return out


def itp_batch_destroy(b):
    load().itp_batch_destroy(b)


# ---- a thin object wrapper -----------------------------------------------------
class ItpGrid:
    """One problem on the GPU: owns an itp_handle."""

    def __init__(self, nx, ny, nz, lx, ly, lz, n_states, n_guard=0, precision=ITP_FP64,
                 cuda_stream=0):
        self.shape = (nz, ny, nx)
        self.n_points = nx * ny * nz
        self.n_states, self.n_guard = n_states, n_guard
        self.m = n_states + n_guard
        self.h = itp_create_grid(nx, ny, nz, lx, ly, lz, n_states, n_guard, precision,
                                 cuda_stream)

    @classmethod
    def borrowed(cls, h, shape, n_states, n_guard):
        """Wrap a handle owned elsewhere (a problem of an ItpBatch)."""
        self = cls.__new__(cls)
        nz, ny, nx = shape
        self.shape = (nz, ny, nx)
        self.n_points = nx * ny * nz
        self.n_states, self.n_guard = n_states, n_guard
        self.m = n_states + n_guard
        self.h = h
        self._owner = False
        return self

    def close(self):
        if self.h and getattr(self, "_owner", True):
            itp_destroy(self.h)
        self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_potential(self, V):
        itp_set_potential(self.h, _f64(V, self.n_points))

    def set_states(self, psi):
        itp_set_states(self.h, _f64(psi, self.m * self.n_points))

    def get_states(self):
        out = np.empty((self.m, self.n_points), dtype=np.float64)
        return itp_get_states(self.h, out)

    def get_phi(self):
        out = np.empty((self.m, self.n_points), dtype=np.float64)
        return itp_get_phi(self.h, out)

    def propagate(self, order, tau):
        itp_propagate(self.h, order, tau)

    def orthonormalize(self):
        itp_orthonormalize(self.h)

    def propagate_romberg6(self, tau):
        itp_propagate_romberg6(self.h, tau)

    def energies(self, ritz=True, fp64=False):
        """ritz: True (values + rotation), "values" (values only) or False
        (diagonal expectation values).  fp64: the mixed path's final
        evaluation in FP64 (ITP_EVAL_FP64)."""
        flags = ITP_RITZ_VALUES if ritz == "values" else (ITP_RITZ if ritz else 0)
        if fp64:
            flags |= ITP_EVAL_FP64
        out = np.empty(self.m, dtype=np.float64)
        return itp_energies(self.h, out, flags)

    def step(self, order, tau, ritz=True):
        self.propagate(order, tau)
        self.orthonormalize()
        return self.energies(ritz)

    def step_graph(self, order, tau, ritz="values"):
        """One step replayed from a CUDA graph (Ritz values or, with
        ritz=False, diagonal energies)."""
        out = np.empty(self.m, dtype=np.float64)
        return itp_step(self.h, order, tau, ITP_RITZ_VALUES if ritz else 0, out)

    def step_host(self, order, tau, psi_in, psi_out=None, ritz="values"):
        """One step from host states psi_in to host states psi_out (new
        array if None), copies overlapped with the device work; returns
        (psi_out, energies)."""
        if psi_out is None:
            psi_out = np.empty((self.m, self.n_points), dtype=np.float64)
        E = np.empty(self.m, dtype=np.float64)
        itp_step_host(self.h, self.m, self.n_points, order, tau, psi_in, psi_out,
                      ITP_RITZ_VALUES if ritz else 0, E)
        return psi_out, E

    def polish(self, order, tau, tol, max_steps):
        out = np.empty(self.m, dtype=np.float64)
        steps = itp_polish(self.h, order, tau, tol, max_steps, out)
        return steps, out

    def synchronize(self):
        itp_synchronize(self.h)

    def test_expire_waits(self, launches):
        itp_test_expire_waits(self.h, launches)

    def solve_adaptive(self, order, tau0, reduce, gamma, max_steps=200, max_levels=12):
        return itp_solve_adaptive(self.h, self.m, order, tau0, reduce, gamma, max_steps,
                                  max_levels)

    def get_tuning(self):
        return itp_get_tuning(self.h)

    def set_tuning(self, pencil_w, split, row_tb, gram_ctas):
        itp_set_tuning(self.h, pencil_w, split, row_tb, gram_ctas)

    def autotune(self, order, tau):
        return itp_autotune(self.h, order, tau)

    @property
    def kernel_launches(self):
        return itp_kernel_launches(self.h)

    def profile(self, enable=True):
        itp_profile(self.h, enable)

    def profile_read(self):
        """{kind name: (launches, total ms)} since the last profile() call."""
        return {name: itp_profile_read(self.h, k) for k, name in enumerate(KERNEL_KINDS)}


class ItpBatch:
    """Independent problems of uneven size advanced together (one CUDA graph
    launch per step of all of them); owns an itp_batch_handle."""

    def __init__(self, dims, boxes, n_states, n_guard=None, precision=ITP_MIXED, cuda_stream=0):
        dims = np.asarray(dims, dtype=np.int64).reshape(-1, 3)
        ng = np.zeros(len(dims), dtype=np.int64) if n_guard is None else np.asarray(n_guard)
        self.b = itp_create_batch(dims, boxes, n_states, n_guard, precision, cuda_stream)
        self.problems = [ItpGrid.borrowed(itp_batch_problem(self.b, p),
                                          (int(d[2]), int(d[1]), int(d[0])), int(n), int(g))
                         for p, (d, n, g) in enumerate(zip(dims, n_states, ng))]
        self.m_total = sum(q.m for q in self.problems)

    def __len__(self):
        return len(self.problems)

    def __getitem__(self, p):
        return self.problems[p]

    def step(self, order, tau, ritz=True, fp64=False):
        """One step of every problem; returns the list of per-problem energies."""
        flags = (ITP_RITZ_VALUES if ritz else 0) | (ITP_STEP_FP64 if fp64 else 0)
        out = np.empty(self.m_total, dtype=np.float64)
        itp_batch_step(self.b, order, tau, flags, out)
        res, off = [], 0
        for q in self.problems:
            res.append(out[off:off + q.m])
            off += q.m
        return res

    @property
    def kernel_launches(self):
        return int(load().itp_batch_kernel_launches(self.b))

    def set_grouping(self, grouped: bool):
        """Grouped launches per pass over problems of one grid (default) or
        one graph branch per problem (itp_batch_set_grouping)."""
        _check_batch(self.b, load().itp_batch_set_grouping(self.b, 1 if grouped else 0))

    @property
    def groups(self):
        return int(load().itp_batch_groups(self.b))

    def close(self):
        if self.b:
            for q in self.problems:
                q.h = None
            itp_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
