"""Thin ctypes binding of the C ABI declared in include/nmf.h.

Argument marshalling only: every step of the computation runs in the CUDA
library.  Array arguments may be numpy arrays (host memory) or CUDA torch
tensors (device memory); both must be C-contiguous float32 (float64 for
outputs that are doubles).  Loading fails loudly if the library is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

NMF_HALS, NMF_MU, NMF_ANLS, NMF_ANLS_BPP = 0, 1, 2, 3
NMF_FP32, NMF_BF16, NMF_BF16_FP32, NMF_AUTO = 0, 1, 2, 3
NMF_VCYCLE, NMF_NESTED, NMF_FMG, NMF_WCYCLE = 0, 1, 2, 3
NMF_OK, NMF_EINVAL, NMF_ENOMEM, NMF_ENOCONV, NMF_ECUDA, NMF_ETIMEOUT, NMF_EBUSY, NMF_ETOOBIG = 0, -1, -2, -3, -4, -5, -6, -7
ALGOS = {"hals": NMF_HALS, "mu": NMF_MU, "anls": NMF_ANLS, "anls_bpp": NMF_ANLS_BPP}
CYCLES = {"vcycle": NMF_VCYCLE, "ni": NMF_NESTED, "fmg": NMF_FMG, "wcycle": NMF_WCYCLE}

STATUS = {0: "NMF_OK", -1: "NMF_EINVAL", -2: "NMF_ENOMEM", -3: "NMF_ENOCONV", -4: "NMF_ECUDA",
          -5: "NMF_ETIMEOUT", -6: "NMF_EBUSY", -7: "NMF_ETOOBIG"}

# (name, restype, argtypes) of every exported entry point of include/nmf.h
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
SIGNATURES = [
    ("nmf_create", _I, [ctypes.POINTER(_P), _I, ctypes.c_size_t, _I]),
    ("nmf_destroy", None, [_P]),
    ("nmf_last_error", ctypes.c_char_p, [_P]),
    ("nmf_solve", _I, [_P, _P, _I64, _I64, _I, _I, _I, _I, _I, _I, _P, _P]),
    ("nmf_solve_ex", _I, [_P, _P, _I64, _I64, _I, _I, _I, _I, _I, _I, _P, _P, _P]),
    ("nmf_error", _I, [_P, _P, _P, _P, _I64, _I64, _I, ctypes.POINTER(ctypes.c_double)]),
    ("nmf_schedule", _I64, [_I, _I, _I, ctypes.POINTER(_I64)]),
    ("nmf_time_schedule", _I, [_I, ctypes.c_double, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I64)]),
    ("nmf_restrict", _I, [_P, _P, _I, _I, _I64, _P]),
    ("nmf_prolong", _I, [_P, _P, _I, _I, _I64, _P]),
    ("nmf_products", _I, [_P, _P, _P, _P, _I64, _I64, _I, _P, _P, _P, _P]),
    ("nmf_sweep", _I, [_P, _P, _I64, _I64, _I, _I, _I, _P, _P]),
    ("nmf_device_info", _I, [_P, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_char_p)]),
    ("nmf_set_stream", _I, [_P, _P]),
    ("nmf_last_launch_count", _I64, [_P]),
    ("nmf_set_limits", _I, [_P, _I, _I64]),
    ("nmf_profile_sweep", _I, [_P, _P, _I64, _I64, _I, _I, _P, _P, _I, ctypes.POINTER(ctypes.c_float)]),
    ("nmf_profile_coarse", _I, [_P, _P, _I64, _I64, _I, _I, _P, _P, _I, ctypes.POINTER(ctypes.c_float)]),
    ("nmf_error_noalloc", _I, [_P, _P, _P, _I64, _I64, _I, _P, ctypes.POINTER(ctypes.c_double)]),
    ("nmf_solve_batch", _I, [_P, _P, _I]),
    ("nmf_solve_grouped", _I, [_P, _P, _I]),
    ("nmf_workspace_bytes", _I64, [_P, _P, _I]),
    ("nmf_release_workspace", _I, [_P]),
    ("nmf_server_create", _I, [ctypes.POINTER(_P), _I, ctypes.c_size_t, _I, _I]),
    ("nmf_server_submit", _I64, [_P, _P]),
    ("nmf_server_poll", _I, [_P, _I64, _I, ctypes.POINTER(ctypes.c_double)]),
    ("nmf_server_stats", _I, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                              ctypes.POINTER(_I64)]),
    ("nmf_server_destroy", None, [_P]),
]


class Problem(ctypes.Structure):
    """nmf_problem of include/nmf.h."""
    _fields_ = [("M", _P), ("m", _I64), ("n", _I64), ("grid_h", _I), ("grid_w", _I), ("r", _I), ("algo", _I),
                ("levels", _I), ("iters", _I), ("cycle", _I), ("rel_tol", ctypes.c_double), ("V", _P), ("W", _P),
                ("status", _I), ("sweeps_run", _I64), ("objective", ctypes.c_double),
                ("level_sweeps", ctypes.POINTER(_I64))]


class Options(ctypes.Structure):
    _fields_ = [("cycle", _I), ("stop_after", _I64), ("trace", ctypes.POINTER(ctypes.c_double)),
                ("trace_len", _I64), ("trace_count", ctypes.POINTER(_I64)), ("level_sweeps", ctypes.POINTER(_I64)),
                ("coarsen_columns", _I)]


def _flat_level_sweeps(level_sweeps, levels: int):
    """(pre, coarse, post) -> the 2 levels - 1 counts in run order (nmf_options.level_sweeps)."""
    pre, coarse, post = level_sweeps
    if len(pre) != levels - 1 or len(post) != levels - 1:
        raise ValueError("level_sweeps needs levels - 1 before- and after-counts")
    return np.array(list(pre) + [coarse] + list(post)[::-1], dtype=np.int64)


class NMFError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.lib_path()


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load the shared library (raise if it is absent; never fall back)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError(f"GB300 NMF library not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(x):
    """Device or host address of a contiguous float array (numpy or torch)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported array type {type(x)}")


def _check_f32(*arrs):
    for a in arrs:
        if a is None:
            continue
        dt = getattr(a, "dtype", None)
        if isinstance(a, np.ndarray):
            if dt != np.float32:
                raise TypeError("float32 arrays required")
        elif str(dt) != "torch.float32":
            raise TypeError("float32 tensors required")


class Handle:
    """An nmf_handle: device workspaces, stream and cached CUDA graphs."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, precision: int = NMF_FP32):
        self.lib = load()
        h = _P()
        rc = self.lib.nmf_create(ctypes.byref(h), device, hbm_budget_bytes, precision)
        if rc != 0:
            raise NMFError(rc, "nmf_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.nmf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _rc(self, rc: int):
        if rc != 0:
            raise NMFError(rc, self.lib.nmf_last_error(self.h).decode())
        return rc

    # --- entry points -------------------------------------------------------
    def solve(self, M, grid_h: int, grid_w: int, V, W, algo="hals", levels: int = 1, iters: int = 100,
              cycle="vcycle", stop_after: int = 0, trace_len: int = 0, coarsen_columns: bool = False,
              level_sweeps=None):
        """nmf_solve_ex: improves V (m x r) and W (r x n) in place; returns the objective trace if asked.
        coarsen_columns: the columns of M are a smooth sequence, coarsened by the V-cycle too.
        level_sweeps: (pre, coarse, post) explicit V-cycle counts, pre[l] / post[l] the sweeps of
        level l + 1 before / after the coarser cycle (as time_schedule returns them)."""
        _check_f32(M, V, W)
        m, n = M.shape
        r = V.shape[1]
        opt = Options()
        opt.cycle = CYCLES[cycle] if isinstance(cycle, str) else int(cycle)
        opt.stop_after = stop_after
        opt.coarsen_columns = 1 if coarsen_columns else 0
        counts = None
        if level_sweeps is not None:
            counts = _flat_level_sweeps(level_sweeps, levels)
            opt.level_sweeps = counts.ctypes.data_as(ctypes.POINTER(_I64))
        trace = None
        count = _I64(0)
        if trace_len > 0:
            trace = np.zeros(trace_len, dtype=np.float64)
            opt.trace = trace.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            opt.trace_len = trace_len
        opt.trace_count = ctypes.pointer(count)
        a = ALGOS[algo] if isinstance(algo, str) else int(algo)
        self._rc(self.lib.nmf_solve_ex(self.h, _ptr(M), m, n, grid_h, grid_w, r, a, levels, iters,
                                       ctypes.byref(opt), _ptr(V), _ptr(W)))
        if trace is not None:
            return trace[: min(count.value, trace_len)]
        return None

    def solve_batch(self, problems, grouped: bool = False):
        """nmf_solve_batch (grouped=True: nmf_solve_grouped).  `problems`: list of dicts with keys
        M, grid_h, grid_w, V, W and optional algo, levels, iters, cycle, rel_tol.  V and W are
        improved in place; returns a list of (status, sweeps_run, objective)."""
        arr = (Problem * len(problems))()
        for q, d in zip(arr, problems):
            fill_problem(q, d)
        fn = self.lib.nmf_solve_grouped if grouped else self.lib.nmf_solve_batch
        rc = fn(self.h, ctypes.cast(arr, _P), len(problems))
        out = [(q.status, q.sweeps_run, q.objective) for q in arr]
        if rc != 0 and all(s == 0 for s, _, _ in out):
            self._rc(rc)
        return out

    def workspace_bytes(self, d) -> int:
        """nmf_workspace_bytes: device bytes for a problem dict, or a list of them solved together."""
        ds = d if isinstance(d, (list, tuple)) else [d]
        arr = (Problem * len(ds))()
        for q, x in zip(arr, ds):
            fill_problem(q, x)
        b = int(self.lib.nmf_workspace_bytes(self.h, ctypes.cast(arr, _P), len(ds)))
        if b < 0:
            self._rc(b)
        return b

    def release_workspace(self):
        self._rc(self.lib.nmf_release_workspace(self.h))

    def solve_plain(self, M, grid_h, grid_w, V, W, algo="hals", levels=1, iters=100):
        """nmf_solve (V-cycle, no options)."""
        _check_f32(M, V, W)
        m, n = M.shape
        a = ALGOS[algo] if isinstance(algo, str) else int(algo)
        return self._rc(self.lib.nmf_solve(self.h, _ptr(M), m, n, grid_h, grid_w, V.shape[1], a, levels, iters,
                                           _ptr(V), _ptr(W)))

    def sweep(self, M, V, W, algo="hals", sweeps: int = 1):
        _check_f32(M, V, W)
        m, n = M.shape
        a = ALGOS[algo] if isinstance(algo, str) else int(algo)
        self._rc(self.lib.nmf_sweep(self.h, _ptr(M), m, n, V.shape[1], a, sweeps, _ptr(V), _ptr(W)))

    def error(self, M, V, W) -> float:
        _check_f32(M, V, W)
        m, n = M.shape
        out = ctypes.c_double(0.0)
        self._rc(self.lib.nmf_error(self.h, _ptr(M), _ptr(V), _ptr(W), m, n, V.shape[1], ctypes.byref(out)))
        return out.value

    def restrict(self, X, grid_h: int, grid_w: int, Y):
        _check_f32(X, Y)
        self._rc(self.lib.nmf_restrict(self.h, _ptr(X), grid_h, grid_w, X.shape[1], _ptr(Y)))

    def prolong(self, Y, grid_h: int, grid_w: int, X):
        _check_f32(X, Y)
        self._rc(self.lib.nmf_prolong(self.h, _ptr(Y), grid_h, grid_w, Y.shape[1], _ptr(X)))

    def products(self, M, V, W, A=None, B=None, C=None, D=None):
        _check_f32(M, V, W, A, B, C, D)
        m, n = M.shape
        self._rc(self.lib.nmf_products(self.h, _ptr(M), _ptr(V), _ptr(W), m, n, V.shape[1], _ptr(A), _ptr(B),
                                       _ptr(C), _ptr(D)))

    def device_info(self):
        sms = _I(0)
        tag = ctypes.c_char_p()
        self._rc(self.lib.nmf_device_info(self.h, ctypes.byref(sms), ctypes.byref(tag)))
        return sms.value, tag.value.decode()


    def set_stream(self, stream_ptr: int | None):
        """nmf_set_stream: run on the given cudaStream_t (an int address), None = own stream."""
        self._rc(self.lib.nmf_set_stream(self.h, stream_ptr or None))

    def set_limits(self, nnls_max_exchanges: int = -1, barrier_spins: int = -1):
        """nmf_set_limits: ANLS exchange cap and grid-barrier spin budget (-1 = defaults)."""
        self._rc(self.lib.nmf_set_limits(self.h, int(nnls_max_exchanges), int(barrier_spins)))

    def last_launch_count(self) -> int:
        return int(self.lib.nmf_last_launch_count(self.h))

    def profile_sweep(self, M, V, W, algo="hals", reps: int = 20) -> list[float]:
        """nmf_profile_sweep: mean ms per launch of [V-step products, V update, W-step products, W update, error]."""
        _check_f32(M, V, W)
        m, n = M.shape
        out = (ctypes.c_float * 5)()
        a = ALGOS[algo] if isinstance(algo, str) else int(algo)
        self._rc(self.lib.nmf_profile_sweep(self.h, _ptr(M), m, n, V.shape[1], a, _ptr(V), _ptr(W), reps, out))
        return list(out)

    def profile_coarse(self, M, V, W, algo="hals", sweeps: int = 100) -> float | None:
        """nmf_profile_coarse: mean ms per sweep of the persistent coarse-level kernel,
        or None when the kernel does not apply to this shape (NMF_EINVAL)."""
        _check_f32(M, V, W)
        m, n = M.shape
        out = ctypes.c_float(0.0)
        a = ALGOS[algo] if isinstance(algo, str) else int(algo)
        rc = self.lib.nmf_profile_coarse(self.h, _ptr(M), m, n, V.shape[1], a, _ptr(V), _ptr(W), sweeps,
                                         ctypes.byref(out))
        if rc == -1:  # NMF_EINVAL
            return None
        self._rc(rc)
        return float(out.value)


def fill_problem(q: Problem, d: dict) -> Problem:
    """Marshal a problem dict (M, grid_h, grid_w, V, W, algo, levels, iters, cycle, rel_tol and
    optionally level_sweeps = (pre, coarse, post)) into q."""
    _check_f32(d["M"], d["V"], d["W"])
    q.M = _ptr(d["M"])
    q.m, q.n = d["M"].shape
    q.grid_h, q.grid_w = d["grid_h"], d["grid_w"]
    q.r = d["V"].shape[1]
    algo = d.get("algo", "hals")
    q.algo = ALGOS[algo] if isinstance(algo, str) else int(algo)
    q.levels = d.get("levels", 1)
    q.iters = d.get("iters", 100)
    cyc = d.get("cycle", "vcycle")
    q.cycle = CYCLES[cyc] if isinstance(cyc, str) else int(cyc)
    q.rel_tol = d.get("rel_tol", 0.0)
    q.V = _ptr(d["V"])
    q.W = _ptr(d["W"])
    if d.get("level_sweeps") is not None:
        # kept in the dict: the library reads it until the solve or the served request ends
        d["_level_sweeps_flat"] = _flat_level_sweeps(d["level_sweeps"], q.levels)
        q.level_sweeps = d["_level_sweeps_flat"].ctypes.data_as(ctypes.POINTER(_I64))
    return q


class Server:
    """nmf_server: continuous-batching request loop (native threads, one stream per slot)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, slots: int = 4, precision: int = NMF_FP32):
        self.lib = load()
        s = _P()
        rc = self.lib.nmf_server_create(ctypes.byref(s), device, hbm_budget_bytes, slots, precision)
        if rc != 0:
            raise NMFError(rc, "nmf_server_create failed")
        self.s = s
        self._keep = {}

    def submit(self, d: dict) -> int:
        """Queue a problem dict; the arrays in it must stay alive until the ticket completes."""
        q = fill_problem(Problem(), d)
        t = int(self.lib.nmf_server_submit(self.s, ctypes.byref(q)))
        if t < 0:
            raise NMFError(t, "nmf_server_submit failed")
        self._keep[t] = (q, d)
        return t

    def poll(self, ticket: int, wait_ms: int = -1):
        """Returns None while running, else (status, sweeps_run, objective, latency_ms)."""
        lat = ctypes.c_double(0.0)
        rc = self.lib.nmf_server_poll(self.s, ticket, wait_ms, ctypes.byref(lat))
        if rc == -6:
            return None
        q, _ = self._keep.pop(ticket)
        return rc, q.sweeps_run, q.objective, lat.value

    def stats(self):
        v = [_I64(0) for _ in range(4)]
        self.lib.nmf_server_stats(self.s, *[ctypes.byref(x) for x in v])
        return dict(zip(("queued", "running", "completed", "bytes_held"), (x.value for x in v)))

    def close(self):
        if getattr(self, "s", None):
            self.lib.nmf_server_destroy(self.s)
            self.s = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def error_noalloc(M, V, W, stream_ptr: int | None = None) -> float:
    """nmf_error_noalloc: ||M - VW||_F for device tensors, with no device allocation by the library."""
    _check_f32(M, V, W)
    lib = load()
    m, n = M.shape
    out = ctypes.c_double(0.0)
    rc = lib.nmf_error_noalloc(_ptr(M), _ptr(V), _ptr(W), m, n, V.shape[1], stream_ptr or None, ctypes.byref(out))
    if rc != 0:
        raise NMFError(rc, "nmf_error_noalloc failed")
    return out.value


def schedule(cycle: str, levels: int, iters: int) -> list[int]:
    """nmf_schedule: sweeps per level (host-only, no GPU needed)."""
    lib = load()
    out = (_I64 * levels)()
    total = lib.nmf_schedule(CYCLES[cycle], levels, iters, out)
    if total < 0:
        raise NMFError(int(total), "nmf_schedule failed")
    return list(out)


def time_schedule(budget: float, costs) -> tuple[list[int], int, list[int]]:
    """nmf_time_schedule: (pre, coarse, post) V-cycle counts for a time budget and per-level
    sweep costs (host-only, no GPU needed)."""
    lib = load()
    L = len(costs)
    if L < 1:
        raise NMFError(NMF_EINVAL, "time_schedule needs at least one level")
    c = (ctypes.c_double * L)(*[float(x) for x in costs])
    out = (_I64 * (2 * L - 1))()
    rc = lib.nmf_time_schedule(L, float(budget), c, out)
    if rc != 0:
        raise NMFError(int(rc), "nmf_time_schedule failed")
    flat = list(out)
    return flat[:L - 1], flat[L - 1], flat[L:][::-1]

