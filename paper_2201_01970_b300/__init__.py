"""Python binding of libcpr_b300.so, the B300 CPR-preconditioned FGMRES library.

Argument marshalling only: every step of the method runs in the library's CUDA
kernels (include/cpr.h documents each call).  Arrays may be numpy arrays (host)
or torch CUDA tensors (device); the library detects which.  There is no CPU
fallback: importing works without a GPU, but every call needs the CUDA
library, and a missing library raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcpr_b300.so")

CPR_OK = 0
CPR_NOT_CONVERGED = 1
CPR_RUNNING = 2
CPR_ERR_INVALID = -1
CPR_ERR_CUDA = -2
CPR_ERR_OOM = -3
CPR_ERR_SINGULAR = -4
CPR_ERR_BREAKDOWN = -5
CPR_ERR_TIMEOUT = -6


class Opts(C.Structure):
    _fields_ = [("theta_color", C.c_double), ("theta_amg", C.c_double), ("mu", C.c_int),
                ("restart", C.c_int), ("max_restarts", C.c_int), ("precond_fp32", C.c_int),
                ("decouple", C.c_int), ("pre", C.c_int), ("post", C.c_int),
                ("coarse_max", C.c_int), ("max_levels", C.c_int), ("seed", C.c_uint64),
                ("stream", C.c_void_p), ("pdl", C.c_int), ("tail", C.c_int), ("bilu_order", C.c_int),
                ("reuse_refresh", C.c_int), ("resetup", C.c_int), ("amg", C.c_int),
                ("amli_iters", C.c_int), ("coloring", C.c_int), ("coloring_rows", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("setup_called", C.c_int),
                ("setup_count", C.c_int), ("levels", C.c_int), ("converged", C.c_int),
                ("rel_res", C.c_double), ("setup_ms", C.c_double), ("solve_ms", C.c_double),
                ("tail_levels", C.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class Bsr3(C.Structure):
    _fields_ = [("nb", C.c_int32), ("nnzb", C.c_int32), ("rowptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p)]


class LevelInfo(C.Structure):
    _fields_ = [("n", C.c_int), ("nnz", C.c_int), ("ncolors", C.c_int), ("nc", C.c_int),
                ("nnz_p", C.c_int)]


class Schedule(C.Structure):
    _fields_ = [("lanes_a", C.c_int), ("lanes_p", C.c_int), ("lanes_r", C.c_int), ("block", C.c_int)]


class CprError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        detail = ""
        try:
            detail = lib().cpr_last_error_detail().decode()
        except Exception:
            pass
        msg = lib().cpr_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {msg} ({code}) {detail}".strip())


_lib = None


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_2201_01970_b300.build.build() (nvcc, sm_103a)")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.cpr_default_opts.argtypes = [C.POINTER(Opts)]
        L.cpr_setup.argtypes = [C.POINTER(vp), C.POINTER(Bsr3), C.POINTER(Opts)]
        L.cpr_update.argtypes = [vp, C.POINTER(Bsr3)]
        L.cpr_update_values.argtypes = [vp, vp]
        L.cpr_solve.argtypes = [vp, vp, vp, C.c_double, C.POINTER(Stats)]
        L.cpr_solve_start.argtypes = [vp, vp, vp, C.c_double]
        L.cpr_solve_poll.argtypes = [vp, C.POINTER(Stats)]
        L.cpr_destroy.argtypes = [vp]
        L.cpr_strerror.argtypes = [C.c_int]
        L.cpr_strerror.restype = C.c_char_p
        L.cpr_last_error_detail.restype = C.c_char_p
        L.cpr_apply.argtypes = [vp, vp, vp]
        L.cpr_vcycle.argtypes = [vp, vp, vp]
        L.cpr_bilu_apply.argtypes = [vp, vp, vp]
        L.cpr_bilu_apply_noalloc.argtypes = [vp, vp, vp]
        L.cpr_set_memory_limit.argtypes = [C.c_uint64]
        L.cpr_memory_in_use.restype = C.c_uint64
        L.cpr_bsr3_spmv.argtypes = [C.POINTER(Bsr3), vp, vp, vp, vp]
        L.cpr_num_levels.argtypes = [vp]
        L.cpr_get_level_info.argtypes = [vp, C.c_int, C.POINTER(LevelInfo)]
        L.cpr_copy_level.argtypes = [vp, C.c_int] + [vp] * 8
        L.cpr_copy_weights.argtypes = [vp, vp]
        L.cpr_copy_bilu.argtypes = [vp, vp, vp, C.POINTER(C.c_int)]
        L.cpr_batch_setup.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(Bsr3), C.POINTER(Opts)]
        L.cpr_batch_update.argtypes = [vp, C.POINTER(Bsr3)]
        L.cpr_batch_solve.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.c_double, C.POINTER(Stats)]
        L.cpr_batch_size.argtypes = [vp]
        L.cpr_launch_count.restype = C.c_uint64
        L.cpr_profile.argtypes = [vp, C.c_int]
        L.cpr_profile_read.argtypes = [vp, C.c_int, C.POINTER(C.c_long), C.POINTER(C.c_double)]
        L.cpr_profile_vcycle_levels.argtypes = [vp, C.c_int, vp, C.c_int]
        L.cpr_get_schedule.argtypes = [vp, C.c_int, C.POINTER(Schedule)]
        L.cpr_set_schedule.argtypes = [vp, C.c_int, C.POINTER(Schedule)]
        L.cpr_autotune.argtypes = [vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        _lib = L
    return _lib


def _check(rc: int, where: str, allow_not_converged: bool = False) -> int:
    if rc == CPR_OK or (allow_not_converged and rc == CPR_NOT_CONVERGED):
        return rc
    raise CprError(rc, where)


def _ptr(a) -> int:
    """Address of a numpy array or torch tensor (contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _as_bsr3(A) -> tuple:
    """A Bsr3 descriptor for an object with nb, rowptr, col, val (numpy or torch)."""
    rowptr, col, val = A.rowptr, A.col, A.val
    if isinstance(rowptr, np.ndarray):
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        col = np.ascontiguousarray(col, dtype=np.int32)
        val = np.ascontiguousarray(val, dtype=np.float64)
    nb = int(A.nb)
    d = Bsr3(nb, int(col.shape[0]), _ptr(rowptr), _ptr(col), _ptr(val))
    return d, (rowptr, col, val)


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().cpr_default_opts(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def _torch_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


class Solver:
    """A cpr_handle: setup(A) at construction, update(A) per Newton step, solve(b)."""

    def __init__(self, A, **opts):
        if "stream" not in opts:
            opts["stream"] = _torch_stream()
        self.opts = default_opts(**opts)
        self._h = C.c_void_p()
        d, keep = _as_bsr3(A)
        _check(lib().cpr_setup(C.byref(self._h), C.byref(d), C.byref(self.opts)), "cpr_setup")
        self.nb, self.nnzb = d.nb, d.nnzb

    def update(self, A) -> None:
        d, keep = _as_bsr3(A)
        _check(lib().cpr_update(self._h, C.byref(d)), "cpr_update")
        self.nb, self.nnzb = d.nb, d.nnzb

    def update_values(self, val) -> None:
        """cpr_update_values: a new Jacobian with the current pattern (its 9 nnzb values only)."""
        if isinstance(val, np.ndarray):
            val = np.ascontiguousarray(val, dtype=np.float64)
        _check(lib().cpr_update_values(self._h, _ptr(val)), "cpr_update_values")

    def solve(self, b, x=None, rtol: float = 1e-6):
        """Solve A x = b; returns (x, stats).  x (initial guess) is overwritten in place."""
        if x is None:
            if isinstance(b, np.ndarray):
                x = np.zeros_like(b, dtype=np.float64)
            else:
                import torch
                x = torch.zeros_like(b)
        st = Stats()
        rc = lib().cpr_solve(self._h, _ptr(b), _ptr(x), float(rtol), C.byref(st))
        _check(rc, "cpr_solve", allow_not_converged=True)
        return x, st.as_dict()

    def solve_start(self, b, x, rtol: float = 1e-6) -> None:
        """Start a solve without waiting (cpr_solve_start); b and x must stay
        alive until poll() reports the end."""
        self._pending = (b, x)
        _check(lib().cpr_solve_start(self._h, _ptr(b), _ptr(x), float(rtol)), "cpr_solve_start")

    def poll(self):
        """Advance a started solve (cpr_solve_poll): None while it runs, else
        (x, stats) once it has finished."""
        st = Stats()
        rc = lib().cpr_solve_poll(self._h, C.byref(st))
        if rc == CPR_RUNNING:
            return None
        x = self._pending[1]
        self._pending = None
        _check(rc, "cpr_solve_poll", allow_not_converged=True)
        return x, st.as_dict()

    # component applications (device tensors)
    def apply(self, v, z) -> None:
        _check(lib().cpr_apply(self._h, _ptr(v), _ptr(z)), "cpr_apply")

    def vcycle(self, b, x) -> None:
        _check(lib().cpr_vcycle(self._h, _ptr(b), _ptr(x)), "cpr_vcycle")

    def bilu_apply(self, r, z) -> None:
        _check(lib().cpr_bilu_apply(self._h, _ptr(r), _ptr(z)), "cpr_bilu_apply")

    def bilu_apply_noalloc(self, r, z) -> None:
        """cpr_bilu_apply_noalloc: z = R r with no device allocation in the call."""
        _check(lib().cpr_bilu_apply_noalloc(self._h, _ptr(r), _ptr(z)), "cpr_bilu_apply_noalloc")

    # inspection (host numpy copies, natural numbering)
    @property
    def nlev(self) -> int:
        return lib().cpr_num_levels(self._h)

    def level(self, l: int) -> dict:
        info = LevelInfo()
        _check(lib().cpr_get_level_info(self._h, l, C.byref(info)), "cpr_get_level_info")
        n, nnz, nnzp = info.n, info.nnz, info.nnz_p
        out = {"n": n, "nnz": nnz, "ncolors": info.ncolors, "nc": info.nc, "nnz_p": nnzp,
               "rowptr": np.zeros(n + 1, np.int32), "col": np.zeros(nnz, np.int32),
               "val": np.zeros(nnz), "color": np.zeros(n, np.int32), "cf": np.zeros(n, np.int32),
               "prow": np.zeros(n + 1, np.int32), "pcol": np.zeros(nnzp, np.int32),
               "pval": np.zeros(nnzp)}
        keys = ["rowptr", "col", "val", "color", "cf", "prow", "pcol", "pval"]
        _check(lib().cpr_copy_level(self._h, l, *[_ptr(out[k]) if out[k].size else None
                                                  for k in keys]), "cpr_copy_level")
        if not info.ncolors:
            out["color"] = None
        if not info.nc:
            out["cf"] = out["prow"] = out["pcol"] = out["pval"] = None
        return out

    def weights(self) -> np.ndarray:
        w = np.zeros(3 * self.nb)
        _check(lib().cpr_copy_weights(self._h, _ptr(w)), "cpr_copy_weights")
        return w

    def bilu(self):
        bc = np.zeros(self.nb, np.int32)
        lu = np.zeros(9 * self.nnzb)
        nc = C.c_int()
        _check(lib().cpr_copy_bilu(self._h, _ptr(bc), _ptr(lu), C.byref(nc)), "cpr_copy_bilu")
        return bc, nc.value, lu

    def profile(self, enable: bool = True, families=None) -> None:
        """Bracket the given PROF_* families (all when None) in later solves."""
        mask = 0
        if enable:
            mask = (1 << 6) - 1 if families is None else sum(1 << f for f in families)
        _check(lib().cpr_profile(self._h, mask), "cpr_profile")

    def profile_vcycle_levels(self, reps: int = 20) -> dict:
        """In-graph device microseconds of the V-cycle, the BILU application,
        the coarse solve and every level's pre/resid/R/P/post parts."""
        nl = self.nlev
        us = np.zeros(3 + 5 * max(nl - 1, 0))
        rc = lib().cpr_profile_vcycle_levels(self._h, reps, _ptr(us), len(us))
        if rc < 0:
            _check(rc, "cpr_profile_vcycle_levels")
        parts = ("pre", "resid", "R", "P", "post")
        return {"vcycle_us": us[0], "bilu_us": us[1], "coarse_us": us[2],
                "levels": [dict(zip(parts, us[3 + 5 * l: 8 + 5 * l])) for l in range(nl - 1)]}

    def schedule(self, level: int) -> dict:
        """The V-cycle schedule of one level: lanes per row of the A, P and R
        kernels and the CTA size."""
        sc = Schedule()
        _check(lib().cpr_get_schedule(self._h, level, C.byref(sc)), "cpr_get_schedule")
        return {k: getattr(sc, k) for k, _ in Schedule._fields_}

    def set_schedule(self, level: int, lanes_a: int, lanes_p: int, lanes_r: int, block: int) -> None:
        sc = Schedule(lanes_a, lanes_p, lanes_r, block)
        _check(lib().cpr_set_schedule(self._h, level, C.byref(sc)), "cpr_set_schedule")

    def autotune(self, reps: int = 10):
        """Run the schedule autotuner; returns (B_P microseconds before, after)."""
        b, a = C.c_double(), C.c_double()
        _check(lib().cpr_autotune(self._h, reps, C.byref(b), C.byref(a)), "cpr_autotune")
        return b.value, a.value

    def profile_read(self, family: int):
        n, ms = C.c_long(), C.c_double()
        _check(lib().cpr_profile_read(self._h, family, C.byref(n), C.byref(ms)), "cpr_profile_read")
        return n.value, ms.value

    @property
    def stream(self) -> int:
        return self.opts.stream or 0

    def close(self) -> None:
        if self._h:
            lib().cpr_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSolver(Solver):
    """A batch handle: many independent systems (block-diagonal preconditioner,
    per-system FGMRES in lockstep)."""

    def __init__(self, systems, **opts):
        if "stream" not in opts:
            opts["stream"] = _torch_stream()
        self.opts = default_opts(**opts)
        self._h = C.c_void_p()
        descs, self._keep = [], []
        for A in systems:
            d, keep = _as_bsr3(A)
            descs.append(d)
            self._keep.append(keep)
        arr = (Bsr3 * len(descs))(*descs)
        _check(lib().cpr_batch_setup(C.byref(self._h), len(descs), arr, C.byref(self.opts)),
               "cpr_batch_setup")
        self.sizes = [d.nb for d in descs]
        self.nb = sum(self.sizes)
        self.nnzb = sum(d.nnzb for d in descs)

    def update(self, systems) -> None:
        descs = [_as_bsr3(A)[0] for A in systems]
        arr = (Bsr3 * len(descs))(*descs)
        _check(lib().cpr_batch_update(self._h, arr), "cpr_batch_update")

    def solve(self, bs, xs=None, rtol: float = 1e-6):
        """Solve every system; returns (xs, list of stats dicts)."""
        n = len(bs)
        if xs is None:
            xs = []
            for b in bs:
                if isinstance(b, np.ndarray):
                    xs.append(np.zeros_like(b, dtype=np.float64))
                else:
                    import torch
                    xs.append(torch.zeros_like(b))
        bp = (C.c_void_p * n)(*[_ptr(b) for b in bs])
        xp = (C.c_void_p * n)(*[_ptr(x) for x in xs])
        st = (Stats * n)()
        rc = lib().cpr_batch_solve(self._h, bp, xp, float(rtol), st)
        _check(rc, "cpr_batch_solve", allow_not_converged=True)
        return xs, [s_.as_dict() for s_ in st]


PROF_SPMV, PROF_VCYCLE, PROF_BILU, PROF_CGS, PROF_RESID2, PROF_SMOOTH0 = range(6)


def launch_count() -> int:
    return int(lib().cpr_launch_count())


def set_memory_limit(nbytes: int) -> None:
    """Cap the device memory the library holds (0: no cap); beyond it calls fail with CPR_ERR_OOM."""
    lib().cpr_set_memory_limit(int(nbytes))


def memory_in_use() -> int:
    """Device bytes the library holds now, over all handles."""
    return int(lib().cpr_memory_in_use())


def bsr3_spmv(A, x, b=None, y=None, stream=None):
    """y = A x (or b - A x) on the device; A's arrays and x, b, y are CUDA tensors."""
    import torch
    d, keep = _as_bsr3(A)
    if y is None:
        y = torch.empty_like(x)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    _check(lib().cpr_bsr3_spmv(C.byref(d), _ptr(x), _ptr(b), _ptr(y), stream), "cpr_bsr3_spmv")
    return y
