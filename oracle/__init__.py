"""ctypes binding of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use it; the CUDA product path never does.

Every function mirrors one step of the method; see the comments in oracle.c for
the passage of the paper each step follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_FLAGS = ["-O3", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-Wall", "-Wno-unused-function"]


def build(force: bool = False, omp: bool = False) -> str:
    """Compile liboracle.so in-tree (gcc, -ffp-contract=off: no fused multiply-add).

    omp=True builds liboracle_omp.so, the same source with OpenMP over the
    loops marked independent (-fopenmp -march=native): the CPU baseline's
    multi-threaded form, bit-identical to the single-threaded library."""
    out = _LIB_OMP if omp else _LIB
    stale = (not os.path.exists(out)
             or os.path.getmtime(out) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = out + f".tmp{os.getpid()}"
        extra = ["-fopenmp", "-march=native"] if omp else []
        subprocess.check_call(["gcc", *_FLAGS, *extra, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, out)
    return out


class Opts(C.Structure):
    _fields_ = [("theta_color", C.c_double), ("theta_amg", C.c_double), ("mu", C.c_int),
                ("restart", C.c_int), ("max_restarts", C.c_int), ("precond_fp32", C.c_int),
                ("decouple", C.c_int), ("pre", C.c_int), ("post", C.c_int),
                ("coarse_max", C.c_int), ("max_levels", C.c_int), ("seed", C.c_uint64),
                ("bilu_order", C.c_int), ("reuse_refresh", C.c_int), ("resetup", C.c_int),
                ("amg", C.c_int), ("amli_iters", C.c_int), ("coloring", C.c_int),
                ("agg_match", C.c_int), ("coloring_rows", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("setup_called", C.c_int),
                ("setup_count", C.c_int), ("levels", C.c_int), ("converged", C.c_int),
                ("rel_res", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_libs = {}


def lib(omp: bool = False):
    """The oracle library: single-threaded, or the OpenMP build (omp=True)."""
    if omp not in _libs:
        L = C.CDLL(build(omp=omp))
        vp = C.c_void_p
        L.o_csr_n.argtypes = [vp]
        L.o_csr_ncol.argtypes = [vp]
        L.o_csr_nnz.argtypes = [vp]
        L.o_csr_copy.argtypes = [vp, _i32p, _i32p, vp]
        L.o_csr_free.argtypes = [vp]
        L.o_bsr3_spmv.argtypes = [C.c_int, _i32p, _i32p, _f64p, _f64p, _f64p]
        for f in ("o_strength_color", "o_strength_rs"):
            getattr(L, f).argtypes = [C.c_int, _i32p, _i32p, _f64p, C.c_double]
            getattr(L, f).restype = vp
        L.o_sym_union.argtypes = [C.c_int, _i32p, _i32p]
        L.o_sym_union.restype = vp
        L.o_jp_color.argtypes = [C.c_int, _i32p, _i32p, C.c_uint64, C.c_int, C.c_int, _i32p]
        L.o_hash.argtypes = [C.c_uint64, C.c_int, C.c_int, C.c_int]
        L.o_hash.restype = C.c_uint32
        L.o_fmix32.argtypes = [C.c_uint32]
        L.o_fmix32.restype = C.c_uint32
        L.o_pmis.argtypes = [C.c_int, _i32p, _i32p, C.c_uint64, C.c_int, C.c_int, _i32p]
        L.o_interp_direct.argtypes = [C.c_int, _i32p, _i32p, _f64p, _i32p, _i32p, _i32p]
        L.o_interp_direct.restype = vp
        L.o_transpose.argtypes = [C.c_int, C.c_int, _i32p, _i32p, vp]
        L.o_transpose.restype = vp
        L.o_spgemm.argtypes = [C.c_int, C.c_int, _i32p, _i32p, _f64p, C.c_int, _i32p, _i32p, _f64p]
        L.o_spgemm.restype = vp
        L.o_mcgs_sweep.argtypes = [C.c_int, _i32p, _i32p, _f64p, _i32p, C.c_int, _f64p, _f64p,
                                   C.c_int]
        L.o_dense_lu_solve.argtypes = [C.c_int, _f64p, _f64p, _f64p]
        L.o_decouple.argtypes = [C.c_int, _i32p, _i32p, _f64p, C.c_int, _f64p, _f64p]
        L.o_bilu0.argtypes = [C.c_int, _i32p, _i32p, _f64p, C.c_uint64, _i32p, _f64p]
        L.o_bilu0_solve.argtypes = [C.c_int, _i32p, _i32p, _f64p, _i32p, C.c_int, _f64p, _f64p]
        L.o_bilu0_natural.argtypes = [C.c_int, _i32p, _i32p, _f64p, _f64p]
        L.o_natural_levels.argtypes = [C.c_int, _i32p, _i32p, _i32p]
        L.o_vertices_grouping.argtypes = [C.c_int, _i32p, _i32p, _f64p, C.c_double, _i32p]
        L.o_aggregate.argtypes = [C.c_int, _i32p, _i32p, _f64p, C.c_double, C.c_int, C.c_int, _i32p]
        L.o_fgmres_identity.argtypes = [C.c_int, _i32p, _i32p, _f64p, _f64p, _f64p, C.c_double,
                                        C.c_int, C.c_int, C.POINTER(Stats), vp]
        L.o_default_opts.argtypes = [C.POINTER(Opts)]
        L.o_setup.argtypes = [C.POINTER(vp), C.c_int, _i32p, _i32p, _f64p, C.POINTER(Opts)]
        L.o_update.argtypes = [vp, C.c_int, _i32p, _i32p, _f64p]
        L.o_solve.argtypes = [vp, _f64p, _f64p, C.c_double, C.POINTER(Stats)]
        L.o_solve_rows.argtypes = [vp, C.c_int, C.c_int, _f64p, _f64p, C.c_double, C.POINTER(Stats)]
        L.o_destroy.argtypes = [vp]
        L.o_num_levels.argtypes = [vp]
        L.o_last_iters.argtypes = [vp]
        L.o_level_info.argtypes = [vp, C.c_int] + [C.POINTER(C.c_int)] * 5
        L.o_level_get.argtypes = [vp, C.c_int, _i32p, _i32p, _f64p, vp, vp, vp, vp, vp]
        L.o_get_weights.argtypes = [vp, _f64p]
        L.o_bilu_ncolors.argtypes = [vp]
        L.o_bilu_get.argtypes = [vp, _i32p, _f64p]
        L.o_cpr_apply.argtypes = [vp, _f64p, _f64p]
        L.o_vcycle.argtypes = [vp, _f64p, _f64p]
        L.o_bilu_apply.argtypes = [vp, _f64p, _f64p]
        _libs[omp] = L
    return _libs[omp]


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().o_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


@dataclass
class CSR:
    n: int
    ncol: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray | None = None

    def dense(self) -> np.ndarray:
        D = np.zeros((self.n, self.ncol))
        for i in range(self.n):
            for p in range(self.rowptr[i], self.rowptr[i + 1]):
                D[i, self.col[p]] = 1.0 if self.val is None else self.val[p]
        return D

    def pattern(self) -> set:
        return {(i, int(self.col[p])) for i in range(self.n)
                for p in range(self.rowptr[i], self.rowptr[i + 1])}


def _take(ptr, with_val=True) -> CSR:
    L = lib()
    n, ncol, nnz = L.o_csr_n(ptr), L.o_csr_ncol(ptr), L.o_csr_nnz(ptr)
    rp = np.zeros(n + 1, np.int32)
    cl = np.zeros(nnz, np.int32)
    v = np.zeros(nnz, np.float64) if with_val else None
    L.o_csr_copy(ptr, rp, cl, v.ctypes.data if with_val else None)
    L.o_csr_free(ptr)
    return CSR(n, ncol, rp, cl, v)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- primitives

def bsr3_spmv(J, x):
    y = np.zeros(3 * J.nb)
    lib().o_bsr3_spmv(J.nb, _i32(J.rowptr), _i32(J.col), _f64(J.val), _f64(x), y)
    return y


def strength_color(rowptr, col, val, theta) -> CSR:
    n = len(rowptr) - 1
    return _take(lib().o_strength_color(n, _i32(rowptr), _i32(col), _f64(val), theta), False)


def sym_union(S: CSR) -> CSR:
    return _take(lib().o_sym_union(S.n, _i32(S.rowptr), _i32(S.col)), False)


def jp_color(G: CSR, seed=0, salt=0, level=0):
    color = np.zeros(G.n, np.int32)
    nc = lib().o_jp_color(G.n, _i32(G.rowptr), _i32(G.col), seed, salt, level, color)
    return color, nc


def threads(omp: bool = False) -> int:
    """Threads the chosen build's parallel loops run on."""
    return int(lib(omp).o_threads())


def fmix32(h) -> int:
    return int(lib().o_fmix32(h))


def hash32(seed, salt, level, i) -> int:
    return int(lib().o_hash(seed, salt, level, i))


def strength_rs(rowptr, col, val, theta=0.25) -> CSR:
    n = len(rowptr) - 1
    return _take(lib().o_strength_rs(n, _i32(rowptr), _i32(col), _f64(val), theta), False)


def pmis(S: CSR, seed=0, salt=1, level=0):
    cf = np.zeros(S.n, np.int32)
    nc = lib().o_pmis(S.n, _i32(S.rowptr), _i32(S.col), seed, salt, level, cf)
    return cf, nc


def interp_direct(rowptr, col, val, S: CSR, cf) -> CSR:
    n = len(rowptr) - 1
    return _take(lib().o_interp_direct(n, _i32(rowptr), _i32(col), _f64(val), _i32(S.rowptr),
                                       _i32(S.col), _i32(cf)))


def transpose(M: CSR) -> CSR:
    v = None if M.val is None else _f64(M.val)
    return _take(lib().o_transpose(M.n, M.ncol, _i32(M.rowptr), _i32(M.col),
                                   None if v is None else v.ctypes.data), M.val is not None)


def spgemm(A: CSR, B: CSR) -> CSR:
    return _take(lib().o_spgemm(A.n, A.ncol, _i32(A.rowptr), _i32(A.col), _f64(A.val), B.ncol,
                                _i32(B.rowptr), _i32(B.col), _f64(B.val)))


def mcgs_sweep(rowptr, col, val, color, ncolors, b, x, descending=False):
    x = _f64(x).copy()
    n = len(rowptr) - 1
    lib().o_mcgs_sweep(n, _i32(rowptr), _i32(col), _f64(val), _i32(color), ncolors, _f64(b), x,
                       int(descending))
    return x


def dense_lu_solve(A, b):
    A = _f64(A)
    x = np.zeros(A.shape[0])
    rc = lib().o_dense_lu_solve(A.shape[0], A, _f64(b), x)
    if rc != 0:
        raise RuntimeError(f"oracle dense LU failed ({rc})")
    return x


def decouple(J, mode=1):
    w = np.zeros(3 * J.nb)
    ap = np.zeros(J.nnzb)
    rc = lib().o_decouple(J.nb, _i32(J.rowptr), _i32(J.col), _f64(J.val), mode, w, ap)
    if rc != 0:
        raise RuntimeError(f"oracle decoupling failed ({rc})")
    return w, ap


def bilu0(J, seed=0):
    bcolor = np.zeros(J.nb, np.int32)
    lu = np.zeros(9 * J.nnzb)
    nc = lib().o_bilu0(J.nb, _i32(J.rowptr), _i32(J.col), _f64(J.val), seed, bcolor, lu)
    if nc < 0:
        raise RuntimeError(f"oracle BILU(0) failed ({nc})")
    return bcolor, nc, lu


def bilu0_natural(J):
    """Natural-order block ILU(0) (the level-scheduled BILU of Sec. 6): factor
    array in A's pattern, as bilu0's."""
    lu = np.zeros(9 * J.nnzb)
    rc = lib().o_bilu0_natural(J.nb, _i32(J.rowptr), _i32(J.col), _f64(J.val), lu)
    if rc < 0:
        raise RuntimeError(f"oracle natural-order BILU(0) failed ({rc})")
    return lu


def natural_levels(J):
    """Level sets of the natural-order block triangular solves: (level per
    block row, number of levels)."""
    level = np.zeros(J.nb, np.int32)
    nlev = lib().o_natural_levels(J.nb, _i32(J.rowptr), _i32(J.col), level)
    return level, nlev


def vertices_grouping(n, rowptr, col, val, theta):
    """The paper's VerticesSplitting/Grouping (Alg. 4-5) on the Eq. 5.1 strong
    connections of a scalar CSR matrix: (group per vertex, number of groups)."""
    color = np.zeros(n, np.int32)
    c = lib().o_vertices_grouping(n, _i32(rowptr), _i32(col), _f64(val), theta, color)
    return color, c


def aggregate(n, rowptr, col, val, beta=0.25, passes=2, match=0):
    """Pairwise aggregation of a scalar CSR matrix: (aggregate per node, number
    of aggregates); passes = 1 for one matching pass, 2 for the double pass;
    match = 0 greedy, 1 handshake rounds."""
    agg = np.zeros(n, np.int32)
    na = lib().o_aggregate(n, _i32(rowptr), _i32(col), _f64(val), beta, passes, match, agg)
    return agg, na


def bilu0_solve(J, bcolor, nbcolors, lu, r):
    z = np.zeros(3 * J.nb)
    lib().o_bilu0_solve(J.nb, _i32(J.rowptr), _i32(J.col), _f64(lu), _i32(bcolor), nbcolors,
                        _f64(r), z)
    return z


def fgmres_identity(J, b, x0=None, rtol=1e-10, m=30, max_restarts=100):
    x = np.zeros(3 * J.nb) if x0 is None else _f64(x0).copy()
    st = Stats()
    hist = np.zeros(m * max_restarts)
    rc = lib().o_fgmres_identity(J.nb, _i32(J.rowptr), _i32(J.col), _f64(J.val), _f64(b), x,
                                 rtol, m, max_restarts, C.byref(st), hist.ctypes.data)
    return x, st.as_dict(), hist[:st.iters], rc


# ---------------------------------------------------------------- the solver

class Solver:
    """CPR-FGMRES with adaptive setup (Alg. 2 + Alg. 3), FP64 on the CPU."""

    def __init__(self, J, omp: bool = False, **opts):
        self._L = lib(omp)
        self.opts = default_opts(**opts)
        self._h = C.c_void_p()
        self._keep = (_i32(J.rowptr), _i32(J.col), _f64(J.val))
        self.nb = J.nb
        self.nnzb = J.nnzb
        rc = self._L.o_setup(C.byref(self._h), J.nb, *self._keep, C.byref(self.opts))
        if rc != 0:
            raise RuntimeError(f"oracle setup failed ({rc})")

    def update(self, J):
        self._keep = (_i32(J.rowptr), _i32(J.col), _f64(J.val))
        rc = self._L.o_update(self._h, J.nb, *self._keep)
        if rc != 0:
            raise RuntimeError(f"oracle update failed ({rc})")
        self.nb, self.nnzb = J.nb, J.nnzb

    def solve(self, b, x0=None, rtol=1e-6):
        x = np.zeros(3 * self.nb) if x0 is None else _f64(x0).copy()
        st = Stats()
        rc = self._L.o_solve(self._h, _f64(b), x, rtol, C.byref(st))
        if rc < 0:
            raise RuntimeError(f"oracle solve failed ({rc})")
        return x, st.as_dict()

    def solve_rows(self, r0, r1, b, x0=None, rtol=1e-6):
        """FGMRES on block rows [r0, r1) of a block-diagonal A (one system of a
        batch) with this handle's B restricted to them."""
        x = np.zeros(3 * (r1 - r0)) if x0 is None else _f64(x0).copy()
        st = Stats()
        rc = self._L.o_solve_rows(self._h, r0, r1, _f64(b), x, rtol, C.byref(st))
        if rc < 0:
            raise RuntimeError(f"oracle solve_rows failed ({rc})")
        return x, st.as_dict()

    # inspection
    @property
    def nlev(self) -> int:
        return self._L.o_num_levels(self._h)

    def level(self, l: int) -> dict:
        n, nnz, ncol, nc, nnzp = (C.c_int() for _ in range(5))
        self._L.o_level_info(self._h, l, C.byref(n), C.byref(nnz), C.byref(ncol), C.byref(nc),
                           C.byref(nnzp))
        n, nnz, ncolors, nc, nnzp = n.value, nnz.value, ncol.value, nc.value, nnzp.value
        rp = np.zeros(n + 1, np.int32)
        cl = np.zeros(nnz, np.int32)
        v = np.zeros(nnz)
        color = np.zeros(n, np.int32)
        cf = np.zeros(n, np.int32)
        prow = np.zeros(n + 1, np.int32)
        pcol = np.zeros(nnzp, np.int32)
        pval = np.zeros(nnzp)
        has_p = nnzp > 0 or nc > 0
        self._L.o_level_get(self._h, l, rp, cl, v, color.ctypes.data if ncolors else None,
                          cf.ctypes.data if has_p else None, prow.ctypes.data if has_p else None,
                          pcol.ctypes.data if has_p else None, pval.ctypes.data if has_p else None)
        out = {"A": CSR(n, n, rp, cl, v), "ncolors": ncolors, "color": color if ncolors else None}
        if has_p:
            out.update(cf=cf, nc=nc, P=CSR(n, nc, prow, pcol, pval))
        return out

    def weights(self):
        w = np.zeros(3 * self.nb)
        self._L.o_get_weights(self._h, w)
        return w

    def bilu(self):
        bc = np.zeros(self.nb, np.int32)
        lu = np.zeros(9 * self.nnzb)
        self._L.o_bilu_get(self._h, bc, lu)
        return bc, self._L.o_bilu_ncolors(self._h), lu

    def cpr_apply(self, v):
        z = np.zeros(3 * self.nb)
        self._L.o_cpr_apply(self._h, _f64(v), z)
        return z

    def vcycle(self, b):
        x = np.zeros(len(b))
        self._L.o_vcycle(self._h, _f64(b), x)
        return x

    def bilu_apply(self, r):
        z = np.zeros(3 * self.nb)
        self._L.o_bilu_apply(self._h, _f64(r), z)
        return z

    @property
    def last_iters(self) -> int:
        return self._L.o_last_iters(self._h)

    def close(self):
        if self._h:
            self._L.o_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
