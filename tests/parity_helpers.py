"""Comparison helpers shared by the GPU parity tests (CUDA path against the
FP64 oracle)."""
import numpy as np

import blackoil_synth as bs

APPLY_TOL = 1e-10   # preconditioner applications: FP64 differs only in summation order
SOLVE_TOL = 1e-8    # whole solves with equal iteration counts


def assert_apply_close(got, ref, tol=APPLY_TOL, what=""):
    """Element by element: |got - ref| <= tol |ref| + tol max|ref|, so a wrong
    value in a few rows cannot hide under a norm of the whole vector."""
    got, ref = np.asarray(got, float), np.asarray(ref, float)
    scale = max(np.abs(ref).max(), 1e-300)
    np.testing.assert_allclose(got, ref, rtol=tol, atol=tol * scale, err_msg=what)


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def compare_hierarchy(o, g):
    """Every level's A, colors, C/F split (or aggregates) and P, the decoupling
    weights and the BILU(0) coloring and factors, bit for bit."""
    assert g.nlev == o.nlev
    for l in range(o.nlev):
        ol, gl = o.level(l), g.level(l)
        A = ol["A"]
        assert gl["n"] == A.n and gl["nnz"] == len(A.col), l
        np.testing.assert_array_equal(gl["rowptr"], A.rowptr)
        np.testing.assert_array_equal(gl["col"], A.col)
        np.testing.assert_array_equal(gl["val"], A.val)
        if l < o.nlev - 1:
            assert gl["ncolors"] == ol["ncolors"]
            np.testing.assert_array_equal(gl["color"], ol["color"])
            np.testing.assert_array_equal(gl["cf"], ol["cf"])
            P = ol["P"]
            np.testing.assert_array_equal(gl["prow"], P.rowptr)
            np.testing.assert_array_equal(gl["pcol"], P.col)
            np.testing.assert_array_equal(gl["pval"], P.val)
    np.testing.assert_array_equal(g.weights(), o.weights())
    gbc, gnc, glu = g.bilu()
    obc, onc, olu = o.bilu()
    assert gnc == onc
    np.testing.assert_array_equal(gbc, obc)
    np.testing.assert_array_equal(glu, olu)


def block_diag(Js):
    """Block-diagonal concatenation of Jacobians, systems in order (what a
    batch handle is set up on)."""
    rowptr, cols, vals, rhs = [np.zeros(1, np.int32)], [], [], []
    off = poff = 0
    for J in Js:
        rowptr.append((J.rowptr[1:] + poff).astype(np.int32))
        cols.append((J.col + off).astype(np.int32))
        vals.append(J.val)
        rhs.append(J.b)
        off += J.nb
        poff += J.nnzb
    return bs.Jacobian(off, np.concatenate(rowptr), np.concatenate(cols), np.concatenate(vals),
                       np.concatenate(rhs))
