"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks one oracle step against something other than the oracle:
library routines (numpy/scipy/networkx), closed forms, the paper's stated
propositions and special cases, or brute force on tiny inputs.
"""
import os

import networkx as nx
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import blackoil_synth as bs
import oracle
from parity_helpers import block_diag

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def csr_dense(rowptr, col, val, n, m=None):
    return sp.csr_matrix((val, col, rowptr), shape=(n, m or n)).toarray()


def read_grid(name):
    rows = [l.split() for l in open(os.path.join(GOLDEN, name)) if not l.startswith("#")]
    return np.array([[int(v) for v in r] for r in rows if r])


@pytest.fixture(scope="module")
def tiny():
    return bs.tiny()


# ------------------------------------------------------------------ SpMV

def test_bsr3_spmv_matches_scipy():
    J = bs.jacobian("20x20x5")
    x = np.random.default_rng(1).standard_normal(J.n)
    y = oracle.bsr3_spmv(J, x)
    ref = J.to_scipy() @ x
    assert np.allclose(y, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


# ------------------------------------------------------------- decoupling

def test_decoupling_weights_and_pressure_matrix(tiny):
    J = tiny
    w, ap = oracle.decouple(J, mode=1)
    blocks = J.val.reshape(-1, 3, 3)
    A = J.to_dense()
    W = np.zeros((J.n, J.nb))
    Pi = np.zeros((J.n, J.nb))
    for i in range(J.nb):
        p = J.rowptr[i] + list(J.col[J.rowptr[i]:J.rowptr[i + 1]]).index(i)
        # w_i = D_i^-T e_1  <=>  D_i^T w_i = e_1
        assert np.allclose(blocks[p].T @ w[3 * i:3 * i + 3], [1, 0, 0], atol=1e-12)
        W[3 * i:3 * i + 3, i] = w[3 * i:3 * i + 3]
        Pi[3 * i, i] = 1.0
    AP = W.T @ A @ Pi                                   # Pi_P^T A Pi_P with weights
    APo = csr_dense(J.rowptr, J.col, ap, J.nb)
    assert np.allclose(APo, AP, rtol=1e-12, atol=1e-12 * np.abs(AP).max())
    # mode 0: injection, A_P = the [0][0] entries
    w0, ap0 = oracle.decouple(J, mode=0)
    assert np.array_equal(w0.reshape(-1, 3), np.tile([1.0, 0, 0], (J.nb, 1)))
    assert np.array_equal(ap0, blocks[:, 0, 0])


# ------------------------------------------------------- strength, coloring

def _graph(G):
    g = nx.Graph()
    g.add_nodes_from(range(G.n))
    for i in range(G.n):
        for p in range(G.rowptr[i], G.rowptr[i + 1]):
            if G.col[p] != i:
                g.add_edge(i, int(G.col[p]))
    return g


def _pressure_level0(J):
    _, ap = oracle.decouple(J, 1)
    return J.rowptr, J.col, ap


def test_strength_special_cases():
    rp, cl, v = bs.random_sparse(40, 0.15, seed=3, neg_offdiag=False)
    n = len(rp) - 1
    S1 = oracle.strength_color(rp, cl, v, 1.0)
    assert S1.rowptr[-1] == 0                          # theta = 1: no strong edge (Sec. 5.2)
    S0 = oracle.strength_color(rp, cl, v, 0.0)
    off = {(i, int(cl[p])) for i in range(n) for p in range(rp[i], rp[i + 1])
           if cl[p] != i and v[p] != 0}
    assert S0.pattern() == off                          # theta = 0: every off-diagonal nonzero
    Sa = oracle.strength_color(rp, cl, v, 0.05).pattern()
    Sb = oracle.strength_color(rp, cl, v, 0.1).pattern()
    assert Sb <= Sa <= off                              # monotone in theta


@pytest.mark.parametrize("theta", [0.0, 0.05, 0.1, 0.3])
def test_jp_coloring_props_and_greedy_equivalence(theta):
    J = bs.jacobian("20x20x5")
    rp, cl, ap = _pressure_level0(J)
    S = oracle.strength_color(rp, cl, ap, theta)
    G = oracle.sym_union(S)
    color, nc = oracle.jp_color(G, seed=7, salt=0, level=0)
    g = _graph(G)
    # Prop. 5.3: everyone colored, finitely many colors; goal (c): no edge inside a color
    assert color.min() == 0 and color.max() == nc - 1
    assert all(color[a] != color[b] for a, b in g.edges)
    # Prop. 5.1: c <= max degree + 1
    assert nc <= max(dict(g.degree).values(), default=0) + 1
    # JP with key (deg, hash, i) == first-fit greedy in descending key order
    key = {i: (g.degree[i], oracle.hash32(7, 0, 0, i), i) for i in range(G.n)}
    order = sorted(range(G.n), key=lambda i: key[i], reverse=True)
    greedy = nx.coloring.greedy_color(g, strategy=lambda gg, colors: iter(order))
    assert all(greedy[i] == color[i] for i in range(G.n))


def test_theta_one_gives_one_color_and_jacobi():
    J = bs.jacobian("20x20x5")
    rp, cl, ap = _pressure_level0(J)
    G = oracle.sym_union(oracle.strength_color(rp, cl, ap, 1.0))
    color, nc = oracle.jp_color(G)
    assert nc == 1                                       # Sec. 5.2: theta = 1 => c = 1
    rng = np.random.default_rng(0)
    b, x0 = rng.standard_normal(J.nb), rng.standard_normal(J.nb)
    x1 = oracle.mcgs_sweep(rp, cl, ap, color, nc, b, x0)
    A = csr_dense(rp, cl, ap, J.nb)
    jac = x0 + (b - A @ x0) / np.diag(A)                 # one Jacobi step
    assert np.allclose(x1, jac, rtol=1e-12, atol=1e-12 * np.abs(jac).max())


def test_prop52_color_blocks_diagonal_at_theta0():
    J = bs.jacobian("20x20x5")
    rp, cl, ap = _pressure_level0(J)
    G = oracle.sym_union(oracle.strength_color(rp, cl, ap, 0.0))
    color, nc = oracle.jp_color(G, seed=3)
    A = csr_dense(rp, cl, ap, J.nb)
    for c in range(nc):
        idx = np.nonzero(color == c)[0]
        blk = A[np.ix_(idx, idx)]
        assert np.count_nonzero(blk - np.diag(np.diag(blk))) == 0


def test_five_point_grid_coloring():
    rp, cl, v = bs.laplacian_2d(9, 7)
    G = oracle.sym_union(oracle.strength_color(rp, cl, v, 0.0))
    color, nc = oracle.jp_color(G, seed=1)
    g = _graph(G)
    assert 2 <= nc <= 5
    assert all(color[a] != color[b] for a, b in g.edges)


def _seq_gs_in_order(A, b, x, order):
    """Sequential GS visiting rows in `order` (scipy triangular solve on the permuted matrix)."""
    Ap = A[np.ix_(order, order)]
    lower = sp.csr_matrix(np.tril(Ap))
    upper = np.triu(Ap, 1)
    xp = spla.spsolve_triangular(lower, b[order] - upper @ x[order], lower=True)
    out = np.empty_like(x)
    out[order] = xp
    return out


def test_mcgs_theta0_equals_sequential_gs_in_color_order():
    J = bs.jacobian("20x20x5")
    rp, cl, ap = _pressure_level0(J)
    G = oracle.sym_union(oracle.strength_color(rp, cl, ap, 0.0))
    color, nc = oracle.jp_color(G, seed=5)
    A = csr_dense(rp, cl, ap, J.nb)
    rng = np.random.default_rng(2)
    b, x0 = rng.standard_normal(J.nb), rng.standard_normal(J.nb)
    order = np.lexsort((np.arange(J.nb), color))
    x1 = oracle.mcgs_sweep(rp, cl, ap, color, nc, b, x0)
    ref = _seq_gs_in_order(A, b, x0, order)
    assert np.allclose(x1, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())
    # descending colors == sequential GS over the reversed color order
    x2 = oracle.mcgs_sweep(rp, cl, ap, color, nc, b, x0, descending=True)
    order_d = np.lexsort((np.arange(J.nb), -color))
    ref2 = _seq_gs_in_order(A, b, x0, order_d)
    assert np.allclose(x2, ref2, rtol=1e-11, atol=1e-11 * np.abs(ref2).max())


@pytest.mark.parametrize("grid", ["redblack_4x4.txt", "fourcolor_4x4.txt"])
def test_structured_grid_colorings_from_the_paper(grid):
    """Sec. 3.2 / Fig. 2: multi-color GS over the red-black (5-point) and the
    four-color (9-point) groupings equals sequential GS in color order."""
    colors = read_grid(grid).ravel().astype(np.int32)
    n = 16
    nine = grid.startswith("four")
    A = np.zeros((n, n))
    for j in range(4):
        for i in range(4):
            c = i + 4 * j
            for dj in (-1, 0, 1):
                for di in (-1, 0, 1):
                    if (di, dj) == (0, 0) or (not nine and di != 0 and dj != 0):
                        continue
                    ii, jj = i + di, j + dj
                    if 0 <= ii < 4 and 0 <= jj < 4:
                        A[c, ii + 4 * jj] = -1.0
            A[c, c] = -A[c].sum() + 0.5
    M = sp.csr_matrix(A)
    M.sort_indices()
    rp, cl, v = M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data
    # the grouping is a valid coloring (goal (c)) with 2 resp. 4 colors
    nc = int(colors.max()) + 1
    assert nc == (4 if nine else 2)
    assert all(colors[a] != colors[b] for a, b in zip(*np.nonzero(A - np.diag(np.diag(A)))))
    rng = np.random.default_rng(4)
    b, x0 = rng.standard_normal(n), rng.standard_normal(n)
    x1 = oracle.mcgs_sweep(rp, cl, v, colors, nc, b, x0)
    ref = _seq_gs_in_order(A, b, x0, np.lexsort((np.arange(n), colors)))
    assert np.allclose(x1, ref, rtol=1e-13, atol=1e-13)


# -------------------------------------------------------------- coarsening

def _pmis_sequential(S, seed, salt, level):
    """Brute force: PMIS's result equals a sequential sweep in descending key
    order where a point becomes C unless a C point of larger key lies in S_i."""
    n = S.n
    T = oracle.transpose(S)
    lam = np.diff(T.rowptr)
    key = [(int(lam[i]), oracle.hash32(seed, salt, level, i), i) for i in range(n)]
    cf = -np.ones(n, int)
    for i in range(n):
        if S.rowptr[i + 1] == S.rowptr[i] and lam[i] == 0:
            cf[i] = 0
    for i in sorted(range(n), key=lambda i: key[i], reverse=True):
        if cf[i] != -1:
            continue
        Si = S.col[S.rowptr[i]:S.rowptr[i + 1]]
        cf[i] = 0 if any(cf[j] == 1 for j in Si) else 1
    return cf


@pytest.mark.parametrize("which", ["laplace", "random", "pressure"])
def test_pmis_properties_and_sequential_equivalence(which):
    if which == "laplace":
        rp, cl, v = bs.laplacian_2d(12, 9, shift=0.01)
    elif which == "random":
        rp, cl, v = bs.random_sparse(60, 0.08, seed=11)
    else:
        rp, cl, v = _pressure_level0(bs.jacobian("20x20x5"))
    S = oracle.strength_rs(rp, cl, v, 0.25)
    cf, nc = oracle.pmis(S, seed=3, salt=1, level=0)
    n = S.n
    assert set(np.unique(cf)) <= {0, 1} and nc == int(cf.sum()) and nc > 0
    T = oracle.transpose(S)
    for i in range(n):
        Si = S.col[S.rowptr[i]:S.rowptr[i + 1]]
        if cf[i] == 0 and len(Si):
            assert any(cf[j] == 1 for j in Si)          # every F point has a strong C point
        if len(Si) == 0 and T.rowptr[i + 1] == T.rowptr[i]:
            assert cf[i] == 0                            # isolated points are F
    assert np.array_equal(cf, _pmis_sequential(S, 3, 1, 0))


def test_rs_strength_special_cases():
    rp, cl, v = bs.laplacian_2d(6, 5, shift=0.1)
    S = oracle.strength_rs(rp, cl, v, 0.25)
    off = {(i, int(cl[p])) for i in range(len(rp) - 1) for p in range(rp[i], rp[i + 1])
           if cl[p] != i}
    assert S.pattern() == off                            # equal couplings: all strong
    # a positive off-diagonal entry is never strong (sign convention)
    v2 = v.copy()
    p = rp[7] + 1 if cl[rp[7]] == 7 else rp[7]
    v2[p] = 0.5
    S2 = oracle.strength_rs(rp, cl, v2, 0.25)
    assert (7, int(cl[p])) not in S2.pattern()


def _zero_rowsum(n_x, n_y, pos_frac, seed):
    """Zero-row-sum matrix with negative (and optionally some positive) couplings."""
    rp, cl, v = bs.laplacian_2d(n_x, n_y)
    rng = np.random.default_rng(seed)
    A = csr_dense(rp, cl, v, len(rp) - 1)
    n = A.shape[0]
    off = A - np.diag(np.diag(A))
    scale = rng.uniform(0.5, 2.0, (n, n))
    off = off * (scale + scale.T) / 2
    flip = (rng.random((n, n)) < pos_frac) & (off != 0)
    off = np.where(flip, 0.1 * np.abs(off), off)
    A = off - np.diag(off.sum(axis=1))
    M = sp.csr_matrix(A)
    M.sort_indices()
    return M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data, A


@pytest.mark.parametrize("pos_frac", [0.0, 0.15])
def test_direct_interpolation_preserves_constants(pos_frac):
    rp, cl, v, A = _zero_rowsum(10, 8, pos_frac, seed=2)
    n = A.shape[0]
    S = oracle.strength_rs(rp, cl, v, 0.25)
    cf, nc = oracle.pmis(S, seed=1)
    P = oracle.interp_direct(rp, cl, v, S, cf)
    Pd = P.dense()
    cidx = np.cumsum(cf) - 1
    for i in range(n):
        if cf[i] == 1:
            assert np.array_equal(Pd[i], np.eye(nc)[cidx[i]])   # C rows are unit rows
    # Stueben: for zero row sums, P 1 = 1 on F rows with strong C points
    ones = Pd @ np.ones(nc)
    has_c = np.array([any(cf[j] == 1 for j in S.col[S.rowptr[i]:S.rowptr[i + 1]])
                      for i in range(n)])
    assert np.allclose(ones[has_c], 1.0, rtol=0, atol=1e-13)
    assert (P.val > 0).all()


def test_transpose_and_galerkin_product_match_dense():
    J = bs.jacobian("20x20x5")
    rp, cl, ap = _pressure_level0(J)
    S = oracle.strength_rs(rp, cl, ap, 0.25)
    cf, nc = oracle.pmis(S, seed=0)
    P = oracle.interp_direct(rp, cl, ap, S, cf)
    R = oracle.transpose(P)
    assert np.array_equal(R.dense(), P.dense().T)
    A = oracle.CSR(J.nb, J.nb, rp, cl, ap)
    Ac = oracle.spgemm(R, oracle.spgemm(A, P))
    ref = P.dense().T @ A.dense() @ P.dense()
    D = Ac.dense()
    assert np.allclose(D, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    nzr = set(zip(*np.nonzero(np.abs(ref) > 1e-12 * np.abs(ref).max())))
    assert nzr <= Ac.pattern()                                   # pattern covers the product
    for i in range(Ac.n):                                        # sorted, unique columns
        c = Ac.col[Ac.rowptr[i]:Ac.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0)


def test_dense_lu_matches_numpy():
    rng = np.random.default_rng(5)
    for n in (1, 7, 64):
        A = rng.standard_normal((n, n)) + n * np.eye(n) * 0.1
        A[0, 0] = 0.0 if n > 1 else 1.0                          # force a pivot swap
        b = rng.standard_normal(n)
        assert np.allclose(oracle.dense_lu_solve(A, b), np.linalg.solve(A, b), rtol=1e-10)


# ------------------------------------------------------------------ BILU(0)

def _bilu_dense_factors(J, bcolor, nbcolors, lu):
    order = np.lexsort((np.arange(J.nb), bcolor))
    pos = np.empty(J.nb, int)
    pos[order] = np.arange(J.nb)
    L = np.eye(J.n)
    U = np.zeros((J.n, J.n))
    blk = lu.reshape(-1, 3, 3)
    for i in range(J.nb):
        for p in range(J.rowptr[i], J.rowptr[i + 1]):
            j = J.col[p]
            sl_i, sl_j = slice(3 * i, 3 * i + 3), slice(3 * j, 3 * j + 3)
            if j == i:
                U[sl_i, sl_j] = np.linalg.inv(blk[p])
            elif pos[j] < pos[i]:
                L[sl_i, sl_j] = blk[p]
            else:
                U[sl_i, sl_j] = blk[p]
    return L, U


def test_bilu0_defining_property(tiny):
    J = tiny
    bcolor, nbc, lu = oracle.bilu0(J, seed=4)
    # coloring of the block graph is valid (theta = 0: no two neighbours share a color)
    for i in range(J.nb):
        for p in range(J.rowptr[i], J.rowptr[i + 1]):
            if J.col[p] != i:
                assert bcolor[J.col[p]] != bcolor[i]
    L, U = _bilu_dense_factors(J, bcolor, nbc, lu)
    LU = L @ U
    A = J.to_dense()
    mask = np.zeros_like(A, bool)
    for i in range(J.nb):
        for p in range(J.rowptr[i], J.rowptr[i + 1]):
            j = J.col[p]
            mask[3 * i:3 * i + 3, 3 * j:3 * j + 3] = True
    # (L U)_ij = A_ij on the block pattern
    assert np.allclose(LU[mask], A[mask], rtol=1e-11, atol=1e-11 * np.abs(A).max())
    r = np.random.default_rng(0).standard_normal(J.n)
    z = oracle.bilu0_solve(J, bcolor, nbc, lu, r)
    assert np.allclose(z, np.linalg.solve(LU, r), rtol=1e-10, atol=1e-12)


def test_bilu0_block_diagonal_is_exact():
    J = bs.tiny(3, 3, 1, wells="none")
    keep = J.col == np.repeat(np.arange(J.nb), np.diff(J.rowptr))
    Jd = bs.Jacobian(J.nb, np.concatenate([[0], np.cumsum(np.ones(J.nb, int))]).astype(np.int32),
                     np.arange(J.nb, dtype=np.int32),
                     J.val.reshape(-1, 9)[keep].ravel().copy(), J.b)
    bcolor, nbc, lu = oracle.bilu0(Jd)
    r = np.random.default_rng(1).standard_normal(Jd.n)
    z = oracle.bilu0_solve(Jd, bcolor, nbc, lu, r)
    assert np.allclose(z, np.linalg.solve(Jd.to_dense(), r), rtol=1e-12)


def _block_mask(J):
    mask = np.zeros((J.n, J.n), bool)
    for i in range(J.nb):
        for p in range(J.rowptr[i], J.rowptr[i + 1]):
            j = J.col[p]
            mask[3 * i:3 * i + 3, 3 * j:3 * j + 3] = True
    return mask


def test_bilu0_natural_defining_property(tiny):
    """Natural-order block ILU(0) (the level-scheduled BILU of Sec. 6): L is
    block lower and U block upper in the natural numbering, (L U)_ij = A_ij on
    A's block pattern, and the solve applies (L U)^-1."""
    J = tiny
    lu = oracle.bilu0_natural(J)
    one = np.zeros(J.nb, np.int32)
    L, U = _bilu_dense_factors(J, one, 1, lu)
    nz_l = np.abs(L.reshape(J.nb, 3, J.nb, 3)).sum(axis=(1, 3)) > 0
    nz_u = np.abs(U.reshape(J.nb, 3, J.nb, 3)).sum(axis=(1, 3)) > 0
    assert not np.triu(nz_l, 1).any() and not np.tril(nz_u, -1).any()   # block lower / upper
    assert np.array_equal(np.diag(L), np.ones(J.n))
    LU = L @ U
    A = J.to_dense()
    mask = _block_mask(J)
    assert np.allclose(LU[mask], A[mask], rtol=1e-11, atol=1e-11 * np.abs(A).max())
    # with wells the pattern is not closed under elimination: the fill ILU(0) drops is real
    assert not np.allclose(LU, A, rtol=1e-6, atol=1e-9 * np.abs(A).max())
    r = np.random.default_rng(2).standard_normal(J.n)
    z = oracle.bilu0_solve(J, one, 1, lu, r)
    assert np.allclose(z, np.linalg.solve(LU, r), rtol=1e-10, atol=1e-12)


def test_bilu0_natural_on_a_chain_is_the_exact_lu():
    """A 1-D grid gives a block-tridiagonal A, whose natural-order elimination
    creates no fill: ILU(0) is the exact block LU and B = A^-1."""
    J = bs.tiny(7, 1, 1, wells="none")
    lu = oracle.bilu0_natural(J)
    r = np.random.default_rng(3).standard_normal(J.n)
    z = oracle.bilu0_solve(J, np.zeros(J.nb, np.int32), 1, lu, r)
    assert np.allclose(z, np.linalg.solve(J.to_dense(), r), rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("wells", ["none", "corners"])
def test_natural_levels(wells):
    """Level sets of the natural-order sweeps equal the topological generations
    (Kahn's layering, networkx) of the DAG with an edge j -> i for every
    neighbour j < i in the symmetrised block pattern; without wells, on an
    nx x ny x nz 7-point grid, level(x, y, z) = x + y + z."""
    nx_, ny_, nz_ = 5, 4, 3
    J = bs.tiny(nx_, ny_, nz_, wells=wells)
    level, nlev = oracle.natural_levels(J)
    D = nx.DiGraph()
    D.add_nodes_from(range(J.nb))
    for i in range(J.nb):
        for p in range(J.rowptr[i], J.rowptr[i + 1]):
            j = int(J.col[p])
            if j != i:
                D.add_edge(min(i, j), max(i, j))
    gens = list(nx.topological_generations(D))
    assert nlev == len(gens)
    for g, nodes in enumerate(gens):
        assert all(level[v] == g for v in nodes)
    if wells == "none":
        c = np.arange(J.nb)
        assert np.array_equal(level, c % nx_ + (c // nx_) % ny_ + c // (nx_ * ny_))
        assert nlev == nx_ + ny_ + nz_ - 2


# ------------------------------------------------------ CPR, Eq. 3.1, FGMRES

def test_cpr_apply_is_eq31_with_exact_pressure_solve(tiny):
    """Eq. 3.1: B = Pi B_P W^T + M^-1 (I - A Pi B_P W^T), B_P = A_P^-1 (one level)."""
    J = tiny
    s = oracle.Solver(J, coarse_max=10 ** 6)
    assert s.nlev == 1
    A = J.to_dense()
    w = s.weights()
    W = np.zeros((J.n, J.nb))
    Pi = np.zeros((J.n, J.nb))
    for i in range(J.nb):
        W[3 * i:3 * i + 3, i] = w[3 * i:3 * i + 3]
        Pi[3 * i, i] = 1.0
    AP = W.T @ A @ Pi
    bc, nbc, lu = s.bilu()
    L, U = _bilu_dense_factors(J, bc, nbc, lu)
    Minv = np.linalg.inv(L @ U)
    C1 = Pi @ np.linalg.inv(AP) @ W.T
    B = C1 + Minv @ (np.eye(J.n) - A @ C1)
    Bo = np.column_stack([s.cpr_apply(e) for e in np.eye(J.n)])
    assert np.allclose(Bo, B, rtol=1e-9, atol=1e-9 * np.abs(B).max())
    # and I - B A = (I - M^-1 A)(I - Pi B_P W^T A)
    I = np.eye(J.n)
    assert np.allclose(I - Bo @ A, (I - Minv @ A) @ (I - C1 @ A), atol=1e-8)
    s.close()


@pytest.mark.parametrize("refresh", [0, 1])
def test_kept_b_second_residual(refresh):
    """Alg. 3 keeps B^(k-1) for A^(k).  Eq. 3.1 in dense form with B_P = A_P^-1,
    W and M = L U all from A^(k-1): reuse_refresh = 0 keeps A^(k-1) in the
    second residual, reuse_refresh = 1 takes A^(k) there."""
    g = bs.GridSpec(4, 4, 2, 0.0, 1.0, 1.0, None, "corners", seed=4)
    J0, J1 = list(bs.jacobian_sequence(g, 2, drift=0.05))
    s = oracle.Solver(J0, coarse_max=10 ** 6, mu=10 ** 6, reuse_refresh=refresh)
    A0 = J0.to_dense()
    w = s.weights()
    W = np.zeros((J0.n, J0.nb))
    Pi = np.zeros((J0.n, J0.nb))
    for i in range(J0.nb):
        W[3 * i:3 * i + 3, i] = w[3 * i:3 * i + 3]
        Pi[3 * i, i] = 1.0
    bc, nbc, lu = s.bilu()
    L, U = _bilu_dense_factors(J0, bc, nbc, lu)
    Minv = np.linalg.inv(L @ U)
    C1 = Pi @ np.linalg.inv(W.T @ A0 @ Pi) @ W.T
    _, st = s.solve(J0.b)
    s.update(J1)
    _, st = s.solve(J1.b)
    assert st["setup_called"] == 0 and st["converged"]
    Ares = J1.to_dense() if refresh else A0
    B = C1 + Minv @ (np.eye(J0.n) - Ares @ C1)
    Bo = np.column_stack([s.cpr_apply(e) for e in np.eye(J0.n)])
    assert np.allclose(Bo, B, rtol=1e-9, atol=1e-9 * np.abs(B).max())
    # the two readings differ: the drift reaches the second residual
    Bother = C1 + Minv @ (np.eye(J0.n) - (A0 if refresh else J1.to_dense()) @ C1)
    assert not np.allclose(Bo, Bother, rtol=1e-6, atol=1e-6 * np.abs(B).max())
    s.close()


def _level_dense(lv, which):
    M = lv[which]
    return csr_dense(M.rowptr, M.col, M.val, M.n, M.ncol)


def test_numeric_resetup():
    """resetup = 1: when Alg. 3 rebuilds B for a Jacobian of the
    same pattern, the levels, C/F splits, interpolation patterns and colorings
    of the last setup are kept and every value is recomputed.  Pins: A_P =
    W^T A^(k) Pi with W_i solving D_i^T w_i = e_1 on A^(k)'s blocks; every
    A_{l+1} = R A_l P (dense); C rows of P are unit rows; and a numeric
    resetup with unchanged values equals the full setup bit for bit."""
    g = bs.GridSpec(6, 6, 4, 0.0, 1.0, 1.0, None, "corners", seed=6)
    J0, J1 = list(bs.jacobian_sequence(g, 2, drift=0.05))
    kw = dict(coarse_max=20, mu=0)
    full0 = oracle.Solver(J0, **kw)
    assert full0.nlev >= 3
    s = oracle.Solver(J0, resetup=1, **kw)
    s.solve(J0.b)
    s.update(J1)
    _, st = s.solve(J1.b)
    assert st["setup_called"] == 1 and st["converged"]
    assert s.nlev == full0.nlev
    # level 0: the decoupling of A^(k)
    blocks = J1.val.reshape(-1, 3, 3)
    w = s.weights()
    W = np.zeros((J1.n, J1.nb))
    Pi = np.zeros((J1.n, J1.nb))
    for i in range(J1.nb):
        p = J1.rowptr[i] + list(J1.col[J1.rowptr[i]:J1.rowptr[i + 1]]).index(i)
        assert np.allclose(blocks[p].T @ w[3 * i:3 * i + 3], [1, 0, 0], atol=1e-12)
        W[3 * i:3 * i + 3, i] = w[3 * i:3 * i + 3]
        Pi[3 * i, i] = 1.0
    AP = W.T @ J1.to_dense() @ Pi
    l0 = s.level(0)
    assert np.allclose(_level_dense(l0, "A"), AP, rtol=1e-12, atol=1e-12 * np.abs(AP).max())
    for l in range(s.nlev - 1):
        a, k = s.level(l), full0.level(l)
        # the kept structure
        np.testing.assert_array_equal(a["cf"], k["cf"])
        np.testing.assert_array_equal(a["color"], k["color"])
        np.testing.assert_array_equal(a["P"].rowptr, k["P"].rowptr)
        np.testing.assert_array_equal(a["P"].col, k["P"].col)
        P = _level_dense(a, "P")
        for i in np.flatnonzero(a["cf"] == 1):
            assert np.count_nonzero(P[i]) == 1 and P[i].max() == 1.0
        # new values, Galerkin-consistent
        assert not np.array_equal(a["P"].val, k["P"].val)
        Ac = P.T @ _level_dense(a, "A") @ P
        An = _level_dense(s.level(l + 1), "A")
        assert np.allclose(An, Ac, rtol=1e-11, atol=1e-11 * np.abs(Ac).max())
    # unchanged values: the numeric resetup is the full setup
    t = oracle.Solver(J0, resetup=1, **kw)
    t.solve(J0.b)
    t.update(J0)
    for l in range(full0.nlev):
        a, k = t.level(l), full0.level(l)
        for key in ("rowptr", "col", "val"):
            np.testing.assert_array_equal(getattr(a["A"], key), getattr(k["A"], key))
        if l < full0.nlev - 1:
            np.testing.assert_array_equal(a["P"].val, k["P"].val)
    np.testing.assert_array_equal(t.bilu()[2], full0.bilu()[2])
    for o in (full0, s, t):
        o.close()


def test_vcycle_two_level_composition(tiny):
    """V(1,0) with an exact coarse solve: x = S b + P A_c^-1 R (b - A S b)."""
    J = tiny
    s = oracle.Solver(J, coarse_max=4, max_levels=2, pre=1, post=0)
    assert s.nlev == 2
    L0, L1 = s.level(0), s.level(1)
    A = L0["A"].dense()
    P = L0["P"].dense()
    Ac = L1["A"].dense()
    assert np.allclose(Ac, P.T @ A @ P, rtol=1e-12, atol=1e-12 * np.abs(Ac).max())
    b = np.random.default_rng(3).standard_normal(J.nb)
    a0 = L0["A"]
    Sb = oracle.mcgs_sweep(a0.rowptr, a0.col, a0.val, L0["color"], L0["ncolors"], b,
                           np.zeros(J.nb))
    ref = Sb + P @ np.linalg.solve(Ac, P.T @ (b - A @ Sb))
    x = s.vcycle(b)
    assert np.allclose(x, ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())
    s.close()


# ------------------------------- Alg. 4-5: VerticesSplitting/Grouping (f1)

def _grid5(nx_, ny_):
    n = nx_ * ny_
    A = np.zeros((n, n))
    for j in range(ny_):
        for i in range(nx_):
            c = i + nx_ * j
            for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                ii, jj = i + di, j + dj
                if 0 <= ii < nx_ and 0 <= jj < ny_:
                    A[c, ii + nx_ * jj] = -1.0
            A[c, c] = -A[c].sum() + 0.5
    M = sp.csr_matrix(A)
    M.sort_indices()
    return M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data


def test_vertices_grouping_gives_red_black_on_the_five_point_grid():
    """Alg. 4-5 at theta = 0 on the 4x4 five-point grid of Fig. 2(a): the first
    split collects one checkerboard class, which leaves the other independent,
    so c = 2 and the groups are the red-black grouping (red = (i + j) even)."""
    rp, cl, v = _grid5(4, 4)
    color, c = oracle.vertices_grouping(16, rp, cl, v, 0.0)
    assert c == 2
    np.testing.assert_array_equal(color, read_grid("redblack_4x4.txt").ravel())


@pytest.mark.parametrize("theta", [0.0, 0.05, 0.1, 0.3, 1.0])
def test_vertices_grouping_properties(theta):
    """Alg. 4-5 on a black-oil pressure matrix: every vertex in one group, no two
    vertices of a group strongly connected (Eq. 5.1, either direction); at
    theta = 0 each A_{V_l V_l} is diagonal (Prop. 5.2); c <= the largest
    degree of S u S^T plus one (Prop. 5.1's bound); theta = 1 gives one group."""
    rp, cl, v = _pressure_level0(bs.jacobian("20x20x5"))
    n = len(rp) - 1
    color, c = oracle.vertices_grouping(n, rp, cl, v, theta)
    assert color.min() == 0 and color.max() == c - 1 and len(np.unique(color)) == c
    Ad = np.abs(sp.csr_matrix((v, cl, rp), shape=(n, n)).toarray())
    Sd = Ad > theta * Ad.sum(axis=1, keepdims=True)     # Eq. 5.1, the row sum with the diagonal
    np.fill_diagonal(Sd, False)
    G = Sd | Sd.T
    same = color[:, None] == color[None, :]
    assert not (G & same).any()
    if theta == 0.0:
        A = sp.csr_matrix((v, cl, rp), shape=(n, n)).toarray()
        np.fill_diagonal(A, 0.0)
        assert not (A[same] != 0.0).any()
    assert c <= G.sum(axis=1).max() + 1
    if theta == 1.0:
        assert c == 1


def test_vertices_grouping_against_jp():
    """The paper's grouping (Alg. 4-5) and the JP coloring as the PGS-SCM
    smoother of the CPR solve on 20x20x5, at theta in {0, 0.05, 0.1, 0.3}: both
    converge; the level-0 group counts and iteration counts are printed
    (pytest -s) for the comparison in the design notes."""
    J = bs.jacobian("20x20x5")
    rows = []
    for theta in (0.0, 0.05, 0.1, 0.3):
        r = [theta]
        for coloring in (0, 1):
            s = oracle.Solver(J, theta_color=theta, coloring=coloring)
            _, st = s.solve(J.b, rtol=1e-6)
            assert st["converged"]
            r += [s.level(0)["ncolors"], st["iters"]]
            s.close()
        rows.append(r)
    print("\ntheta  JP colors/iters  Alg.4-5 colors/iters")
    for theta, c0, i0, c1, i1 in rows:
        print(f"{theta:5.2f}  {c0:3d} / {i0:3d}        {c1:3d} / {i1:3d}")


# -------------------------------------------- UA-AMG and the AMLI-cycle (f2)

def _chain(n):
    rows, cols, vals = [], [], []
    for i in range(n):
        for j, v in ((i - 1, -1.0), (i, 2.0), (i + 1, -1.0)):
            if 0 <= j < n:
                rows.append(i)
                cols.append(j)
                vals.append(v)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    return A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data


def test_pairwise_aggregation_on_a_chain():
    """A 1-D Laplacian: the end node has the fewest nodes depending on it, so
    matching runs left to right in pairs {2k, 2k+1}; the pair operator is again
    a chain, so the second pass gives aggregates of four consecutive nodes."""
    rp, cl, v = _chain(16)
    agg1, n1 = oracle.aggregate(16, rp, cl, v, passes=1)
    assert n1 == 8 and np.array_equal(agg1, np.arange(16) // 2)
    agg2, n2 = oracle.aggregate(16, rp, cl, v, passes=2)
    assert n2 == 4 and np.array_equal(agg2, np.arange(16) // 4)


@pytest.mark.parametrize("which", ["laplacian", "pressure"])
def test_pairwise_aggregation_properties(which):
    """Every node in exactly one aggregate; one pass forms pairs or singletons,
    each pair strongly coupled (c_ij < 0 and -c_ij >= 0.25 max_k -c_ik, from one
    of its nodes, c the symmetric part); two passes give at most four nodes,
    each aggregate connected in the symmetrised pattern; the count at least
    halves twice on the Laplacian."""
    if which == "laplacian":
        rp, cl, v = bs.laplacian_2d(12, 10)
    else:
        rp, cl, v = _pressure_level0(bs.jacobian(bs.GridSpec(8, 8, 3, seed=2)))
    n = len(rp) - 1
    A = sp.csr_matrix((v, cl, rp), shape=(n, n))
    C = ((A + A.T) * 0.5).toarray()
    np.fill_diagonal(C, 0.0)
    maxneg = np.maximum((-C).max(axis=1), 0.0)

    def strong(i, j):
        return C[i, j] < 0 and -C[i, j] >= 0.25 * maxneg[i]

    agg1, n1 = oracle.aggregate(n, rp, cl, v, passes=1)
    sizes = np.bincount(agg1, minlength=n1)
    assert sizes.sum() == n and sizes.min() >= 1 and sizes.max() <= 2
    for a in np.flatnonzero(sizes == 2):
        i, j = np.flatnonzero(agg1 == a)
        assert strong(i, j) or strong(j, i)
    agg2, n2 = oracle.aggregate(n, rp, cl, v, passes=2)
    sizes = np.bincount(agg2, minlength=n2)
    assert sizes.sum() == n and sizes.min() >= 1 and sizes.max() <= 4
    G = nx.Graph((i, int(j)) for i in range(n) for j in cl[rp[i]:rp[i + 1]] if j != i)
    for a in range(n2):
        assert nx.is_connected(G.subgraph(np.flatnonzero(agg2 == a).tolist()))
    if which == "laplacian":
        assert n2 <= n // 3


def test_handshake_matching_on_a_weighted_chain():
    """agg_match = 1 (handshake rounds) on a chain whose couplings grow weaker
    to the right, -(n - i) between i and i + 1: the strongest remaining edge is
    always the leftmost, so the pairs are {2k, 2k + 1}, and the pair operator
    is again such a chain, giving aggregates of four."""
    n = 16
    A = np.zeros((n, n))
    for i in range(n - 1):
        A[i, i + 1] = A[i + 1, i] = -(n - i)
    A[np.arange(n), np.arange(n)] = -A.sum(axis=1) + 1.0
    M = sp.csr_matrix(A)
    M.sort_indices()
    rp, cl, v = M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data
    agg1, n1 = oracle.aggregate(n, rp, cl, v, passes=1, match=1)
    assert n1 == 8 and np.array_equal(agg1, np.arange(n) // 2)
    agg2, n2 = oracle.aggregate(n, rp, cl, v, passes=2, match=1)
    assert n2 == 4 and np.array_equal(agg2, np.arange(n) // 4)


@pytest.mark.parametrize("which", ["laplacian", "pressure"])
def test_handshake_matching_properties(which):
    """Handshake rounds: pairs are strongly coupled in at least one direction;
    the matching is maximal (no two single nodes strongly coupled); two passes
    give connected aggregates of at most four nodes."""
    if which == "laplacian":
        rp, cl, v = bs.laplacian_2d(12, 10)
    else:
        rp, cl, v = _pressure_level0(bs.jacobian(bs.GridSpec(8, 8, 3, seed=2)))
    n = len(rp) - 1
    A = sp.csr_matrix((v, cl, rp), shape=(n, n))
    C = ((A + A.T) * 0.5).toarray()
    np.fill_diagonal(C, 0.0)
    maxneg = np.maximum((-C).max(axis=1), 0.0)
    strong = (C < 0) & (-C >= 0.25 * maxneg[:, None])
    cand = strong | strong.T
    agg1, n1 = oracle.aggregate(n, rp, cl, v, passes=1, match=1)
    sizes = np.bincount(agg1, minlength=n1)
    assert sizes.sum() == n and sizes.max() <= 2
    for a in np.flatnonzero(sizes == 2):
        i, j = np.flatnonzero(agg1 == a)
        assert cand[i, j]
    single = sizes[agg1] == 1
    assert not (cand & single[:, None] & single[None, :]).any()
    agg2, n2 = oracle.aggregate(n, rp, cl, v, passes=2, match=1)
    sizes = np.bincount(agg2, minlength=n2)
    assert sizes.sum() == n and sizes.max() <= 4
    G = nx.Graph((i, int(j)) for i in range(n) for j in cl[rp[i]:rp[i + 1]] if j != i)
    for a in range(n2):
        assert nx.is_connected(G.subgraph(np.flatnonzero(agg2 == a).tolist()))


@pytest.mark.parametrize("which", ["laplacian", "pressure", "heterogeneous"])
def test_handshake_with_attachment_properties(which):
    """agg_match = 2: the handshake pairs of agg_match = 1, and every node left
    alone that has a candidate joins the pair of its candidate of smallest edge
    key (c_ij, smaller hash, larger hash, index), recomputed here by brute
    force; nodes without a candidate stay alone; aggregates are numbered by
    the smallest node of their pair (or the lone node)."""
    if which == "laplacian":
        rp, cl, v = bs.laplacian_2d(12, 10)
    elif which == "pressure":
        rp, cl, v = _pressure_level0(bs.jacobian(bs.GridSpec(8, 8, 3, seed=2)))
    else:
        rp, cl, v = _pressure_level0(bs.jacobian(bs.GridSpec(10, 9, 4, 0.0, 2.0, 0.1, None, "corners", seed=7)))
    n = len(rp) - 1
    A = sp.csr_matrix((v, cl, rp), shape=(n, n))
    C = ((A + A.T) * 0.5).toarray()
    np.fill_diagonal(C, 0.0)
    maxneg = np.maximum((-C).max(axis=1), 0.0)
    strong = (C < 0) & (-C >= 0.25 * maxneg[:, None])
    cand = strong | strong.T
    hb = oracle.fmix32(3 * 1000003)            # the pass hash o_aggregate uses
    h = np.array([oracle.fmix32(i ^ hb) for i in range(n)], dtype=np.int64)
    pairs, npairs = oracle.aggregate(n, rp, cl, v, passes=1, match=1)
    agg, na = oracle.aggregate(n, rp, cl, v, passes=1, match=2)
    psize = np.bincount(pairs, minlength=npairs)
    lone = psize[pairs] == 1
    host = {}
    for i in np.flatnonzero(lone):
        js = np.flatnonzero(cand[i])
        if len(js):
            key = [(C[i, j], min(h[i], h[j]), max(h[i], h[j]), j) for j in js]
            host[i] = min(key)[3]
            assert psize[pairs[host[i]]] == 2          # every candidate of a lone node is paired
    leaders = sorted({int(np.flatnonzero(pairs == a).min()) for a in range(npairs)} - set(host))
    assert na == len(leaders)
    num = {ld: k for k, ld in enumerate(leaders)}
    for i in range(n):
        if i in host:
            assert agg[i] == agg[host[i]]
        else:
            assert agg[i] == num[int(np.flatnonzero(pairs == pairs[i]).min())]
    if which == "heterogeneous":
        assert len(host) > 0                      # the case the attachment is for


def test_ua_attachment_coarsens_and_solves():
    """amg = 1 with agg_match = 2 on a heterogeneous anisotropic grid (the
    benchmark generator's ln k ~ N(0, 2), kz/kx = 0.1): no singleton with a
    candidate survives, each level coarsens by at least 3x, the levels are
    Galerkin with unit-row P, and the CPR solve reaches the direct solution."""
    J = bs.jacobian(bs.GridSpec(12, 12, 6, 0.0, 2.0, 0.1, None, "corners", seed=11))
    s = oracle.Solver(J, amg=1, agg_match=2, coarse_max=16)
    assert s.nlev >= 3
    for l in range(s.nlev - 1):
        L0, L1 = s.level(l), s.level(l + 1)
        assert L1["A"].n * 3 <= L0["A"].n
        P = L0["P"].dense()
        assert np.array_equal(P.sum(axis=1), np.ones(P.shape[0]))
        Ac = L1["A"].dense()
        assert np.allclose(Ac, P.T @ L0["A"].dense() @ P, rtol=1e-12, atol=1e-12 * np.abs(Ac).max())
    x, st = s.solve(J.b, rtol=1e-10)
    assert st["converged"]
    assert np.allclose(x, np.linalg.solve(J.to_dense(), J.b), rtol=1e-7, atol=1e-9)
    s.close()


def test_ua_with_handshake_matching_solves():
    """amg = 1 with agg_match = 1: Galerkin levels of unit-row P and a CPR
    solve reaching the direct solution."""
    J = bs.jacobian(bs.GridSpec(8, 8, 4, seed=3))
    s = oracle.Solver(J, amg=1, agg_match=1, coarse_max=16)
    assert s.nlev >= 2
    for l in range(s.nlev - 1):
        L0, L1 = s.level(l), s.level(l + 1)
        P = L0["P"].dense()
        assert np.array_equal(P.sum(axis=1), np.ones(P.shape[0]))
        Ac = L1["A"].dense()
        assert np.allclose(Ac, P.T @ L0["A"].dense() @ P, rtol=1e-12, atol=1e-12 * np.abs(Ac).max())
    x, st = s.solve(J.b, rtol=1e-10)
    assert st["converged"]
    assert np.allclose(x, np.linalg.solve(J.to_dense(), J.b), rtol=1e-7, atol=1e-9)
    s.close()


def test_ua_hierarchy_is_galerkin():
    """amg = 1: P_l has one unit entry per row (the node's aggregate, at most
    four nodes each) and A_{l+1} = P_l^T A_l P_l."""
    J = bs.jacobian(bs.GridSpec(10, 10, 4, seed=1))
    s = oracle.Solver(J, amg=1, coarse_max=30)
    assert s.nlev >= 3
    for l in range(s.nlev - 1):
        L0, L1 = s.level(l), s.level(l + 1)
        P = L0["P"].dense()
        assert np.array_equal(P.sum(axis=1), np.ones(P.shape[0])) and set(np.unique(P)) <= {0.0, 1.0}
        assert np.array_equal(np.argmax(P, axis=1), L0["cf"])
        assert np.bincount(L0["cf"]).max() <= 4
        A, Ac = L0["A"].dense(), L1["A"].dense()
        assert np.allclose(Ac, P.T @ A @ P, rtol=1e-12, atol=1e-12 * np.abs(Ac).max())
    s.close()


def test_ua_numeric_resetup():
    """amg = 1 with resetup = 1: a rebuild keeps the aggregates (so P) and
    recomputes A_{l+1} = P^T A_l P; with unchanged values it equals the full
    setup bit for bit, and on the next Jacobian the levels stay Galerkin."""
    g = bs.GridSpec(10, 10, 4, seed=2)
    J0, J1 = list(bs.jacobian_sequence(g, 2, drift=0.05))
    kw = dict(amg=1, coarse_max=30, mu=0)
    full = oracle.Solver(J0, **kw)
    s = oracle.Solver(J0, resetup=1, **kw)
    s.solve(J0.b)
    s.update(J0)
    for l in range(full.nlev):
        np.testing.assert_array_equal(s.level(l)["A"].val, full.level(l)["A"].val)
    s.update(J1)
    _, st = s.solve(J1.b, rtol=1e-8)
    assert st["setup_called"] == 1 and st["converged"] and s.nlev == full.nlev
    for l in range(s.nlev - 1):
        a = s.level(l)
        np.testing.assert_array_equal(a["cf"], full.level(l)["cf"])
        P = a["P"].dense()
        Ac = P.T @ a["A"].dense() @ P
        An = s.level(l + 1)["A"].dense()
        assert np.allclose(An, Ac, rtol=1e-11, atol=1e-11 * np.abs(Ac).max())
    full.close()
    s.close()


def _two_level_dense(lv, lvc, Acinv):
    """x = S b + P Ac^-1 P^T (b - A S b) as a matrix (pre = 1, post = 0)."""
    a = lv["A"]
    A, P = a.dense(), lv["P"].dense()
    n = A.shape[0]
    S = np.column_stack([oracle.mcgs_sweep(a.rowptr, a.col, a.val, lv["color"], lv["ncolors"], e,
                                           np.zeros(n)) for e in np.eye(n)])
    return S + P @ Acinv @ P.T @ (np.eye(n) - A @ S)


def test_amli_cycle_two_levels_is_the_two_level_cycle():
    """With the coarsest level next, the AMLI-cycle's coarse problem is solved
    exactly: x = S b + P A_c^-1 P^T (b - A S b)."""
    J = bs.tiny()
    s = oracle.Solver(J, amg=1, coarse_max=12, max_levels=2, pre=1, post=0)
    assert s.nlev == 2
    L0, L1 = s.level(0), s.level(1)
    B = _two_level_dense(L0, L1, np.linalg.inv(L1["A"].dense()))
    b = np.random.default_rng(5).standard_normal(J.nb)
    assert np.allclose(s.vcycle(b), B @ b, rtol=1e-10, atol=1e-10 * np.abs(B @ b).max())
    s.close()


def test_amli_cycle_coarse_correction_minimises_the_residual():
    """Three levels, two GCR steps on level 1 with the (linear) two-level cycle
    B_1 of levels 1-2 as preconditioner: the correction e minimises
    ||r_1 - A_1 e|| over span{B_1 r_1, B_1 A_1 B_1 r_1} (least squares here),
    and x = S_0 b + P_0 e.  The cycle is homogeneous and not additive."""
    J = bs.jacobian(bs.GridSpec(6, 6, 3, seed=4))
    s = oracle.Solver(J, amg=1, coarse_max=8, max_levels=3, pre=1, post=0, amli_iters=2)
    assert s.nlev == 3
    L0, L1, L2 = s.level(0), s.level(1), s.level(2)
    B1 = _two_level_dense(L1, L2, np.linalg.inv(L2["A"].dense()))
    a0 = L0["A"]
    A0, P0, A1 = a0.dense(), L0["P"].dense(), L1["A"].dense()
    rng = np.random.default_rng(6)
    b = rng.standard_normal(J.nb)
    S0b = oracle.mcgs_sweep(a0.rowptr, a0.col, a0.val, L0["color"], L0["ncolors"], b, np.zeros(J.nb))
    r1 = P0.T @ (b - A0 @ S0b)
    V = np.column_stack([B1 @ r1, B1 @ A1 @ B1 @ r1])
    y = np.linalg.lstsq(A1 @ V, r1, rcond=None)[0]
    ref = S0b + P0 @ (V @ y)
    x = s.vcycle(b)
    assert np.allclose(x, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())
    assert np.array_equal(s.vcycle(4.0 * b), 4.0 * x)
    b2 = rng.standard_normal(J.nb)
    assert not np.allclose(s.vcycle(b + b2), x + s.vcycle(b2), rtol=1e-6, atol=1e-9)
    s.close()


def test_cpr_solve_with_ua_amg():
    """The CPR solve with the UA-AMG first stage reaches the direct solution."""
    J = bs.jacobian(bs.GridSpec(8, 8, 4, seed=3))
    s = oracle.Solver(J, amg=1, coarse_max=16)
    x, st = s.solve(J.b, rtol=1e-10)
    assert st["converged"]
    assert np.allclose(x, np.linalg.solve(J.to_dense(), J.b), rtol=1e-7, atol=1e-9)
    s.close()


@pytest.mark.parametrize("coarse_max", [10 ** 6, 8])
def test_whole_solve_reaches_direct_solution(tiny, coarse_max):
    J = tiny
    s = oracle.Solver(J, coarse_max=coarse_max)
    x, st = s.solve(J.b, rtol=1e-12)
    ref = np.linalg.solve(J.to_dense(), J.b)
    assert st["converged"]
    assert np.linalg.norm(x - ref) <= 1e-8 * np.linalg.norm(ref)
    s.close()


def test_fgmres_identity_exact_in_n_steps():
    rng = np.random.default_rng(8)
    J = bs.tiny(3, 3, 1, wells="none", seed=3)             # 9 block rows, n = 27 <= 30
    x, st, hist, rc = oracle.fgmres_identity(J, J.b, rtol=1e-13, m=30, max_restarts=1)
    ref = np.linalg.solve(J.to_dense(), J.b)
    assert rc == 0 and st["iters"] <= J.n and st["restarts"] == 1
    assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)
    assert np.all(np.diff(hist) <= 1e-15)                     # GMRES residuals never increase
    x0 = rng.standard_normal(J.n)
    x2, st2, _, rc2 = oracle.fgmres_identity(J, J.b, x0=x0, rtol=1e-13, m=30, max_restarts=1)
    assert rc2 == 0 and np.linalg.norm(x2 - ref) <= 1e-10 * np.linalg.norm(ref)


def test_zero_rhs_and_initial_guess():
    J = bs.tiny()
    s = oracle.Solver(J)
    x, st = s.solve(np.zeros(J.n))
    assert st["iters"] == 0 and st["converged"] and not x.any()
    # a nonzero initial guess reaches the same solution (criterion relative to r_0, Alg. 2)
    ref = np.linalg.solve(J.to_dense(), J.b)
    x0 = np.random.default_rng(0).standard_normal(J.n)
    x, st = s.solve(J.b, x0=x0, rtol=1e-12)
    assert st["converged"] and np.linalg.norm(x - ref) <= 1e-8 * np.linalg.norm(ref)
    s.close()


# ------------------------------------------------------------- adaptive rule

@pytest.mark.parametrize("mu", [0, 5, 10 ** 6])
def test_adaptive_setup_rule(mu):
    """Alg. 3: reuse B^(k-1) iff k > 1 and It^(k-1) <= mu; mu = 0 is plain CPR."""
    g = bs.GridSpec(6, 6, 3, 0.0, 1.0, 1.0, None, "corners", seed=2)
    seq = list(bs.jacobian_sequence(g, 6, drift=0.05))
    s = oracle.Solver(seq[0], mu=mu)
    calls, iters = [1], []
    _, st = s.solve(seq[0].b)
    iters.append(st["iters"])
    for J in seq[1:]:
        s.update(J)
        _, st = s.solve(J.b)
        calls.append(st["setup_called"])
        iters.append(st["iters"])
        assert st["converged"]
    expect = [1] + [int(iters[k - 1] > mu) for k in range(1, len(seq))]
    assert calls == expect
    if mu == 0:
        assert calls == [1] * len(seq)
    if mu == 10 ** 6:
        assert calls == [1] + [0] * (len(seq) - 1)
    s.close()


def test_pattern_change_forces_setup():
    """Remark 4.2: a new size forces a new setup whatever mu says."""
    s = oracle.Solver(bs.tiny(4, 4, 2), mu=10 ** 6)
    s.solve(bs.tiny(4, 4, 2).b)
    J2 = bs.tiny(5, 4, 2)
    s.update(J2)
    x, st = s.solve(J2.b)
    assert st["setup_called"] == 1 and st["converged"]
    s.close()


# ------------------------------------------------------- hash and V-cycle pins

def test_fmix32_against_published_murmur3_vectors():
    """MurmurHash3_x86_32 of the empty key is fmix32(seed) (no blocks, no tail,
    length 0), so its published test vectors pin the finalizer: seed 1 gives
    0x514E28B7, seed 0xFFFFFFFF gives 0x81F16F39, seed 0 gives 0.  The
    per-vertex hash is then fmix32(i ^ fmix32(seed32 + 1000003 salt + level))."""
    assert oracle.fmix32(1) == 0x514E28B7
    assert oracle.fmix32(0xFFFFFFFF) == 0x81F16F39
    assert oracle.fmix32(0) == 0
    for i in (0, 1, 7, 123456):
        assert oracle.hash32(1, 0, 0, i) == oracle.fmix32(i ^ 0x514E28B7)
    # salt and level enter the base as seed32 + 1000003 * salt + level
    assert oracle.hash32(0, 1, 5, 9) == oracle.fmix32(9 ^ oracle.fmix32(1000003 + 5))


def _mcgs_dense(A, color, ncolors, b, x, descending):
    """One multi-color Gauss-Seidel sweep (Alg. 6) from the matrix splitting:
    the rows of each color take x_I <- (b_I - (A - D)_I x) / d_I with x as of
    the start of the color (Jacobi within a color)."""
    x = x.copy()
    d = np.diag(A)
    off = A - np.diag(d)
    order = range(ncolors - 1, -1, -1) if descending else range(ncolors)
    for c in order:
        I = color == c
        x[I] = (b[I] - off[I] @ x) / d[I]
    return x


def _vcycle_dense(levels, l, b, post_descending=True):
    """V(1,1) from zero on dense level matrices: pre-smoothing colors ascending,
    residual, R = P^T, the coarser level recursively (exact at the coarsest),
    prolongation, post-smoothing colors descending."""
    A = levels[l]["A"]
    if l == len(levels) - 1:
        return np.linalg.solve(A, b)
    col, nc, P = levels[l]["color"], levels[l]["ncolors"], levels[l]["P"]
    x = _mcgs_dense(A, col, nc, b, np.zeros_like(b), False)
    xc = _vcycle_dense(levels, l + 1, P.T @ (b - A @ x), post_descending)
    x = x + P @ xc
    return _mcgs_dense(A, col, nc, b, x, post_descending)


def test_vcycle_three_level_composition():
    """The oracle's V(1,1) on three levels against the dense composition above:
    colors ascending before the coarse correction and descending after it, the
    middle level smoothed on both sides, an exact solve only on the coarsest.
    Ascending post-smoothing would give a different result, by far more than
    the tolerance, so the test fixes the order as well as the recursion."""
    J = bs.tiny(6, 5, 3)
    s = oracle.Solver(J, coarse_max=8, max_levels=3)
    assert s.nlev == 3
    levels = []
    for l in range(3):
        L = s.level(l)
        d = {"A": L["A"].dense()}
        if l < 2:
            assert L["ncolors"] >= 2
            d.update(color=L["color"], ncolors=L["ncolors"], P=L["P"].dense())
        levels.append(d)
    b = np.random.default_rng(5).standard_normal(J.nb)
    ref = _vcycle_dense(levels, 0, b)
    x = s.vcycle(b)
    np.testing.assert_allclose(x, ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())
    wrong = _vcycle_dense(levels, 0, b, post_descending=False)
    assert np.abs(wrong - ref).max() > 1e-6 * np.abs(ref).max()
    s.close()


def test_solve_rows_on_a_block_diagonal_system():
    """FGMRES on one system of a block-diagonal concatenation with the shared B
    restricted to its rows: B of a vector supported on one system is zero on
    the others (exactly), a coarse-LU-only B reaches that system's direct
    solution, and with the default hierarchy the solve converges on the true
    residual of the system alone."""
    J1, J2 = bs.tiny(4, 4, 2, seed=1), bs.tiny(5, 3, 2, seed=2)
    C = block_diag([J1, J2])
    o = oracle.Solver(C, coarse_max=8)
    v = np.zeros(C.n)
    v[3 * J1.nb:] = np.random.default_rng(1).standard_normal(J2.n)
    z = o.cpr_apply(v)
    assert not z[:3 * J1.nb].any() and np.abs(z[3 * J1.nb:]).max() > 0
    x, st = o.solve_rows(J1.nb, C.nb, J2.b, rtol=1e-6)
    assert st["converged"]
    assert np.linalg.norm(J2.b - oracle.bsr3_spmv(J2, x)) < 1e-6 * np.linalg.norm(J2.b)
    o.close()
    exact = oracle.Solver(C, coarse_max=4096)
    assert exact.nlev == 1
    x, st = exact.solve_rows(0, J1.nb, J1.b, rtol=1e-12)
    ref = np.linalg.solve(J1.to_dense(), J1.b)
    np.testing.assert_allclose(x, ref, rtol=1e-8, atol=1e-8 * np.abs(ref).max())
    with pytest.raises(RuntimeError):
        exact.solve_rows(0, J1.nb + 1, np.zeros(3 * J1.nb + 3))   # couples into the next system
    exact.close()


def test_openmp_build_is_bit_identical():
    """The CPU baseline's multi-threaded oracle (OpenMP over rows within a
    color, SpMV rows and element-wise vector updates) computes every value in
    the single-threaded order: B v, the BILU(0) solve, the V-cycle and whole
    solves agree bit for bit, multicolor and natural-order BILU alike."""
    for J, kw in ((bs.jacobian("20x20x5"), {}), (bs.jacobian(bs.GridSpec(37, 23, 9, seed=5)), {}),
                  (bs.jacobian("20x20x5"), {"bilu_order": 1})):
        a, b = oracle.Solver(J, **kw), oracle.Solver(J, omp=True, **kw)
        v = np.random.default_rng(2).standard_normal(J.n)
        np.testing.assert_array_equal(a.cpr_apply(v), b.cpr_apply(v))
        np.testing.assert_array_equal(a.bilu_apply(v), b.bilu_apply(v))
        np.testing.assert_array_equal(a.vcycle(v[:J.nb]), b.vcycle(v[:J.nb]))
        xa, sa = a.solve(J.b, rtol=1e-8)
        xb, sb = b.solve(J.b, rtol=1e-8)
        assert sa == sb
        np.testing.assert_array_equal(xa, xb)
        a.close()
        b.close()
