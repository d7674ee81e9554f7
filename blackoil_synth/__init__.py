"""Seeded synthetic black-oil Jacobians in 3x3 block-sparse-row (BSR) form.

This module is the ONLY code shared by the CUDA path's tests/benchmark and the
FP64 oracle: it draws random numbers and assembles matrices from them, and holds
none of the solver's arithmetic (no decoupling, strength, coarsening, smoothing or
Krylov step).  Both sides receive identical bytes.

The structure follows the fully implicit black-oil Jacobian of Eq. 2.7/2.8
(Sec. 2.2): one 3x3 block row per cell (unknowns P, S_w, S_o / S_g) and one
block row per implicit well (bottom-hole pressure in slot 0, identity in the
two dummy slots).  The paper's SPE10 data is not available, so values are
synthetic with SPE10's shape:

* cells c = i + nx*(j + ny*k) on an nx x ny x nz grid, 7-point stencil;
* ln k drawn per cell (normal, or alternating bands of layers for a
  channelised field); harmonic face transmissibility T = 2 k_a k_b/(k_a+k_b),
  z faces scaled by kz/kx;
* pressure column (column 0) of row alpha: -T*lambda_alpha off the diagonal,
  lambda_alpha*sum(T) + acc on it, lambda = (1.0, 0.8, 0.5), acc ~ U(1e-2,1e-1);
* saturation diagonals acc + 0.5*sum(T);
* every other saturation-column entry U(-0.1,0.1) times the diagonal entry of
  its row (in diagonal and off-diagonal blocks);
* wells: WI = k of the perforated cell, coupled through slot 0 both ways
  (scaled by lambda_alpha in the cell rows, which also gain lambda_alpha*WI on
  their diagonal), well row [0][0] = sum(WI);
* right-hand side U(-1,1).

A Newton sequence (``step`` > 0) multiplies every generator input (T, acc,
couplings, WI) by (1 + drift*U(-1,1)) once per step, cumulatively, with a
generator seeded by (seed, step); the pattern never changes.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

LAMBDA = np.array([1.0, 0.8, 0.5])


@dataclass(frozen=True)
class GridSpec:
    """Parameters of one synthetic reservoir workload."""
    nx: int
    ny: int
    nz: int
    lnk_mean: float = 0.0
    lnk_std: float = 1.0
    kz_over_kx: float = 1.0
    # channelised layers: bands of `band` layers alternate between the two
    # (mean, std) pairs; None = one normal field
    bands: tuple | None = None
    wells: str = "corners"          # "corners" | "five_spot" | "none"
    seed: int = 0

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz


# The workloads (sizes, permeability fields and wells) the tests and the
# benchmark use.  Keys name the grid.
CONFIGS = {
    "20x20x5": GridSpec(20, 20, 5, 0.0, 1.0, 1.0, None, "corners"),
    "128x128x32": GridSpec(128, 128, 32, 0.0, 2.0, 0.1, None, "five_spot"),
    "60x220x85": GridSpec(60, 220, 85, 0.0, 1.0, 1.0, (5, (3.0, 1.0), (-2.0, 1.0)), "corners"),
}


def batch_specs(nsys: int = 64, seed: int = 0) -> list[GridSpec]:
    """Independent systems for batched solves: nx, ny drawn uniformly from
    16..64 with nz = 16 (16^3 to 64x64x16 cells), ln k ~ N(0, 1.5), corner wells."""
    rng = np.random.Generator(np.random.PCG64([seed, 64]))
    out = []
    for k in range(nsys):
        nx, ny = (int(v) for v in rng.integers(16, 65, 2))
        out.append(GridSpec(nx, ny, 16, 0.0, 1.5, 1.0, None, "corners", seed=1000 + k))
    return out


def ensemble_specs(nmembers: int = 32, seed: int = 0, full: bool = True) -> list[GridSpec]:
    """Ensemble members for the serving workload: grids from 32x32x8 to
    128x128x32 (nx = ny from {32, 48, 64, 96, 128}, nz from {8, 16, 32}), or,
    with full=False, from 32x32x8 to 64x64x16; ln k ~ N(0, 1), corner wells."""
    rng = np.random.Generator(np.random.PCG64([seed, 32]))
    sizes, layers = ([32, 48, 64, 96, 128], [8, 16, 32]) if full else ([32, 48, 64], [8, 16])
    out = []
    for k in range(nmembers):
        n = int(rng.choice(sizes))
        nz = int(rng.choice(layers))
        out.append(GridSpec(n, n, nz, 0.0, 1.0, 1.0, None, "corners", seed=2000 + k))
    return out


def well_columns(g: GridSpec) -> list[tuple[int, int]]:
    """(i, j) surface locations of the wells; each perforates every layer."""
    if g.wells == "none":
        return []
    if g.wells == "corners":            # injector + producer on corner columns
        return [(0, 0), (g.nx - 1, g.ny - 1)]
    if g.wells == "five_spot":          # 3 x 3 lattice
        xs = sorted({0, g.nx // 2, g.nx - 1})
        ys = sorted({0, g.ny // 2, g.ny - 1})
        return [(i, j) for j in ys for i in xs]
    raise ValueError(g.wells)


@dataclass
class Jacobian:
    """One 3x3-BSR system.  Arrays are host numpy arrays (int32 / float64)."""
    nb: int
    rowptr: np.ndarray      # int32 [nb+1]
    col: np.ndarray         # int32 [nnzb], sorted within each row, diagonal present
    val: np.ndarray         # float64 [nnzb*9], row-major 3x3 blocks
    b: np.ndarray           # float64 [3*nb]
    spec: GridSpec | None = None
    step: int = 0
    ncells: int = 0
    nwells: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def nnzb(self) -> int:
        return int(self.col.shape[0])

    @property
    def n(self) -> int:
        return 3 * self.nb

    def to_dense(self) -> np.ndarray:
        """Dense (3nb x 3nb) copy; for tiny systems only."""
        A = np.zeros((3 * self.nb, 3 * self.nb))
        v = self.val.reshape(-1, 3, 3)
        for i in range(self.nb):
            for p in range(self.rowptr[i], self.rowptr[i + 1]):
                j = self.col[p]
                A[3 * i:3 * i + 3, 3 * j:3 * j + 3] = v[p]
        return A

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.bsr_matrix((self.val.reshape(-1, 3, 3), self.col, self.rowptr),
                             shape=(3 * self.nb, 3 * self.nb))


class _Pattern:
    """Block pattern and the index maps the value assembly needs (built once per grid)."""

    def __init__(self, g: GridSpec):
        nx, ny, nz = g.nx, g.ny, g.nz
        nc = g.ncells
        self.nc = nc
        wells = well_columns(g)
        self.nw = len(wells)
        cid = np.arange(nc).reshape(nz, ny, nx)   # cid[k, j, i]
        # neighbour offsets in ascending column order: -z, -y, -x, (self), +x, +y, +z
        ii = np.broadcast_to(np.arange(nx)[None, None, :], (nz, ny, nx)).ravel()
        jj = np.broadcast_to(np.arange(ny)[None, :, None], (nz, ny, nx)).ravel()
        kk = np.broadcast_to(np.arange(nz)[:, None, None], (nz, ny, nx)).ravel()
        self.ii, self.jj, self.kk = ii, jj, kk
        slots = [
            ("z-", kk > 0, -nx * ny),
            ("y-", jj > 0, -nx),
            ("x-", ii > 0, -1),
            ("self", np.ones(nc, bool), 0),
            ("x+", ii < nx - 1, 1),
            ("y+", jj < ny - 1, nx),
            ("z+", kk < nz - 1, nx * ny),
        ]
        # perforations: well w perforates cells (i_w, j_w, k) for all k
        perf_cell = []
        perf_well = []
        for w, (iw, jw) in enumerate(wells):
            for k in range(nz):
                perf_cell.append(int(cid[k, jw, iw]))
                perf_well.append(w)
        perf_cell = np.array(perf_cell, dtype=np.int64)
        perf_well = np.array(perf_well, dtype=np.int64)
        self.perf_cell, self.perf_well = perf_cell, perf_well
        cell_well = np.full(nc, -1, dtype=np.int64)
        cell_well[perf_cell] = perf_well
        self.cell_well = cell_well

        # row lengths
        cnt = np.zeros(nc + self.nw, dtype=np.int64)
        for _, m, _ in slots:
            cnt[:nc] += m
        cnt[:nc] += cell_well >= 0
        for w in range(self.nw):
            cnt[nc + w] = np.count_nonzero(perf_well == w) + 1
        rowptr = np.zeros(nc + self.nw + 1, dtype=np.int64)
        np.cumsum(cnt, out=rowptr[1:])
        self.rowptr = rowptr
        nnzb = int(rowptr[-1])
        col = np.empty(nnzb, dtype=np.int64)
        # slot position of each (cell, slot)
        pos = rowptr[:nc].copy()
        self.slot_pos = {}
        for name, m, off in slots:
            cells = np.nonzero(m)[0]
            p = pos[cells]
            col[p] = cells + off
            self.slot_pos[name] = (cells, p)
            pos[cells] += 1
        # cell -> well block (well columns are > every cell column, so last)
        pc = perf_cell
        self.cw_pos = pos[pc].copy()
        col[self.cw_pos] = nc + perf_well
        pos[pc] += 1
        # well rows: perforated cells ascending, then the diagonal
        self.wc_pos = np.empty(len(pc), dtype=np.int64)
        self.wdiag_pos = np.empty(self.nw, dtype=np.int64)
        for w in range(self.nw):
            sel = np.nonzero(perf_well == w)[0]
            order = sel[np.argsort(pc[sel])]
            p0 = rowptr[nc + w]
            self.wc_pos[order] = p0 + np.arange(len(order))
            col[p0:p0 + len(order)] = pc[order]
            self.wdiag_pos[w] = p0 + len(order)
            col[p0 + len(order)] = nc + w
        self.col = col
        self.nnzb = nnzb
        self.nb = nc + self.nw
        # faces: x faces between (i,j,k) and (i+1,j,k), etc.; index by the lower cell
        self.nfx = (nx - 1) * ny * nz
        self.nfy = nx * (ny - 1) * nz
        self.nfz = nx * ny * (nz - 1)


def _lnk(g: GridSpec, rng: np.random.Generator) -> np.ndarray:
    z = rng.standard_normal(g.ncells)
    if g.bands is None:
        return g.lnk_mean + g.lnk_std * z
    band, (m0, s0), (m1, s1) = g.bands
    kk = np.arange(g.ncells) // (g.nx * g.ny)
    first = ((kk // band) % 2) == 0
    return np.where(first, m0 + s0 * z, m1 + s1 * z)


class _Inputs:
    """The generator's inputs (the quantities that drift between Newton steps)."""

    def __init__(self, g: GridSpec, pat: _Pattern):
        rng = np.random.Generator(np.random.PCG64(g.seed))
        nx, ny, nz = g.nx, g.ny, g.nz
        k = np.exp(_lnk(g, rng)).reshape(nz, ny, nx)
        self.acc = rng.uniform(1e-2, 1e-1, g.ncells)
        self.coup = rng.uniform(-0.1, 0.1, (pat.nnzb, 3, 2))
        self.rhs_base = rng.uniform(-1.0, 1.0, 3 * pat.nb)

        def harm(a, b):
            return 2.0 * a * b / (a + b)

        self.Tx = harm(k[:, :, :-1], k[:, :, 1:]).ravel()            # [nz, ny, nx-1]
        self.Ty = harm(k[:, :-1, :], k[:, 1:, :]).ravel()            # [nz, ny-1, nx]
        self.Tz = (harm(k[:-1], k[1:]) * g.kz_over_kx).ravel()       # [nz-1, ny, nx]
        self.WI = k.ravel()[pat.perf_cell].copy()

    def drift(self, g: GridSpec, step: int, rel: float):
        rng = np.random.Generator(np.random.PCG64([g.seed, step]))
        for name in ("Tx", "Ty", "Tz", "acc", "coup", "WI"):
            a = getattr(self, name)
            a *= 1.0 + rel * rng.uniform(-1.0, 1.0, a.shape)
        return rng


_PATTERN_CACHE: dict = {}


def _pattern(g: GridSpec) -> _Pattern:
    """The last grid's pattern is kept; safe to call from several threads (a
    miss may build the pattern twice, never returns another grid's)."""
    key = (g.nx, g.ny, g.nz, g.wells)
    pat = _PATTERN_CACHE.get(key)
    if pat is None:
        pat = _Pattern(g)
        _PATTERN_CACHE.clear()
        _PATTERN_CACHE[key] = pat
    return pat


def jacobian_sequence(g: GridSpec, nsteps: int, drift: float = 0.05):
    """Yield the Jacobians of Newton steps 0..nsteps-1 (values drift cumulatively)."""
    pat = _pattern(g)
    inp = _Inputs(g, pat)
    for s in range(nsteps):
        if s == 0:
            rhs = inp.rhs_base
        else:
            rng = inp.drift(g, s, drift)
            rhs = rng.uniform(-1.0, 1.0, 3 * pat.nb)
        yield _assemble(g, pat, inp, rhs, s)


def jacobian(g: GridSpec | str, step: int = 0, drift: float = 0.05) -> Jacobian:
    """The Jacobian of Newton step `step` of workload `g` (a GridSpec or a CONFIGS key)."""
    if isinstance(g, str):
        g = CONFIGS[g]
    last = None
    for last in jacobian_sequence(g, step + 1, drift):
        pass
    return last


def _assemble(g: GridSpec, pat: _Pattern, inp: _Inputs, rhs: np.ndarray, step: int) -> Jacobian:
    nx, ny, nz = g.nx, g.ny, g.nz
    nc = pat.nc
    val = np.zeros((pat.nnzb, 3, 3))
    lam = LAMBDA
    # transmissibility of each neighbour slot, and the row sums
    Tsum = np.zeros(nc)
    slotT = {}
    ii, jj, kk = pat.ii, pat.jj, pat.kk
    for name, (cells, p) in pat.slot_pos.items():
        if name == "self":
            continue
        i, j, k = ii[cells], jj[cells], kk[cells]
        if name == "x-":
            T = inp.Tx[(k * ny + j) * (nx - 1) + (i - 1)]
        elif name == "x+":
            T = inp.Tx[(k * ny + j) * (nx - 1) + i]
        elif name == "y-":
            T = inp.Ty[(k * (ny - 1) + (j - 1)) * nx + i]
        elif name == "y+":
            T = inp.Ty[(k * (ny - 1) + j) * nx + i]
        elif name == "z-":
            T = inp.Tz[((k - 1) * ny + j) * nx + i]
        else:  # z+
            T = inp.Tz[(k * ny + j) * nx + i]
        slotT[name] = (cells, p, T)
        np.add.at(Tsum, cells, T)
    WIcell = np.zeros(nc)
    WIcell[pat.perf_cell] = inp.WI
    acc = inp.acc
    # diagonal blocks of cells
    cells, pd = pat.slot_pos["self"]
    d = np.zeros((nc, 3, 3))
    for a in range(3):
        d[:, a, 0] = lam[a] * (Tsum + WIcell) + acc
    d[:, 1, 1] = acc + 0.5 * Tsum
    d[:, 2, 2] = acc + 0.5 * Tsum
    cp = inp.coup[pd]                         # [nc, 3, 2]
    rowdiag = np.stack([d[:, 0, 0], d[:, 1, 1], d[:, 2, 2]], axis=1)   # [nc, 3]
    d[:, 0, 1] = cp[:, 0, 0] * rowdiag[:, 0]
    d[:, 0, 2] = cp[:, 0, 1] * rowdiag[:, 0]
    d[:, 1, 2] = cp[:, 1, 1] * rowdiag[:, 1]
    d[:, 2, 1] = cp[:, 2, 0] * rowdiag[:, 2]
    val[pd] = d
    # off-diagonal cell-cell blocks
    for name, (cells, p, T) in slotT.items():
        blk = np.zeros((len(cells), 3, 3))
        blk[:, :, 0] = -T[:, None] * lam[None, :]
        cpp = inp.coup[p]
        rd = rowdiag[cells]
        blk[:, :, 1] = cpp[:, :, 0] * rd
        blk[:, :, 2] = cpp[:, :, 1] * rd
        val[p] = blk
    # cell -> well blocks and well rows
    if pat.nw:
        pc = pat.perf_cell
        WI = inp.WI
        blk = np.zeros((len(pc), 3, 3))
        blk[:, :, 0] = -WI[:, None] * lam[None, :]
        val[pat.cw_pos] = blk
        wblk = np.zeros((len(pc), 3, 3))
        wblk[:, 0, 0] = -WI
        val[pat.wc_pos] = wblk
        wsum = np.zeros(pat.nw)
        np.add.at(wsum, pat.perf_well, WI)
        for w in range(pat.nw):
            val[pat.wdiag_pos[w]] = np.diag([wsum[w], 1.0, 1.0])
    return Jacobian(
        nb=pat.nb,
        rowptr=pat.rowptr.astype(np.int32),
        col=pat.col.astype(np.int32),
        val=np.ascontiguousarray(val.reshape(-1)),
        b=np.ascontiguousarray(rhs.copy()),
        spec=g, step=step, ncells=nc, nwells=pat.nw,
    )


def tiny(nx: int = 4, ny: int = 4, nz: int = 2, seed: int = 0, wells: str = "corners",
         lnk_std: float = 1.0) -> Jacobian:
    """A small system for brute-force checks (4x4x2 + 2 wells = 34 block rows)."""
    return jacobian(GridSpec(nx, ny, nz, 0.0, lnk_std, 1.0, None, wells, seed))


# ---------------------------------------------------------------------------
# Scalar test matrices (for the pressure-level pins): plain textbook operators.

def laplacian_2d(nx: int, ny: int, shift: float = 0.0) -> tuple:
    """5-point 2-D Laplacian (Dirichlet-free, zero row sum plus `shift` on the
    diagonal) as CSR arrays (rowptr int32, col int32, val float64)."""
    n = nx * ny
    rows, cols, vals = [], [], []
    for j in range(ny):
        for i in range(nx):
            c = i + nx * j
            nb = []
            if j > 0:
                nb.append(c - nx)
            if i > 0:
                nb.append(c - 1)
            if i < nx - 1:
                nb.append(c + 1)
            if j < ny - 1:
                nb.append(c + nx)
            ent = [(q, -1.0) for q in nb] + [(c, float(len(nb)) + shift)]
            ent.sort()
            for q, v in ent:
                rows.append(c)
                cols.append(q)
                vals.append(v)
    return _coo_to_csr(n, rows, cols, vals)


def random_sparse(n: int, density: float, seed: int, spd_shift: float = 1.0,
                  symmetric_pattern: bool = True, neg_offdiag: bool = True) -> tuple:
    """A random sparse matrix with a nonzero diagonal, as CSR arrays."""
    rng = np.random.Generator(np.random.PCG64(seed))
    M = (rng.random((n, n)) < density).astype(float)
    np.fill_diagonal(M, 0.0)
    if symmetric_pattern:
        M = np.maximum(M, M.T)
    V = rng.uniform(0.1, 1.0, (n, n)) * M
    if not neg_offdiag:
        V *= np.where(rng.random((n, n)) < 0.3, -1.0, 1.0)
        V = -V
    else:
        V = -V
    diag = np.abs(V).sum(axis=1) + spd_shift
    A = V + np.diag(diag)
    rows, cols = np.nonzero((M + np.eye(n)) > 0)
    return _coo_to_csr(n, rows.tolist(), cols.tolist(), A[rows, cols].tolist())


def _coo_to_csr(n, rows, cols, vals):
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(n + 1, dtype=np.int32)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr).astype(np.int32)
    return rowptr, cols.astype(np.int32), vals
