"""Seeded synthetic water boxes and the block-sparse matrices built on them.

The paper's sign-method and DBCSR workloads are liquid water described with an
atom-blocked Gaussian basis: DBCSR block sizes follow the basis of each atom
(5 for H and 13 for O with DZVP, DBCSR section "DBCSR library"), and the
Kohn-Sham matrices are sparse because matrix elements decay with the distance
between atoms.  The Kohn-Sham matrices themselves need a full electronic
structure code, so this module builds stand-ins with the same shapes, block
sizes and sparsity structure:

* water molecules at 1 g/cc (box edge 9.86 A for 32 molecules), placed by
  random sequential addition with a minimum O-O distance of 2.5 A and a
  uniformly random orientation (Shoemake quaternion); rigid geometry with
  O-H = 0.9572 A and H-O-H = 104.52 degrees; atoms ordered O, H, H per molecule;
* a *decay matrix*: block (I, J) is present iff the minimum-image distance
  r_IJ < 8 A; its entries are u * exp(-0.3 r_IJ^2) with u uniform in [-1, 1);
  block (J, I) is the transpose of block (I, J); a diagonal block is
  (U + U^T)/2 + 2 I;
* an *overlap matrix* S for a non-orthogonal basis: 1 + sigma * |D|, where D is a
  decay matrix on the same pattern drawn from an independent stream, without the
  diagonal shift (entries taken in absolute value, as overlaps of nearby s-like
  functions are positive), and sigma = 0.9 / (largest row sum of |D|).  By the
  Gershgorin bound the eigenvalues of S lie in [0.1, 1.9], so S is symmetric positive
  definite (on water boxes they fall in about [0.9, 1.6]).  By Sylvester's law of
  inertia and Ostrowski's theorem the generalized problem H c = S c e keeps the gapped
  Hamiltonian's occupied count at mu = 0, with eigenvalues in [-17.5, -0.13] or
  [0.13, 17.5];
* a *gapped Hamiltonian*: for every molecule the intra-molecular d x d part of
  the decay matrix is diagonalised and its eigenvalues replaced by
  -1 + 0.25 t (the 4 lowest) and +1 + 0.25 t (the other d - 4), t evenly
  spaced in [-1, 1]; the inter-molecular blocks are scaled by
  gamma = 0.5 / (largest absolute row sum of the inter-molecular part).  By
  Weyl's inequality and the Gershgorin bound every eigenvalue lies in
  [-1.75, -0.25] or [0.25, 1.75], so mu = 0 sits in a gap and the density
  matrix holds exactly 4 occupied states per molecule.

Random numbers come from counter-based SplitMix64 (``synth.splitmix``): every
matrix entry has a fixed counter, so results do not depend on the order in
which blocks are generated.  This module draws inputs only; it holds none of
the sign method's arithmetic (no block products, filtering or iteration).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import splitmix

R_OH = 0.9572            # A, rigid water O-H bond length (gas-phase value)
THETA_HOH = 104.52       # degrees
MIN_OO = 2.5             # A, minimum O-O distance in the placement
BOX_32 = 9.86            # A, edge of a 32-molecule box at 1 g/cc
R_CUT = 8.0              # A, block present iff r_IJ < R_CUT
DECAY = 0.3              # 1/A^2, entries ~ exp(-DECAY r^2)
DIAG_SHIFT = 2.0         # added to the diagonal of diagonal blocks
N_OCC_PER_MOL = 4        # occupied states per water (8 valence electrons / 2)

# sub-stream tags
_TAG_POS, _TAG_ORI, _TAG_VAL = 1, 2, 3
_TAG_OVERLAP = 4


@dataclasses.dataclass
class BlockMatrix:
    """A square block-sparse matrix in block-CSR form.

    ``blk_size[I]`` is the edge of block row/column I.  Row I holds the blocks
    ``col[row_ptr[I]:row_ptr[I+1]]`` (ascending).  Block b of the CSR order
    has ``blk_size[row(b)] * blk_size[col[b]]`` entries, stored row-major and
    packed one after the other in ``data``.
    """

    blk_size: np.ndarray   # int32 [nblk]
    row_ptr: np.ndarray    # int64 [nblk + 1]
    col: np.ndarray        # int32 [nnzb]
    data: np.ndarray       # float64 [sum of block areas]

    @property
    def nblk(self) -> int:
        return int(self.blk_size.shape[0])

    @property
    def nnzb(self) -> int:
        return int(self.col.shape[0])

    @property
    def n(self) -> int:
        return int(self.blk_size.sum())

    def rows(self) -> np.ndarray:
        return np.repeat(np.arange(self.nblk, dtype=np.int32), np.diff(self.row_ptr))

    def blk_off(self) -> np.ndarray:
        """Offset (in elements) of every block in ``data``."""
        area = self.blk_size[self.rows()].astype(np.int64) * self.blk_size[self.col].astype(np.int64)
        off = np.zeros(self.nnzb + 1, dtype=np.int64)
        np.cumsum(area, out=off[1:])
        return off[:-1]

    def copy(self) -> "BlockMatrix":
        return BlockMatrix(self.blk_size.copy(), self.row_ptr.copy(), self.col.copy(), self.data.copy())


@dataclasses.dataclass
class WaterBox:
    n_mol: int
    box: float                # cubic box edge, A
    pos: np.ndarray           # [3 n_mol, 3] atom positions in [0, box)
    species: np.ndarray       # [3 n_mol] 0 = O, 1 = H

    @property
    def n_atoms(self) -> int:
        return 3 * self.n_mol


def box_edge(n_mol: int) -> float:
    """Edge of a cubic box holding ``n_mol`` waters at 1 g/cc."""
    return BOX_32 * (n_mol / 32.0) ** (1.0 / 3.0)


def _min_image(d: np.ndarray, box: float) -> np.ndarray:
    return d - box * np.round(d / box)


def place_waters(n_mol: int, seed: int, box: float | None = None, max_attempts_per_mol: int = 2000) -> WaterBox:
    """Random sequential addition of rigid waters with min-image O-O >= 2.5 A."""
    box = box_edge(n_mol) if box is None else float(box)
    s_pos = splitmix.substream(seed, _TAG_POS)
    ncell = max(1, int(box // MIN_OO))
    use_cells = ncell >= 3
    cell = box / ncell
    cells: dict[tuple[int, int, int], list[int]] = {}
    opos = np.zeros((n_mol, 3))
    counter = 0
    budget = max_attempts_per_mol * max(n_mol, 1)
    batch = 3 * 4096
    pool = splitmix.uniform01(s_pos, np.arange(batch, dtype=np.uint64))
    pool_base = 0
    min2 = MIN_OO * MIN_OO
    placed = 0
    while placed < n_mol:
        if counter - pool_base + 3 > batch:
            pool_base = counter
            pool = splitmix.uniform01(s_pos, np.arange(pool_base, pool_base + batch, dtype=np.uint64))
        u = pool[counter - pool_base: counter - pool_base + 3]
        counter += 3
        if counter // 3 > budget:
            raise RuntimeError(f"water placement jammed after {budget} attempts ({placed}/{n_mol} placed)")
        p = (u[0] * box, u[1] * box, u[2] * box)
        ok = True
        if use_cells:
            c = (int(p[0] // cell) % ncell, int(p[1] // cell) % ncell, int(p[2] // cell) % ncell)
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        key = ((c[0] + dx) % ncell, (c[1] + dy) % ncell, (c[2] + dz) % ncell)
                        for q in cells.get(key, ()):
                            d2 = 0.0
                            for ax in range(3):
                                d = p[ax] - opos[q, ax]
                                d -= box * round(d / box)
                                d2 += d * d
                            if d2 < min2:
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
        else:
            if placed:
                d = _min_image(opos[:placed] - np.array(p), box)
                ok = bool(np.all((d * d).sum(axis=1) >= min2))
        if not ok:
            continue
        opos[placed] = p
        if use_cells:
            cells.setdefault(c, []).append(placed)
        placed += 1

    # orientations: Shoemake's uniform random unit quaternion from 3 uniforms
    s_ori = splitmix.substream(seed, _TAG_ORI)
    u = splitmix.uniform01(s_ori, np.arange(3 * n_mol, dtype=np.uint64)).reshape(n_mol, 3)
    a, b = np.sqrt(1.0 - u[:, 0]), np.sqrt(u[:, 0])
    qx, qy = a * np.sin(2 * np.pi * u[:, 1]), a * np.cos(2 * np.pi * u[:, 1])
    qz, qw = b * np.sin(2 * np.pi * u[:, 2]), b * np.cos(2 * np.pi * u[:, 2])
    rot = np.empty((n_mol, 3, 3))
    rot[:, 0, 0] = 1 - 2 * (qy * qy + qz * qz)
    rot[:, 0, 1] = 2 * (qx * qy - qz * qw)
    rot[:, 0, 2] = 2 * (qx * qz + qy * qw)
    rot[:, 1, 0] = 2 * (qx * qy + qz * qw)
    rot[:, 1, 1] = 1 - 2 * (qx * qx + qz * qz)
    rot[:, 1, 2] = 2 * (qy * qz - qx * qw)
    rot[:, 2, 0] = 2 * (qx * qz - qy * qw)
    rot[:, 2, 1] = 2 * (qy * qz + qx * qw)
    rot[:, 2, 2] = 1 - 2 * (qx * qx + qy * qy)
    half = math.radians(THETA_HOH) / 2
    frame = np.array([[0.0, 0.0, 0.0],
                      [R_OH * math.sin(half), R_OH * math.cos(half), 0.0],
                      [-R_OH * math.sin(half), R_OH * math.cos(half), 0.0]])
    atoms = opos[:, None, :] + np.einsum("mij,aj->mai", rot, frame)
    pos = np.mod(atoms.reshape(-1, 3), box)
    species = np.tile(np.array([0, 1, 1], dtype=np.int8), n_mol)
    return WaterBox(n_mol=n_mol, box=box, pos=pos, species=species)


def neighbour_pairs(wb: WaterBox, rcut: float = R_CUT):
    """All atom pairs I <= J with minimum-image distance r_IJ < rcut, sorted by (I, J).

    Returns (I, J, r) as int32, int32, float64 arrays (I == J pairs have r = 0).
    """
    pos, box, n = wb.pos, wb.box, wb.n_atoms
    if box > 2.0 * rcut + 1.0:
        from scipy.spatial import cKDTree
        tree = cKDTree(pos, boxsize=box)
        pr = tree.query_pairs(rcut, output_type="ndarray").astype(np.int64)
        i, j = np.minimum(pr[:, 0], pr[:, 1]), np.maximum(pr[:, 0], pr[:, 1])
    else:
        ii, jj = np.triu_indices(n, k=1)
        i, j = ii.astype(np.int64), jj.astype(np.int64)
    d = _min_image(pos[i] - pos[j], box)
    r = np.sqrt((d * d).sum(axis=1))
    keep = r < rcut
    i, j, r = i[keep], j[keep], r[keep]
    diag = np.arange(n, dtype=np.int64)
    i = np.concatenate([i, diag])
    j = np.concatenate([j, diag])
    r = np.concatenate([r, np.zeros(n)])
    order = np.lexsort((j, i))
    return i[order].astype(np.int32), j[order].astype(np.int32), r[order]


def atom_block_sizes(wb: WaterBox, basis: tuple[int, int]) -> np.ndarray:
    b_o, b_h = basis
    return np.where(wb.species == 0, b_o, b_h).astype(np.int32)


def _csr_from_upper(nblk: int, ui: np.ndarray, uj: np.ndarray):
    """CSR layout of the symmetric pattern given by upper pairs (ui <= uj).

    Returns row_ptr, col, and for every upper pair the CSR index of block (i, j)
    and of its mirror (j, i) (equal for diagonal pairs).
    """
    nup = ui.shape[0]
    off = ui != uj
    rows = np.concatenate([ui, uj[off]]).astype(np.int64)
    cols = np.concatenate([uj, ui[off]]).astype(np.int64)
    src = np.concatenate([np.arange(nup), np.nonzero(off)[0]])
    mirror = np.concatenate([np.zeros(nup, bool), np.ones(int(off.sum()), bool)])
    order = np.lexsort((cols, rows))
    csr_pos = np.empty_like(order)
    csr_pos[order] = np.arange(order.shape[0])
    pos_up = np.empty(nup, dtype=np.int64)
    pos_lo = np.empty(nup, dtype=np.int64)
    pos_up[src[~mirror]] = csr_pos[~mirror]
    pos_lo[:] = pos_up
    pos_lo[src[mirror]] = csr_pos[mirror]
    counts = np.bincount(rows, minlength=nblk)
    row_ptr = np.zeros(nblk + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, cols[order].astype(np.int32), pos_up, pos_lo


def _chunks(idx: np.ndarray, area: int):
    step = max(1, (1 << 24) // max(area, 1))
    for s in range(0, idx.shape[0], step):
        yield idx[s:s + step]


def decay_matrix(wb: WaterBox, basis: tuple[int, int], seed: int,
                 rcut: float = R_CUT, decay: float = DECAY, shift: float = DIAG_SHIFT):
    """The decay-construction matrix on a water box (see module docstring).

    Random stream: the upper blocks (I <= J) taken in (I, J) order, each
    contributing its m*n entries row-major, draw consecutive counters of the
    value sub-stream of ``seed``.

    Returns (BlockMatrix, (ui, uj, r, pos_up, pos_lo)) where the tuple describes
    every upper pair and the CSR index of it and of its mirror.
    """
    bs = atom_block_sizes(wb, basis)
    ui, uj, r = neighbour_pairs(wb, rcut)
    row_ptr, col, pos_up, pos_lo = _csr_from_upper(bs.shape[0], ui, uj)
    m = BlockMatrix(bs, row_ptr, col, np.empty(0))
    boff = m.blk_off()
    area_csr = bs[m.rows()].astype(np.int64) * bs[col].astype(np.int64)
    data = np.empty(int(area_csr.sum()), dtype=np.float64)
    m.data = data

    uarea = bs[ui].astype(np.int64) * bs[uj].astype(np.int64)
    ustart = np.zeros(ui.shape[0], dtype=np.int64)
    np.cumsum(uarea[:-1], out=ustart[1:])
    s_val = splitmix.substream(seed, _TAG_VAL)
    nnzb = col.shape[0]
    rows = m.rows()
    # source upper pair of every CSR block and whether the block is its mirror
    src = np.empty(nnzb, dtype=np.int64)
    src[pos_up] = np.arange(ui.shape[0])
    mirror = np.zeros(nnzb, dtype=bool)
    offd = ui != uj
    src[pos_lo[offd]] = np.nonzero(offd)[0]
    mirror[pos_lo[offd]] = True
    fac_blk = np.exp(-decay * r * r)[src]
    mb = bs[rows].astype(np.int64)
    nb = bs[col].astype(np.int64)
    # walk the output in CSR order, a chunk of whole blocks at a time: element
    # (a, c) of block b draws counter ustart[src] + a*nb + c, or, for a mirrored
    # block, the counter of element (c, a) of its source: ustart[src] + c*mb + a
    chunk = 1 << 20
    b0 = 0
    while b0 < nnzb:
        b1 = int(np.searchsorted(boff, boff[b0] + chunk, side="right"))
        b1 = max(b1, b0 + 1)
        b1 = min(b1, nnzb)
        e0, e1 = int(boff[b0]), int(boff[b1 - 1] + area_csr[b1 - 1])
        cnt_b = area_csr[b0:b1]
        blk = np.repeat(np.arange(b0, b1), cnt_b)
        local = np.arange(e1 - e0, dtype=np.int64) - np.repeat(boff[b0:b1] - e0, cnt_b)
        nbe = nb[blk]
        a_ = local // nbe
        c_ = local - a_ * nbe
        ctr = ustart[src[blk]] + np.where(mirror[blk], c_ * mb[blk] + a_, local)
        data[e0:e1] = splitmix.uniform_pm1(s_val, ctr.astype(np.uint64)) * fac_blk[blk]
        b0 = b1
    # diagonal blocks: (U + U^T) / 2 + shift * 1 (U drawn as above, exp(0) = 1)
    dg = np.nonzero(rows == col)[0]
    for bm_ in np.unique(bs):
        sel = dg[bs[rows[dg]] == bm_]
        if sel.size == 0:
            continue
        area = int(bm_) * int(bm_)
        idx = boff[sel][:, None] + np.arange(area, dtype=np.int64)[None, :]
        u = data[idx].reshape(-1, bm_, bm_)
        d = 0.5 * (u + np.transpose(u, (0, 2, 1))) + shift * np.eye(bm_)[None, :, :]
        data[idx] = d.reshape(-1, area)
    return m, (ui, uj, r, pos_up, pos_lo)


def _abs_row_sums(A: BlockMatrix, select: np.ndarray) -> np.ndarray:
    """Sum over the selected blocks of |entries| along every matrix row."""
    bs = A.blk_size
    rows = A.rows()
    boff = A.blk_off()
    roff = np.zeros(bs.shape[0] + 1, dtype=np.int64)
    np.cumsum(bs, out=roff[1:])
    rowsum = np.zeros(A.n)
    for bm in np.unique(bs):
        for bn in np.unique(bs):
            sel = np.nonzero(select & (bs[rows] == bm) & (bs[A.col] == bn))[0]
            area = int(bm) * int(bn)
            ar = np.arange(area, dtype=np.int64)
            for ch in _chunks(sel, area):
                v = np.abs(A.data[boff[ch][:, None] + ar[None, :]]).reshape(-1, bm, bn).sum(axis=2)
                tgt = roff[rows[ch]][:, None] + np.arange(bm)[None, :]
                np.add.at(rowsum, tgt.ravel(), v.ravel())
    return rowsum


def overlap_matrix(wb: WaterBox, basis: tuple[int, int], seed: int, spread: float = 0.9) -> BlockMatrix:
    """Synthetic overlap S = 1 + sigma |D| on the decay pattern (see module docstring):
    eigenvalues in [1 - spread, 1 + spread]."""
    D, _ = decay_matrix(wb, basis, splitmix.substream(seed, _TAG_OVERLAP), shift=0.0)
    rowsum = _abs_row_sums(D, np.ones(D.col.shape[0], dtype=bool))
    sigma = spread / float(rowsum.max())
    data = np.abs(D.data) * sigma
    rows = D.rows()
    boff = D.blk_off()
    for b in np.nonzero(rows == D.col)[0]:
        m = int(D.blk_size[rows[b]])
        data[boff[b]:boff[b] + m * m:m + 1] += 1.0
    return BlockMatrix(D.blk_size, D.row_ptr, D.col, data)


@dataclasses.dataclass
class Hamiltonian:
    H: BlockMatrix
    gamma: float            # scale applied to the inter-molecular decay blocks
    n_occ: int              # occupied states = 4 per molecule
    n_mol: int
    n_atoms: int
    mu: float = 0.0         # mid-gap chemical potential


def gapped_hamiltonian(wb: WaterBox, basis: tuple[int, int], seed: int) -> Hamiltonian:
    """Gapped synthetic Kohn-Sham stand-in on a water box (see module docstring)."""
    A, (ui, uj, r, pos_up, pos_lo) = decay_matrix(wb, basis, seed)
    bs = A.blk_size
    b_o, b_h = basis
    d = b_o + 2 * b_h
    n_mol = wb.n_mol
    rows = A.rows()
    boff = A.blk_off()
    roff = np.zeros(bs.shape[0] + 1, dtype=np.int64)
    np.cumsum(bs, out=roff[1:])
    mol_r = rows // 3
    mol_c = A.col // 3
    intra = mol_r == mol_c

    # gamma: inverse of the largest absolute row sum of the inter-molecular part
    rowsum = np.zeros(A.n)
    for bm in np.unique(bs):
        for bn in np.unique(bs):
            sel = np.nonzero((~intra) & (bs[rows] == bm) & (bs[A.col] == bn))[0]
            area = int(bm) * int(bn)
            ar = np.arange(area, dtype=np.int64)
            for ch in _chunks(sel, area):
                v = np.abs(A.data[boff[ch][:, None] + ar[None, :]]).reshape(-1, bm, bn).sum(axis=2)
                tgt = roff[rows[ch]][:, None] + np.arange(bm)[None, :]
                np.add.at(rowsum, tgt.ravel(), v.ravel())
    gmax = float(rowsum.max()) if rowsum.size else 0.0
    gamma = 0.5 / gmax if gmax > 0 else 0.0

    # intra-molecular dense parts -> spectrum replaced
    loc = np.array([0, b_o, b_o + b_h, d])
    Hm = np.zeros((n_mol, d, d))
    isel = np.nonzero(intra)[0]
    ai = rows[isel] % 3
    aj = A.col[isel] % 3
    mol = mol_r[isel]
    for a in range(3):
        for b in range(3):
            s = isel[(ai == a) & (aj == b)]
            bm, bn = loc[a + 1] - loc[a], loc[b + 1] - loc[b]
            ar = np.arange(bm * bn, dtype=np.int64)
            blocks = A.data[boff[s][:, None] + ar[None, :]].reshape(-1, bm, bn)
            Hm[mol[(ai == a) & (aj == b)], loc[a]:loc[a + 1], loc[b]:loc[b + 1]] = blocks
    Hm = 0.5 * (Hm + np.transpose(Hm, (0, 2, 1)))
    _, Q = np.linalg.eigh(Hm)
    target = np.concatenate([-1.0 + 0.25 * np.linspace(-1.0, 1.0, N_OCC_PER_MOL),
                             1.0 + 0.25 * np.linspace(-1.0, 1.0, d - N_OCC_PER_MOL)])
    Hn = np.einsum("mij,j,mkj->mik", Q, target, Q)
    Hn = 0.5 * (Hn + np.transpose(Hn, (0, 2, 1)))

    data = A.data * gamma
    for a in range(3):
        for b in range(3):
            sel = (ai == a) & (aj == b)
            s = isel[sel]
            bm, bn = loc[a + 1] - loc[a], loc[b + 1] - loc[b]
            ar = np.arange(bm * bn, dtype=np.int64)
            data[boff[s][:, None] + ar[None, :]] = Hn[mol[sel], loc[a]:loc[a + 1], loc[b]:loc[b + 1]].reshape(-1, bm * bn)
    H = BlockMatrix(bs, A.row_ptr, A.col, data)
    return Hamiltonian(H=H, gamma=gamma, n_occ=N_OCC_PER_MOL * n_mol, n_mol=n_mol, n_atoms=wb.n_atoms)

