"""Test matrices as FP64 CSR (oracle side).

CSR convention: ``rowptr`` int64 (D+1), ``col`` int32, ``val`` float64, the
columns of every row strictly ascending, the diagonal entry always stored
(value 0 where the matrix has none), so ``nnz`` counts the pattern including
the diagonal.

Hubbard matrix (Sec. 3.2 and Sec. 4.1: D = C(n_sites, n_fermions)^2 for equal
spin populations; Table 2 lists its row lengths).  Reading of the basis, which
the paper leaves to ScaMaC: per spin, occupation bitstrings over the sites
(bit i = site i) with the fixed particle number, ranked in increasing integer
order; row index = rank_up * dim_dn + rank_dn; creation operators ordered all
spin-up before all spin-down, sites ascending.  Then a hop c^+_{i s} c_{j s}
carries the sign (-1)^(number of spin-s fermions strictly between i and j),
the spin-up fermions passed by a spin-down hop cancel in pairs, and

    H = -t sum_<ij>,s (c^+_is c_js + h.c.) + U sum_i n_i,up n_i,dn .

Bonds: (i, i+1) for open boundaries, plus (0, L-1) for periodic ones (L >= 3).

3D Anderson model (stand-in for the narrow-band stencil matrices of Sec. 3.2):
cubic L^3 lattice, row i = x + L (y + L z), periodic, hopping -t to the six
neighbours and on-site energy eps_i = W (u_i - 1/2) from the disorder stream.
"""
from math import comb

import numpy as np

from . import splitmix


def _csr_from_coo(D, rows, cols, vals):
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    if len(rows) > 1:
        dup = (rows[1:] == rows[:-1]) & (cols[1:] == cols[:-1])
        if dup.any():
            raise ValueError("duplicate entries in generated matrix")
    counts = np.bincount(rows, minlength=D)
    rowptr = np.zeros(D + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return rowptr, cols.astype(np.int32), vals.astype(np.float64)


# --------------------------------------------------------------------------
# Hubbard
# --------------------------------------------------------------------------

def spin_basis(n_sites, n_part):
    """All bitstrings over n_sites with n_part bits set, ascending."""
    allc = np.arange(1 << n_sites, dtype=np.int64)
    pop = np.zeros_like(allc)
    for b in range(n_sites):
        pop += (allc >> b) & 1
    return allc[pop == n_part]


def _popcount(a):
    a = np.asarray(a, dtype=np.int64)
    c = np.zeros_like(a)
    for b in range(20):
        c += (a >> b) & 1
    return c


def hubbard_bonds(n_sites, bc):
    bonds = [(i, i + 1) for i in range(n_sites - 1)]
    if bc == "periodic":
        if n_sites < 3:
            raise ValueError("periodic Hubbard chain needs n_sites >= 3")
        bonds.append((0, n_sites - 1))
    elif bc != "open":
        raise ValueError("bc must be 'open' or 'periodic'")
    return bonds


def hubbard_dim(n_sites, n_up, n_dn):
    return comb(n_sites, n_up) * comb(n_sites, n_dn)


def _hubbard_entries(n_sites, n_up, n_dn, t, U, bc, rows):
    """COO entries (row, col, val) of the given rows of the Hubbard matrix."""
    bu, bd = spin_basis(n_sites, n_up), spin_basis(n_sites, n_dn)
    dim_dn = len(bd)
    rank_u = -np.ones(1 << n_sites, dtype=np.int64)
    rank_u[bu] = np.arange(len(bu))
    rank_d = -np.ones(1 << n_sites, dtype=np.int64)
    rank_d[bd] = np.arange(len(bd))
    rows = np.asarray(rows, dtype=np.int64)
    ru, rd = rows // dim_dn, rows % dim_dn
    su, sd = bu[ru], bd[rd]
    R, C, Vv = [rows], [rows], [U * _popcount(su & sd).astype(np.float64)]
    for (i, j) in hubbard_bonds(n_sites, bc):
        between = ((1 << j) - 1) ^ ((1 << (i + 1)) - 1)   # sites i < s < j
        flip = (1 << i) | (1 << j)
        for spin in (0, 1):
            s = su if spin == 0 else sd
            can = (((s >> i) & 1) ^ ((s >> j) & 1)) == 1
            s2 = s[can] ^ flip
            sign = 1.0 - 2.0 * (_popcount(s[can] & between) & 1)
            if spin == 0:
                col = rank_u[s2] * dim_dn + rd[can]
            else:
                col = ru[can] * dim_dn + rank_d[s2]
            R.append(rows[can]); C.append(col); Vv.append(-t * sign)
    return np.concatenate(R), np.concatenate(C), np.concatenate(Vv)


def hubbard(n_sites, n_up, n_dn, t=1.0, U=4.0, bc="open"):
    D = hubbard_dim(n_sites, n_up, n_dn)
    r, c, v = _hubbard_entries(n_sites, n_up, n_dn, t, U, bc, np.arange(D))
    return _csr_from_coo(D, r, c, v)


def hubbard_rows(n_sites, n_up, n_dn, t, U, bc, rows):
    """Sorted (col, val) of each requested row, for sampled checks at full size."""
    out = []
    for row in np.asarray(rows, dtype=np.int64):
        r, c, v = _hubbard_entries(n_sites, n_up, n_dn, t, U, bc, [row])
        o = np.argsort(c)
        out.append((c[o].astype(np.int32), v[o]))
    return out


# --------------------------------------------------------------------------
# 3D Anderson model, tight-binding chain, diagonal
# --------------------------------------------------------------------------

def anderson_disorder(L, W, seed):
    D = L ** 3
    u = splitmix.uniform(seed, splitmix.STREAM_DISORDER, np.arange(D))
    return W * (u - 0.5)


def _anderson_cols(L, rows):
    x = rows % L
    y = (rows // L) % L
    z = rows // (L * L)
    def idx(xx, yy, zz):
        return xx + L * (yy + L * zz)
    return np.stack([rows,
                     idx((x + 1) % L, y, z), idx((x - 1) % L, y, z),
                     idx(x, (y + 1) % L, z), idx(x, (y - 1) % L, z),
                     idx(x, y, (z + 1) % L), idx(x, y, (z - 1) % L)], axis=1)


def anderson3d(L, W, seed, t=1.0):
    if L < 3:
        raise ValueError("the periodic 7-point stencil needs L >= 3")
    D = L ** 3
    rows = np.arange(D, dtype=np.int64)
    cols = _anderson_cols(L, rows)
    vals = np.full(cols.shape, -t, dtype=np.float64)
    vals[:, 0] = anderson_disorder(L, W, seed)
    order = np.argsort(cols, axis=1, kind="stable")
    cols = np.take_along_axis(cols, order, axis=1)
    vals = np.take_along_axis(vals, order, axis=1)
    rowptr = np.arange(0, 7 * D + 1, 7, dtype=np.int64)
    return rowptr, cols.reshape(-1).astype(np.int32), vals.reshape(-1)


def anderson_rows(L, W, seed, t, rows):
    rows = np.asarray(rows, dtype=np.int64)
    cols = _anderson_cols(L, rows)
    eps = W * (splitmix.uniform(seed, splitmix.STREAM_DISORDER, rows) - 0.5)
    out = []
    for k in range(len(rows)):
        v = np.full(7, -t)
        v[0] = eps[k]
        o = np.argsort(cols[k], kind="stable")
        out.append((cols[k][o].astype(np.int32), v[o]))
    return out


def anderson_instance(s):
    """Size and disorder of batched instance s: L in 16..48, W in [2, 16]."""
    uL = splitmix.uniform(s, splitmix.STREAM_INST_L, [0])[0]
    uW = splitmix.uniform(s, splitmix.STREAM_INST_W, [0])[0]
    return 16 + int(np.floor(33.0 * uL)), 2.0 + 14.0 * uW


def roadgraph(side, q=0.3, seed=0):
    """Road-like planar graph Laplacian L = D_g - A on a side x side grid.

    Node i = x + side*y.  A random spanning tree: every node except (0, 0)
    keeps one edge to a parent that precedes it -- row 0 links left; column 0
    links down; elsewhere left if u < 1/2 else down (u from stream 7, counter
    i).  Every other grid edge (the left and the down edge of node i) is added
    with probability q (stream 8, counters 2i and 2i+1), so the mean degree is
    about 2 (1 + q): connected, planar, irregular.
    """
    N = side * side
    i = np.arange(N, dtype=np.int64)
    x, y = i % side, i // side
    u_par = splitmix.uniform(seed, splitmix.STREAM_ROAD_TREE, i)
    par_left = (y == 0) & (x > 0) | (y > 0) & (x > 0) & (u_par < 0.5)
    par_down = (y > 0) & ((x == 0) | (u_par >= 0.5))
    u_l = splitmix.uniform(seed, splitmix.STREAM_ROAD_EXTRA, 2 * i)
    u_d = splitmix.uniform(seed, splitmix.STREAM_ROAD_EXTRA, 2 * i + 1)
    left = par_left | ((x > 0) & ~par_left & (u_l < q))
    down = par_down | ((y > 0) & ~par_down & (u_d < q))
    a = np.concatenate([i[left], i[down]])
    b = np.concatenate([i[left] - 1, i[down] - side])
    deg = np.bincount(a, minlength=N) + np.bincount(b, minlength=N)
    rows = np.concatenate([a, b, i])
    cols = np.concatenate([b, a, i])
    vals = np.concatenate([-np.ones(len(a)), -np.ones(len(a)), deg.astype(np.float64)])
    return _csr_from_coo(N, rows, cols, vals)


def chain(n, t=1.0):
    """Open tight-binding chain: -t on the first off-diagonals, 0 diagonal."""
    rows, cols, vals = [np.arange(n)], [np.arange(n)], [np.zeros(n)]
    i = np.arange(n - 1)
    rows += [i, i + 1]; cols += [i + 1, i]; vals += [np.full(n - 1, -t)] * 2
    return _csr_from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def diagonal(values):
    values = np.asarray(values, dtype=np.float64)
    n = len(values)
    return np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), values.copy()


# --------------------------------------------------------------------------
# spec strings ("hubbard:n_sites=8,n_up=4,n_dn=4,t=1,U=4,bc=open")
# --------------------------------------------------------------------------

def parse_spec(spec):
    kind, _, rest = spec.partition(":")
    kv = {}
    for item in filter(None, rest.split(",")):
        k, _, v = item.partition("=")
        kv[k.strip()] = v.strip()
    return kind.strip(), kv


def build(spec):
    kind, kv = parse_spec(spec)
    if kind == "hubbard":
        return hubbard(int(kv["n_sites"]), int(kv["n_up"]), int(kv["n_dn"]),
                       float(kv.get("t", 1)), float(kv.get("U", 4)), kv.get("bc", "open"))
    if kind == "anderson3d":
        return anderson3d(int(kv["L"]), float(kv.get("W", 0)), int(kv.get("seed", 0)),
                          float(kv.get("t", 1)))
    if kind == "chain":
        return chain(int(kv["n"]), float(kv.get("t", 1)))
    if kind == "roadgraph":
        return roadgraph(int(kv["side"]), float(kv.get("q", 0.3)), int(kv.get("seed", 0)))
    raise ValueError(f"unknown matrix kind {kind!r}")


def to_scipy(csr):
    import scipy.sparse as sp
    rowptr, col, val = csr
    D = len(rowptr) - 1
    return sp.csr_matrix((val, col, rowptr), shape=(D, D))
