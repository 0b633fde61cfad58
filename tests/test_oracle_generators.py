"""Pins of the oracle's RNG and matrix generators (no GPU)."""
import os
from math import comb

import numpy as np
import pytest

from oracle import matrices as mat
from oracle import splitmix

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix_published_sequence():
    vals = [int(l, 16) for l in open(os.path.join(GOLD, "splitmix64.txt")) if l.startswith("0x")]
    got = [int(splitmix.mix64(np.uint64((k + 1) * 0x9E3779B97F4A7C15 % 2**64))) for k in range(3)]
    assert got == vals


def test_uniform_and_irwin_hall_moments():
    u = splitmix.uniform(7, splitmix.STREAM_DISORDER, np.arange(200000))
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1 / 12) < 0.002
    g = splitmix.irwin_hall(3, splitmix.STREAM_START, np.arange(100000))
    assert abs(g.mean()) < 0.02 and abs(g.var() - 1.0) < 0.02
    # streams and seeds decorrelate
    a = splitmix.uniform(1, 1, np.arange(1000)); b = splitmix.uniform(1, 2, np.arange(1000))
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.1


def test_hubbard_dimension_and_symmetry():
    for L, nu, nd in [(6, 3, 3), (8, 4, 4), (7, 2, 3)]:
        rp, c, v = mat.hubbard(L, nu, nd, 1.0, 4.0, "open")
        assert len(rp) - 1 == comb(L, nu) * comb(L, nd)
        A = mat.to_scipy((rp, c, v))
        assert abs(A - A.T).max() == 0.0
        assert all(np.all(np.diff(c[rp[i]:rp[i + 1]]) > 0) for i in range(0, len(rp) - 1, 37))


def test_hubbard_config1_counts():
    # 8-site chain, 4+4, open: D = C(8,4)^2 = 4900, 8 off-diagonal entries per row on average,
    # trace = U * D * N_up * N_dn / L.
    rp, c, v = mat.hubbard(8, 4, 4, 1.0, 4.0, "open")
    D = len(rp) - 1
    assert D == 4900
    row = np.repeat(np.arange(D), np.diff(rp))
    assert (c != row).sum() / D == pytest.approx(8.0, abs=1e-12)
    assert v[c == row].sum() == pytest.approx(4.0 * D * 16 / 8)


def _sector_hops(L, N, bc):
    """Mean number of hops per row for each spin sector, counted on generated rows."""
    dim = comb(L, N)
    rows_up = np.arange(dim) * dim               # vary the up configuration, dn fixed
    rows_dn = np.arange(dim)                     # vary the dn configuration, up fixed
    up = [np.sum(c // dim != r // dim) for r, (c, _) in zip(rows_up, mat.hubbard_rows(L, N, N, 1, 0, bc, rows_up))]
    dn = [np.sum(c % dim != r % dim) for r, (c, _) in zip(rows_dn, mat.hubbard_rows(L, N, N, 1, 0, bc, rows_dn))]
    return np.mean(up) + np.mean(dn)


def test_hubbard_table2_nnz_per_row():
    # Table 2 prints D and n_nzr for Hubbard14 / Hubbard16 (open chain, half filling).
    for line in open(os.path.join(GOLD, "table2_hubbard.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, L, nu, nd, D, nnzr = line.split()
        L, nu, nd, D = int(L), int(nu), int(nd), int(D)
        assert mat.hubbard_dim(L, nu, nd) == D
        if L <= 14:                              # 16 sites: 12870 rows per sector, still cheap
            assert round(_sector_hops(L, nu, "open"), 2) == float(nnzr)


def _levels(L, bc, N):
    k = np.arange(L)
    if bc == "open":
        return np.sort(-2.0 * np.cos((k + 1) * np.pi / (L + 1)))
    # With the fermion sign (-1)^(N-1) on the ring-closing hop the operator is the
    # plain periodic one, so the single-particle levels are periodic for every N;
    # dropping the sign would give antiperiodic levels for even N.
    return np.sort(-2.0 * np.cos(2 * np.pi * k / L))


def _free_fermion_spectrum(L, nu, nd, bc):
    from itertools import combinations
    eu, ed = _levels(L, bc, nu), _levels(L, bc, nd)
    su = [sum(eu[list(s)]) for s in combinations(range(L), nu)]
    sd = [sum(ed[list(s)]) for s in combinations(range(L), nd)]
    return np.sort(np.add.outer(su, sd).ravel())


@pytest.mark.parametrize("L,nu,nd,bc", [(6, 3, 3, "open"), (6, 2, 2, "periodic"),
                                         (6, 3, 3, "periodic"), (5, 2, 3, "periodic")])
def test_hubbard_U0_is_free_fermions(L, nu, nd, bc):
    A = mat.to_scipy(mat.hubbard(L, nu, nd, 1.0, 0.0, bc)).toarray()
    ev = np.linalg.eigvalsh(A)
    assert np.abs(ev - _free_fermion_spectrum(L, nu, nd, bc)).max() < 1e-12


def test_hubbard_t0_counts_double_occupancy():
    A = mat.to_scipy(mat.hubbard(5, 2, 3, 0.0, 3.0, "open")).toarray()
    assert np.count_nonzero(A - np.diag(np.diag(A))) == 0
    vals, counts = np.unique(np.diag(A), return_counts=True)
    # double occupancies d: C(5,d) C(5-d, 2-d) C(5-2+d... brute force over configurations
    from itertools import combinations
    exp = {}
    for su in combinations(range(5), 2):
        for sd in combinations(range(5), 3):
            d = len(set(su) & set(sd))
            exp[3.0 * d] = exp.get(3.0 * d, 0) + 1
    assert dict(zip(vals, counts)) == exp


def test_hubbard_half_filling_particle_hole_symmetry():
    L, U = 6, 4.0
    ev = np.linalg.eigvalsh(mat.to_scipy(mat.hubbard(L, 3, 3, 1.0, U, "open")).toarray())
    assert np.abs(ev + ev[::-1] - U * L / 2).max() < 1e-11


def test_anderson_clean_lattice_and_disorder():
    L = 5
    A = mat.to_scipy(mat.anderson3d(L, 0.0, 0)).toarray()
    k = 2 * np.pi * np.arange(L) / L
    e = -2 * (np.cos(k)[:, None, None] + np.cos(k)[None, :, None] + np.cos(k)[None, None, :])
    assert np.abs(np.linalg.eigvalsh(A) - np.sort(e.ravel())).max() < 1e-12
    rp, c, v = mat.anderson3d(4, 2.0, 1)
    row = np.repeat(np.arange(64), 7)
    eps = v[c == row]
    u = splitmix.uniform(1, splitmix.STREAM_DISORDER, np.arange(64))
    assert np.array_equal(eps, 2.0 * (u - 0.5))
    assert eps.min() >= -1.0 and eps.max() < 1.0
    assert np.all(v[c != row] == -1.0)
    A = mat.to_scipy((rp, c, v))
    assert abs(A - A.T).max() == 0.0


def test_anderson_rows_match_full():
    rp, c, v = mat.anderson3d(6, 3.0, 5)
    rows = [0, 5, 77, 215]
    for r, (cc, vv) in zip(rows, mat.anderson_rows(6, 3.0, 5, 1.0, rows)):
        assert np.array_equal(cc, c[rp[r]:rp[r + 1]]) and np.array_equal(vv, v[rp[r]:rp[r + 1]])


def test_chain_spectrum():
    n = 50
    ev = np.linalg.eigvalsh(mat.to_scipy(mat.chain(n)).toarray())
    assert np.abs(ev - np.sort(-2 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1)))).max() < 1e-13


def test_anderson_instances_in_range():
    Ls, Ws = zip(*[mat.anderson_instance(s) for s in range(64)])
    assert min(Ls) >= 16 and max(Ls) <= 48 and min(Ws) >= 2 and max(Ws) <= 16
    assert len(set(Ls)) > 10


def test_roadgraph_is_a_connected_planar_laplacian():
    import scipy.sparse.csgraph as csg
    side, q = 40, 0.3
    rp, c, v = mat.roadgraph(side, q, 5)
    N = side * side
    A = mat.to_scipy((rp, c, v))
    assert abs(A - A.T).max() == 0.0
    assert np.abs(np.asarray(A.sum(axis=1))).max() == 0.0          # Laplacian rows sum to zero
    off = A.copy(); off.setdiag(0); off.eliminate_zeros()
    i, j = off.nonzero()
    d = np.abs(i - j)
    assert np.all((d == 1) | (d == side))                           # grid edges only
    assert np.all((d != 1) | (np.minimum(i, j) % side != side - 1))  # no wrap-around
    assert csg.connected_components(off)[0] == 1
    n_edges = off.nnz // 2
    tree_extra = n_edges - (N - 1)
    other = 2 * side * (side - 1) - (N - 1)
    assert abs(tree_extra / other - q) < 0.05                        # extra edges with probability q
    ev = np.linalg.eigvalsh(A.toarray())
    assert abs(ev[0]) < 1e-10 and ev[1] > 1e-6                       # one zero mode: connected
    assert ev[-1] <= 8.0 + 1e-12                                     # Gershgorin: 2 * max degree


def test_instance_sizes_agree_with_input_generator():
    import fd_inputs
    for s in range(64):
        assert fd_inputs.anderson_instance(s) == mat.anderson_instance(s)


@pytest.mark.parametrize("L,nu,nd,bc", [(6, 3, 3, "open"), (7, 3, 2, "periodic"), (8, 4, 1, "periodic"),
                                        (5, 0, 2, "open"), (6, 2, 0, "periodic")])
def test_hubbard_is_a_kronecker_sum(L, nu, nd, bc):
    # with all up operators ordered before all down ones, a hop of either spin
    # passes only fermions of its own spin, so the matrix factorises as
    # H = H_up x 1 + 1 x H_dn + U n_double in the row order rank_up * dim_dn + rank_dn
    import scipy.sparse as sp
    t, U = 1.3, 4.2
    h_up = mat.to_scipy(mat.hubbard(L, nu, 0, t, 0.0, bc))
    h_dn = mat.to_scipy(mat.hubbard(L, nd, 0, t, 0.0, bc))
    bu, bd = mat.spin_basis(L, nu), mat.spin_basis(L, nd)
    n_double = np.array([bin(int(a) & int(b)).count("1") for a in bu for b in bd], dtype=np.float64)
    K = sp.kron(h_up, sp.identity(len(bd))) + sp.kron(sp.identity(len(bu)), h_dn) + sp.diags(U * n_double)
    H = mat.to_scipy(mat.hubbard(L, nu, nd, t, U, bc))
    assert H.shape == K.shape
    assert abs(H - K).max() == 0.0
