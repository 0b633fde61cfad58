"""Pins of the oracle's communication metrics (Sec. 3.1): closed forms for the
chain and the periodic stencil, brute force on small random patterns, and the
paper's own Table 7 for the 24-site spin chain."""
import os

import numpy as np
import pytest

import fd_inputs
from oracle import comm
from oracle import matrices as mat

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _brute(csr, n_p):
    rowptr, col, val = csr
    D = len(rowptr) - 1
    out_vc, out_vm = [], []
    for p in range(n_p):
        a, b = p * D // n_p, (p + 1) * D // n_p
        seen = set()
        for i in range(a, b):
            for k in range(rowptr[i], rowptr[i + 1]):
                if val[k] != 0:
                    seen.add(int(col[k]))
        out_vm.append(sum(1 for j in seen if a <= j < b))
        out_vc.append(sum(1 for j in seen if not a <= j < b))
    return np.array(out_vc), np.array(out_vm)


@pytest.mark.parametrize("n,n_p", [(100, 2), (101, 3), (1000, 7), (64, 8)])
def test_chain_closed_form(n, n_p):
    # rows [a, b) of an open chain read a - 1 and b from other processes and every
    # own entry (each row's neighbour inside the range); the zero diagonal is no access
    csr = mat.chain(n)
    n_vc, n_vm = comm.counts(csr, n_p)
    a, b = comm.uniform_ranges(n, n_p)
    assert list(n_vc) == [(1 if p > 0 else 0) + (1 if p < n_p - 1 else 0) for p in range(n_p)]
    assert list(n_vm) == list(b - a)
    chi1, chi2, chi3, _, _ = comm.metrics(csr, n_p)
    assert chi2 == pytest.approx(2 * (n_p - 1) / n)
    assert chi3 == pytest.approx(n_p * (2 if n_p > 2 else 1) / n)
    assert chi1 == pytest.approx(max(n_vc / (b - a)))


@pytest.mark.parametrize("L,n_p", [(8, 2), (8, 4), (12, 3), (12, 6)])
def test_periodic_stencil_slabs(L, n_p):
    # slabs of L / N_p planes: two neighbouring planes of L^2 entries are remote
    # (the periodic wrap included), every own row is read (nonzero disorder diagonal)
    csr = mat.anderson3d(L, 2.0, 1)
    chi1, chi2, chi3, n_vc, n_vm = comm.metrics(csr, n_p)
    assert list(n_vc) == [2 * L * L] * n_p
    assert list(n_vm) == [L ** 3 // n_p] * n_p
    for c in (chi1, chi2, chi3):
        assert c == pytest.approx(2 * n_p / L)


@pytest.mark.parametrize("D,n_p,seed", [(50, 1, 0), (97, 3, 1), (200, 8, 2), (31, 31, 3)])
def test_counts_match_brute_force(D, n_p, seed):
    csr = fd_inputs.random_symmetric_csr(D, 4.0, seed)
    n_vc, n_vm = comm.counts(csr, n_p)
    bvc, bvm = _brute(csr, n_p)
    assert np.array_equal(n_vc, bvc) and np.array_equal(n_vm, bvm)
    if n_p == 1:
        assert comm.metrics(csr, 1)[:3] == (0.0, 0.0, 0.0)


def test_spin_chain_matches_tables_7_and_9():
    # the 24-site chain with 12 particles: the hopping pattern of SpinChainXXZ
    csr = mat.build("hubbard:n_sites=24,n_up=12,n_dn=0,t=1,U=4,bc=open")
    assert len(csr[0]) - 1 == 2704156
    rows = np.loadtxt(os.path.join(GOLD, "table7_spinchain_chi.txt"))
    for n_p, chi13, chi2 in rows:
        c1, c2, c3, _, _ = comm.metrics(csr, int(n_p))
        assert abs(c3 - chi13) <= 0.005 + 1e-12, (n_p, c3, chi13)
        assert abs(c1 - chi13) <= 0.005 + 1e-12, (n_p, c1, chi13)
        assert abs(c2 - chi2) <= 0.005 + 1e-12, (n_p, c2, chi2)
    # Table 9: the same counts as volumes of 64 FP64 vectors, to half a unit of
    # the last printed digit (0.1 MiB)
    for n_p, avg, mx in np.loadtxt(os.path.join(GOLD, "table9_commvol_spinchain24.txt")):
        n_vc, _ = comm.counts(csr, int(n_p))
        a, m = comm.volumes(n_vc, int(n_p), 64, 8)
        assert abs(a / 2 ** 20 - avg) <= 0.05 + 1e-9, (n_p, a / 2 ** 20, avg)
        assert abs(m / 2 ** 20 - mx) <= 0.05 + 1e-9, (n_p, m / 2 ** 20, mx)


def test_volumes_closed_form():
    # open chain: interior processes read 2 remote entries, the ends 1
    csr = mat.chain(1000)
    n_vc, _ = comm.counts(csr, 4)
    avg, mx = comm.volumes(n_vc, 4, 64, 8)
    assert avg == 64 * 8 * (1 + 2 + 2 + 1) / 4
    assert mx == 64 * 8 * 2
    chi1, chi2, chi3, _, _ = comm.metrics(csr, 4)
    assert avg == pytest.approx(64 * 1000 * 8 * chi2 / 4)
    assert mx == pytest.approx(64 * 1000 * 8 * chi3 / 4)
