"""Communication metrics on the GPU (Sec. 3.1) against the oracle (bit-exact
counts) and against the paper's Tables 2 and 7."""
import os

import numpy as np
import pytest

import fd_inputs
from oracle import comm
from oracle import matrices as mat

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def fd():
    import paper_2209_01974_gb300 as fd
    return fd


@pytest.fixture(scope="module")
def ctx(fd):
    return fd.fd_create(0)


SPECS = ["hubbard:n_sites=8,n_up=4,n_dn=4,t=1,U=4,bc=open",
         "hubbard:n_sites=10,n_up=3,n_dn=5,t=1,U=4,bc=periodic",
         "anderson3d:L=10,W=2,seed=1",
         "roadgraph:side=40,q=0.3,seed=0",
         "chain:n=1001"]


@pytest.mark.parametrize("spec", SPECS)
@pytest.mark.parametrize("n_p", [1, 2, 3, 7, 16, 64])
def test_counts_match_oracle(fd, ctx, spec, n_p):
    A = fd.fd_build_matrix(ctx, spec, C=64, sigma=1)
    csr = mat.build(spec)
    c1, c2, c3, n_vc, n_vm = fd.fd_comm_metrics(ctx, A, n_p)
    o1, o2, o3, ovc, ovm = comm.metrics(csr, n_p)
    assert np.array_equal(n_vc, ovc) and np.array_equal(n_vm, ovm)
    assert (c1, c2, c3) == pytest.approx((o1, o2, o3), rel=1e-15, abs=0)


def test_ragged_csr_matches_oracle(fd, ctx):
    csr = fd_inputs.random_symmetric_csr(5000, 6.0, 11, max_row=200)
    A = fd.fd_matrix_from_csr(ctx, *csr, C=32, sigma=1)
    for n_p in (2, 5, 33):
        _, _, _, n_vc, n_vm = fd.fd_comm_metrics(ctx, A, n_p)
        ovc, ovm = comm.counts(csr, n_p)
        assert np.array_equal(n_vc, ovc) and np.array_equal(n_vm, ovm)


def test_rejects_sorted_rows_and_bad_np(fd, ctx):
    A = fd.fd_build_matrix(ctx, "roadgraph:side=40,q=0.3,seed=0", C=64, sigma=64)
    with pytest.raises(fd.FDError):
        fd.fd_comm_metrics(ctx, A, 4)
    B = fd.fd_build_matrix(ctx, "chain:n=100", C=32, sigma=1)
    with pytest.raises(fd.FDError):
        fd.fd_comm_metrics(ctx, B, 0)
    with pytest.raises(fd.FDError):
        fd.fd_comm_metrics(ctx, B, 101)


@pytest.mark.parametrize("spec,gold", [
    ("hubbard:n_sites=24,n_up=12,n_dn=0,t=1,U=4,bc=open", "table7_spinchain_chi.txt"),
    ("hubbard:n_sites=14,n_up=7,n_dn=7,t=1,U=4,bc=open", "table2_hubbard_chi.txt"),
])
def test_paper_tables(fd, ctx, spec, gold):
    A = fd.fd_build_matrix(ctx, spec, C=64, sigma=1)
    for n_p, chi13, chi2 in np.loadtxt(os.path.join(GOLD, gold)):
        c1, c2, c3, _, _ = fd.fd_comm_metrics(ctx, A, int(n_p))
        assert abs(c1 - chi13) <= 0.005 + 1e-12, (n_p, c1, chi13)
        assert abs(c3 - chi13) <= 0.005 + 1e-12, (n_p, c3, chi13)
        assert abs(c2 - chi2) <= 0.005 + 1e-12, (n_p, c2, chi2)


def table3_rows():
    rows = []
    for line in open(os.path.join(GOLD, "table3_commvol_hubbard14.txt")):
        if line.strip() and not line.startswith("#"):
            n_p, avg, mx, unit = line.split()
            rows.append((int(n_p), float(avg), float(mx), 2.0 ** 30 if unit == "GiB" else 2.0 ** 20))
    return rows


def check_table3(counts):
    # counts(n_p) -> n_vc per process; volumes of 64 FP64 vectors against the
    # printed values, to half a unit of their last printed digit
    for n_p, avg, mx, scale in table3_rows():
        a, m = comm.volumes(counts(n_p), n_p, 64, 8)
        assert abs(a / scale - avg) <= 0.005 + 1e-9, (n_p, a / scale, avg)
        assert abs(m / scale - mx) <= 0.005 + 1e-9, (n_p, m / scale, mx)


def test_paper_table3_volumes(fd, ctx):
    A = fd.fd_build_matrix(ctx, "hubbard:n_sites=14,n_up=7,n_dn=7,t=1,U=4,bc=open", C=64, sigma=1)
    check_table3(lambda n_p: fd.fd_comm_metrics(ctx, A, n_p)[3])
