"""Device matrix generation and SELL-C-sigma storage: bit-exact against the oracle."""
import numpy as np
import pytest

import fd_inputs
from oracle import lanczos
from oracle import matrices as mat

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fd():
    import paper_2209_01974_gb300 as fd
    return fd


@pytest.fixture(scope="module")
def ctx(fd):
    return fd.fd_create(0)


SPECS = [
    "hubbard:n_sites=8,n_up=4,n_dn=4,t=1,U=4,bc=open",
    "hubbard:n_sites=6,n_up=2,n_dn=2,t=1,U=4,bc=periodic",
    "hubbard:n_sites=7,n_up=3,n_dn=2,t=0.5,U=2.5,bc=periodic",
    "anderson3d:L=8,W=2,seed=1",
    "anderson3d:L=5,W=16,seed=7,t=1",
    "chain:n=1000,t=1",
]


@pytest.mark.parametrize("spec", SPECS)
@pytest.mark.parametrize("C,sigma", [(32, 1), (64, 128)])
def test_generated_matrix_is_bit_exact(fd, ctx, spec, C, sigma):
    A = fd.fd_build_matrix(ctx, spec, C=C, sigma=sigma)
    rp, c, v = fd.fd_matrix_to_csr(ctx, A)
    orp, oc, ov = mat.build(spec)
    assert np.array_equal(rp, orp)
    assert np.array_equal(c, oc)
    assert np.array_equal(v.view(np.uint64), ov.view(np.uint64))
    info = A.info
    g = lanczos.gershgorin((orp, oc, ov))
    assert info["gersh_lo"] == pytest.approx(g[0], rel=1e-13, abs=1e-13)
    assert info["gersh_hi"] == pytest.approx(g[1], rel=1e-13, abs=1e-13)


def test_sigma_permutation_is_a_valid_window_sort(fd, ctx):
    csr = fd_inputs.random_symmetric_csr(3001, 6, 11, max_row=40)
    for sigma in (1, 32, 1000, 4096):
        A = fd.fd_matrix_from_csr(ctx, *csr, C=32, sigma=sigma)
        perm = fd.fd_matrix_perm(ctx, A)
        assert np.array_equal(np.sort(perm), np.arange(3001))
        lens = np.diff(csr[0])
        for w0 in range(0, 3001, sigma):
            seg = perm[w0:w0 + sigma]
            assert np.all((seg >= w0) & (seg < w0 + sigma))
            l = lens[seg]
            assert np.all(np.diff(l) <= 0)
            for val in np.unique(l):           # equal lengths keep their original order
                s = seg[l == val]
                assert np.all(np.diff(s) > 0)
        rp, c, v = fd.fd_matrix_to_csr(ctx, A)
        assert np.array_equal(rp, csr[0]) and np.array_equal(c, csr[1]) and np.array_equal(v, csr[2])


def test_from_csr_without_diagonal_round_trips(fd, ctx):
    rp, c, v = mat.chain(50)
    keep = c != np.repeat(np.arange(50), np.diff(rp))
    rp2 = np.concatenate([[0], np.cumsum([keep[rp[i]:rp[i + 1]].sum() for i in range(50)])])
    A = fd.fd_matrix_from_csr(ctx, rp2, c[keep], v[keep])
    r, cc, vv = fd.fd_matrix_to_csr(ctx, A)
    assert np.array_equal(r, rp2) and np.array_equal(cc, c[keep]) and np.array_equal(vv, v[keep])


def test_malformed_csr_is_rejected(fd, ctx):
    rp, c, v = mat.chain(10)
    bad = c.copy(); bad[5] = 99
    with pytest.raises(fd.FDError) as e:
        fd.fd_matrix_from_csr(ctx, rp, bad, v)
    assert e.value.status == fd.FD_ERR_ARG
    rp2 = rp.copy(); rp2[3] = rp2[4] + 1
    with pytest.raises(fd.FDError):
        fd.fd_matrix_from_csr(ctx, rp2, c, v)
    with pytest.raises(fd.FDError):
        fd.fd_build_matrix(ctx, "hubbard:n_sites=40,n_up=2,n_dn=2")
    with pytest.raises(fd.FDError):
        fd.fd_build_matrix(ctx, "nosuchmatrix:x=1")


def test_full_size_stencil_sampled_rows(fd, ctx):
    # 3D Anderson L = 128 (2,097,152 rows), disorder W = 2, seed 1
    A = fd.fd_build_matrix(ctx, "anderson3d:L=128,W=2,seed=1")
    rp, c, v = fd.fd_matrix_to_csr(ctx, A)
    assert len(rp) - 1 == 128 ** 3 and rp[-1] == 7 * 128 ** 3
    rows = np.random.default_rng(0).choice(128 ** 3, 64, replace=False)
    for r, (oc, ov) in zip(rows, mat.anderson_rows(128, 2.0, 1, 1.0, rows)):
        assert np.array_equal(c[rp[r]:rp[r + 1]], oc)
        assert np.array_equal(v[rp[r]:rp[r + 1]], ov)


def test_full_size_hubbard14_ring_sampled_rows(fd, ctx):
    # Hubbard ring of 14 sites, 7 + 7 electrons (11,778,624 rows), periodic with fermion sign
    A = fd.fd_build_matrix(ctx, "hubbard:n_sites=14,n_up=7,n_dn=7,t=1,U=4,bc=periodic")
    rp, c, v = fd.fd_matrix_to_csr(ctx, A)
    D = 3432 ** 2
    assert len(rp) - 1 == D
    # every ring bond can hop iff exactly one of its sites is occupied:
    # mean off-diagonal count 2 * 14 * 2 * C(12,6) / C(14,7), plus the diagonal
    assert (rp[-1] - D) / D == pytest.approx(2 * 14 * 2 * 924 / 3432, abs=1e-12)
    rows = np.random.default_rng(1).choice(D, 40, replace=False)
    for r, (oc, ov) in zip(rows, mat.hubbard_rows(14, 7, 7, 1.0, 4.0, "periodic", rows)):
        assert np.array_equal(c[rp[r]:rp[r + 1]], oc)
        assert np.array_equal(v[rp[r]:rp[r + 1]], ov)
