"""Lehmann bounds and the Lehmann interval mode of the FD loop on the GPU,
against the oracle (oracle/lehmann.py, oracle/fd.py) and dense eigensolvers."""
import numpy as np
import pytest

import fd_inputs
from oracle import fd as ofd
from oracle import lehmann
from oracle import matrices as mat

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fd():
    import paper_2209_01974_gb300 as fd
    return fd


@pytest.fixture(scope="module")
def ctx(fd):
    return fd.fd_create(0)


def _t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _check_bounds(got, ref, scale):
    assert len(got[0]) == len(ref[0]) and len(got[1]) == len(ref[1])
    for g, r in zip(got, ref):
        # a bound rho + 1/mu is as accurate as mu relative to |1/mu| (the
        # distance from rho), plus the rounding of the operator
        assert np.all(np.abs(g - r) <= 1e-9 * (np.abs(r - 0.0) + scale))


@pytest.mark.parametrize("ns", [1, 7, 16, 40])
def test_bounds_match_oracle_random_matrix(fd, ctx, ns):
    rp, col, val = fd_inputs.random_symmetric_csr(3000, 6, 11 + ns, max_row=40)
    A = fd.fd_matrix_from_csr(ctx, rp, col, val)
    S = mat.to_scipy((rp, col, val))
    V0 = fd_inputs.random_block(3000, ns, 5 + ns)
    rho = 0.137
    got = fd.fd_lehmann_bounds(ctx, A, _t(V0), rho)
    ref = lehmann.lehmann_bounds(S, V0, rho)
    _check_bounds(got, ref, abs(S).sum(axis=1).max())


def test_bounds_match_oracle_on_filtered_hubbard_block(fd, ctx):
    # a block filtered towards the shift, the situation inside FD: bounds tight
    spec = "hubbard:n_sites=8,n_up=4,n_dn=4,t=1,U=4,bc=open"
    csr = mat.build(spec)
    S = mat.to_scipy(csr)
    lam, X = np.linalg.eigh(S.toarray())
    rho = 0.05
    idx = np.argsort(np.abs(lam - rho))[:24]
    V0 = X[:, idx] + 1e-6 * fd_inputs.random_block(S.shape[0], 24, 3)
    A = fd.fd_build_matrix(ctx, spec)
    got = fd.fd_lehmann_bounds(ctx, A, _t(V0), rho)
    ref = lehmann.lehmann_bounds(S, V0, rho)
    _check_bounds(got, ref, np.abs(lam).max())
    # and they enclose the true eigenvalues nearest rho
    below = np.sort(lam[lam < rho])[::-1]
    above = np.sort(lam[lam > rho])
    assert np.all(below[:len(got[0])] >= got[0] - 1e-10)
    assert np.all(above[:len(got[1])] <= got[1] + 1e-10)


def test_bounds_break_down_on_exact_eigenvector_at_the_shift(fd, ctx):
    d = np.linspace(-2.0, 3.0, 200)
    A = fd.fd_matrix_from_csr(ctx, *mat.diagonal(d))
    V0 = np.zeros((200, 2))
    V0[17, 0] = 1.0
    V0[:, 1] = fd_inputs.random_block(200, 1, 2)[:, 0]
    with pytest.raises(fd.FDError) as e:
        fd.fd_lehmann_bounds(ctx, A, _t(V0), float(d[17]))
    assert e.value.status == fd.FD_ERR_BREAKDOWN


def _nearest(ev, tau, k):
    return np.sort(ev[np.lexsort((ev, np.abs(ev - tau)))[:k]])


@pytest.mark.parametrize("spec,a,b,nt,nb,deg", [
    ("chain:n=2000", -0.05, 0.05, 8, 16, 50),
    ("anderson3d:L=12,W=4,seed=9", -0.2, 0.2, 10, 16, 60),
    ("hubbard:n_sites=6,n_up=3,n_dn=3,t=1,U=4,bc=periodic", 2.0, 3.0, 6, 8, 30),
    ("anderson3d:L=10,W=16,seed=2", -0.01, 0.01, 12, 16, 100),
])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_lehmann_solves_match_dense(fd, ctx, spec, a, b, nt, nb, deg, prec):
    csr = mat.build(spec)
    ev = np.linalg.eigvalsh(mat.to_scipy(csr).toarray())
    A = fd.fd_build_matrix(ctx, spec)
    th, rho, res = fd.fd_solve(ctx, A, a, b, nt, nb, deg, 1e-9, intervals="lehmann", precision=prec)
    assert res["converged"] == 1 and rho.max() <= 1e-9
    assert np.abs(th - _nearest(ev, 0.5 * (a + b), nt)).max() <= 1e-10 * np.abs(ev).max()


def test_lehmann_config1_agrees_with_oracle_loop(fd, ctx):
    spec = "hubbard:n_sites=8,n_up=4,n_dn=4,t=1,U=4,bc=open"
    A = fd.fd_build_matrix(ctx, spec)
    th, rho, res = fd.fd_solve(ctx, A, -0.5, 0.5, 20, 32, 100, 1e-9, intervals="lehmann")
    o = ofd.fd_solve(mat.build(spec), -0.5, 0.5, 20, 32, 100, 1e-9, intervals="lehmann")
    assert res["converged"] == 1 and o.converged
    lam_max = 20.3
    assert np.abs(th - o.theta).max() <= 1e-10 * lam_max
    # the same start block, bounds and interval rule: the same outer iterations
    assert abs(res["iterations"] - o.iterations) <= 1


def test_interval_mode_is_checked(fd, ctx):
    A = fd.fd_build_matrix(ctx, "chain:n=100")
    with pytest.raises(fd.FDError) as e:
        fd.fd_solve(ctx, A, -0.1, 0.1, 4, 8, 20, 1e-9, intervals=7)
    assert e.value.status == fd.FD_ERR_ARG
