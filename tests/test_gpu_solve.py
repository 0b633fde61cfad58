"""Full FD solves on the GPU: eigenvalues against dense diagonalisation and the oracle."""
import numpy as np
import pytest

from oracle import fd as ofd
from oracle import matrices as mat

pytestmark = pytest.mark.gpu

CONFIG1 = "hubbard:n_sites=8,n_up=4,n_dn=4,t=1,U=4,bc=open"


@pytest.fixture(scope="module")
def fd():
    import paper_2209_01974_gb300 as fd
    return fd


@pytest.fixture(scope="module")
def ctx(fd):
    return fd.fd_create(0)


@pytest.fixture(scope="module")
def dense1():
    A = mat.to_scipy(mat.build(CONFIG1)).toarray()
    ev = np.linalg.eigvalsh(A)
    return A, ev


def _nearest(ev, tau, k):
    return np.sort(ev[np.lexsort((ev, np.abs(ev - tau)))[:k]])


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_config1_solve_matches_dense(fd, ctx, dense1, precision):
    import torch
    H, ev = dense1
    A = fd.fd_build_matrix(ctx, CONFIG1)
    X = torch.zeros((4900, 20), dtype=torch.float64, device="cuda")
    th, rho, res = fd.fd_solve(ctx, A, -0.5, 0.5, 20, 32, 100, 1e-9, X=X, precision=precision)
    assert res["converged"] == 1
    assert rho.max() <= 1e-9
    normH = np.abs(ev).max()
    assert np.abs(th - _nearest(ev, 0.0, 20)).max() <= 1e-10 * normH
    Xh = X.cpu().numpy()
    assert np.abs(H @ Xh - Xh * th[None, :]).max() <= 1e-9
    assert np.abs(Xh.T @ Xh - np.eye(20)).max() < 1e-10
    if precision == "f32":
        assert res["n_spmmv_f32"] > 0


def test_config1_solve_agrees_with_oracle_loop(fd, ctx, dense1):
    A = fd.fd_build_matrix(ctx, CONFIG1)
    th, rho, res = fd.fd_solve(ctx, A, -0.5, 0.5, 20, 32, 100, 1e-9)
    o = ofd.fd_solve(mat.build(CONFIG1), -0.5, 0.5, 20, 32, 100, 1e-9)
    assert o.converged
    assert np.abs(th - o.theta).max() <= 1e-10 * np.abs(dense1[1]).max()
    # same start block, bounds and heuristic: the same number of outer iterations
    assert abs(res["iterations"] - o.iterations) <= 1


@pytest.mark.parametrize("spec,a,b,nt,nb,deg", [
    ("chain:n=2000", -0.05, 0.05, 8, 16, 50),
    ("anderson3d:L=12,W=4,seed=9", -0.2, 0.2, 10, 16, 60),
    ("hubbard:n_sites=6,n_up=3,n_dn=3,t=1,U=4,bc=periodic", 2.0, 3.0, 6, 8, 30),
])
def test_small_solves_match_dense(fd, ctx, spec, a, b, nt, nb, deg):
    csr = mat.build(spec)
    ev = np.linalg.eigvalsh(mat.to_scipy(csr).toarray())
    A = fd.fd_build_matrix(ctx, spec)
    th, rho, res = fd.fd_solve(ctx, A, a, b, nt, nb, deg, 1e-9)
    assert res["converged"] == 1 and rho.max() <= 1e-9
    assert np.abs(th - _nearest(ev, 0.5 * (a + b), nt)).max() <= 1e-10 * np.abs(ev).max()


def test_noconv_reports_status(fd, ctx):
    A = fd.fd_build_matrix(ctx, CONFIG1)
    with pytest.raises(fd.FDError) as e:
        fd.fd_solve(ctx, A, -0.5, 0.5, 20, 32, 10, 1e-9, max_outer=2)
    assert e.value.status == fd.FD_ERR_NOCONV
    th, rho, res = fd.fd_solve(ctx, A, -0.5, 0.5, 20, 32, 10, 1e-9, max_outer=2, raise_noconv=False)
    assert res["converged"] == 0 and res["iterations"] == 2


def test_fig2_diagonal_matrix_on_gpu(fd, ctx):
    """The example of Fig. 2: 1000 equidistant eigenvalues in [-1, 1], the 10
    nearest the centre of [-0.01, 0.01] with N_s = 20 search vectors."""
    lam = -1 + 2 * np.arange(1000) / 999
    A = fd.fd_matrix_from_csr(ctx, *mat.diagonal(lam))
    th, rho, res = fd.fd_solve(ctx, A, -0.01, 0.01, 10, 4, 20, 1e-9, ns=20)
    assert res["converged"] == 1 and rho.max() <= 1e-9
    assert np.abs(th - _nearest(lam, 0.0, 10)).max() <= 1e-12


def test_solve_rejects_degenerate_sizes(fd, ctx):
    A = fd.fd_build_matrix(ctx, "chain:n=10")
    with pytest.raises(fd.FDError) as e:
        fd.fd_solve(ctx, A, -0.1, 0.1, 8, 16, 20, 1e-9)        # N_s = 32 > D = 10
    assert e.value.status == fd.FD_ERR_ARG
    with pytest.raises(fd.FDError):
        fd.fd_solve(ctx, A, 0.1, -0.1, 2, 2, 20, 1e-9)         # a > b
    with pytest.raises(fd.FDError):
        fd.fd_matrix_from_csr(ctx, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))  # D = 0
