"""Fused Chebyshev filter (Alg. 2) and SpMMV on the GPU against the oracle, element by element."""
import numpy as np
import pytest

import fd_inputs
from gpu_util import U32, U64, filter_tolerance
from oracle import chebyshev as ch
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


def _torch():
    import torch
    return torch


def _run_filter(fd, ctx, A, V0, mu, alpha, beta, dtype, ld=None, col0=0):
    torch = _torch()
    D, nb = V0.shape
    ld = ld or nb
    big = torch.zeros((D, ld), dtype=dtype, device="cuda")
    big[:, col0:col0 + nb] = torch.from_numpy(V0).to(dtype)
    V = big[:, col0:col0 + nb]
    W1 = torch.empty((D, nb), dtype=dtype, device="cuda")
    W2 = torch.empty((D, nb), dtype=dtype, device="cuda")
    fd.fd_filter(ctx, A, V, mu, alpha, beta, W1, W2)
    torch.cuda.synchronize()
    out = big.cpu().numpy().astype(np.float64)
    # columns outside the block are untouched
    rest = np.delete(out, np.s_[col0:col0 + nb], axis=1)
    assert np.all(rest == 0.0)
    return out[:, col0:col0 + nb]


def _params(csr, n, seed=0):
    lo, hi = lanczos.gershgorin(csr)
    alpha, beta = ch.scale_params(lo - 0.01, hi + 0.01)
    w = np.random.default_rng(seed).uniform(-0.6, 0.4)
    mu = ch.filter_coeffs(w, w + 0.3, n)
    return mu, alpha, beta


CASES = [
    ("hubbard:n_sites=8,n_up=4,n_dn=4,t=1,U=4,bc=open", 32, 1),
    ("anderson3d:L=11,W=3,seed=5", 64, 1),                 # D = 1331: ragged last chunk
    ("chain:n=777,t=1", 64, 8),                             # sigma > 1: permuted rows
]


@pytest.mark.parametrize("spec,C,sigma", CASES)
@pytest.mark.parametrize("nb", [2, 4, 8, 16, 32, 64, 128])
@pytest.mark.parametrize("n", [2, 3, 25])
def test_filter_f64_matches_oracle(fd, ctx, spec, C, sigma, nb, n):
    csr = mat.build(spec)
    A = fd.fd_build_matrix(ctx, spec, C=C, sigma=sigma)
    D = len(csr[0]) - 1
    V0 = fd_inputs.random_block(D, nb, nb + n)
    mu, alpha, beta = _params(csr, n)
    got = _run_filter(fd, ctx, A, V0, mu, alpha, beta, _torch().float64)
    ref = ch.cheb_filter(mat.to_scipy(csr), V0, mu, alpha, beta)
    tol = filter_tolerance(csr, mu, alpha, beta, V0, U64)
    assert np.all(np.abs(got - ref) <= tol)


@pytest.mark.parametrize("nb", [4, 16, 64, 128])
@pytest.mark.parametrize("n", [2, 3, 40])
def test_filter_f32_matches_oracle(fd, ctx, nb, n):
    spec = "hubbard:n_sites=7,n_up=3,n_dn=3,t=1,U=4,bc=periodic"
    csr = mat.build(spec)
    A = fd.fd_build_matrix(ctx, spec)
    D = len(csr[0]) - 1
    V0 = fd_inputs.random_block(D, nb, 3 * nb + n).astype(np.float32).astype(np.float64)
    mu, alpha, beta = _params(csr, n, 3)
    got = _run_filter(fd, ctx, A, V0, mu, alpha, beta, _torch().float32)
    ref = ch.cheb_filter(mat.to_scipy(csr), V0, mu, alpha, beta)
    tol = filter_tolerance(csr, mu, alpha, beta, V0, U32)
    assert np.all(np.abs(got - ref) <= tol)


@pytest.mark.parametrize("sigma", [1, 64, 1024])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_filter_ragged_permuted_matrix(fd, ctx, sigma, dtype):
    torch = _torch()
    csr = fd_inputs.random_symmetric_csr(2501, 9, 4, max_row=60)
    A = fd.fd_matrix_from_csr(ctx, *csr, C=32, sigma=sigma)
    V0 = fd_inputs.random_block(2501, 32, 7)
    mu, alpha, beta = _params(csr, 17, 5)
    if dtype == "f32":
        V0 = V0.astype(np.float32).astype(np.float64)
    got = _run_filter(fd, ctx, A, V0, mu, alpha, beta, torch.float64 if dtype == "f64" else torch.float32,
                      ld=96, col0=32)
    ref = ch.cheb_filter(mat.to_scipy(csr), V0, mu, alpha, beta)
    tol = filter_tolerance(csr, mu, alpha, beta, V0, U64 if dtype == "f64" else U32)
    assert np.all(np.abs(got - ref) <= tol)


def test_spmmv_matches_oracle(fd, ctx):
    torch = _torch()
    for sigma in (1, 256):
        csr = fd_inputs.random_symmetric_csr(4099, 5, 2, max_row=30)
        A = fd.fd_matrix_from_csr(ctx, *csr, sigma=sigma)
        X0 = fd_inputs.random_block(4099, 64, 1)
        X = torch.from_numpy(X0).cuda()
        Y = torch.empty_like(X)
        fd.fd_spmmv(ctx, A, X, Y)
        ref = mat.to_scipy(csr) @ X0
        rowabs = abs(mat.to_scipy(csr)) @ np.abs(X0)
        nnz_row = np.diff(csr[0]).max()
        assert np.all(np.abs(Y.cpu().numpy() - ref) <= nnz_row * U64 * rowabs + 1e-300)


def test_filter_rejects_bad_arguments(fd, ctx):
    torch = _torch()
    A = fd.fd_build_matrix(ctx, "chain:n=64")
    V = torch.zeros((64, 8), dtype=torch.float64, device="cuda")
    W1, W2 = torch.zeros_like(V), torch.zeros_like(V)
    with pytest.raises(fd.FDError) as e:
        fd.fd_filter(ctx, A, V, [1.0, 0.5], 1.0, 0.0, W1, W2)      # degree 1 < 2
    assert e.value.status == fd.FD_ERR_ARG
    V6 = torch.zeros((64, 6), dtype=torch.float64, device="cuda")
    with pytest.raises(fd.FDError):
        fd.fd_filter(ctx, A, V6, [1.0, 0.5, 0.1], 1.0, 0.0, W1[:, :6], W2[:, :6])  # nb = 6
    with pytest.raises(fd.FDError):
        fd.fd_filter(ctx, A, V, [1.0, np.nan, 0.1], 1.0, 0.0, W1, W2)


def test_full_size_stencil_one_sweep(fd, ctx):
    """3D Anderson L = 128, nb = 64, FP64 and FP32, degree 3: every element vs the oracle."""
    torch = _torch()
    spec = "anderson3d:L=128,W=2,seed=1"
    csr = mat.build(spec)
    A = fd.fd_build_matrix(ctx, spec)
    D = 128 ** 3
    V0 = fd_inputs.random_block(D, 64, 2024)
    alpha, beta = ch.scale_params(-7.01, 7.01)
    mu = ch.filter_coeffs(-0.1, 0.1, 3)
    ref = ch.cheb_filter(mat.to_scipy(csr), V0, mu, alpha, beta)
    for dt, u in ((torch.float64, U64), (torch.float32, U32)):
        V0d = V0 if dt == torch.float64 else V0.astype(np.float32).astype(np.float64)
        refd = ref if dt == torch.float64 else ch.cheb_filter(mat.to_scipy(csr), V0d, mu, alpha, beta)
        got = _run_filter(fd, ctx, A, V0d, mu, alpha, beta, dt)
        tol = filter_tolerance(csr, mu, alpha, beta, V0d, u)
        assert np.all(np.abs(got - refd) <= tol)


# windows inside the interval, touching -1 or +1, beyond it (clipped), at the
# spectrum's edge, and a narrow one at the centre
COEFF_WINDOWS = [(-0.3, 0.45), (-1.0, -0.6), (0.7, 1.0), (-1.5, -0.2), (0.2, 3.0),
                 (-0.99999, -0.9999), (0.9995, 0.99999), (-0.001, 0.002)]


@pytest.mark.parametrize("n", [2, 3, 100, 5000])
@pytest.mark.parametrize("win", COEFF_WINDOWS)
def test_filter_coeffs_match_oracle(fd, n, win):
    # the library's coefficients (Sec. 2 window series, Jackson damping,
    # p(window centre) = 1) element by element against the oracle's
    got = fd.fd_filter_coeffs(win[0], win[1], n)
    ref = ch.filter_coeffs(win[0], win[1], n)
    assert got.shape == ref.shape == (n + 1,)
    assert np.all(np.isfinite(got))
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_filter_coeffs_reject_bad_arguments(fd):
    for args in [(0.1, 0.1, 10), (0.2, 0.1, 10), (-0.5, 0.5, 1), (np.nan, 0.5, 10)]:
        with pytest.raises(fd.FDError) as e:
            fd.fd_filter_coeffs(*args)
        assert e.value.status == fd.FD_ERR_ARG
