"""Float-float sweeps (FD_FF) on the GPU against the FP64 oracle, element by
element.  A float-float value is hi + lo with two floats; its sums and
products (error-free transformations in FP32) round within a few 2^-48 of
the magnitudes involved, so the derived filter bound is taken with
u = 2^-45, against 2^-53 for FP64 and 2^-24 for FP32."""
import numpy as np
import pytest

import fd_inputs
from gpu_util import U32, filter_tolerance
from oracle import chebyshev as ch
from oracle import lanczos
from oracle import matrices as mat

pytestmark = pytest.mark.gpu

U_FF = 2.0 ** -45


@pytest.fixture(scope="module")
def fd():
    import paper_2209_01974_gb300 as fd
    return fd


@pytest.fixture(scope="module")
def ctx(fd):
    return fd.fd_create(0)


def _ff_block(fd, ctx, V64):
    import torch
    D, n = V64.shape
    out = torch.empty((D, n, 2), dtype=torch.float32, device="cuda")
    fd.fd_copy_block(ctx, V64, out)
    return out


def _to_f64(fd, ctx, Vff):
    import torch
    D, n, _ = Vff.shape
    out = torch.empty((D, n), dtype=torch.float64, device="cuda")
    fd.fd_copy_block(ctx, Vff, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _params(csr, n, seed=0):
    lo, hi = lanczos.gershgorin(csr)
    alpha, beta = ch.scale_params(lo - 0.01, hi + 0.01)
    w = np.random.default_rng(seed).uniform(-0.6, 0.4)
    return ch.filter_coeffs(w, w + 0.3, n), alpha, beta


def test_split_round_trip(fd, ctx):
    """FP64 -> (hi, lo) -> FP64: hi is the nearest float, lo the nearest float
    to the remainder, so the round trip is within 2^-48 |x| and exact for
    values with at most 48 significant bits."""
    import torch
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1000, 8)) * np.exp(rng.uniform(-20, 20, (1000, 8)))
    x[:, 0] = rng.integers(-2 ** 40, 2 ** 40, 1000) * 2.0 ** -30  # at most 41 significant bits: exact
    X = torch.from_numpy(x).cuda()
    ff = _ff_block(fd, ctx, X)
    pairs = ff.cpu().numpy().astype(np.float64)
    assert np.array_equal(pairs[..., 0], x.astype(np.float32).astype(np.float64))
    back = _to_f64(fd, ctx, ff)
    assert np.all(np.abs(back - x) <= 2.0 ** -48 * np.abs(x))
    assert np.array_equal(back[:, 0], x[:, 0])


CASES = [
    ("anderson3d:L=11,W=3,seed=5", 64, 1),   # D = 1331: ragged last chunk, random diagonal
    ("chain:n=777,t=1", 64, 8),               # sigma > 1: permuted rows
    ("hubbard:n_sites=8,n_up=4,n_dn=4,t=1,U=4,bc=open", 32, 1),
]


@pytest.mark.parametrize("spec,C,sigma", CASES)
@pytest.mark.parametrize("nb", [2, 16, 64])
@pytest.mark.parametrize("n", [2, 3, 60])
def test_filter_ff_matches_oracle(fd, ctx, spec, C, sigma, nb, n):
    import torch
    csr = mat.build(spec)
    A = fd.fd_build_matrix(ctx, spec, C=C, sigma=sigma)
    D = len(csr[0]) - 1
    V0 = fd_inputs.random_block(D, nb, 7 * nb + n)
    mu, alpha, beta = _params(csr, n)
    V = _ff_block(fd, ctx, torch.from_numpy(V0).cuda())
    W1, W2 = torch.empty_like(V), torch.empty_like(V)
    fd.fd_filter(ctx, A, V, mu, alpha, beta, W1, W2)
    got = _to_f64(fd, ctx, V)
    ref = ch.cheb_filter(mat.to_scipy(csr), V0, mu, alpha, beta)
    assert np.all(np.abs(got - ref) <= filter_tolerance(csr, mu, alpha, beta, V0, U_FF))
    if n == 60:
        # far inside the FP32 bound: the sweep really carries the low words
        assert np.abs(got - ref).max() <= 1e-6 * filter_tolerance(csr, mu, alpha, beta, V0, U32).max()


@pytest.mark.parametrize("nb", [2, 16, 128])
def test_spmmv_ff_matches_oracle(fd, ctx, nb):
    import torch
    spec = "anderson3d:L=9,W=12,seed=2"
    csr = mat.build(spec)
    A = fd.fd_build_matrix(ctx, spec, C=32, sigma=4)
    D = len(csr[0]) - 1
    X0 = fd_inputs.random_block(D, nb, 99)
    X = _ff_block(fd, ctx, torch.from_numpy(X0).cuda())
    Y = torch.empty_like(X)
    fd.fd_spmmv(ctx, A, X, Y)
    got = _to_f64(fd, ctx, Y)
    S = mat.to_scipy(csr)
    ref = S @ X0
    bound = 12 * U_FF * (abs(S) @ np.abs(X0))
    assert np.all(np.abs(got - ref) <= bound)


@pytest.mark.parametrize("spec", ["hubbard:n_sites=8,n_up=4,n_dn=4,t=1,U=4,bc=open",
                                  "hubbard:n_sites=7,n_up=3,n_dn=2,t=1,U=4.3,bc=periodic"])
@pytest.mark.parametrize("nb", [2, 16])
def test_filter_ff_matrix_free_matches_oracle(fd, ctx, spec, nb):
    """The matrix-free Hubbard operator (kron=1) in float-float against the
    oracle within the derived bound, and against the stored matrix's
    float-float filter within twice it."""
    import torch
    csr = mat.build(spec)
    D = len(csr[0]) - 1
    V0 = fd_inputs.random_block(D, nb, 31 + nb)
    mu, alpha, beta = _params(csr, 30)
    out = []
    for s_ in (spec + ",kron=1", spec):
        A = fd.fd_build_matrix(ctx, s_)
        V = _ff_block(fd, ctx, torch.from_numpy(V0).cuda())
        W1, W2 = torch.empty_like(V), torch.empty_like(V)
        fd.fd_filter(ctx, A, V, mu, alpha, beta, W1, W2)
        out.append(_to_f64(fd, ctx, V))
    ref = ch.cheb_filter(mat.to_scipy(csr), V0, mu, alpha, beta)
    tol = filter_tolerance(csr, mu, alpha, beta, V0, U_FF)
    assert np.all(np.abs(out[0] - ref) <= tol)
    assert np.all(np.abs(out[0] - out[1]) <= 2 * tol)


def test_solve_ff_finish_on_matrix_free(fd, ctx):
    spec = "hubbard:n_sites=8,n_up=4,n_dn=4,t=1,U=4,bc=open"
    A = fd.fd_build_matrix(ctx, spec + ",kron=1")
    th0, r0, res0 = fd.fd_solve(ctx, fd.fd_build_matrix(ctx, spec), -0.5, 0.5, 20, 32, 100, 1e-9)
    th, r, res = fd.fd_solve(ctx, A, -0.5, 0.5, 20, 32, 100, 1e-9, precision="f32", finish="ff")
    assert res["converged"] and np.all(r <= 1e-9) and res["n_spmmv_ff"] > 0
    assert np.abs(np.sort(th) - np.sort(th0)).max() <= 1e-10 * max(1.0, np.abs(th0).max())


@pytest.mark.parametrize("form", [{"precision": "ff"}, {"precision": "f32", "finish": "ff"}])
def test_solve_ff_forms_match_f64(fd, ctx, form):
    """Config 1 (8-site Hubbard chain, 20 pairs nearest [-0.5, 0.5]): the
    float-float forms reach the same eigenvalues as the FP64 form, residuals
    <= 1e-9, with their sweeps counted."""
    spec = "hubbard:n_sites=8,n_up=4,n_dn=4,t=1,U=4,bc=open"
    A = fd.fd_build_matrix(ctx, spec)
    th0, r0, res0 = fd.fd_solve(ctx, A, -0.5, 0.5, 20, 32, 100, 1e-9)
    th, r, res = fd.fd_solve(ctx, A, -0.5, 0.5, 20, 32, 100, 1e-9, **form)
    assert res["converged"] and res0["converged"]
    assert np.all(r <= 1e-9)
    assert np.abs(np.sort(th) - np.sort(th0)).max() <= 1e-10 * max(1.0, np.abs(th0).max())
    assert res["n_spmmv_ff"] > 0
    if form["precision"] == "ff":
        assert res["n_spmmv_f32"] == 0
