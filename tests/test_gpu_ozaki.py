"""FP64 Gram and rotation products on the tcgen05 tensor cores (Ozaki splitting) against
FP64 references, and the CholQR / Rayleigh-Ritz steps built on them."""
import numpy as np
import pytest

import fd_inputs
from oracle import matrices as mat
from oracle import ortho, rayleigh_ritz

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


@pytest.fixture(scope="module")
def fd():
    import paper_2209_01974_gb300 as fd
    return fd


@pytest.fixture(scope="module")
def ctx(fd):
    c = fd.fd_create(0)
    yield c
    fd.fd_set_gemm_mode(c, "auto")


def _t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _block(D, n, seed, spread=6):
    rng = np.random.default_rng(seed)
    V = rng.standard_normal((D, n)) * np.logspace(0, spread, n)[None, :]
    V[rng.random((D, n)) < 0.05] = 0.0
    return V


def _bound(X, Y):
    # split error per term < (2^-55 truncation + 2^-53.2 dropped digit pairs) 2^(e+f)
    # <= 2^-50.9 |X|max |Y|max, the reference's own rounding <= K u |X|max |Y|max:
    # together under 8 K u |X|max |Y|max = K 2^-50 |X|max |Y|max
    K = X.shape[0]
    return 8 * K * U * np.outer(np.abs(X).max(0), np.abs(Y).max(0))


@pytest.mark.parametrize("D,m,n", [(20000, 96, 96), (7777, 130, 70), (300, 64, 64)])
def test_ozaki_gram_is_fp64_accurate(fd, ctx, D, m, n):
    X = _block(D, m, 1)
    Y = X if m == n else _block(D, n, 2, 3)
    fd.fd_set_gemm_mode(ctx, "ozaki")
    C = fd.fd_gram(ctx, _t(X), _t(Y)).cpu().numpy()
    ref = X.T @ Y
    assert np.all(np.abs(C - ref) <= _bound(X, Y))
    # relative to what FP64 FMA arithmetic achieves on the same data
    fd.fd_set_gemm_mode(ctx, "fp64")
    C64 = fd.fd_gram(ctx, _t(X), _t(Y)).cpu().numpy()
    assert np.all(np.abs(C64 - ref) <= _bound(X, Y))


@pytest.mark.parametrize("upper", [False, True])
def test_ozaki_rotation_is_fp64_accurate(fd, ctx, upper):
    D, n = 9001, 96
    V = _block(D, n, 3, 4)
    M = np.random.default_rng(4).standard_normal((n, n)) * np.logspace(0, 3, n)[:, None]
    if upper:
        M = np.triu(M)
    ref = V @ M
    fd.fd_set_gemm_mode(ctx, "ozaki")
    Vt = _t(V)
    fd.fd_rotate(ctx, Vt, _t(M), upper)
    got = Vt.cpu().numpy()
    bound = 8 * n * U * np.outer(np.abs(V).max(1), np.abs(M).max(0))
    assert np.all(np.abs(got - ref) <= bound)


def test_ozaki_cholqr_and_rr_match_fp64_mode(fd, ctx):
    import torch
    D, ns = 30000, 64
    V0 = fd_inputs.random_block(D, ns, 9) @ np.diag(np.logspace(0, 4, ns))
    out = {}
    for mode in ("fp64", "ozaki"):
        fd.fd_set_gemm_mode(ctx, mode)
        V = _t(V0)
        R = torch.zeros((ns, ns), dtype=torch.float64, device="cuda")
        assert fd.fd_orthonormalize(ctx, V, R) == 2
        Q = V.cpu().numpy()
        assert np.abs(Q.T @ Q - np.eye(ns)).max() < 1e-14
        out[mode] = (Q, R.cpu().numpy())
    assert np.abs(out["fp64"][0] - out["ozaki"][0]).max() < 1e-10
    assert np.abs(out["fp64"][1] - out["ozaki"][1]).max() < 1e-12 * np.abs(out["fp64"][1]).max()
    Qo, Ro, _ = ortho.cholqr2(V0)
    assert np.abs(out["ozaki"][1] - Ro).max() <= 1e-12 * np.abs(Ro).max()


def test_ozaki_rayleigh_ritz(fd, ctx):
    import torch
    spec = "anderson3d:L=40,W=4,seed=3"
    csr = mat.build(spec)
    D = 40 ** 3
    V0, _ = np.linalg.qr(fd_inputs.random_block(D, 64, 5))
    A = fd.fd_build_matrix(ctx, spec)
    fd.fd_set_gemm_mode(ctx, "ozaki")
    V = _t(V0)
    th, rho = fd.fd_rayleigh_ritz(ctx, A, V, torch.empty_like(V))
    tho, _, _, rhoo = rayleigh_ritz.rayleigh_ritz(mat.to_scipy(csr), V0)
    assert np.abs(th - tho).max() <= 1e-12 * np.abs(tho).max()
    assert np.abs(rho - rhoo).max() <= 1e-11 * np.abs(tho).max()


def test_ozaki_nonfinite_input_takes_fp64_path(fd, ctx):
    fd.fd_set_gemm_mode(ctx, "ozaki")
    bad = fd_inputs.random_block(5000, 64, 1)
    bad[7, 3] = np.nan
    with pytest.raises(fd.FDError) as e:
        fd.fd_orthonormalize(ctx, _t(bad))
    assert e.value.status == fd.FD_ERR_BREAKDOWN


def test_bounded_wait_gives_up_and_context_stays_usable(fd, ctx):
    # an mbarrier nobody arrives on: the same bounded wait as the tensor-core
    # products gives up after 0.1 s and the call reports FD_ERR_TIMEOUT
    assert fd.fd_check_bounded_wait(ctx, 100000) == fd.FD_ERR_TIMEOUT
    assert fd.fd_check_bounded_wait(ctx, 0) == fd.FD_ERR_ARG
    # the context and the device still work afterwards
    X = _block(20000, 96, 5)
    fd.fd_set_gemm_mode(ctx, "ozaki")
    C = fd.fd_gram(ctx, _t(X), _t(X)).cpu().numpy()
    assert np.all(np.abs(C - X.T @ X) <= _bound(X, X))


def test_full_size_gram_and_cholqr2(fd, ctx):
    # the bench's block, 2,097,152 x 384: sampled Gram entries against CPU dot
    # products, then the orthonormality of CholQR2 (tensor-core products) checked
    # with the FP64-arithmetic Gram
    import torch
    D, ns = 2097152, 384
    g = torch.Generator(device="cuda").manual_seed(7)
    V = torch.randn((D, ns), dtype=torch.float64, device="cuda", generator=g)
    V[:, 100] *= 1e3  # columns of very different scale
    fd.fd_set_gemm_mode(ctx, "auto")
    G = fd.fd_gram(ctx, V, V).cpu().numpy()
    pairs = [(0, 0), (0, 383), (100, 100), (100, 7), (250, 251), (383, 17)]
    cols = {c: V[:, c].cpu().numpy() for c in {c for p in pairs for c in p}}
    for i, j in pairs:
        x, y = cols[i], cols[j]
        ref = float(np.dot(x, y))
        # split error + the CPU sum's own rounding: under 8 K u max|x| max|y|
        assert abs(G[i, j] - ref) <= 8 * D * U * np.abs(x).max() * np.abs(y).max()
    fd.fd_orthonormalize(ctx, V)
    fd.fd_set_gemm_mode(ctx, "fp64")
    Q = fd.fd_gram(ctx, V, V).cpu().numpy()
    fd.fd_set_gemm_mode(ctx, "auto")
    # the FP64 check Gram rounds each entry by about sqrt(D) u (blocked sums)
    assert np.abs(Q - np.eye(ns)).max() <= 1e-12
    del V
    torch.cuda.empty_cache()
