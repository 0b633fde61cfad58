"""Cholesky-QR, Rayleigh-Ritz, Lanczos interval and KPM moments on the GPU against the oracle."""
import numpy as np
import pytest

import fd_inputs
from oracle import chebyshev as ch
from oracle import kpm, lanczos, ortho, rayleigh_ritz
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


@pytest.mark.parametrize("D,ns", [(5000, 96), (3001, 40), (20000, 448), (777, 2)])
def test_cholqr2_orthonormal_and_matches_oracle(fd, ctx, D, ns):
    import torch
    V0 = fd_inputs.random_block(D, ns, ns) @ np.diag(np.logspace(0, 4, ns))
    V = _t(V0)
    R = torch.zeros((ns, ns), dtype=torch.float64, device="cuda")
    passes = fd.fd_orthonormalize(ctx, V, R)
    assert passes == 2
    Q = V.cpu().numpy()
    assert np.abs(Q.T @ Q - np.eye(ns)).max() < 1e-14 * max(1, ns / 100)
    Qo, Ro, _ = ortho.cholqr2(V0)
    assert np.abs(R.cpu().numpy() - Ro).max() <= 1e-12 * np.abs(Ro).max()
    assert np.abs(Q - Qo).max() <= 1e-10


def test_cholqr_reports_a_block_it_cannot_orthonormalise(fd, ctx):
    # condition 1e20: the last pass's R is far from the identity -> breakdown,
    # in both Cholesky-QR entry points (the oracle raises Breakdown likewise)
    rng = np.random.default_rng(2)
    U, _ = np.linalg.qr(rng.standard_normal((4000, 32)))
    W, _ = np.linalg.qr(rng.standard_normal((32, 32)))
    V0 = U @ np.diag(np.logspace(0, -20, 32)) @ W
    for call in (fd.fd_orthonormalize, fd.fd_orthonormalize_noalloc):
        with pytest.raises(fd.FDError) as e:
            call(ctx, _t(V0))
        assert e.value.status == fd.FD_ERR_BREAKDOWN and "rank deficient" in str(e.value)


def test_cholqr_shifted_path_and_breakdown(fd, ctx):
    import torch
    rng = np.random.default_rng(2)
    U, _ = np.linalg.qr(rng.standard_normal((4000, 32)))
    W, _ = np.linalg.qr(rng.standard_normal((32, 32)))
    V0 = U @ np.diag(np.logspace(0, -12, 32)) @ W
    V = _t(V0)
    assert fd.fd_orthonormalize(ctx, V) == 3
    Q = V.cpu().numpy()
    assert np.abs(Q.T @ Q - np.eye(32)).max() < 1e-13
    bad = fd_inputs.random_block(100, 4, 1)
    bad[3, 2] = np.nan
    with pytest.raises(fd.FDError) as e:
        fd.fd_orthonormalize(ctx, _t(bad))
    assert e.value.status == fd.FD_ERR_BREAKDOWN


@pytest.mark.parametrize("spec,ns", [("hubbard:n_sites=8,n_up=4,n_dn=4,t=1,U=4,bc=open", 96),
                                     ("anderson3d:L=10,W=4,seed=3", 64),
                                     ("chain:n=300", 20)])
def test_rayleigh_ritz_matches_oracle(fd, ctx, spec, ns):
    import torch
    csr = mat.build(spec)
    D = len(csr[0]) - 1
    V0, _ = np.linalg.qr(fd_inputs.random_block(D, ns, 5))
    A = fd.fd_build_matrix(ctx, spec)
    V = _t(V0)
    AV = torch.empty_like(V)
    th, rho = fd.fd_rayleigh_ritz(ctx, A, V, AV)
    tho, Vo, Wo, rhoo = rayleigh_ritz.rayleigh_ritz(mat.to_scipy(csr), V0)
    normH = np.abs(tho).max()
    assert np.abs(th - tho).max() <= 1e-12 * normH
    assert np.abs(rho - rhoo).max() <= 1e-11 * normH
    # Ritz vectors: equal up to sign where the Ritz values are separated
    Vg = V.cpu().numpy()
    gap = np.minimum(np.abs(np.diff(tho, prepend=-np.inf)), np.abs(np.diff(tho, append=np.inf)))
    ok = gap > 1e-6 * normH
    d = np.abs(np.abs(np.sum(Vg * Vo, axis=0)) - 1.0)
    assert np.all(d[ok] < 1e-9)


def test_rr_exact_invariant_subspace(fd, ctx):
    import torch
    spec = "hubbard:n_sites=6,n_up=3,n_dn=3,t=1,U=4,bc=open"
    csr = mat.build(spec)
    ev, X = np.linalg.eigh(mat.to_scipy(csr).toarray())
    sub = X[:, 100:132] @ np.linalg.qr(np.random.default_rng(1).standard_normal((32, 32)))[0]
    A = fd.fd_build_matrix(ctx, spec)
    V = _t(sub)
    th, rho = fd.fd_rayleigh_ritz(ctx, A, V, torch.empty_like(V))
    assert np.abs(th - ev[100:132]).max() < 1e-12
    assert rho.max() < 1e-12


@pytest.mark.parametrize("spec", ["hubbard:n_sites=8,n_up=4,n_dn=4,t=1,U=4,bc=open",
                                  "anderson3d:L=12,W=2,seed=1", "chain:n=500"])
def test_spectral_bounds_match_oracle(fd, ctx, spec):
    csr = mat.build(spec)
    A = fd.fd_build_matrix(ctx, spec)
    lo, hi = fd.fd_spectral_bounds(ctx, A, 20, 0)
    olo, ohi = lanczos.inclusion_interval(csr, 20, 0)
    assert lo == pytest.approx(olo, abs=1e-9 * max(1, abs(olo)))
    assert hi == pytest.approx(ohi, abs=1e-9 * max(1, abs(ohi)))
    if len(csr[0]) <= 5001:
        ev = np.linalg.eigvalsh(mat.to_scipy(csr).toarray())
        assert lo <= ev[0] and hi >= ev[-1]


@pytest.mark.parametrize("R", [4, 16, 64])
def test_kpm_moments_match_oracle(fd, ctx, R):
    spec = "anderson3d:L=10,W=3,seed=2"
    csr = mat.build(spec)
    A = fd.fd_build_matrix(ctx, spec)
    alpha, beta = ch.scale_params(-8.0, 8.0)
    mu = fd.fd_kpm_moments(ctx, A, 48, R, 7, alpha, beta)
    muo = kpm.kpm_moments(mat.to_scipy(csr), 48, R, 7, alpha, beta)
    assert np.abs(mu - muo).max() < 1e-11
