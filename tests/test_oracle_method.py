"""Pins of the oracle's filter, Lanczos interval, CholQR, Rayleigh-Ritz, KPM and FD loop."""
import os

import numpy as np
import pytest
import scipy.integrate as si
import scipy.linalg as sla

import fd_inputs
from oracle import chebyshev as ch
from oracle import fd, kpm, lanczos, ortho, rayleigh_ritz
from oracle import matrices as mat

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Chebyshev / Jackson

def test_jackson_kernel_properties():
    for n in (2, 10, 100, 501):
        g = ch.jackson(n)
        assert g[0] == pytest.approx(1.0, abs=1e-14)
        assert np.all(np.diff(g) < 0) and g[-1] > 0


def test_jackson_kernel_closed_forms():
    # g_1 = cos(pi/(N+1)), N = n + 1; and every g_k is the normalised
    # autocorrelation at lag k of the sine window a_v = sin(pi v/(N+1)),
    # v = 1..N, whose squared Fourier sum is the (positive) Jackson kernel.
    # Either fails for N off by one.
    for n in (2, 10, 100, 501):
        N = n + 1
        g = ch.jackson(n)
        assert g[1] == pytest.approx(np.cos(np.pi / (N + 1)), abs=1e-15)
        a = np.sin(np.pi * np.arange(1, N + 1) / (N + 1))
        ac = np.array([a[:N - k] @ a[k:] for k in range(n + 1)]) / (a @ a)
        assert np.abs(g - ac).max() < 1e-13


def test_window_coeffs_match_quadrature():
    x_l, x_r, n = -0.3, 0.45, 12
    c = ch.window_coeffs(x_l, x_r, n)
    for k in range(n + 1):
        f = lambda t: np.cos(k * t)
        val = si.quad(f, np.arccos(x_r), np.arccos(x_l), epsabs=1e-14)[0] / np.pi
        assert c[k] == pytest.approx(val * (1 if k == 0 else 2), abs=1e-13)


def test_cheb_eval_matches_numpy_chebval():
    mu = np.random.default_rng(0).standard_normal(40)
    x = np.linspace(-1, 1, 101)
    assert np.abs(ch.cheb_eval(mu, x) - np.polynomial.chebyshev.chebval(x, mu)).max() < 1e-12


def test_jackson_filter_is_nonnegative_and_peaks_in_window():
    mu = ch.filter_coeffs(-0.2, 0.1, 300)
    x = np.linspace(-1, 1, 4001)
    p = ch.cheb_eval(mu, x)
    assert p.min() > -1e-12
    assert ch.cheb_eval(mu, -0.05) == pytest.approx(1.0)
    assert p[np.abs(x + 0.05) > 0.3].max() < 1e-4 and p[np.abs(x + 0.05) > 0.7].max() < 1e-6


def test_filter_on_diagonal_matrix_scales_rows():
    lam = np.linspace(-3, 5, 200)
    A = mat.to_scipy(mat.diagonal(lam))
    alpha, beta = ch.scale_params(-3.5, 5.5)
    mu = ch.filter_coeffs(alpha * 0.5 + beta, alpha * 1.5 + beta, 60)
    V = fd_inputs.random_block(200, 5, 1)
    out = ch.cheb_filter(A, V, mu, alpha, beta)
    expect = ch.cheb_eval(mu, alpha * lam + beta)[:, None] * V
    assert np.abs(out - expect).max() < 1e-12


def test_filter_on_chain_eigenvectors():
    n = 64
    A = mat.to_scipy(mat.chain(n))
    k = np.arange(1, n + 1)
    j = np.arange(1, n + 1)
    X = np.sqrt(2 / (n + 1)) * np.sin(np.pi * np.outer(j, k) / (n + 1))   # columns: eigenvectors
    lam = -2 * np.cos(k * np.pi / (n + 1))
    alpha, beta = ch.scale_params(-2.1, 2.1)
    mu = ch.filter_coeffs(-0.3, 0.3, 40)
    out = ch.cheb_filter(A, X, mu, alpha, beta)
    assert np.abs(out - X * ch.cheb_eval(mu, alpha * lam + beta)[None, :]).max() < 1e-12


def test_filter_rejects_degree_below_two():
    with pytest.raises(ValueError):
        ch.cheb_filter(mat.to_scipy(mat.chain(5)), np.ones((5, 1)), np.ones(2), 1.0, 0.0)


# ---------------------------------------------------------------- spectral interval

@pytest.mark.parametrize("spec", ["hubbard:n_sites=6,n_up=3,n_dn=3,t=1,U=4,bc=open",
                                  "anderson3d:L=6,W=4,seed=2", "chain:n=300"])
def test_inclusion_interval_contains_spectrum(spec):
    csr = mat.build(spec)
    ev = np.linalg.eigvalsh(mat.to_scipy(csr).toarray())
    lo, hi = lanczos.inclusion_interval(csr, 20, 0)
    assert lo <= ev[0] and hi >= ev[-1]
    g = lanczos.gershgorin(csr)
    assert g[0] <= lo and hi <= g[1]


def test_gershgorin_brute_force():
    csr = fd_inputs.random_symmetric_csr(50, 4, 3)
    A = mat.to_scipy(csr).toarray()
    r = np.abs(A).sum(1) - np.abs(np.diag(A))
    assert lanczos.gershgorin(csr) == pytest.approx(((np.diag(A) - r).min(), (np.diag(A) + r).max()))


# ---------------------------------------------------------------- CholQR2

def test_cholqr2_orthonormal_and_matches_lapack_r():
    V = fd_inputs.random_block(3000, 40, 5) @ np.diag(np.logspace(0, 5, 40))
    Q, R, passes = ortho.cholqr2(V)
    assert passes == 2
    assert np.abs(Q.T @ Q - np.eye(40)).max() < 1e-14
    assert np.abs(Q @ R - V).max() < 1e-12 * np.abs(V).max()
    Rl = np.linalg.qr(V, mode="r")
    s = np.sign(np.diag(Rl))
    assert np.abs(s[:, None] * Rl - R).max() < 1e-10 * np.abs(R).max()


def test_cholqr_shifted_fallback_on_ill_conditioned_block():
    rng = np.random.default_rng(2)
    U, _ = np.linalg.qr(rng.standard_normal((2000, 30)))
    W, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    V = U @ np.diag(np.logspace(0, -12, 30)) @ W          # cond 1e12: plain Cholesky fails
    with pytest.raises(ortho.Breakdown):
        ortho.cholqr_pass(V.copy(), allow_shift=False)
    Q, R, passes = ortho.cholqr2(V)
    assert passes == 3
    assert np.abs(Q.T @ Q - np.eye(30)).max() < 1e-13


def test_cholqr_nan_breaks_down():
    V = fd_inputs.random_block(100, 4, 1)
    V[3, 2] = np.nan
    with pytest.raises(ortho.Breakdown):
        ortho.cholqr2(V)


# ---------------------------------------------------------------- Rayleigh-Ritz

def test_rayleigh_ritz_exact_invariant_subspace():
    csr = mat.hubbard(6, 3, 3, 1.0, 4.0, "open")
    A = mat.to_scipy(csr)
    ev, X = np.linalg.eigh(A.toarray())
    sub = X[:, 100:130] @ np.linalg.qr(np.random.default_rng(1).standard_normal((30, 30)))[0]
    theta, V, W, rho = rayleigh_ritz.rayleigh_ritz(A, sub)
    assert np.abs(theta - ev[100:130]).max() < 1e-12
    assert rho.max() < 1e-12


def test_rayleigh_ritz_residual_definition():
    A = mat.to_scipy(mat.chain(80))
    V, _ = np.linalg.qr(fd_inputs.random_block(80, 6, 4))
    theta, Vr, W, rho = rayleigh_ritz.rayleigh_ritz(A, V)
    for i in range(6):
        assert rho[i] == pytest.approx(np.linalg.norm(A @ Vr[:, i] - theta[i] * Vr[:, i]), rel=1e-12)
    # Ritz values interlace the spectrum
    ev = np.linalg.eigvalsh(A.toarray())
    assert theta.min() >= ev[0] - 1e-12 and theta.max() <= ev[-1] + 1e-12


# ---------------------------------------------------------------- KPM

def test_kpm_moments_exact_trace_and_count():
    csr = mat.anderson3d(6, 2.0, 3)
    A = mat.to_scipy(csr)
    D = A.shape[0]
    ev = np.linalg.eigvalsh(A.toarray())
    alpha, beta = ch.scale_params(-8.0, 8.0)
    x = alpha * ev + beta
    M = 48
    exact = np.array([np.mean(np.cos(m * np.arccos(x))) for m in range(M)])
    R = 64
    mu = kpm.kpm_moments(A, M, R, 1, alpha, beta)
    # stochastic trace: error ~ sqrt(2 / (R D)) per moment
    assert np.abs(mu - exact).max() < 6 * np.sqrt(2.0 / (R * D))
    cnt_exact = kpm.eigen_count(exact, D, alpha * -1 + beta, alpha * 1 + beta)
    true = np.sum((ev >= -1) & (ev <= 1))
    assert abs(cnt_exact - true) < 0.15 * true


def test_kpm_clean_lattice_moments_closed_form():
    # 1D chain with periodic... use the open chain: T_m moments are means over its cos levels
    A = mat.to_scipy(mat.chain(200))
    k = np.arange(1, 201)
    lam = -2 * np.cos(k * np.pi / 201)
    alpha, beta = ch.scale_params(-2.5, 2.5)
    exact = [np.mean(np.cos(m * np.arccos(alpha * lam + beta))) for m in range(20)]
    mu = kpm.kpm_moments(A, 20, 400, 9, alpha, beta)
    assert np.abs(mu - exact).max() < 6 * np.sqrt(2.0 / (400 * 200))


# ---------------------------------------------------------------- FD loop

def test_fig2_experiment():
    rows = [l.split() for l in open(os.path.join(GOLD, "fig2_experiment.txt")) if not l.startswith("#")]
    lam = -1 + 2 * np.arange(1000) / 999
    csr = mat.diagonal(lam)
    tgt = np.sort(np.argsort(np.abs(lam))[:10])
    for r in rows:
        search, conv = (float(r[0]), float(r[1])), r[2] == "yes"
        _, hist = fd.fd_fixed_intervals(csr, (-0.01, 0.01), search, 10, 20, 9)
        ok = [np.sum(X[tgt, :] ** 2, axis=1).min() > 1 - 1e-7 for _, X, _ in hist]
        if conv:
            first = ok.index(True) + 1
            assert first <= int(r[3])          # within the paper's eight applications
        else:
            assert not any(ok)


def test_fd_config1_matches_dense_eigensolver():
    csr = mat.hubbard(8, 4, 4, 1.0, 4.0, "open")
    r = fd.fd_solve(csr, -0.5, 0.5, 20, 32, 100, 1e-9)
    assert r.converged and r.resid.max() <= 1e-9
    A = mat.to_scipy(csr).toarray()
    ev = np.linalg.eigvalsh(A)
    want = np.sort(ev[np.lexsort((ev, np.abs(ev)))[:20]])
    normH = np.abs(ev).max()
    assert np.abs(r.theta - want).max() <= 1e-10 * normH
    # eigenvectors: residual certificate with the dense matrix
    assert np.abs(A @ r.X - r.X * r.theta[None, :]).max() < 1e-9


def test_cholqr_reports_a_block_it_cannot_orthonormalise():
    # condition 1e12: the shifted third pass recovers an orthonormal basis;
    # condition 1e20: no pass can, and the last pass's R shows it (Breakdown
    # instead of a basis that is not orthonormal)
    rng = np.random.default_rng(2)
    U, _ = np.linalg.qr(rng.standard_normal((4000, 32)))
    W, _ = np.linalg.qr(rng.standard_normal((32, 32)))
    Q, R, p = ortho.cholqr2(U @ np.diag(np.logspace(0, -12, 32)) @ W)
    assert p == 3 and np.abs(Q.T @ Q - np.eye(32)).max() < 1e-13
    with pytest.raises(ortho.Breakdown):
        ortho.cholqr2(U @ np.diag(np.logspace(0, -20, 32)) @ W)


def test_fd_recovers_from_an_inclusion_interval_that_misses_the_spectrum_ends(monkeypatch):
    # [-4, 19] misses both ends of the 8-site chain's [-4.2358, 20.2358]: the
    # filter amplifies the eigenvectors beyond, the Ritz step finds them and the
    # interval moves out past them; the wanted eigenvalues still come out
    csr = mat.build("hubbard:n_sites=8,n_up=4,n_dn=4,t=1,U=4,bc=open")
    lam = np.linalg.eigvalsh(mat.to_scipy(csr).toarray())
    monkeypatch.setattr(fd.lanczos, "inclusion_interval", lambda csr, m=20, seed=0: (-4.0, 19.0))
    r = fd.fd_solve(csr, -0.5, 0.5, 20, 32, 100, 1e-9)
    want = np.sort(lam[np.lexsort((lam, np.abs(lam)))[:20]])
    assert r.converged and r.resid.max() <= 1e-9
    assert r.bounds[0] <= lam[0] and r.bounds[1] >= lam[-1]
    assert np.abs(r.theta - want).max() <= 1e-10 * np.abs(lam).max()
