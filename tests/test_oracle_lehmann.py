"""Pins of the oracle's Lehmann bounds: the enclosure holds for any subspace,
is exact on invariant subspaces, matches the one-vector closed form, and
tightens monotonically on nested subspaces."""
import numpy as np
import pytest

from oracle import lehmann
from oracle import matrices as mat


def _sym(D, seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((D, D))
    return 0.5 * (M + M.T)


def _nearest(lam, rho):
    below = np.sort(lam[lam < rho])[::-1]
    above = np.sort(lam[lam > rho])
    return below, above


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("m", [1, 4, 12])
def test_bounds_enclose_for_any_subspace(seed, m):
    D = 60
    A = _sym(D, seed)
    lam = np.linalg.eigvalsh(A)
    rng = np.random.default_rng(100 + seed)
    rho = float(rng.uniform(lam[5], lam[-6]))
    # a random subspace, and one filtered towards rho (the situation of FD)
    for V in (rng.standard_normal((D, m)),
              np.linalg.solve(A - rho * np.eye(D), np.linalg.solve(A - rho * np.eye(D),
                                                                      rng.standard_normal((D, m))))):
        below, above = lehmann.lehmann_bounds(A, V, rho)
        lb, la = _nearest(lam, rho)
        tol = 1e-9 * np.abs(lam).max()
        for k in range(min(len(below), len(lb))):
            assert lb[k] >= below[k] - tol
        for k in range(min(len(above), len(la))):
            assert la[k] <= above[k] + tol
        assert len(below) + len(above) == m


def test_exact_on_invariant_subspace():
    A = mat.to_scipy(mat.build("hubbard:n_sites=6,n_up=3,n_dn=2,t=1,U=4,bc=open")).toarray()
    lam, X = np.linalg.eigh(A)
    rho = 1.2345
    idx = np.argsort(np.abs(lam - rho))[:10]
    below, above = lehmann.lehmann_bounds(A, X[:, idx], rho)
    lb, la = _nearest(lam[idx], rho)
    scale = np.abs(lam).max()
    assert np.allclose(below, lb, atol=1e-11 * scale, rtol=0)
    assert np.allclose(above, la, atol=1e-11 * scale, rtol=0)


def test_one_vector_closed_form():
    d = np.array([-3.0, -1.0, 0.5, 2.0, 4.0])
    A = np.diag(d)
    v = np.array([0.3, -0.2, 0.9, 0.1, 0.05])
    rho = 0.0
    mu = np.sum((d - rho) * v * v) / np.sum((d - rho) ** 2 * v * v)
    below, above = lehmann.lehmann_bounds(A, v[:, None], rho)
    got = below[0] if mu < 0 else above[0]
    assert got == pytest.approx(rho + 1.0 / mu, rel=1e-14)
    assert len(below) + len(above) == 1
    # mu > 0 here: an upper bound for the nearest eigenvalue above rho (0.5)
    assert mu > 0 and above[0] >= 0.5


def test_nested_subspaces_tighten():
    D = 80
    A = _sym(D, 7)
    rng = np.random.default_rng(8)
    rho = 0.1
    V = rng.standard_normal((D, 20))
    b1, a1 = lehmann.lehmann_bounds(A, V[:, :8], rho)
    b2, a2 = lehmann.lehmann_bounds(A, V, rho)
    tol = 1e-10
    for k in range(min(len(b1), len(b2))):
        assert b2[k] >= b1[k] - tol   # lower bounds below rho only rise
    for k in range(min(len(a1), len(a2))):
        assert a2[k] <= a1[k] + tol   # upper bounds above rho only fall


# ---------------------------------------------------------------- interval rule
def _count(lam, lo, hi):
    return int(np.sum((lam >= lo) & (lam <= hi)))


@pytest.mark.parametrize("seed", range(5))
def test_target_interval_holds_n_target_eigenvalues_when_bounds_are_used(seed):
    # on a subspace filtered towards tau the Lehmann bounds are informative:
    # each target edge is a Lehmann bound, so the target interval holds at
    # least k_b + k_a eigenvalues; always search contains target contains tau
    D, ns, nt = 120, 16, 6
    A = _sym(D, 20 + seed)
    lam = np.linalg.eigvalsh(A)
    rng = np.random.default_rng(30 + seed)
    tau = float(rng.uniform(lam[30], lam[-30]))
    B = np.linalg.inv(A - tau * np.eye(D))
    for k, V in enumerate((rng.standard_normal((D, ns)), B @ B @ B @ rng.standard_normal((D, ns)))):
        Q, _ = np.linalg.qr(V)
        theta = np.linalg.eigvalsh(Q.T @ A @ Q)
        below, above = lehmann.lehmann_bounds(A, Q, tau)
        (t_l, t_r), (s_l, s_r) = lehmann.lehmann_intervals(below, above, theta, tau, nt, ns)
        kb, ka = lehmann.nearest_counts(theta, tau, nt)
        assert s_l <= t_l <= t_r <= s_r
        used_l = kb > 0 and t_l == below[kb - 1]
        used_r = ka > 0 and t_r == above[ka - 1]
        if k == 1:
            assert used_l and used_r
        if used_l and used_r:
            assert _count(lam, t_l, t_r) >= kb + ka


def test_loose_bounds_fall_back_to_the_ritz_hull():
    # a random subspace: bounds far outside the search hull, Ritz hull kept
    D, ns, nt = 200, 12, 4
    A = _sym(D, 41)
    rng = np.random.default_rng(42)
    Q, _ = np.linalg.qr(rng.standard_normal((D, ns)))
    theta = np.linalg.eigvalsh(Q.T @ A @ Q)
    tau = float(np.median(theta))
    below, above = lehmann.lehmann_bounds(A, Q, tau)
    (t_l, t_r), (s_l, s_r) = lehmann.lehmann_intervals(below, above, theta, tau, nt, ns)
    near = theta[np.lexsort((theta, np.abs(theta - tau)))]
    kb, ka = lehmann.nearest_counts(theta, tau, nt)
    if not (s_l < below[kb - 1]):
        assert t_l == near[:nt].min()
    if not (above[ka - 1] < s_r):
        assert t_r == near[:nt].max()


def test_intervals_on_invariant_subspace_are_eigenvalue_hulls():
    A = mat.to_scipy(mat.build("hubbard:n_sites=6,n_up=3,n_dn=3,t=1,U=4,bc=open")).toarray()
    lam, X = np.linalg.eigh(A)
    tau = 8.05
    idx = np.sort(np.argsort(np.abs(lam - tau), kind="stable")[:16])
    theta = lam[idx]
    below, above = lehmann.lehmann_bounds(A, X[:, idx], tau)
    (t_l, t_r), (s_l, s_r) = lehmann.lehmann_intervals(below, above, theta, tau, 5, 16)
    near = theta[np.lexsort((theta, np.abs(theta - tau)))]
    scale = np.abs(lam).max()
    assert t_l == pytest.approx(near[:5].min(), abs=1e-11 * scale)
    assert t_r == pytest.approx(near[:5].max(), abs=1e-11 * scale)
    assert s_l == pytest.approx(near[:12].min(), abs=1e-11 * scale)
    assert s_r == pytest.approx(near[:12].max(), abs=1e-11 * scale)


def test_nearest_counts():
    assert lehmann.nearest_counts([-3.0, -1.0, 0.5, 2.0], 0.0, 2) == (1, 1)
    assert lehmann.nearest_counts([-0.1, 0.1, 0.2], 0.0, 2) == (1, 1)   # tie: smaller first
    assert lehmann.nearest_counts([0.0, 1.0], 0.0, 2) == (0, 1)          # at tau: neither side


def test_fd_with_lehmann_intervals_matches_dense():
    # the 8-site Hubbard chain (config 1) with the Lehmann interval rule
    csr = mat.build("hubbard:n_sites=8,n_up=4,n_dn=4,t=1,U=4,bc=open")
    from oracle import fd
    lam = np.linalg.eigvalsh(mat.to_scipy(csr).toarray())
    r = fd.fd_solve(csr, -0.5, 0.5, 20, 32, 100, 1e-9, intervals="lehmann")
    want = np.sort(lam[np.lexsort((lam, np.abs(lam)))[:20]])
    assert r.converged and r.resid.max() <= 1e-9
    assert np.abs(r.theta - want).max() <= 1e-10 * np.abs(lam).max()
