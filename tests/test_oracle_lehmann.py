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
