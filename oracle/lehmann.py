"""Lehmann bounds for the eigenvalues nearest a shift (Lehmann 1963; the paper
takes its target and search intervals from Lehmann intervals, Sec. 2).

Test infrastructure only: the CUDA library never imports this module.

The paper gives no formulas; this is Lehmann's theorem written out.  For a
symmetric A, a basis V (D x m, full rank) of the search space and a shift rho
that is no eigenvalue of A, let W = (A - rho) V.  Rayleigh-Ritz for
B = (A - rho)^-1 on span(W) has the projected matrices
    W^T B W = V^T (A - rho) V =: A1,     W^T W = ((A - rho) V)^T ((A - rho) V) =: A2,
so its Ritz values mu are the eigenvalues of the pencil A1 x = mu A2 x.  Ritz
values bound the extreme eigenvalues of B from inside, and the eigenvalues of B
are 1 / (lambda - rho).  Hence, with the negative mu in increasing order and
the positive mu in decreasing order,
    lambda_below[k] >= rho + 1 / mu_neg[k]   (the k-th eigenvalue below rho, nearest first)
    lambda_above[k] <= rho + 1 / mu_pos[k]   (the k-th eigenvalue above rho, nearest first)
for every k the subspace provides: guaranteed outer bounds, where the Ritz
values of A itself give bounds from the other side.
"""
import numpy as np
import scipy.linalg as sla


def lehmann_bounds(A, V, rho):
    """(below, above): lower bounds of the eigenvalues of A below rho and upper
    bounds of those above rho, nearest to rho first.  A: dense or sparse
    symmetric (D x D), V: D x m basis, rho: float, no eigenvalue of A."""
    V = np.asarray(V, dtype=np.float64)
    W = A @ V - rho * V
    A1 = V.T @ W
    A1 = 0.5 * (A1 + A1.T)
    A2 = W.T @ W
    A2 = 0.5 * (A2 + A2.T)
    mu = sla.eigh(A1, A2, eigvals_only=True)
    neg = np.sort(mu[mu < 0])          # most negative first: nearest below rho
    pos = np.sort(mu[mu > 0])[::-1]    # largest first: nearest above rho
    return rho + 1.0 / neg, rho + 1.0 / pos
