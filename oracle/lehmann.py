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


def nearest_counts(theta, tau, k):
    """Among the k Ritz values nearest tau (ties: the smaller value first), how
    many lie below tau and how many above it."""
    theta = np.asarray(theta, dtype=np.float64)
    sel = theta[np.lexsort((theta, np.abs(theta - tau)))[:k]]
    return int(np.sum(sel < tau)), int(np.sum(sel > tau))


def lehmann_intervals(below, above, theta, tau, n_target, ns):
    """Target and search intervals of the FD iteration from the Ritz values and
    the Lehmann bounds at the shift tau (the paper takes both intervals from
    Lehmann intervals, Sec. 2, and gives no rule; this is the reading the build
    uses).

    Search interval: the hull of the ceil(0.75 ns) Ritz values nearest tau
    (ties: smaller value first), the N_s eigenvalues the filter must keep.
    Target interval: with k_b, k_a the numbers of the n_target nearest Ritz
    values that lie below and above tau, each edge is the Lehmann bound
    below[k_b - 1] (above[k_a - 1]) when that bound lies inside the search
    interval, else the edge of the hull of the n_target nearest Ritz values.
    By Lehmann's theorem [below[k_b - 1], above[k_a - 1]] holds at least
    k_b + k_a eigenvalues, so once the bounds are informative the target
    interval provably holds the n_target wanted eigenvalues, also when a
    spurious Ritz value has taken the place of one of them; while the subspace
    is poor the bounds lie far outside and the Ritz hull is used.  Returns
    (target, search)."""
    theta = np.asarray(theta, dtype=np.float64)
    order = np.lexsort((theta, np.abs(theta - tau)))
    tgt = theta[order[:n_target]]
    srch = theta[order[:int(np.ceil(0.75 * ns))]]
    t_l, t_r = float(tgt.min()), float(tgt.max())
    s_l, s_r = float(min(srch.min(), t_l)), float(max(srch.max(), t_r))
    kb, ka = nearest_counts(theta, tau, n_target)
    if 0 < kb <= len(below) and s_l < below[kb - 1] <= t_l:
        t_l = float(below[kb - 1])
    if 0 < ka <= len(above) and t_r <= above[ka - 1] < s_r:
        t_r = float(above[ka - 1])
    return (t_l, t_r), (s_l, s_r)
