"""Spectral inclusion interval from a few Lanczos steps (Sec. 2, Alg. 1 steps 1-2).

m Lanczos steps with full reorthogonalisation (cheap at m = 20) from the start
vector of the Lanczos stream give the tridiagonal T_m, its extreme eigenpairs
(theta_min, s_min), (theta_max, s_max) and the last off-diagonal beta_m.  The
paper asks for an inclusion interval but states no margin.  Reading used here:
each extreme Ritz value is pushed outwards by its Lanczos residual bound
|beta_m e_m^T s| plus 1% of the Ritz span, and the result is clipped to the
Gershgorin interval, which is a guaranteed inclusion interval:

    lam_l = max(g_l, theta_min - |beta_m s_min[m]| - 0.01 w)
    lam_r = min(g_r, theta_max + |beta_m s_max[m]| + 0.01 w),   w = theta_max - theta_min

(a Ritz value found outside [lam_l, lam_r] later widens the interval; see fd).
"""
import numpy as np

from . import splitmix


def lanczos_bounds(A, m=20, seed=0):
    D = A.shape[0]
    r = splitmix.irwin_hall(seed, splitmix.STREAM_LANCZOS, np.arange(D))
    Q = np.zeros((D, min(m, D)))
    alphas, betas = [], []
    q = r / np.linalg.norm(r)
    beta = 0.0
    for j in range(min(m, D)):
        Q[:, j] = q
        w = A @ q
        a = q @ w
        alphas.append(a)
        for _ in range(2):                      # full reorthogonalisation, twice
            w = w - Q[:, :j + 1] @ (Q[:, :j + 1].T @ w)
        beta = np.linalg.norm(w)
        if j == min(m, D) - 1 or beta <= 1e-14 * max(1.0, abs(a)):
            break
        betas.append(beta)
        q = w / beta
    k = len(alphas)
    T = np.diag(alphas) + np.diag(betas[:k - 1], 1) + np.diag(betas[:k - 1], -1)
    th, S = np.linalg.eigh(T)
    tmin, tmax = th[0], th[-1]
    w = max(tmax - tmin, 1e-10 * max(1.0, abs(tmin), abs(tmax)))
    lo = tmin - abs(beta * S[-1, 0]) - 0.01 * w
    hi = tmax + abs(beta * S[-1, -1]) + 0.01 * w
    return lo, hi


def inclusion_interval(csr, m=20, seed=0):
    """Lanczos interval clipped to the Gershgorin interval."""
    from .matrices import to_scipy
    lo, hi = lanczos_bounds(to_scipy(csr), m, seed)
    g_l, g_r = gershgorin(csr)
    return max(g_l, lo), min(g_r, hi)


def gershgorin(csr):
    """[min_i (a_ii - r_i), max_i (a_ii + r_i)], r_i = sum_{j != i} |a_ij|."""
    rowptr, col, val = csr
    D = len(rowptr) - 1
    row = np.repeat(np.arange(D), np.diff(rowptr))
    diag = np.zeros(D)
    on = col == row
    np.add.at(diag, row[on], val[on])
    rad = np.zeros(D)
    np.add.at(rad, row[~on], np.abs(val[~on]))
    return float((diag - rad).min()), float((diag + rad).max())
