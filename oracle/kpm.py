"""Kernel-polynomial density-of-states moments (Sec. 4.1: the DOS of Figs. 6-7
is computed with KPM; D * int_a^b rho = number of eigenvalues in [a, b]).

Plain definition: with R random vectors r_j (entries from the normal-like
KPM stream, element (i, j) at counter i*R + j) and A~ = alpha A + beta I,

    mu_m = (1 / (R D)) sum_j r_j^T T_m(A~) r_j ,   m = 0 .. M-1,

evaluated with the three-term recurrence T_{m+1} = 2 A~ T_m - T_{m-1}.
The Jackson-damped DOS gives the eigenvalue count in [a, b] as
    D * sum_m g_m mu_m c_m([x_a, x_b])
with c_m the window coefficients of oracle.chebyshev.
"""
import numpy as np

from . import chebyshev, splitmix


def random_vectors(D, R, seed):
    e = np.arange(D * R, dtype=np.int64)
    return splitmix.irwin_hall(seed, splitmix.STREAM_KPM, e).reshape(D, R)


def kpm_moments(A, n_moments, n_random, seed, alpha, beta):
    D = A.shape[0]
    r = random_vectors(D, n_random, seed)
    mu = np.zeros(n_moments)
    x_prev = r
    mu[0] = np.sum(r * x_prev)
    if n_moments > 1:
        x = alpha * (A @ r) + beta * r
        mu[1] = np.sum(r * x)
        for m in range(2, n_moments):
            x_next = 2.0 * (alpha * (A @ x) + beta * x) - x_prev
            mu[m] = np.sum(r * x_next)
            x_prev, x = x, x_next
    return mu / (n_random * D)


def eigen_count(mu, D, x_a, x_b):
    n = len(mu) - 1
    return D * float(np.sum(chebyshev.jackson(n) * mu * chebyshev.window_coeffs(x_a, x_b, n)))
