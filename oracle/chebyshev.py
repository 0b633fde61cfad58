"""Chebyshev filter polynomial and its evaluation (Sec. 2, Alg. 2).

The filter is p(x) = sum_{k=0..n} mu_k T_k(x) on the scaled matrix
A~ = alpha A + beta I, where alpha, beta map the spectral inclusion interval
[lam_l, lam_r] onto [-1, 1] (Sec. 2).  The coefficients are the Chebyshev
expansion of the indicator of a window [x_l, x_r] (Sec. 2 builds the filter
from the Chebyshev series of a window function), damped by the Jackson kernel (the kernel
polynomial method the paper cites for KPM, Sec. 4.1):

    theta = arccos(x)
    c_0 = (theta_l - theta_r) / pi
    c_k = 2 (sin k theta_l - sin k theta_r) / (k pi)
    g_k = [(N - k + 1) cos(pi k/(N+1)) + sin(pi k/(N+1)) cot(pi/(N+1))] / (N+1),  N = n + 1
    mu_k = g_k c_k, scaled so that p at the window centre equals 1.

Alg. 2 (reconstructed from Sec. 2 and the kappa = 5 count of Eq. EstimateT:
W1 is read once, W2 and V are read and written in the fused step):
    W2 <- V ; W1 <- A~ V ; V <- mu_0 W2 + mu_1 W1
    for k = 2..n:  W2 <- 2 A~ W1 - W2 ;  V <- V + mu_k W2 ;  swap(W1, W2)
"""
import numpy as np


def scale_params(lam_l, lam_r):
    """alpha, beta with alpha*lam + beta mapping [lam_l, lam_r] -> [-1, 1]."""
    w = lam_r - lam_l
    return 2.0 / w, -(lam_r + lam_l) / w


def jackson(n):
    N = n + 1
    k = np.arange(n + 1, dtype=np.float64)
    a = np.pi / (N + 1)
    return ((N - k + 1) * np.cos(a * k) + np.sin(a * k) / np.tan(a)) / (N + 1)


def window_coeffs(x_l, x_r, n):
    """Chebyshev coefficients of the indicator of [x_l, x_r] (within [-1, 1])."""
    x_l, x_r = max(-1.0, x_l), min(1.0, x_r)
    th_l, th_r = np.arccos(x_l), np.arccos(x_r)
    k = np.arange(1, n + 1, dtype=np.float64)
    c = np.empty(n + 1)
    c[0] = (th_l - th_r) / np.pi
    c[1:] = 2.0 * (np.sin(k * th_l) - np.sin(k * th_r)) / (k * np.pi)
    return c


def cheb_eval(mu, x):
    """p(x) = sum mu_k T_k(x) for scalar or array x in [-1, 1] (T_k(cos t) = cos k t)."""
    x = np.clip(np.asarray(x, dtype=np.float64), -1.0, 1.0)
    th = np.arccos(x)
    k = np.arange(len(mu))
    return np.cos(np.multiply.outer(th, k)) @ mu


def filter_coeffs(x_l, x_r, n):
    """Jackson-damped window coefficients, normalised to p(window centre) = 1."""
    mu = jackson(n) * window_coeffs(x_l, x_r, n)
    xc = 0.5 * (max(-1.0, x_l) + min(1.0, x_r))
    return mu / cheb_eval(mu, xc)


def cheb_filter(A, V, mu, alpha, beta):
    """V -> p(A~) V with Alg. 2 (A is a scipy CSR matrix; V a D x m array, copied)."""
    n = len(mu) - 1
    if n < 2:
        raise ValueError("Alg. 2 takes a Chebyshev expansion of degree n >= 2")
    V = np.array(V, dtype=np.float64, copy=True)

    def At(X):
        return alpha * (A @ X) + beta * X

    W2 = V.copy()
    W1 = At(V)
    V = mu[0] * W2 + mu[1] * W1
    for k in range(2, n + 1):
        W2 = 2.0 * At(W1) - W2
        V = V + mu[k] * W2
        W1, W2 = W2, W1
    return V


def cheb_step(A, W1, W2, V, mu_k, alpha, beta):
    """One fused generic step k >= 3 of Alg. 2, returned as (W2_new, V_new)."""
    W2n = 2.0 * (alpha * (A @ W1) + beta * W1) - W2
    return W2n, V + mu_k * W2n
