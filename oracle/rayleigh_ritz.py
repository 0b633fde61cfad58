"""Rayleigh-Ritz step and residual norms (Sec. 2, Alg. 1: after each
orthogonalisation one more SpMV yields the Ritz values; the convergence test
uses the residual rho = ||A v - lambda v||_2).

For an orthonormal D x N_s block V:
    W = A V ;  H = V^T W, symmetrised (H + H^T)/2 ;  H = Q diag(theta) Q^T
    (theta ascending) ;  V <- V Q ;  W <- W Q ;  rho_i = ||W_i - theta_i V_i||_2 .
"""
import numpy as np


def rayleigh_ritz(A, V):
    W = A @ V
    H = V.T @ W
    H = 0.5 * (H + H.T)
    theta, Q = np.linalg.eigh(H)
    V = V @ Q
    W = W @ Q
    rho = np.linalg.norm(W - V * theta[None, :], axis=0)
    return theta, V, W, rho
