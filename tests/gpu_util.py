"""Helpers of the GPU parity tests: derived tolerances and oracle adapters."""
import numpy as np

U64 = 2.0 ** -53
U32 = 2.0 ** -24


def filter_tolerance(csr, mu, alpha, beta, V, u):
    """Per-column worst-case bound on |p(A~)V computed - exact| for Alg. 2.

    One fused step rounds a row dot product of at most nnz_row + 3 terms, so
    its error is at most (nnz_row + 3) u r max|x| with r the largest absolute
    row sum of A~ (Gershgorin).  A perturbation made at step j reaches step k
    multiplied by U_{k-j}(A~), |U_m| <= m + 1 on [-1, 1], so x_k carries at
    most (k^2/2 + k + 1) such errors, each with |x| <= ||V_c||_2 (|T_k| <= 1 on
    the spectrum).  Summing |mu_k| times that over k gives the bound; the FP32
    path adds the rounding of A and V to FP32, which the +3 already covers.
    """
    rowptr, col, val = csr
    D = len(rowptr) - 1
    nnz_row = int(np.diff(rowptr).max())
    row = np.repeat(np.arange(D), np.diff(rowptr))
    absrow = np.zeros(D)
    np.add.at(absrow, row, np.abs(alpha * val))
    r = max(1.0, float((absrow + abs(beta)).max()))
    k = np.arange(len(mu))
    growth = float(np.sum(np.abs(mu) * (k * k / 2.0 + k + 1.0)))
    colnorm = np.linalg.norm(np.asarray(V, dtype=np.float64), axis=0)
    return (nnz_row + 3) * u * r * growth * colnorm[None, :]
