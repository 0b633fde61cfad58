"""Orthonormalisation of the search block (Sec. 2, Alg. 1 step 3).

The paper orthogonalises with TSQR and names SVQB as the alternative; this
build uses Cholesky-QR twice (CholQR2), falling back to the shifted Cholesky-QR
of Fukaya et al. (SIAM J. Sci. Comput. 2020) when a Cholesky factorisation
breaks down.  One pass:

    G = V^T V ;  G = R^T R (Cholesky, R upper) ;  V <- V R^-1 .

If the Cholesky of G meets a pivot that is not > 0 (or not finite), the pass
is redone on G + s I with s = 11 (D N_s + N_s (N_s + 1)) u tr(G), u = 2^-53
(tr(G) >= ||G||_2 stands in for ||V||_2^2), and one extra plain pass is added:
two passes normally, three once a shift was used.
"""
import numpy as np
import scipy.linalg as sla

U64 = 2.0 ** -53


class Breakdown(Exception):
    pass


def _chol_upper(G):
    try:
        R = np.linalg.cholesky(G).T
    except np.linalg.LinAlgError:
        return None
    if not np.all(np.isfinite(R)):
        return None
    return R


def cholqr_pass(V, allow_shift=True):
    """One (possibly shifted) Cholesky-QR pass; returns (V R^-1, R, shifted)."""
    D, ns = V.shape
    G = V.T @ V
    G = 0.5 * (G + G.T)
    R = _chol_upper(G)
    shifted = False
    if R is None:
        if not allow_shift or not np.all(np.isfinite(G)):
            raise Breakdown("Cholesky of the Gram matrix failed")
        s = 11.0 * (D * ns + ns * (ns + 1)) * U64 * np.trace(G)
        R = _chol_upper(G + s * np.eye(ns))
        if R is None:
            raise Breakdown("shifted Cholesky failed")
        shifted = True
    Q = sla.solve_triangular(R, V.T, trans="T", lower=False).T
    return Q, R, shifted


def cholqr2(V):
    """Orthonormal basis Q of span(V) and R with V = Q R (CholQR2 / shifted CholQR3).

    The last pass factors the Gram matrix of a block that the earlier passes
    have already orthonormalised, so its R is close to the identity.  A
    diagonal entry off by more than a factor 4 means those passes failed (the
    block is numerically rank deficient beyond what the shifted passes
    recover, e.g. a filter that amplified some directions by 1e16 over the
    rest): Breakdown, rather than a block that is not orthonormal."""
    Q = np.array(V, dtype=np.float64, copy=True)
    Rtot = np.eye(Q.shape[1])
    passes, any_shift = 0, False
    R = None
    while passes < 2 or (any_shift and passes < 3):
        Q, R, sh = cholqr_pass(Q)
        any_shift |= sh
        Rtot = R @ Rtot
        passes += 1
    d = np.abs(np.diag(R))
    if not np.all((d > 0.25) & (d < 4.0)):
        raise Breakdown("the search block is numerically rank deficient: orthonormalisation failed")
    return Q, Rtot, passes
