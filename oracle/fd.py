"""The FD outer loop (Sec. 2, Alg. 1), plain FP64.

Alg. 1 is printed as an image; its steps are read from Sec. 2:
  1-2. spectral inclusion interval [lam_l, lam_r] from a few Lanczos steps;
       alpha, beta map it onto [-1, 1];
  then N_s random search vectors, and repeat:
  3.   orthonormalise the search block (here CholQR2, oracle.ortho);
  4.   one more SpMMV gives the Ritz pairs and the residuals
       rho = ||A v - theta v||_2 (oracle.rayleigh_ritz);
  5.   stop when the N_t Ritz values nearest the target tau all have rho <= tol;
  6.   choose the target and search intervals and the polynomial degree;
  8.   apply the Chebyshev filter to all N_s vectors (oracle.chebyshev).

Readings where the paper is silent (intervals="ritz" replaces the paper's
Lehmann intervals by a Ritz-value heuristic; intervals="lehmann" takes them
from Lehmann bounds, oracle.lehmann.lehmann_intervals):
  * N_s = nb * ceil(4 N_t / nb) (Sec. 2: N_s/N_t ~ 4), at most D;
  * tau = (a + b)/2 for the window [a, b]; the N_t wanted pairs are those whose
    Ritz values are nearest tau (ties: smaller value first);
  * target interval [t_l, t_r] = hull of the N_t nearest Ritz values, search
    interval [s_l, s_r] = hull of the ceil(0.75 N_s) nearest ones;
  * filter window [t_l - m_l (t_l - s_l), t_r + m_r (s_r - t_r)] (m_l = m_r =
    1/2 by default), first window [a, b];
  * degree n = clamp(ceil(c_n pi / dtheta), n_min, n_max) where dtheta is the
    smaller Chebyshev-angle distance between a target edge and the matching
    search edge (c_n = 4 by default); n_min is the configured degree, which
    the first filter uses;
  * a Ritz value outside [lam_l, lam_r] moves that side out to the Ritz
    value plus 1% of the interval width (at least 2% beyond the old edge)
    before the next filter: outside [-1, 1] the Chebyshev polynomials grow
    like cosh(n acosh|x|), so a side left inside the spectrum lets the filter
    amplify the eigenvectors beyond it past what orthonormalisation can hold.
"""
import math
from dataclasses import dataclass, field

import numpy as np

from . import chebyshev, lanczos, lehmann, ortho, rayleigh_ritz, splitmix
from .matrices import to_scipy


@dataclass
class FDResult:
    converged: bool
    theta: np.ndarray            # N_t Ritz values, ascending
    X: np.ndarray                # D x N_t Ritz vectors (sign: largest |entry| > 0)
    resid: np.ndarray            # their residual norms
    iterations: int
    n_spmmv: int                 # SpMMVs counted per vector column block of width N_s
    bounds: tuple
    log: list = field(default_factory=list)


def default_ns(n_target, nb, D):
    return min(D, nb * math.ceil(4 * n_target / nb))


def start_block(D, ns, seed):
    e = np.arange(D * ns, dtype=np.int64)
    return splitmix.irwin_hall(seed, splitmix.STREAM_START, e).reshape(D, ns)


def nearest_order(theta, tau):
    return np.lexsort((theta, np.abs(theta - tau)))


def window_and_degree(target, search, alpha, beta, n_min, n_max, c_n=4.0, m_l=0.5, m_r=0.5):
    """Filter window and degree from a target interval and a search interval
    that contains it (step 6): window edges a fraction m of the way from the
    target edges to the search edges; degree c_n pi / dtheta, dtheta the
    smaller Chebyshev-angle distance between a target edge and its search
    edge, clamped to [n_min, n_max]."""
    (t_l, t_r), (s_l, s_r) = target, search
    s_l, s_r = min(s_l, t_l), max(s_r, t_r)
    th = lambda lam: math.acos(min(1.0, max(-1.0, alpha * lam + beta)))
    dth = min(th(s_l) - th(t_l), th(t_r) - th(s_r))
    n = n_max if dth <= 0.0 else int(math.ceil(c_n * math.pi / dth))
    n = max(n_min, min(n_max, n))
    return (t_l - m_l * (t_l - s_l), t_r + m_r * (s_r - t_r)), n


def choose_filter(theta, tau, n_target, ns, alpha, beta, n_min, n_max,
                  c_n=4.0, m_l=0.5, m_r=0.5):
    """Window [w_l, w_r] and degree n from the current Ritz values (step 6)."""
    order = nearest_order(theta, tau)
    tgt = theta[order[:n_target]]
    srch = theta[order[:math.ceil(0.75 * ns)]]
    t_l, t_r = tgt.min(), tgt.max()
    s_l, s_r = min(srch.min(), t_l), max(srch.max(), t_r)
    window, n = window_and_degree((t_l, t_r), (s_l, s_r), alpha, beta, n_min, n_max, c_n, m_l, m_r)
    return window, n, (t_l, t_r), (s_l, s_r)


def fd_solve(csr, a, b, n_target, nb, degree, tol, ns=None, max_outer=60, seed=0,
             lanczos_steps=20, n_max=100000, c_n=4.0, m_l=0.5, m_r=0.5, intervals="ritz"):
    """intervals: "ritz" (hulls of the nearest Ritz values) or "lehmann" (the
    Lehmann bounds at the shift tau, oracle.lehmann.lehmann_intervals)."""
    A = to_scipy(csr)
    D = A.shape[0]
    ns = ns or default_ns(n_target, nb, D)
    lam_l, lam_r = lanczos.inclusion_interval(csr, lanczos_steps, seed)
    delta = None
    tau = 0.5 * (a + b)
    V = start_block(D, ns, seed)
    window, n = (a, b), degree
    n_spmmv, log = 0, []
    theta = rho = None
    for it in range(max_outer):
        V, _, _ = ortho.cholqr2(V)
        theta, V, W, rho = rayleigh_ritz.rayleigh_ritz(A, V)
        n_spmmv += 1
        order = nearest_order(theta, tau)
        sel = order[:n_target]
        done = bool(np.all(rho[sel] <= tol))
        log.append(dict(it=it, degree=n, window=window, max_resid=float(rho[sel].max()),
                        n_conv=int((rho[sel] <= tol).sum())))
        if done:
            break
        if delta is None:
            delta = 0.01 * (lam_r - lam_l)
        if theta.min() < lam_l:
            lam_l = min(lam_l - 2 * delta, theta.min() - delta)
        if theta.max() > lam_r:
            lam_r = max(lam_r + 2 * delta, theta.max() + delta)
        alpha, beta = chebyshev.scale_params(lam_l, lam_r)
        if it > 0:
            if intervals == "lehmann":
                below, above = lehmann.lehmann_bounds(A, V, tau)
                tgt, srch = lehmann.lehmann_intervals(below, above, theta, tau, n_target, ns)
                window, n = window_and_degree(tgt, srch, alpha, beta, degree, n_max, c_n, m_l, m_r)
            else:
                window, n, _, _ = choose_filter(theta, tau, n_target, ns, alpha, beta, degree,
                                                n_max, c_n, m_l, m_r)
        mu = chebyshev.filter_coeffs(alpha * window[0] + beta, alpha * window[1] + beta, n)
        V = chebyshev.cheb_filter(A, V, mu, alpha, beta)
        n_spmmv += n
    sel = np.sort(nearest_order(theta, tau)[:n_target])
    X = V[:, sel].copy()
    idx = np.argmax(np.abs(X), axis=0)
    X *= np.sign(X[idx, np.arange(X.shape[1])])[None, :]
    return FDResult(bool(np.all(rho[sel] <= tol)), theta[sel], X, rho[sel], len(log),
                    n_spmmv, (lam_l, lam_r), log)


def fd_fixed_intervals(csr, target, search, n_t, ns, iterations, c_n=4.0, seed=0,
                       lanczos_steps=20, m=0.5):
    """FD with fixed target/search intervals (the set-up of Fig. 2).

    Returns, per filter application, the Ritz values and Ritz vectors nearest
    the target centre after orthonormalisation and Rayleigh-Ritz.
    """
    A = to_scipy(csr)
    D = A.shape[0]
    lam_l, lam_r = lanczos.inclusion_interval(csr, lanczos_steps, seed)
    alpha, beta = chebyshev.scale_params(lam_l, lam_r)
    tau = 0.5 * (target[0] + target[1])
    th = lambda lam: math.acos(min(1.0, max(-1.0, alpha * lam + beta)))
    dth = min(th(search[0]) - th(target[0]), th(target[1]) - th(search[1]))
    n = int(math.ceil(c_n * math.pi / dth))
    w = (target[0] - m * (target[0] - search[0]), target[1] + m * (search[1] - target[1]))
    mu = chebyshev.filter_coeffs(alpha * w[0] + beta, alpha * w[1] + beta, n)
    V = start_block(D, ns, seed)
    hist = []
    for _ in range(iterations):
        V = chebyshev.cheb_filter(A, V, mu, alpha, beta)
        V, _, _ = ortho.cholqr2(V)
        theta, V, W, rho = rayleigh_ritz.rayleigh_ritz(A, V)
        sel = np.sort(nearest_order(theta, tau)[:n_t])
        hist.append((theta[sel], V[:, sel], rho[sel]))
    return n, hist
