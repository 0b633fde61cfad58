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


def local_filter(entries, samples, fetch, mu, alpha, beta):
    """Alg. 2 restricted to the rows it needs for the output rows `samples`.

    entries(rows) -> (row, col, val) COO entries of those rows of H (diagonal
    included); fetch(idx) -> the input block's rows idx (host array).  With
    S_0 = samples and S_{j+1} = S_j and its neighbours, x_k is computed on
    S_{n-k}, so only the n-hop neighbourhood of the samples is touched; the
    oracle's order of operations (Alg. 2) is kept.  Returns the exact output
    rows and m = sum_k |mu_k| m_k with m_0 = |x_0|, m_1 = M m_0,
    m_k = 2 M m_{k-1} + m_{k-2}, M = |alpha| |H| + |beta| I: a computed
    recurrence whose every step rounds at most g relative to its own
    magnitudes has error <= k g m_k at step k (induction on the recurrence),
    so (n + 1) g m bounds the whole filter's error."""
    import scipy.sparse as sp
    n = len(mu) - 1
    sets = [np.unique(np.asarray(samples, dtype=np.int64))]
    ops = []
    for _ in range(n):
        r, c, v = entries(sets[-1])
        nxt = np.union1d(sets[-1], c)
        pr = np.searchsorted(sets[-1], r)
        pc = np.searchsorted(nxt, c)
        ops.append((sp.csr_matrix((v, (pr, pc)), shape=(len(sets[-1]), len(nxt))),
                    np.searchsorted(nxt, sets[-1])))
        sets.append(nxt)
    x0 = np.asarray(fetch(sets[n]), dtype=np.float64)

    def apply(j, x, sign_abs=False):
        # Atilde (or M) on S_j from x on S_{j+1}
        op, own = ops[j]
        if sign_abs:
            return abs(alpha) * (abs(op) @ x) + abs(beta) * x[own]
        return alpha * (op @ x) + beta * x[own]

    def restrict(j_from, j_to, x):
        # x on S_{j_from} -> x on S_{j_to} (j_to < j_from)
        return x[np.searchsorted(sets[j_from], sets[j_to])]

    xs, ms = [x0], [np.abs(x0)]       # x_k lives on S_{n-k}
    for k in range(1, n + 1):
        j = n - k
        if k == 1:
            xs.append(apply(j, xs[0]))
            ms.append(apply(j, ms[0], True))
        else:
            xs.append(2.0 * apply(j, xs[k - 1]) - restrict(n - k + 2, j, xs[k - 2]))
            ms.append(2.0 * apply(j, ms[k - 1], True) + restrict(n - k + 2, j, ms[k - 2]))
    out = sum(mu[k] * restrict(n - k, 0, xs[k]) for k in range(n + 1))
    mag = sum(abs(mu[k]) * restrict(n - k, 0, ms[k]) for k in range(n + 1))
    return out, mag
