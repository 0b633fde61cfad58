"""Communication metrics of distributed SpMV (Sec. 3.1), from the sparsity pattern.

Test infrastructure only: the CUDA library never imports this module.

Rows are distributed uniformly over N_p processes: process p owns rows
[a_p, b_p) with a_p = floor(p D / N_p) (the paper only states b - a ~ D / N_p;
this split reproduces its Table 7 exactly).  For each process (Sec. 3.1):
  n_vm = |{ j in [a, b) : A_ij != 0 for some i in [a, b) }|   local vector entries
  n_vc = |{ j not in [a, b) : A_ij != 0 for some i in [a, b) }| remote entries
and the three metrics
  chi_1 = max_p n_vc / n_vm,   chi_2 = sum_p n_vc / D,   chi_3 = N_p max_p n_vc / D,
all zero for N_p = 1.  The pattern is the set of stored entries with a nonzero
value (an explicitly stored zero, such as a zero diagonal, is not an access).
"""
import numpy as np


def uniform_ranges(D, n_p):
    """Row ranges [a_p, b_p) of the uniform distribution."""
    a = (np.arange(n_p + 1, dtype=np.int64) * D) // n_p
    return a[:-1], a[1:]


def counts(csr, n_p):
    """(n_vc, n_vm) per process, int64 arrays of length n_p."""
    rowptr, col, val = csr
    D = len(rowptr) - 1
    a, b = uniform_ranges(D, n_p)
    rowptr = np.asarray(rowptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    nonzero = np.asarray(val) != 0
    n_vc = np.zeros(n_p, dtype=np.int64)
    n_vm = np.zeros(n_p, dtype=np.int64)
    read = np.zeros(D, dtype=bool)  # vector entries process p reads
    for p in range(n_p):
        lo, hi = rowptr[a[p]], rowptr[b[p]]
        read[:] = False
        read[col[lo:hi][nonzero[lo:hi]]] = True
        n_vm[p] = np.count_nonzero(read[a[p]:b[p]])
        n_vc[p] = np.count_nonzero(read) - n_vm[p]
    return n_vc, n_vm


def metrics(csr, n_p):
    """(chi_1, chi_2, chi_3, n_vc, n_vm) for the uniform distribution over n_p."""
    D = len(csr[0]) - 1
    n_vc, n_vm = counts(csr, n_p)
    if n_p == 1:
        return 0.0, 0.0, 0.0, n_vc, n_vm
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(n_vm > 0, n_vc / np.maximum(n_vm, 1), np.where(n_vc > 0, np.inf, 0.0))
    chi1 = float(r.max())
    chi2 = float(n_vc.sum()) / D
    chi3 = n_p * float(n_vc.max()) / D
    return chi1, chi2, chi3, n_vc, n_vm


def volumes(n_vc, n_p, n_b, S_d):
    """Average and maximal communication volume per process and SpMV in bytes
    (Sec. 3.1, Eqs. VCAve and VCMax): V = n_b S_d n_vc per process, so
    V_ave = n_b S_d sum_p n_vc / N_p = n_b D S_d chi_2 / N_p and
    V_max = n_b S_d max_p n_vc = n_b D S_d chi_3 / N_p."""
    n_vc = np.asarray(n_vc, dtype=np.int64)
    return n_b * S_d * float(n_vc.sum()) / n_p, float(n_b * S_d * int(n_vc.max()))
