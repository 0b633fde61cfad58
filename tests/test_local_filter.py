"""The restricted Alg. 2 of the full-size parity tests (tests/gpu_util.local_filter)
equals the oracle's whole-matrix filter on the rows it returns, and its
magnitude bound covers a perturbed run (no GPU)."""
import numpy as np
import pytest

import fd_inputs
from gpu_util import local_filter
from oracle import chebyshev as ch
from oracle import matrices as mat


@pytest.mark.parametrize("n", [2, 3, 4, 7])
def test_local_filter_equals_full_filter(n):
    csr = mat.hubbard(8, 4, 3, 1.0, 4.0, "periodic")
    A = mat.to_scipy(csr)
    D = A.shape[0]
    V0 = fd_inputs.random_block(D, 5, n)
    alpha, beta = ch.scale_params(-16.5, 28.5)
    mu = ch.filter_coeffs(alpha * 1.0 + beta, alpha * 2.0 + beta, n)
    full = ch.cheb_filter(A, V0, mu, alpha, beta)
    rows = np.array([0, 3, 17, 100, D - 1])

    def entries(r):
        return mat._hubbard_entries(8, 4, 3, 1.0, 4.0, "periodic", r)

    got, mag = local_filter(entries, rows, lambda idx: V0[idx], mu, alpha, beta)
    assert np.abs(got - full[rows]).max() <= 1e-13 * np.abs(full).max()
    # the magnitude sum dominates the exact values it bounds
    assert np.all(mag >= np.abs(got) - 1e-12)
