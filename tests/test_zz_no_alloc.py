"""fd_orthonormalize_noalloc: Cholesky-QR for callers that cannot let the
library allocate device memory (their GPU memory belongs to another allocator,
or they size their memory once at start-up).  Checked through the C ABI
against fd_orthonormalize on two calls in a row.  This file is collected last,
so a run that stops at the first failure has already run every other test."""
import numpy as np
import pytest

import fd_inputs

pytestmark = pytest.mark.gpu


def _t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def test_noalloc_matches_allocating_entry_point_twice():
    import torch

    import paper_2209_01974_gb300 as fd
    ctx = fd.fd_create(0)
    for call, (D, ns, seed) in enumerate([(20000, 96, 3), (5003, 40, 4)]):
        V0 = fd_inputs.random_block(D, ns, seed) @ np.diag(np.logspace(0, 4, ns))
        Va, Vb = _t(V0), _t(V0)
        Ra = torch.zeros((ns, ns), dtype=torch.float64, device="cuda")
        Rb = torch.zeros_like(Ra)
        pa = fd.fd_orthonormalize(ctx, Va, Ra)
        pb = fd.fd_orthonormalize_noalloc(ctx, Vb, Rb)
        assert pa == pb == 2, call
        Qa, Qb = Va.cpu().numpy(), Vb.cpu().numpy()
        assert np.abs(Qb.T @ Qb - np.eye(ns)).max() < 1e-14
        assert np.abs(Qa - Qb).max() <= 1e-10
        assert np.abs(Ra.cpu().numpy() - Rb.cpu().numpy()).max() <= 1e-12 * np.abs(Ra.cpu().numpy()).max()


def test_noalloc_rejects_blocks_beyond_its_maximum():
    import torch

    import paper_2209_01974_gb300 as fd
    ctx = fd.fd_create(0)
    V = torch.zeros((1000, 258), dtype=torch.float64, device="cuda")
    with pytest.raises(fd.FDError) as e:
        fd.fd_orthonormalize_noalloc(ctx, V)
    assert e.value.status == fd.FD_ERR_ARG and "maximum" in str(e.value)
