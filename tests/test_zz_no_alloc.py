"""fd_orthonormalize_noalloc: Cholesky-QR for callers that cannot let the
library allocate device memory (their GPU memory belongs to another allocator,
or they size their memory once at start-up).  Checked through the C ABI
against fd_orthonormalize on two calls in a row, against the oracle's CholQR2
on blocks large enough that fd_orthonormalize itself would take the
tensor-core products (D >= 65536, ns >= 64), and audited: a fresh context
holds no workspace and has made no cudaMalloc call before or after.  This file
is collected last, so a run that stops at the first failure has already run
every other test."""
import numpy as np
import pytest

import fd_inputs
from oracle import ortho

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


@pytest.mark.parametrize("mode", ["auto", "ozaki"])
def test_noalloc_large_block_matches_oracle_and_allocates_nothing(mode):
    # D >= 65536 and ns >= 64: fd_orthonormalize would use the tensor-core
    # products and their digit workspaces here; the allocation-free entry
    # point must not, in either gemm mode
    import torch

    import paper_2209_01974_gb300 as fd
    ctx = fd.fd_create(0)
    fd.fd_set_gemm_mode(ctx, mode)
    assert ctx.workspace == (0, 0)
    for call, (D, ns, seed) in enumerate([(70001, 64, 11), (131072, 128, 12)]):
        V0 = fd_inputs.random_block(D, ns, seed) @ np.diag(np.logspace(0, 3, ns))
        V = _t(V0)
        R = torch.zeros((ns, ns), dtype=torch.float64, device="cuda")
        passes = fd.fd_orthonormalize_noalloc(ctx, V, R)
        torch.cuda.synchronize()
        assert ctx.workspace == (0, 0), (mode, call)
        Qo, Ro, po = ortho.cholqr2(V0)
        assert passes == po == 2
        Q = V.cpu().numpy()
        assert np.abs(Q.T @ Q - np.eye(ns)).max() < 1e-14 * max(1, ns / 100)
        assert np.abs(R.cpu().numpy() - Ro).max() <= 1e-12 * np.abs(Ro).max()
        assert np.abs(Q - Qo).max() <= 1e-10


def test_noalloc_rejects_blocks_beyond_its_maximum():
    import torch

    import paper_2209_01974_gb300 as fd
    ctx = fd.fd_create(0)
    V = torch.zeros((1000, 258), dtype=torch.float64, device="cuda")
    with pytest.raises(fd.FDError) as e:
        fd.fd_orthonormalize_noalloc(ctx, V)
    assert e.value.status == fd.FD_ERR_ARG and "maximum" in str(e.value)
