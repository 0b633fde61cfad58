"""Failure detection with faults made on the host (none faults or hangs the
GPU): an allocation refused by a workspace cap, an inclusion interval that
misses part of the spectrum, and a corrupted matrix caught by the debug
index checks before any step kernel reads it."""
import numpy as np
import pytest

import fd_inputs
from oracle import matrices as mat
from oracle import ortho

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fd():
    import paper_2209_01974_gb300 as fd
    return fd


def _t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def test_workspace_cap_refuses_allocation_with_oom(fd):
    ctx = fd.fd_create(0)
    fd.fd_set_workspace_limit(ctx, 4096)
    V = _t(fd_inputs.random_block(20000, 96, 1))
    with pytest.raises(fd.FDError) as e:
        fd.fd_orthonormalize(ctx, V)
    assert e.value.status == fd.FD_ERR_OOM and "limit" in str(e.value)
    assert ctx.workspace[0] <= 4096
    fd.fd_set_workspace_limit(ctx, 0)          # lifted: the same call succeeds
    assert fd.fd_orthonormalize(ctx, V) == 2


def test_refused_digit_workspace_falls_back_to_fp64(fd):
    # the tensor-core products need 16 bytes per operand element for their
    # digits (268 MB here); with a 96 MB cap they are refused and the FP64
    # products run instead, with the same result
    D, ns = 131072, 128
    V0 = fd_inputs.random_block(D, ns, 8) @ np.diag(np.logspace(0, 3, ns))
    Qo, Ro, _ = ortho.cholqr2(V0)
    import torch
    free = fd.fd_create(0)
    fd.fd_set_gemm_mode(free, "ozaki")
    V = _t(V0)
    fd.fd_orthonormalize(free, V)
    assert free.workspace[0] > 200 << 20        # uncapped: the digit tiles were allocated
    capped = fd.fd_create(0)
    fd.fd_set_gemm_mode(capped, "ozaki")
    fd.fd_set_workspace_limit(capped, 96 << 20)
    V = _t(V0)
    R = torch.zeros((ns, ns), dtype=torch.float64, device="cuda")
    assert fd.fd_orthonormalize(capped, V, R) == 2
    assert capped.workspace[0] <= 96 << 20
    Q = V.cpu().numpy()
    assert np.abs(Q.T @ Q - np.eye(ns)).max() < 1e-14 * max(1, ns / 100)
    assert np.abs(R.cpu().numpy() - Ro).max() <= 1e-12 * np.abs(Ro).max()
    assert np.abs(Q - Qo).max() <= 1e-10


def test_too_narrow_inclusion_interval_is_widened(fd):
    # the 8-site chain's spectrum is [-4.2358, 20.2358]; starting from
    # [-4, 19] misses both ends: Ritz values outside widen the interval and the
    # solve still finds the wanted eigenvalues (the filter amplifies the
    # eigenvectors outside, but the Ritz step still resolves the window)
    spec = "hubbard:n_sites=8,n_up=4,n_dn=4,t=1,U=4,bc=open"
    ctx = fd.fd_create(0)
    A = fd.fd_build_matrix(ctx, spec)
    lam = np.linalg.eigvalsh(mat.to_scipy(mat.build(spec)).toarray())
    th, rho, res = fd.fd_solve(ctx, A, -0.5, 0.5, 20, 32, 100, 1e-9, lam_l=-4.0, lam_r=19.0)
    # moved out past the Ritz values found outside, which the filter has
    # amplified until they are the extreme eigenvalues
    assert res["lam_l"] < -4.0 and res["lam_r"] > 19.0
    assert res["lam_l"] <= lam[0] and res["lam_r"] >= lam[-1]
    want = np.sort(lam[np.lexsort((lam, np.abs(lam)))[:20]])
    assert res["converged"] == 1 and rho.max() <= 1e-9
    assert np.abs(th - want).max() <= 1e-10 * np.abs(lam).max()
    with pytest.raises(fd.FDError) as e:
        fd.fd_solve(ctx, A, -0.5, 0.5, 20, 32, 100, 1e-9, lam_l=3.0, lam_r=1.0)
    assert e.value.status == fd.FD_ERR_ARG


@pytest.mark.parametrize("bad", [10 ** 6, -3])
def test_debug_checks_report_a_corrupted_matrix(fd, bad):
    import torch
    ctx = fd.fd_create(0)
    fd.fd_set_debug_checks(ctx, True)
    A = fd.fd_build_matrix(ctx, "chain:n=1000")
    X = torch.zeros((1000, 8), dtype=torch.float64, device="cuda")
    Y = torch.empty_like(X)
    fd.fd_spmmv(ctx, A, X, Y)                   # a sound matrix passes the checks
    fd.fd_debug_set_sell_column(ctx, A, 37, bad)
    with pytest.raises(fd.FDError) as e:
        fd.fd_spmmv(ctx, A, X, Y)
    assert e.value.status == fd.FD_ERR_BOUNDS
    mu = np.array([0.5, 0.3, 0.2])
    with pytest.raises(fd.FDError) as e:
        fd.fd_filter(ctx, A, X, mu, 0.4, 0.0, torch.empty_like(X), torch.empty_like(X))
    assert e.value.status == fd.FD_ERR_BOUNDS
    with pytest.raises(fd.FDError) as e:
        fd.fd_solve(ctx, A, -0.1, 0.1, 4, 8, 20, 1e-9)
    assert e.value.status == fd.FD_ERR_BOUNDS
    A.free()                                    # never used without the checks
    torch.cuda.synchronize()                    # the context is still sound
    B = fd.fd_build_matrix(ctx, "chain:n=1000")
    fd.fd_spmmv(ctx, B, X, Y)
