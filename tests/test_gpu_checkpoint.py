"""Checkpoint and resume of the FD loop (runs of the paper last up to 26 h,
Table 6): a solve stopped after k outer iterations, saved to a file, reloaded
in a fresh context with a freshly built matrix and resumed, repeats the
uninterrupted solve exactly."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CASES = [("hubbard:n_sites=8,n_up=4,n_dn=4,t=1,U=4,bc=open", -0.5, 0.5, 20, 32, 100, "f64", "ritz", 2),
         ("anderson3d:L=14,W=12,seed=5", -0.01, 0.01, 16, 16, 100, "f32", "lehmann", 3)]


@pytest.mark.parametrize("spec,a,b,nt,nb,deg,prec,iv,k", CASES)
def test_resumed_solve_repeats_uninterrupted_solve(tmp_path, spec, a, b, nt, nb, deg, prec, iv, k):
    import paper_2209_01974_gb300 as fd
    ctx = fd.fd_create(0)
    A = fd.fd_build_matrix(ctx, spec)
    th0, rho0, r0 = fd.fd_solve(ctx, A, a, b, nt, nb, deg, 1e-9, precision=prec, intervals=iv)
    assert r0["converged"] == 1 and r0["iterations"] > k
    th1, rho1, r1, ck = fd.fd_solve_checkpointed(ctx, A, a, b, nt, nb, deg, 1e-9, k, precision=prec,
                                                 intervals=iv)
    assert ck.state.converged == 0 and ck.state.iteration == k
    path = str(tmp_path / "fd_ckpt.npz")
    ck.save(path)
    del ck
    ctx2 = fd.fd_create(0)
    A2 = fd.fd_build_matrix(ctx2, spec)
    ck2 = fd.Checkpoint.load(path)
    th2, rho2, r2, ck2 = fd.fd_solve_checkpointed(ctx2, A2, a, b, nt, nb, deg, 1e-9, 1000, ck2,
                                                  precision=prec, intervals=iv)
    assert ck2.state.converged == 1 and r2["converged"] == 1
    assert r2["iterations"] == r0["iterations"] and r2["n_spmmv"] == r0["n_spmmv"]
    assert r2["final_degree"] == r0["final_degree"]
    assert np.array_equal(th2, th0) and np.array_equal(rho2, rho0)


def test_checkpoint_of_another_problem_is_rejected():
    import paper_2209_01974_gb300 as fd
    ctx = fd.fd_create(0)
    A = fd.fd_build_matrix(ctx, "chain:n=500")
    _, _, _, ck = fd.fd_solve_checkpointed(ctx, A, -0.05, 0.05, 4, 8, 40, 1e-9, 1)
    assert ck.state.iteration == 1
    B = fd.fd_build_matrix(ctx, "chain:n=400")
    with pytest.raises(fd.FDError) as e:
        fd.fd_solve_checkpointed(ctx, B, -0.05, 0.05, 4, 8, 40, 1e-9, 1, ck)
    assert e.value.status == fd.FD_ERR_ARG
